// k_rates4_d58.cu - instantiations of the fused four-phonon kernel (double, 5..8 atoms per cell,
// fixed σ); split across translation units so that they compile in parallel.
#include "k_rates4.cuh"

namespace fc4 {

cudaError_t launch4_d_5_8(int na, const Tables &t, const RateArgs &a, int ch, int threads, cudaStream_t s) {
    return launch4_atoms<double, false, 5, 8>(na, t, a, ch, threads, s);
}

}  // namespace fc4
