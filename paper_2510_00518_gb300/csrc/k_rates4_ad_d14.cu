// k_rates4_ad_d14.cu - instantiations of the fused four-phonon kernel (double, 1..4 atoms per cell,
// adaptive σ); split across translation units so that they compile in parallel.
#include "k_rates4.cuh"

namespace fc4 {

cudaError_t launch4_ad_d_1_4(int na, const Tables &t, const RateArgs &a, int ch, int threads, cudaStream_t s) {
    return launch4_atoms<double, true, 1, 4>(na, t, a, ch, threads, s);
}

}  // namespace fc4
