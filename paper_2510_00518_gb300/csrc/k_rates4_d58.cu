// k_rates4_d58.cu - instantiations of the fused four-phonon kernel (double, 5..8 atoms per cell);
// split across translation units so that they compile in parallel.
#include "k_rates4.cuh"

namespace fc4 {

cudaError_t launch4_d_5_8(int na, const Tables &t, const RateArgs &a, int ch, int threads,
                               cudaStream_t s) {
    switch (na) {
    case 5: return launch4<double, 5>(t, a, ch, threads, s);
    case 6: return launch4<double, 6>(t, a, ch, threads, s);
    case 7: return launch4<double, 7>(t, a, ch, threads, s);
    case 8: return launch4<double, 8>(t, a, ch, threads, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace fc4
