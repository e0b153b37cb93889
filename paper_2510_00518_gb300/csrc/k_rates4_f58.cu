// k_rates4_f58.cu - instantiations of the fused four-phonon kernel (float, 5..8 atoms per cell);
// split across translation units so that they compile in parallel.
#include "k_rates4.cuh"

namespace fc4 {

cudaError_t launch4_f_5_8(int na, const Tables &t, const RateArgs &a, int ch, int threads,
                               cudaStream_t s) {
    switch (na) {
    case 5: return launch4<float, 5>(t, a, ch, threads, s);
    case 6: return launch4<float, 6>(t, a, ch, threads, s);
    case 7: return launch4<float, 7>(t, a, ch, threads, s);
    case 8: return launch4<float, 8>(t, a, ch, threads, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace fc4
