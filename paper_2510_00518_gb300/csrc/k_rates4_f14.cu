// k_rates4_f14.cu - instantiations of the fused four-phonon kernel (float, 1..4 atoms per cell);
// split across translation units so that they compile in parallel.
#include "k_rates4.cuh"

namespace fc4 {

cudaError_t launch4_f_1_4(int na, const Tables &t, const RateArgs &a, int ch, int threads,
                               cudaStream_t s) {
    switch (na) {
    case 1: return launch4<float, 1>(t, a, ch, threads, s);
    case 2: return launch4<float, 2>(t, a, ch, threads, s);
    case 3: return launch4<float, 3>(t, a, ch, threads, s);
    case 4: return launch4<float, 4>(t, a, ch, threads, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace fc4
