// k_rates4_d14.cu - instantiations of the fused four-phonon kernel (double, 1..4 atoms per cell);
// split across translation units so that they compile in parallel.
#include "k_rates4.cuh"

namespace fc4 {

cudaError_t launch4_d_1_4(int na, const Tables &t, const RateArgs &a, int ch, int threads,
                               cudaStream_t s) {
    switch (na) {
    case 1: return launch4<double, 1>(t, a, ch, threads, s);
    case 2: return launch4<double, 2>(t, a, ch, threads, s);
    case 3: return launch4<double, 3>(t, a, ch, threads, s);
    case 4: return launch4<double, 4>(t, a, ch, threads, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch4_d_5_8(int, const Tables &, const RateArgs &, int, int, cudaStream_t);
cudaError_t launch4_f_1_4(int, const Tables &, const RateArgs &, int, int, cudaStream_t);
cudaError_t launch4_f_5_8(int, const Tables &, const RateArgs &, int, int, cudaStream_t);

cudaError_t launch_rates4(const Tables &t, const RateArgs &a, int ch, int fp64, int threads,
                          cudaStream_t s) {
    if (threads <= 0) threads = 128;
    if (threads % 32 || threads > 256) return cudaErrorInvalidValue;
    const int na = t.n_atoms;
    if (fp64) return na <= 4 ? launch4_d_1_4(na, t, a, ch, threads, s) : launch4_d_5_8(na, t, a, ch, threads, s);
    return na <= 4 ? launch4_f_1_4(na, t, a, ch, threads, s) : launch4_f_5_8(na, t, a, ch, threads, s);
}

}  // namespace fc4
