// k_rates4_d14.cu - instantiations of the fused four-phonon kernel (double, 1..4 atoms per cell);
// split across translation units so that they compile in parallel.
#include "k_rates4_tile.cuh"

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

cudaError_t launch4_tile_f(int na, const Tables &, const RateArgs &, int, cudaStream_t);
cudaError_t launch4_tile_d(int na, const Tables &, const RateArgs &, int, cudaStream_t);

// The tiled kernel (k_rates4_tile.cuh) serves cells of <= 2 atoms whose tile fits in shared
// memory; every other case uses the general kernel.
size_t rates4_wbuf_per_mode(const Tables &t, int fp64) {
    const int na = t.n_atoms;
    if (na > 2) return 0;
    const size_t smem = fp64 ? (na == 1 ? tile_smem_bytes<double, 1>(t) : tile_smem_bytes<double, 2>(t))
                             : (na == 1 ? tile_smem_bytes<float, 1>(t) : tile_smem_bytes<float, 2>(t));
    if (smem > 200 * 1024) return 0;
    return fp64 ? (na == 1 ? tile_w_bytes_per_mode<double, 1>(t) : tile_w_bytes_per_mode<double, 2>(t))
                : (na == 1 ? tile_w_bytes_per_mode<float, 1>(t) : tile_w_bytes_per_mode<float, 2>(t));
}

cudaError_t launch_rates4(const Tables &t, RateArgs &a, int ch, int fp64, int threads,
                          cudaStream_t s) {
    const int na = t.n_atoms;
    const size_t per_mode = rates4_wbuf_per_mode(t, fp64);
    if (per_mode && a.wbuf && a.wbuf_bytes >= per_mode) {
        a.n_part[ch] = t.N;
        return fp64 ? launch4_tile_d(na, t, a, ch, s) : launch4_tile_f(na, t, a, ch, s);
    }
    a.n_part[ch] = t.N;
    if (threads <= 0) threads = 128;
    if (threads % 32 || threads > 256) return cudaErrorInvalidValue;
    if (fp64) return na <= 4 ? launch4_d_1_4(na, t, a, ch, threads, s) : launch4_d_5_8(na, t, a, ch, threads, s);
    return na <= 4 ? launch4_f_1_4(na, t, a, ch, threads, s) : launch4_f_5_8(na, t, a, ch, threads, s);
}

}  // namespace fc4
