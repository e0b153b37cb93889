// k_rates4_d14.cu - the four-phonon dispatcher (tiled or general kernel, precision, fixed or
// adaptive σ) and the instantiations of the general kernel for double, 1..4 atoms, fixed σ.
#include "k_rates4_tile.cuh"

namespace fc4 {

cudaError_t launch4_d_1_4(int na, const Tables &t, const RateArgs &a, int ch, int threads, cudaStream_t s) {
    return launch4_atoms<double, false, 1, 4>(na, t, a, ch, threads, s);
}

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
    const bool ad = a.adaptive != 0;
    if (a.part_d) {                        // iterative BTE: the tiled kernels only
        if (!(per_mode && a.wbuf && a.wbuf_bytes >= per_mode)) return cudaErrorInvalidValue;
        a.n_part[ch] = t.N;
        return fp64 ? launch4_tile_bte_d(na, t, a, ch, s) : launch4_tile_bte_f(na, t, a, ch, s);
    }
    if (per_mode && a.wbuf && a.wbuf_bytes >= per_mode) {
        a.n_part[ch] = t.N;
        if (ad) return fp64 ? launch4_tile_ad_d(na, t, a, ch, s) : launch4_tile_ad_f(na, t, a, ch, s);
        return fp64 ? launch4_tile_d(na, t, a, ch, s) : launch4_tile_f(na, t, a, ch, s);
    }
    a.n_part[ch] = t.N;
    if (threads <= 0) threads = 128;
    if (threads % 32 || threads > 256) return cudaErrorInvalidValue;
    const bool lo = na <= 4;
    if (ad) {
        if (fp64) return lo ? launch4_ad_d_1_4(na, t, a, ch, threads, s) : launch4_ad_d_5_8(na, t, a, ch, threads, s);
        return lo ? launch4_ad_f_1_4(na, t, a, ch, threads, s) : launch4_ad_f_5_8(na, t, a, ch, threads, s);
    }
    if (fp64) return lo ? launch4_d_1_4(na, t, a, ch, threads, s) : launch4_d_5_8(na, t, a, ch, threads, s);
    return lo ? launch4_f_1_4(na, t, a, ch, threads, s) : launch4_f_5_8(na, t, a, ch, threads, s);
}

}  // namespace fc4
