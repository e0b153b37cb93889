// k_rates4_f58.cu - instantiations of the fused four-phonon kernel (float, 5..8 atoms per cell,
// fixed σ); split across translation units so that they compile in parallel.
#include "k_rates4_batch.cuh"

namespace fc4 {

cudaError_t launch4_f_5_8(int na, const Tables &t, const RateArgs &a, int ch, int threads, cudaStream_t s) {
    return launch4_atoms<float, false, 5, 8>(na, t, a, ch, threads, s);
}

cudaError_t launch4_batch_f_5_8(int na, const int4 *items, int n_items, int *counter, size_t smem,
                                cudaStream_t s) {
    return launch4_batch_atoms<float, 5, 8>(na, items, n_items, counter, smem, s);
}

cudaError_t batch_upload_f_5_8(const Tables *tabs, const RateArgs *args, int n, cudaStream_t s) {
    return batch_upload(tabs, args, n, s);
}

}  // namespace fc4
