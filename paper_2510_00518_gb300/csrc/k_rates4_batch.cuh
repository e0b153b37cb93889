// k_rates4_batch.cuh - persistent four-phonon launch over many contexts of one cell size (FP32,
// fixed σ), included by the translation units that instantiate the general kernel in FP32.
//
// Each block takes the next work item (context, channel, unit) from a list ordered from the
// largest meshes down, through a global counter zeroed before the launch, and runs the unit with
// the general kernel's body (rates4_unit), until the list is exhausted.  The contexts' tables and
// call arguments sit in this translation unit's constant memory: every thread of a block reads
// the same context, so the reads are uniform constant-cache hits, as for a kernel parameter (from
// global memory the persistent form ran 1.2x slower than one launch per crystal).
#pragma once
#include "k_rates4.cuh"

namespace fc4 {

constexpr int kMaxBatchContexts = 40;
static __constant__ Tables c_batch_tabs[kMaxBatchContexts];
static __constant__ RateArgs c_batch_args[kMaxBatchContexts];

template <typename R, int NA>
__global__ void __launch_bounds__(128, 4)
rates4_batch_kernel(const int4 *__restrict__ items, int n_items, int *counter) {
    __shared__ int s_item;
    for (;;) {
        __syncthreads();                                 // the previous unit is done with shared memory
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int i = s_item;
        if (i >= n_items) break;
        const int4 it = items[i];                        // (context, channel, unit, -)
        rates4_unit<R, NA, false>(c_batch_tabs[it.x], c_batch_args[it.x], it.y, it.z);
    }
}

// Copy the contexts' tables and arguments into this unit's constant memory (stream-ordered).
inline cudaError_t batch_upload(const Tables *tabs, const RateArgs *args, int n, cudaStream_t s) {
    if (n > kMaxBatchContexts) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyToSymbolAsync(c_batch_tabs, tabs, sizeof(Tables) * n, 0, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbolAsync(c_batch_args, args, sizeof(RateArgs) * n, 0, cudaMemcpyHostToDevice, s);
}

// The persistent kernel on a grid that fills the device (resident blocks per SM x SMs).
template <typename R, int NA>
cudaError_t launch4_batch(const int4 *items, int n_items, int *counter, size_t smem, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(rates4_batch_kernel<R, NA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rates4_batch_kernel<R, NA>, 128, smem)) != cudaSuccess)
        return e;
    const int grid = std::max(1, std::min(n_items, sms * std::max(per_sm, 1)));
    rates4_batch_kernel<R, NA><<<grid, 128, smem, s>>>(items, n_items, counter);
    return cudaGetLastError();
}

template <typename R, int NA, int HI>
cudaError_t launch4_batch_atoms(int na, const int4 *items, int n_items, int *counter, size_t smem, cudaStream_t s) {
    if (na == NA) return launch4_batch<R, NA>(items, n_items, counter, smem, s);
    if constexpr (NA < HI) return launch4_batch_atoms<R, NA + 1, HI>(na, items, n_items, counter, smem, s);
    else return cudaErrorInvalidValue;
}

}  // namespace fc4
