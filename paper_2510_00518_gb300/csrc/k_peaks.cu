// k_peaks.cu - calibration kernels: the FP32 and FP64 fused multiply-add rates of the current
// device, the denominators of the rate kernels' roofline (their arithmetic runs on the CUDA
// cores, whose peak no library figure gives).
//
// Every thread runs kChains independent FMA chains (enough independent work to hide the FMA
// latency at full occupancy) for a fixed number of iterations; the grid holds 8 blocks of 256
// threads per SM.  Flops = 2 x threads x chains x iterations, timed with CUDA events after a
// warm-up launch.  The chains' sum is stored so that the work cannot be removed.
#include <cuda_runtime.h>

#include "fc4.h"

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(int iters, T a, T b, T *out) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)-12345.0) out[0] = s;           // never true for the chosen a, b; keeps the chains live
}

template <typename T>
cudaError_t time_peak(int iters, cudaStream_t s, double *tflops) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int grid = 8 * sms;
    cudaEvent_t ev0, ev1;
    if ((e = cudaEventCreate(&ev0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&ev1)) != cudaSuccess) { cudaEventDestroy(ev0); return e; }
    const T a = (T)0.999999, b = (T)1e-7;
    fma_peak_kernel<T><<<grid, kPeakThreads, 0, s>>>(iters, a, b, nullptr);          // warm-up
    cudaEventRecord(ev0, s);
    fma_peak_kernel<T><<<grid, kPeakThreads, 0, s>>>(iters, a, b, nullptr);
    cudaEventRecord(ev1, s);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * grid * kPeakThreads * (double)kChains * 16.0 * iters;
    *tflops = ms > 0.0f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    return cudaSuccess;
}

}  // namespace

extern "C" fc4_status fc4_device_peaks(double out[2], void *stream) {
    if (!out) return FC4_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    if (time_peak<float>(4096, s, &out[0]) != cudaSuccess) return FC4_ERR_CUDA;
    if (time_peak<double>(128, s, &out[1]) != cudaSuccess) return FC4_ERR_CUDA;
    return FC4_OK;
}
