// fc4_device.cuh - device-side helpers shared by the kernels of libfc4: complex arithmetic for
// double2 / float2, integer mesh arithmetic, the exact FP64 energy-window test, deterministic
// block scans and reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fc4 {

constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------------------ complex

template <typename R> struct CplxOf;
template <> struct CplxOf<double> { using type = double2; };
template <> struct CplxOf<float> { using type = float2; };
template <typename R> using Cplx = typename CplxOf<R>::type;

__host__ __device__ __forceinline__ double2 cmake(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 cmake(float a, float b) { return make_float2(a, b); }

template <typename C> __device__ __forceinline__ C czero() { C z; z.x = 0; z.y = 0; return z; }
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// acc + a * b
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C acc) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
    return acc;
}
// acc + s * a (s real)
template <typename C, typename R> __device__ __forceinline__ C crfma(R s, C a, C acc) {
    acc.x = fma(s, a.x, acc.x);
    acc.y = fma(s, a.y, acc.y);
    return acc;
}
template <typename C> __device__ __forceinline__ C cconj_if(C a, bool c) { if (c) a.y = -a.y; return a; }
template <typename C> __device__ __forceinline__ double cabs2(C a) {
    return (double)a.x * (double)a.x + (double)a.y * (double)a.y;
}

// ------------------------------------------------------------------------------ mesh

__device__ __forceinline__ int mod_pos(int x, int n) {
    int r = x % n;
    return r < 0 ? r + n : r;
}

// index of the mesh point with integer coordinates c (any integers), first axis fastest
__device__ __forceinline__ int q_index(int c0, int c1, int c2, int n0, int n1, int n2) {
    return mod_pos(c0, n0) + n0 * (mod_pos(c1, n1) + n1 * mod_pos(c2, n2));
}

// x mod n for x in [-2n, 3n) (sums of up to three mesh coordinates with signs): no division
__device__ __forceinline__ int mod_near(int x, int n) {
    x = x < 0 ? x + n : x;
    x = x < 0 ? x + n : x;
    x = x >= n ? x - n : x;
    x = x >= n ? x - n : x;
    return x;
}

__device__ __forceinline__ int q_index_near(int c0, int c1, int c2, int n0, int n1, int n2) {
    return mod_near(c0, n0) + n0 * (mod_near(c1, n1) + n1 * mod_near(c2, n2));
}

// phase index of exp(i q.R) = exp(2πi k / L): k = Σ_a q_a R_a (L / n_a) mod L, where rl holds
// the precomputed R_a (L / n_a) reduced modulo L
__device__ __forceinline__ int phase_index(int4 q, int4 rl, int L) {
    return mod_pos(q.x * rl.x + q.y * rl.y + q.z * rl.z, L);
}

// ------------------------------------------------------------------------------ window

// Energy mismatch Δ of channel ch, IEEE FP64 with the fixed parenthesisation of the interface
// (explicit round-to-nearest intrinsics: never reassociated or contracted).
__device__ __forceinline__ double delta_exact(int ch, double w, double w1, double w2, double w3) {
    switch (ch) {
    case 0: return __dsub_rn(__dadd_rn(w, w1), w2);
    case 1: return __dsub_rn(w, __dadd_rn(w1, w2));
    case 2: return __dadd_rn(__dsub_rn(w, w3), __dadd_rn(w1, w2));
    case 3: return __dsub_rn(__dadd_rn(w, w1), __dadd_rn(w2, w3));
    default: {
        double a = w1, b = w2, c = w3, t;
        if (a > b) { t = a; a = b; b = t; }
        if (b > c) { t = b; b = c; c = t; }
        if (a > b) { t = a; a = b; b = t; }
        return __dsub_rn(w, __dadd_rn(__dadd_rn(a, b), c));
    }
    }
}

// Bose-Einstein occupation factor of channel ch (forward minus backward rates over partners)
template <typename R>
__device__ __forceinline__ R occupation_factor(int ch, R n1, R n2, R n3) {
    const R one = R(1);
    switch (ch) {
    case 0: return n1 - n2;
    case 1: return one + n1 + n2;
    case 2: return n1 * n2 * (one + n3) - (one + n1) * (one + n2) * n3;
    case 3: return n1 * (one + n2) * (one + n3) - (one + n1) * n2 * n3;
    default: return (one + n1) * (one + n2) * (one + n3) - n1 * n2 * n3;
    }
}

// ------------------------------------------------------------------------------ adaptive width

// Adaptive Gaussian width of two modes from their group velocities v_a, v_b (Å rad/ps), the
// reciprocal vectors b (rows, 1/Å) and the mesh n:
//   σ = s sqrt(Σ_k ((Δv . b_k) / n_k)² / 6),  Δv = v_a - v_b,
// in IEEE FP64 with every operation rounded to nearest in the order written (never contracted or
// reassociated), so that the window decision σ > 0 and |Δ| <= 2σ is reproducible bit for bit.
__device__ __forceinline__ double sigma_adaptive_exact(const double *va, const double *vb, const double *b,
                                                       const int *n, double s) {
    const double d0 = __dsub_rn(va[0], vb[0]), d1 = __dsub_rn(va[1], vb[1]), d2 = __dsub_rn(va[2], vb[2]);
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double x = __dadd_rn(__dadd_rn(__dmul_rn(d0, b[3 * k]), __dmul_rn(d1, b[3 * k + 1])),
                             __dmul_rn(d2, b[3 * k + 2]));
        x = __ddiv_rn(x, (double)n[k]);
        acc = __dadd_rn(acc, __dmul_rn(x, x));
    }
    return __dmul_rn(s, __dsqrt_rn(__ddiv_rn(acc, 6.0)));
}

// |ΔP| for the FP32 prefilter and the mixed-precision weight, where P_k = (v . b_k) / n_k is stored
// per mode as an FP32 hi/lo pair: the hi parts of two close velocities subtract exactly, so the
// difference is accurate to a few ulp of itself plus ~2^-45 max|P|.
__device__ __forceinline__ float vel_diff_norm32(float4 ha, float4 la, float4 hb, float4 lb) {
    const float x = (ha.x - hb.x) + (la.x - lb.x);
    const float y = (ha.y - hb.y) + (la.y - lb.y);
    const float z = (ha.z - hb.z) + (la.z - lb.z);
    return __fsqrt_rn(x * x + y * y + z * z);
}

// ------------------------------------------------------------------------------ block helpers

// Exclusive scan of one int per thread across the block (blockDim.x a multiple of 32, <= 1024).
// Deterministic.  s_warp must hold 32 ints.  Returns the prefix; *total gets the block sum.
__device__ __forceinline__ int block_exclusive_scan(int v, int *s_warp, int *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < nw ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFull, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) s_warp[lane] = t;
    }
    __syncthreads();
    int off = (wid ? s_warp[wid - 1] : 0) + x - v;
    *total = s_warp[nw - 1];
    __syncthreads();
    return off;
}

// Deterministic block sum (fixed butterfly per warp, warps added in order by thread 0).
// s_red must hold 32 values; the result is valid in thread 0.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *s_red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (lane == 0) s_red[wid] = v;
    __syncthreads();
    T r = T(0);
    if (threadIdx.x == 0)
        for (int w = 0; w < nw; ++w) r += s_red[w];
    __syncthreads();
    return r;
}

// Several deterministic block sums in one pass (two barriers); results valid in thread 0.
// s_d must hold 32 * ND doubles, s_n 32 * NL long longs.
template <int ND, int NL>
__device__ __forceinline__ void block_sum_multi(double (&d)[ND], long long (&n)[NL], double *s_d, long long *s_n) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < ND; ++k) d[k] += __shfl_xor_sync(kFull, d[k], o);
#pragma unroll
        for (int k = 0; k < NL; ++k) n[k] += __shfl_xor_sync(kFull, n[k], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < ND; ++k) s_d[32 * k + wid] = d[k];
#pragma unroll
        for (int k = 0; k < NL; ++k) s_n[32 * k + wid] = n[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < ND; ++k) {
            double r = 0.0;
            for (int w = 0; w < nw; ++w) r += s_d[32 * k + w];
            d[k] = r;
        }
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            long long r = 0;
            for (int w = 0; w < nw; ++w) r += s_n[32 * k + w];
            n[k] = r;
        }
    }
    __syncthreads();
}

}  // namespace fc4
