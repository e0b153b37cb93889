// fc4_window.cuh - energy window and Gaussian with adaptive broadening, shared by the rate kernels
// and the process lists.
//
// The width of a process comes from the two legs its free partner sum moves together (3ph: λ' and
// λ'', 4ph: λ'' and λ'''): σ = s sqrt(Σ_k ((Δv . b_k) / n_k)² / 6).  A process is kept iff
// σ > σ_min = 1e-9 rad/ps and |Δ| <= 2σ, both in FP64 in the order of the definition (velocities
// equal by symmetry differ by rounding noise only; the 1/σ weight of such a width is meaningless).  The FP32 prefilter works on
// P_k = (v . b_k) / n_k stored per mode as hi/lo pairs and on the FP32 mismatch; with
//   |Δ32 - Δ| <= 13 u ω_max  and  |2σ32 - 2σ| <= 10 u 2σ32 + 2^-41 (2s/√6) Q   (u = 2^-24,
//   Q >= max_k |P_k| and the FP64 rounding of the oracle's own σ, see the host's margin),
// a candidate is kept for sure when |Δ32| <= (1 - 32u) 2σ32 - e0 and 2σ32 > g_min (which
// implies σ > σ_min), rejected for sure when
// |Δ32| > (1 + 32u) 2σ32 + e0, and decided by the exact FP64 test otherwise; e0 = 64 u ω_max +
// 2^-40 (2s/√6) Q also absorbs the rounding of the thresholds.  Kept sets therefore equal those
// of the exact test bit for bit.
#pragma once
#include "fc4_device.cuh"
#include "fc4_kernels.h"

namespace fc4 {

constexpr double kSqrtPi = 1.7724538509055160273;
constexpr float kInvSqrtPiF = 0.56418958354775628695f;

// 2σ of the pair (ma, mb) in FP32 (prefilter)
__device__ __forceinline__ float two_sigma32(const Tables &t, const RateArgs &a, int ma, int mb) {
    return a.ad_c32 * vel_diff_norm32(t.vp32[ma], t.vp32lo[ma], t.vp32[mb], t.vp32lo[mb]);
}

// exact FP64 σ of the pair (ma, mb)
__device__ __forceinline__ double sigma_exact(const Tables &t, const RateArgs &a, int ma, int mb) {
    return sigma_adaptive_exact(t.vel + 3 * (size_t)ma, t.vel + 3 * (size_t)mb, t.recip, t.mesh, a.ad_scale);
}

// FP32 prefilter with adaptive σ: 2 keep, 1 ambiguous, 0 reject
__device__ __forceinline__ int window_adaptive32(const RateArgs &a, float ad, float g32) {
    if (ad <= fmaf(a.ad_rlo, g32, -a.ad_e0) && g32 > a.ad_gmin) return 2;
    return ad <= fmaf(a.ad_rhi, g32, a.ad_e0) ? 1 : 0;
}

// Exact decision (out of line: it is rare).  m3 < 0 for the three-phonon channels.
static __device__ __noinline__ bool window_exact_adaptive(const Tables &t, const RateArgs &a, int ch, int m0,
                                                          int m1, int m2, int m3, int ma, int mb) {
    const double sg = sigma_exact(t, a, ma, mb);
    if (!(sg > kAdaptiveSigmaMin)) return false;
    const double d = delta_exact(ch, t.om[m0], t.om[m1], t.om[m2], m3 >= 0 ? t.om[m3] : 0.0);
    return fabs(d) <= __dmul_rn(2.0, sg);
}

// Gaussian exp(-Δ²/σ²) / (σ sqrt(π)) with the pair's adaptive σ: FP64 and FP32 (mixed weights)
__device__ __forceinline__ double gauss_adaptive(const Tables &t, const RateArgs &a, double d, int ma, int mb) {
    const double sg = sigma_exact(t, a, ma, mb);
    return exp(-(d * d) / (sg * sg)) / (sg * kSqrtPi);
}

__device__ __forceinline__ float gauss_adaptive32(const Tables &t, const RateArgs &a, float d, int ma, int mb) {
    float sg = a.ad_s32 * vel_diff_norm32(t.vp32[ma], t.vp32lo[ma], t.vp32[mb], t.vp32lo[mb]);
    if (!(sg > 0.0f)) sg = (float)sigma_exact(t, a, ma, mb);   // |ΔP| below FP32 resolution
    const float rs = __frcp_rn(sg);
    const float r = d * rs;
    return __expf(-(r * r)) * (kInvSqrtPiF * rs);
}

// Sampling estimate of the four-phonon sums (fc4_set_sampling): the partner pair (λ, q', q'')
// enters with probability f, decided by SplitMix64's output function (Steele, Lea and Flood,
// OOPSLA 2014) of the counter seed + (key + 1) x 0x9e3779b97f4a7c15, key = (mode N + q') N + q'';
// the pair is in the sample iff the hash is below floor(f 2^64).
__device__ __forceinline__ bool pair_sampled(const RateArgs &a, int m0, int q1, int q2, int N) {
    const unsigned long long key = ((unsigned long long)m0 * (unsigned long long)N + (unsigned long long)q1) *
                                       (unsigned long long)N + (unsigned long long)q2;
    unsigned long long z = a.sample_seed + (key + 1ull) * 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return (z ^ (z >> 31)) < a.sample_threshold;
}

// Window row of one (q'', λ''') for the four-phonon channels with adaptive σ: bit j'' set iff kept.
template <int NB>
static __device__ __noinline__ unsigned window_adaptive4_row(const Tables &t, const RateArgs &a, int ch, int s2,
                                                             float base32, int m0, int m1, int q2, int m3,
                                                             unsigned v2) {
    const float w3 = t.om32[m3];
    const float4 h3 = t.vp32[m3], l3 = t.vp32lo[m3];
    unsigned keep = 0;
    for (int j2 = 0; j2 < NB; ++j2) {
        if (!((v2 >> j2) & 1u)) continue;
        const int m2 = q2 * NB + j2;
        const float ad = fabsf((base32 + (float)s2 * t.om32[m2]) - w3);
        const float g32 = a.ad_c32 * vel_diff_norm32(t.vp32[m2], t.vp32lo[m2], h3, l3);
        const int w = window_adaptive32(a, ad, g32);
        if (w == 2 || (w == 1 && window_exact_adaptive(t, a, ch, m0, m1, m2, m3, m2, m3))) keep |= 1u << j2;
    }
    return keep;
}

}  // namespace fc4
