// k_rates4.cuh - fused four-phonon kernel: enumeration, energy window, matrix element V4,
// weight and per-(λ, q') reduction, for one channel (++, +-, --).
//
// The paper (Algorithms 3-4) enumerates the kept processes on the CPU, ships index lists to
// the GPU and evaluates V per process.  Here the same work is fused and factored so that the
// dense parts are shared.  One thread block owns a unit (λ = (q, j), q') and loops over the
// partner branch j'.  With q''' = q + s1 q' + s2 q'', the phase of a cluster factorises as
//   exp(i(s1 q'.R1 + s2 q''.R2 - q'''.R3)) = exp(-i q.R3) exp(i s1 q'.(R1 - R3)) exp(i s2 q''.(R2 - R3)),
// so with a "key" r = (leg-2 atom c, leg-3 atom d, R2 - R3) the element is
//   V = Σ_r P_r(q'')^s2 Σ_γδ W_r[γδ] e^s2_λ''(cγ) e*_λ'''(dδ),
//   W_r[γδ] = Σ_{clusters in r} exp(-i q.R3 + i s1 q'.(R1 - R3)) / sqrt(m) Σ_αβ Φ[αβγδ] e_λ(aα) e^s1_λ'(bβ),
// W built once per (λ, q', j') in shared memory.  Partners q'' are enumerated one per thread,
// the window is tested with an FP32 prefilter of proven error bound (ambiguous cases are
// decided by the exact FP64 Δ), kept (q'', j''', j''-mask) items are compacted in order by a
// block scan, and each item computes Y[cγ] = Σ_r P_r Σ_δ W_r[γδ] e*_λ'''(dδ) once for all its
// j'' (V = Σ_cγ e^s2_λ''(cγ) Y[cγ]).
#pragma once
#include <algorithm>

#include "fc4_window.cuh"

namespace fc4 {

template <typename R>
struct Sel {
    static __device__ __forceinline__ const Cplx<R> *ev(const Tables &t);
    static __device__ __forceinline__ const Cplx<R> *rt(const Tables &t);
    static __device__ __forceinline__ const Cplx<R> *P4(const Tables &t);
    static __device__ __forceinline__ const R *phi4(const Tables &t);
    static __device__ __forceinline__ const R *ism4(const Tables &t);
    static __device__ __forceinline__ const R *occ(const Tables &t);
    static __device__ __forceinline__ const R *invw(const Tables &t);
    static __device__ __forceinline__ const R *om(const Tables &t);
    static __device__ __forceinline__ const R *bteF(const RateArgs &a);
};
template <> struct Sel<double> {
    static __device__ __forceinline__ const double2 *ev(const Tables &t) { return t.ev; }
    static __device__ __forceinline__ const double2 *rt(const Tables &t) { return t.rt; }
    static __device__ __forceinline__ const double2 *P4(const Tables &t) { return t.P4; }
    static __device__ __forceinline__ const double *phi4(const Tables &t) { return t.phi4; }
    static __device__ __forceinline__ const double *ism4(const Tables &t) { return t.c4_ism; }
    static __device__ __forceinline__ const double *occ(const Tables &t) { return t.occ; }
    static __device__ __forceinline__ const double *invw(const Tables &t) { return t.invw; }
    static __device__ __forceinline__ const double *om(const Tables &t) { return t.om; }
    static __device__ __forceinline__ const double *bteF(const RateArgs &a) { return a.bte_F; }
};
template <> struct Sel<float> {
    static __device__ __forceinline__ const float2 *ev(const Tables &t) { return t.ev32; }
    static __device__ __forceinline__ const float2 *rt(const Tables &t) { return t.rt32; }
    static __device__ __forceinline__ const float2 *P4(const Tables &t) { return t.P4_32; }
    static __device__ __forceinline__ const float *phi4(const Tables &t) { return t.phi4_32; }
    static __device__ __forceinline__ const float *ism4(const Tables &t) { return t.c4_ism32; }
    static __device__ __forceinline__ const float *occ(const Tables &t) { return t.occ32; }
    static __device__ __forceinline__ const float *invw(const Tables &t) { return t.invw32; }
    static __device__ __forceinline__ const float *om(const Tables &t) { return t.om32; }
    static __device__ __forceinline__ const float *bteF(const RateArgs &a) { return a.bte_F32; }
};

// Exact FP64 decision for the rare candidates inside the prefilter's ambiguity band (kept out of
// line: the unrolled branch loops stay small).
static __device__ __noinline__ bool window_exact4(int ch, double w0, double w1, double w2, double w3,
                                            double two_sigma) {
    return fabs(delta_exact(ch, w0, w1, w2, w3)) <= two_sigma;
}

// symmetry factor of the 4ph channels: 1/2 (++, +-), 1/6 (--)
template <typename R> __device__ __forceinline__ R sym4(int ch) { return ch == 4 ? R(1) / R(6) : R(0.5); }

constexpr int kQChunk = 1024;      // partner q'' handled per compaction round

// Error-free sum: a + b = s + e exactly (Knuth's TwoSum, round-to-nearest FP32).
__device__ __forceinline__ float two_sum(float a, float b, float &e) {
    const float s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
    return s;
}

// Δ = ω + s1 ω' + s2 ω'' - ω''' from hi/lo FP32 splits of each ω (|error| ~ 2^-44 ω_max): the
// Gaussian's argument in the mixed path without FP64 instructions.
__device__ __forceinline__ float delta_comp(float h0, float l0, float h1, float l1, float h2, float l2,
                                            float h3, float l3, int s1, int s2) {
    float e1, e2, e3;
    const float x1 = two_sum(h0, (float)s1 * h1, e1);
    const float x2 = two_sum(x1, (float)s2 * h2, e2);
    const float x3 = two_sum(x2, -h3, e3);
    const float lo = ((l0 + (float)s1 * l1) + ((float)s2 * l2 - l3));
    return x3 + ((e1 + e2) + (e3 + lo));
}

// Triangular domain of a (q', q'') pair (partner-swap symmetry of the summand): -1 the pair is the
// swap of one evaluated elsewhere; 0 no symmetry used (weight 1); 1 weight 2; 2 +- with q'' = q'''
// (keep j'' <= j'''); 3 ++ / -- with q'' = q' (keep j'' >= j').
__device__ __forceinline__ int tri_code(const RateArgs &a, int ch, int q1, int q2, int q3) {
    if (ch == 3) {
        if (!(a.tri & 1)) return 0;
        return q2 > q3 ? -1 : (q2 < q3 ? 1 : 2);
    }
    if (!(a.tri & 2)) return 0;
    return q2 < q1 ? -1 : (q2 > q1 ? 1 : 3);
}

// tri_code of a (q', q'') pair of mode m0 under the sampling estimate: a representative stands for
// its own pair and, off the diagonal (code 1), for its swapped pair ((λ, q', q''') for +-,
// (λ, q'', q') for ++ and --); it keeps weight 2 when both are in the sample, becomes weight 1
// (code 0) when one is, and is skipped (-1) when neither is.
__device__ __forceinline__ int tri_code_sampled(const RateArgs &a, int ch, int m0, int q1, int q2, int q3, int N) {
    const int tri = tri_code(a, ch, q1, q2, q3);
    if (a.sample_all || tri < 0) return tri;
    const int sa = pair_sampled(a, m0, q1, q2, N) ? 1 : 0;
    if (tri != 1) return sa ? tri : -1;
    const int sb = (ch == 3 ? pair_sampled(a, m0, q1, q3, N) : pair_sampled(a, m0, q2, q1, N)) ? 1 : 0;
    return sa + sb == 2 ? 1 : sa + sb == 1 ? 0 : -1;
}

// weight of an evaluated process: 2 for a swapped pair, 1 on the diagonal or without symmetry
__device__ __forceinline__ int tri_weight(int tri, int j1, int j2, int j3) {
    return tri == 0 ? 1 : tri == 1 ? 2 : tri == 2 ? (j2 < j3 ? 2 : 1) : (j2 > j1 ? 2 : 1);
}

// Window masks of one q'': bit j'' of mask[j'''] is set iff the process is kept (restricted to the
// triangular domain).  FP32 prefilter with the proven bound; candidates inside the band are
// decided by the exact FP64 Δ.
template <int NB, bool ADA>
__device__ __forceinline__ int window_masks(const Tables &t, const RateArgs &a, int ch, int s2,
                                            float base32, int m0, int m1, double w0, double w1, int q2,
                                            int q3, unsigned (&mask)[NB]) {
    const unsigned v2 = t.vmask[q2], v3 = t.vmask[q3];
    const int q1 = m1 / NB, j1 = m1 - q1 * NB;
    const int tri = tri_code_sampled(a, ch, m0, q1, q2, q3, t.N);
    if (tri < 0) {
#pragma unroll
        for (int j3 = 0; j3 < NB; ++j3) mask[j3] = 0u;
        return 0;
    }
    // branch pairs of the domain: j'' <= j''' (tri 2) or j'' >= j' (tri 3)
    auto dom = [&](int j3) -> unsigned {
        return tri == 2 ? (2u << j3) - 1u : tri == 3 ? ~((1u << j1) - 1u) : ~0u;
    };
    if constexpr (ADA) {
        int n = 0;
        for (int j3 = 0; j3 < NB; ++j3) {
            mask[j3] = ((v3 >> j3) & 1u) ? window_adaptive4_row<NB>(t, a, ch, s2, base32, m0, m1, q2, q3 * NB + j3, v2) & dom(j3)
                                         : 0u;
            n += (mask[j3] != 0);
        }
        return n;
    }
    float t2[NB], w3f[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        t2[j] = base32 + (float)s2 * t.om32[q2 * NB + j];
        w3f[j] = t.om32[q3 * NB + j];
    }
    int n = 0;
#pragma unroll
    for (int j3 = 0; j3 < NB; ++j3) {
        unsigned m = 0;
        if ((v3 >> j3) & 1u) {
#pragma unroll
            for (int j2 = 0; j2 < NB; ++j2) {
                if (!((v2 >> j2) & 1u)) continue;
                const float ad = fabsf(t2[j2] - w3f[j3]);
                bool keep;
                if (ad <= a.lo32) keep = true;
                else if (ad > a.hi32) keep = false;
                else keep = window_exact4(ch, w0, w1, t.om[q2 * NB + j2], t.om[q3 * NB + j3], a.two_sigma);
                m |= (unsigned)keep << j2;
            }
        }
        mask[j3] = m & dom(j3);
        n += (mask[j3] != 0);
    }
    return n;
}

// Kahan-compensated FP32 accumulator (mixed path) / plain FP64 accumulator (FP64 path).
template <typename R> struct Acc {
    double s = 0.0;
    __device__ __forceinline__ void add(R x) { s += (double)x; }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct Acc<float> {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// One (λ, q') unit of the general kernel, run by the whole block (the body of rates4_kernel and of
// the batched persistent kernel, which takes its units from a work list over many contexts).
template <typename R, int NA, bool ADA>
__device__ __forceinline__ void rates4_unit(const Tables &t, const RateArgs &a, int ch, int unit) {
    using C = Cplx<R>;
    constexpr int NB = 3 * NA;
    // X-route (FP32, <= 2 atoms): X[c,d][γδ] = Σ_r P_r W_r[γδ] once per q'', then 36 complex
    // MACs per (q'', j''') item.  Otherwise Y[cγ] is contracted key by key per item.
    constexpr bool XROUTE = (sizeof(R) == 4) && (NA <= 2);
    const int s1 = (ch == 4) ? -1 : 1;
    const int s2 = (ch == 2) ? 1 : -1;
    const int N = t.N;

    extern __shared__ __align__(16) unsigned char smem[];
    C *sW = reinterpret_cast<C *>(smem);                        // [n_keys * 9]
    C *sCon = sW + t.n_keys * 9;                                // [nc4 * 9]  per-cluster terms
    C *sE = sCon + t.nc4 * 9;                                   // [NA*NA*9]  e_λ(aα) e^s1_λ'(bβ)
    C *se0 = sE + NA * NA * 9;                                  // [NB]       e_λ
    unsigned long long *sQ = reinterpret_cast<unsigned long long *>(se0 + NB + (NB & 1));  // [kQChunk]
    __shared__ int s_scan[32];
    __shared__ double s_red[32];
    __shared__ long long s_redn[32];

    const int ms = unit / N, q1 = unit - ms * N;
    const int m0 = a.modes[ms];
    const int q0 = m0 / NB, j0 = m0 - q0 * NB;
    const C *ev = Sel<R>::ev(t);
    const C *rt = Sel<R>::rt(t);
    const C *P4 = Sel<R>::P4(t);
    const R *phi4 = Sel<R>::phi4(t);
    const R *ism4 = Sel<R>::ism4(t);
    const R *occ = Sel<R>::occ(t);
    const R *invw = Sel<R>::invw(t);

    Acc<R> acc_g, acc_wp;
    long long acc_n = 0, acc_items = 0, acc_ent = 0, acc_ev = 0, acc_cev = 0;

    const bool active = !(q0 == 0 && j0 < 3);
    if (active) {
        const int4 c0 = t.qc[q0], c1 = t.qc[q1];
        const int b0 = c0.x + s1 * c1.x, b1 = c0.y + s1 * c1.y, b2 = c0.z + s1 * c1.z;
        const double w0 = t.om[m0];
        const float w0f = t.om32[m0];
        const unsigned vm1 = t.vmask[q1];
        for (int k = threadIdx.x; k < NB; k += blockDim.x) se0[k] = ev[(q0 * NB + k) * NB + j0];

        for (int j1 = 0; j1 < NB; ++j1) {
            if (!((vm1 >> j1) & 1u)) continue;
            const int m1 = q1 * NB + j1;
            __syncthreads();                       // previous j1 finished with the shared tables
            for (int k = threadIdx.x; k < NA * NA * 9; k += blockDim.x) {
                const int ab = k / 9, ij = k - ab * 9;
                const int at = ab / NA, bt = ab - at * NA;
                const int al = ij / 3, be = ij - al * 3;
                C y = cconj_if(ev[(q1 * NB + 3 * bt + be) * NB + j1], s1 < 0);
                sE[k] = cmul(se0[3 * at + al], y);
            }
            __syncthreads();
            // per-cluster terms exp(-i q.R3 + i s1 q'.(R1 - R3)) / sqrt(m) Σ_αβ Φ[αβγδ] E[αβ]
            for (int k = threadIdx.x; k < t.nc4 * 9; k += blockDim.x) {
                const int c = k / 9, gd = k - c * 9;
                const int4 at = t.c4_at[c];
                const int idx = mod_pos(s1 * phase_index(c1, t.c4_r13[c], t.L) -
                                            phase_index(c0, t.c4_r3[c], t.L), t.L);
                const R *ph4 = phi4 + 81 * c + gd;
                const C *E = sE + (at.x * NA + at.y) * 9;
                C v = czero<C>();
#pragma unroll
                for (int ab = 0; ab < 9; ++ab) v = crfma(ph4[9 * ab], E[ab], v);
                const C p = cmul(rt[idx], v);
                sCon[k] = cmake(p.x * ism4[c], p.y * ism4[c]);
            }
            __syncthreads();
            // W_r[γδ]: clusters of a key summed in order (deterministic)
            for (int k = threadIdx.x; k < t.n_keys * 9; k += blockDim.x) {
                const int r = k / 9, gd = k - r * 9;
                C acc = czero<C>();
                for (int c = t.key_start[r]; c < t.key_start[r + 1]; ++c) acc = cadd(acc, sCon[c * 9 + gd]);
                sW[k] = acc;
            }
            __syncthreads();

            const float base32 = w0f + (float)s1 * t.om32[m1];
            const double w1 = t.om[m1];
            // ++ and -- on their triangle (q'' >= q') start at q'' = q'
            for (int qb = (ch != 3 && (a.tri & 2)) ? q1 : 0; qb < N; qb += kQChunk) {
                const int qe = min(N, qb + kQChunk);
                // pass 1: window masks of this thread's q''; the X-route keeps those with a kept
                // process in a small local list (q'' packed with the 36 mask bits) and counts them
                constexpr int kPer = kQChunk / 64;              // blockDim >= 64
                unsigned long long ent[XROUTE ? kPer : 1];
                int n_act = 0;
                for (int q2 = qb + threadIdx.x; q2 < qe; q2 += blockDim.x) {
                    const int4 c2 = t.qc[q2];
                    const int q3 = q_index(b0 + s2 * c2.x, b1 + s2 * c2.y, b2 + s2 * c2.z,
                                           t.mesh[0], t.mesh[1], t.mesh[2]);
                    unsigned mask[NB];
                    if (tri_code_sampled(a, ch, m0, q1, q2, q3, N) >= 0) acc_cev += NB * NB;   // visited
                    if (window_masks<NB, ADA>(t, a, ch, s2, base32, m0, m1, w0, w1, q2, q3, mask) > 0) {
                        if constexpr (XROUTE) {
                            unsigned long long e = (unsigned long long)q2 << 40;
#pragma unroll
                            for (int j3 = 0; j3 < NB; ++j3) e |= (unsigned long long)mask[j3] << (NB * j3);
                            ent[n_act] = e;
                        }
                        ++n_act;
                    }
                }
                int total;
                int off = block_exclusive_scan(n_act, s_scan, &total);
                // pass 2: write them in order
                if constexpr (XROUTE) {
                    for (int k = 0; k < n_act; ++k) sQ[off + k] = ent[k];
                } else if (n_act) {
                    for (int q2 = qb + threadIdx.x; q2 < qe; q2 += blockDim.x) {
                        const int4 c2 = t.qc[q2];
                        const int q3 = q_index(b0 + s2 * c2.x, b1 + s2 * c2.y, b2 + s2 * c2.z,
                                               t.mesh[0], t.mesh[1], t.mesh[2]);
                        unsigned mask[NB];
                        if (window_masks<NB, ADA>(t, a, ch, s2, base32, m0, m1, w0, w1, q2, q3, mask) > 0) sQ[off++] = q2;
                    }
                }
                __syncthreads();

                for (int it = threadIdx.x; it < total; it += blockDim.x) {
                    ++acc_ent;
                    const unsigned long long e = sQ[it];
                    const int iq2 = XROUTE ? (int)(e >> 40) : (int)e;
                    const int4 c2 = t.qc[iq2];
                    const int q3 = q_index(b0 + s2 * c2.x, b1 + s2 * c2.y, b2 + s2 * c2.z,
                                           t.mesh[0], t.mesh[1], t.mesh[2]);
                    unsigned mask[NB];
                    const int tri = tri_code_sampled(a, ch, m0, q1, iq2, q3, N);
                    if constexpr (XROUTE) {
#pragma unroll
                        for (int j3 = 0; j3 < NB; ++j3) mask[j3] = (unsigned)(e >> (NB * j3)) & ((1u << NB) - 1u);
                    } else {
                        window_masks<NB, ADA>(t, a, ch, s2, base32, m0, m1, w0, w1, iq2, q3, mask);
                    }
                    const C *P = P4 + (size_t)iq2 * t.n_keys;
                    C X[XROUTE ? NA : 1][XROUTE ? NA : 1][9];
                    if constexpr (XROUTE) {
#pragma unroll
                        for (int c = 0; c < NA; ++c)
#pragma unroll
                            for (int d = 0; d < NA; ++d) {
#pragma unroll
                                for (int k = 0; k < 9; ++k) X[c][d][k] = czero<C>();
                                const int r0 = t.grp_start[c * NA + d], r1 = t.grp_start[c * NA + d + 1];
                                for (int r = r0; r < r1; ++r) {
                                    const C ph = cconj_if(P[r], s2 < 0);
                                    const C *Wr = sW + 9 * r;
#pragma unroll
                                    for (int k = 0; k < 9; ++k) X[c][d][k] = cfma(ph, Wr[k], X[c][d][k]);
                                }
                            }
                    }
#pragma unroll 1
                    for (int j3 = 0; j3 < NB; ++j3) {
                        unsigned m = mask[j3];
                        if (!m) continue;
                        ++acc_items;
                        C Y[NA][3];
#pragma unroll
                        for (int c = 0; c < NA; ++c)
#pragma unroll
                            for (int g = 0; g < 3; ++g) Y[c][g] = czero<C>();
                        if constexpr (XROUTE) {
                            // Y[cγ] = Σ_dδ X[c,d][γδ] e*_λ'''(dδ)
#pragma unroll
                            for (int d = 0; d < NA; ++d) {
                                C e3[3];
#pragma unroll
                                for (int dl = 0; dl < 3; ++dl) e3[dl] = cconj(ev[(q3 * NB + 3 * d + dl) * NB + j3]);
#pragma unroll
                                for (int c = 0; c < NA; ++c)
#pragma unroll
                                    for (int g = 0; g < 3; ++g)
#pragma unroll
                                        for (int dl = 0; dl < 3; ++dl) Y[c][g] = cfma(X[c][d][3 * g + dl], e3[dl], Y[c][g]);
                            }
                        } else {
                            // Y[cγ] = Σ_d Σ_{r in (c,d)} P_r^s2 Σ_δ W_r[γδ] e*_λ'''(dδ)
#pragma unroll
                            for (int c = 0; c < NA; ++c) {
#pragma unroll
                                for (int d = 0; d < NA; ++d) {
                                    const int r0 = t.grp_start[c * NA + d], r1 = t.grp_start[c * NA + d + 1];
                                    if (r0 == r1) continue;
                                    C e3[3];
#pragma unroll
                                    for (int dl = 0; dl < 3; ++dl) e3[dl] = cconj(ev[(q3 * NB + 3 * d + dl) * NB + j3]);
                                    for (int r = r0; r < r1; ++r) {
                                        const C ph = cconj_if(P[r], s2 < 0);
                                        const C *Wr = sW + 9 * r;
#pragma unroll
                                        for (int g = 0; g < 3; ++g) {
                                            C u = cmul(Wr[3 * g], e3[0]);
                                            u = cfma(Wr[3 * g + 1], e3[1], u);
                                            u = cfma(Wr[3 * g + 2], e3[2], u);
                                            Y[c][g] = cfma(ph, u, Y[c][g]);
                                        }
                                    }
                                }
                            }
                        }
                        const int m3 = q3 * NB + j3;
                        const R n3 = occ[m3], iw3 = invw[m3];
                        while (m) {
                            const int j2 = __ffs(m) - 1;
                            m &= m - 1;
                            const int m2 = iq2 * NB + j2;
                            C V = czero<C>();
#pragma unroll
                            for (int c = 0; c < NA; ++c)
#pragma unroll
                                for (int g = 0; g < 3; ++g)
                                    V = cfma(cconj_if(ev[(iq2 * NB + 3 * c + g) * NB + j2], s2 < 0), Y[c][g], V);
                            R w;
                            if constexpr (sizeof(R) == 8) {
                                const double d = delta_exact(ch, w0, w1, t.om[m2], t.om[m3]);
                                double g;
                                if constexpr (ADA) g = gauss_adaptive(t, a, d, m2, m3);
                                else g = exp(-(d * d) * a.inv_sigma2) * a.gnorm;
                                w = sym4<double>(ch) * occupation_factor<double>(ch, occ[m1], occ[m2], n3) *
                                    g * invw[m0] * invw[m1] * invw[m2] * iw3;
                            } else {
                                const float df = delta_comp(t.om32[m0], t.om32lo[m0], t.om32[m1], t.om32lo[m1],
                                                            t.om32[m2], t.om32lo[m2], t.om32[m3], t.om32lo[m3], s1, s2);
                                float g;
                                if constexpr (ADA) g = gauss_adaptive32(t, a, df, m2, m3);
                                else g = __expf(-(df * df) * a.inv_sigma2_32) * a.gnorm32;
                                w = sym4<float>(ch) * occupation_factor<float>(ch, occ[m1], occ[m2], n3) * g *
                                    (invw[m0] * invw[m1]) * (invw[m2] * iw3);
                            }
                            const int wt = tri_weight(tri, j1, j2, j3);
                            w *= (R)wt;
                            acc_wp.add(w);
                            acc_g.add(w * (V.x * V.x + V.y * V.y));
                            acc_n += wt;
                            acc_ev += 1;
                        }
                    }
                }
                __syncthreads();                   // sQ reused by the next chunk
            }
        }
    }
    const double g = block_sum(acc_g.value(), s_red);
    const double wp = block_sum(acc_wp.value(), s_red);
    const long long n = block_sum(acc_n, s_redn);
    const long long ni = block_sum(acc_items, s_redn);
    const long long ne = block_sum(acc_ent, s_redn);
    const long long nev = block_sum(acc_ev, s_redn);
    const long long ncv = block_sum(acc_cev, s_redn);
    if (threadIdx.x == 0) {
        const size_t o = ((size_t)ch * a.n_modes + ms) * N + q1;
        a.part_g[o] = g;
        a.part_wp[o] = wp;
        a.part_n[o] = n;
        a.part_items[o] = ni;
        a.part_ent[o] = ne;
        if (a.part_ev) a.part_ev[o] = nev;
        if (a.part_cev) a.part_cev[o] = ncv;
    }
}

template <typename R, int NA, bool ADA>
__global__ void __launch_bounds__(128, 4)
rates4_kernel(const __grid_constant__ Tables t, const __grid_constant__ RateArgs a, int ch) {
    rates4_unit<R, NA, ADA>(t, a, ch, blockIdx.x);
}

template <typename R, int NA, bool ADA>
cudaError_t launch4(const Tables &t, const RateArgs &a, int ch, int threads, cudaStream_t s) {
    using C = Cplx<R>;
    constexpr int NB = 3 * NA;
    size_t smem = sizeof(C) * ((size_t)t.n_keys * 9 + (size_t)t.nc4 * 9 + NA * NA * 9 + NB) +
                  sizeof(C) + sizeof(unsigned long long) * (size_t)kQChunk;
    smem = (smem + 15) & ~size_t(15);
    cudaError_t e = cudaFuncSetAttribute(rates4_kernel<R, NA, ADA>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long units = (long long)a.n_modes * t.N;
    if (units > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (units == 0) return cudaSuccess;
    rates4_kernel<R, NA, ADA><<<(unsigned)units, threads, smem, s>>>(t, a, ch);
    e = cudaGetLastError();
    if (e == cudaSuccess && a.n_kernels) ++*a.n_kernels;
    return e;
}

// Dynamic shared memory of the general kernel for one context's tables.
template <typename R, int NA>
size_t general_smem_bytes(const Tables &t) {
    using C = Cplx<R>;
    constexpr int NB = 3 * NA;
    size_t smem = sizeof(C) * ((size_t)t.n_keys * 9 + (size_t)t.nc4 * 9 + NA * NA * 9 + NB) +
                  sizeof(C) + sizeof(unsigned long long) * (size_t)kQChunk;
    return (smem + 15) & ~size_t(15);
}

template <typename R, int NA, int HI>
size_t general_smem_atoms(int na, const Tables &t) {
    if (na == NA) return general_smem_bytes<R, NA>(t);
    if constexpr (NA < HI) return general_smem_atoms<R, NA + 1, HI>(na, t);
    else return 0;
}

// Dispatch over the atom count NA..HI (instantiations split across translation units so that they
// compile in parallel; ADA selects the adaptive-σ window and Gaussian at compile time so that the
// fixed-σ kernels carry none of its registers).
template <typename R, bool ADA, int NA, int HI>
cudaError_t launch4_atoms(int na, const Tables &t, const RateArgs &a, int ch, int threads, cudaStream_t s) {
    if (na == NA) return launch4<R, NA, ADA>(t, a, ch, threads, s);
    if constexpr (NA < HI) return launch4_atoms<R, ADA, NA + 1, HI>(na, t, a, ch, threads, s);
    else return cudaErrorInvalidValue;
}

// general-kernel launchers, one per translation unit: precision x adaptive x atoms 1-4 / 5-8
#define FC4_GENERAL_LAUNCHER(name) \
    cudaError_t name(int na, const Tables &t, const RateArgs &a, int ch, int threads, cudaStream_t s);
FC4_GENERAL_LAUNCHER(launch4_d_1_4)
FC4_GENERAL_LAUNCHER(launch4_d_5_8)
FC4_GENERAL_LAUNCHER(launch4_f_1_4)
FC4_GENERAL_LAUNCHER(launch4_f_5_8)
FC4_GENERAL_LAUNCHER(launch4_ad_d_1_4)
FC4_GENERAL_LAUNCHER(launch4_ad_d_5_8)
FC4_GENERAL_LAUNCHER(launch4_ad_f_1_4)
FC4_GENERAL_LAUNCHER(launch4_ad_f_5_8)
#undef FC4_GENERAL_LAUNCHER

// tiled-path launchers (<= 2 atoms)
cudaError_t launch4_tile_f(int na, const Tables &t, const RateArgs &a, int ch, cudaStream_t s);
cudaError_t launch4_tile_d(int na, const Tables &t, const RateArgs &a, int ch, cudaStream_t s);
cudaError_t launch4_tile_ad_f(int na, const Tables &t, const RateArgs &a, int ch, cudaStream_t s);
cudaError_t launch4_tile_ad_d(int na, const Tables &t, const RateArgs &a, int ch, cudaStream_t s);
cudaError_t launch4_tile_bte_f(int na, const Tables &t, const RateArgs &a, int ch, cudaStream_t s);
cudaError_t launch4_tile_bte_d(int na, const Tables &t, const RateArgs &a, int ch, cudaStream_t s);

}  // namespace fc4
