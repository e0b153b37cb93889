// k_rates4_tile.cuh - four-phonon path for small cells (<= 2 atoms), in two kernels.
//
// w4_kernel writes W_r[γδ](λ, q', j') for every partner branch j' of a unit (λ, q') to a global
// buffer (HBM is otherwise idle here; one pass over the clusters per unit).  rates4_tile_kernel
// then owns the unit: it copies that W to shared memory, sweeps q'' in rounds of 128 threads x
// kQPT q'' (over the unit's triangle where the partner-swap symmetry holds), tests the window
// against every j' at once (branch-free FP32 prefilter, rare ambiguous candidates decided by the
// exact FP64 Δ), compacts the (q'', j', masks) entries with a block scan, and evaluates them:
//   FP32: X[c,d][γδ] = Σ_{r in (c,d)} P_r^s2 W_r[γδ] once per entry, Y = X e*''' per j''' (36 MACs);
//   FP64: Y[cγ] = Σ_r P_r^s2 Σ_δ W_r[γδ] e*'''(dδ) per j''' (register-light).
// The same window decision, weights and accumulation as the general kernel (k_rates4.cuh).
#pragma once
#include "k_rates4.cuh"

namespace fc4 {

constexpr int kTileQ = 128;
// Partner points q'' per thread and compaction round, and blocks per SM.  Fixed σ: 4 for the
// sparse ++ and -- channels (more window work per round), 2 for +- (fewer registers held across
// its dense entry work), 4 blocks of 128 threads per SM (128 registers).  Adaptive σ carries the
// pair widths and the per-process width through the same loops: at 128 registers it spilled
// (~500 bytes), so it runs 3 blocks per SM (168 registers) with 2 and 1 q'' per round; measured on
// the 16^3 precision workload this took a 5-q batch from 792 to 614 ms, while the fixed-σ kernels
// lose 1-3 % with either change.
constexpr int kQPTSparse = 4, kQPTDense = 2;
constexpr int kQPTSparseAd = 2, kQPTDenseAd = 1;
template <bool ADA> constexpr int qpt_of(bool dense) {
    return ADA ? (dense ? kQPTDenseAd : kQPTSparseAd) : (dense ? kQPTDense : kQPTSparse);
}
// q'' per chunk of the +- triangle list (the q'' <= q''' of a unit, built in shared memory)
constexpr int kTriChunk = 1024;


// W[j'][r][γδ] of units (λ, q') for every partner branch j', written to global memory (layout
// [unit][j'][r][γδ]).  One block per (λ, group of kW4Group q'): Φ contracted with e_λ and the mass
// factor, Φ~_c[β][γδ] = Σ_α Φ_c[αβγδ] e_λ(aα) / sqrt(m), is built once in shared memory.  Per q' the
// cluster phases are folded first, per key r and leg-1 atom b,
//   Ψ_rb[β][γδ] = Σ_{c in r, b(c) = b} exp(i(s1 q'.(R1 - R3) - q.R3)) Φ~_c[β][γδ]   (fixed order),
// and then W_r[γδ] = Σ_b Σ_β e^s1_λ'(bβ) Ψ_rb[β][γδ] for every j' (coalesced writes): the phase
// work is shared by all partner branches.
constexpr int kW4Group = 8;

constexpr int kW4Threads = 256;

template <typename R, int NA>
__global__ void __launch_bounds__(kW4Threads)
w4_kernel(const __grid_constant__ Tables t, const __grid_constant__ RateArgs a, int ch, int mode0,
          Cplx<R> *wout) {
    using C = Cplx<R>;
    constexpr int NB = 3 * NA;
    const int s1 = (ch == 4) ? -1 : 1;
    const int N = t.N, nk = t.n_keys, nc4 = t.nc4;
    const int ngrp = (N + kW4Group - 1) / kW4Group;
    extern __shared__ __align__(16) unsigned char smem[];
    C *sPt = reinterpret_cast<C *>(smem);                       // [nc4][3][9]
    C *sPh = sPt + nc4 * 27;                                    // [nc4]
    C *sE1 = sPh + nc4;                                         // [NB][NB]  e^s1_λ'(comp) per j'
    C *se0 = sE1 + NB * NB;                                     // [NB]
    C *sPsi = se0 + NB;                                         // [nk][NA][27]
    const int ml = blockIdx.x / ngrp, qg = blockIdx.x - ml * ngrp;
    const int m0 = a.modes[mode0 + ml];
    const int q0 = m0 / NB, j0 = m0 - q0 * NB;
    const C *ev = Sel<R>::ev(t);
    const C *rt = Sel<R>::rt(t);
    const R *phi4 = Sel<R>::phi4(t);
    const R *ism4 = Sel<R>::ism4(t);
    const int4 c0 = t.qc[q0];
    for (int k = threadIdx.x; k < NB; k += blockDim.x) se0[k] = ev[(q0 * NB + k) * NB + j0];
    __syncthreads();
    for (int k = threadIdx.x; k < nc4 * 27; k += blockDim.x) {
        const int c = k / 27, rem = k - c * 27;
        const int be = rem / 9, gd = rem - be * 9;
        const int a0 = t.c4_at[c].x;
        const R *ph4 = phi4 + 81 * c + be * 9 + gd;
        C v = czero<C>();
#pragma unroll
        for (int al = 0; al < 3; ++al) v = crfma(ph4[27 * al], se0[3 * a0 + al], v);
        sPt[k] = cmake(v.x * ism4[c], v.y * ism4[c]);
    }
    const int q1_end = min(N, (qg + 1) * kW4Group);
    for (int q1 = qg * kW4Group; q1 < q1_end; ++q1) {
        const int4 c1 = t.qc[q1];
        __syncthreads();                                         // sPt ready / previous q' done
        for (int c = threadIdx.x; c < nc4; c += blockDim.x)
            sPh[c] = rt[mod_pos(s1 * phase_index(c1, t.c4_r13[c], t.L) - phase_index(c0, t.c4_r3[c], t.L), t.L)];
        for (int k = threadIdx.x; k < NB * NB; k += blockDim.x) {
            const int j1 = k / NB, comp = k - j1 * NB;
            sE1[k] = cconj_if(ev[(q1 * NB + comp) * NB + j1], s1 < 0);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < nk * NA * 27; k += blockDim.x) {
            const int rb = k / 27, bgd = k - rb * 27;            // rb = r NA + b
            C acc = czero<C>();
            for (int i = t.kb_start[rb]; i < t.kb_start[rb + 1]; ++i) {
                const int c = t.kb_idx[i];
                acc = cfma(sPh[c], sPt[c * 27 + bgd], acc);
            }
            sPsi[k] = acc;
        }
        __syncthreads();
        C *wo = wout + ((size_t)ml * N + q1) * NB * nk * 9;
        for (int k = threadIdx.x; k < NB * nk * 9; k += blockDim.x) {
            const int j1 = k / (nk * 9), rem = k - j1 * (nk * 9);
            const int r = rem / 9, gd = rem - r * 9;
            const C *e1 = sE1 + j1 * NB;
            const C *ps = sPsi + r * NA * 27 + gd;
            C acc = czero<C>();
#pragma unroll
            for (int b = 0; b < NA; ++b)
#pragma unroll
                for (int be = 0; be < 3; ++be) acc = cfma(e1[3 * b + be], ps[b * 27 + be * 9], acc);
            wo[k] = acc;
        }
    }
}

// BTE = true also accumulates the off-diagonal term of the iterative Boltzmann equation,
//   Δ_λ = Σ_p γ_p Σ_k s_k (ω_k / ω_λ) F_k  (partner signs: ++ (-, -, +), +- (-, +, +), -- (+, +, +)),
// into a.part_d; the partner combination is symmetric under the swap the triangular domain uses.
template <typename R, int NA, bool ADA, int kQPT, bool BTE = false, bool NOCOMP = false>
__global__ void __launch_bounds__(kTileQ, ADA ? 3 : 4)
rates4_tile_kernel(const __grid_constant__ Tables t, const __grid_constant__ RateArgs a, int ch,
                   int mode0, const Cplx<R> *__restrict__ wall) {
    using C = Cplx<R>;
    constexpr int NB = 3 * NA;
    constexpr bool XROUTE = (sizeof(R) == 4);
    const int s1 = (ch == 4) ? -1 : 1;
    const int s2 = (ch == 2) ? 1 : -1;
    const int N = t.N, nk = t.n_keys;

    extern __shared__ __align__(16) unsigned char smem[];
    C *sW = reinterpret_cast<C *>(smem);                        // [NB][nk][9]
    unsigned long long *sQ = reinterpret_cast<unsigned long long *>(sW + NB * nk * 9);   // [kTileQ * NB * kQPT]
    float *s_g = reinterpret_cast<float *>(sQ + kTileQ * NB * kQPT);   // adaptive σ: [NB * NB][kTileQ] widths
    __shared__ int s_scan[32];
    __shared__ double s_red[(BTE ? 5 : 2) * 32];
    __shared__ long long s_redn[5 * 32];
    __shared__ unsigned short s_tri[kTriChunk];                 // +- triangle: q'' - chunk start

    const int unit = blockIdx.x;                                // (mode - mode0) * N + q'
    const int ml = unit / N, q1 = unit - ml * N;
    const int ms = mode0 + ml;
    const int m0 = a.modes[ms];
    const int q0 = m0 / NB, j0 = m0 - q0 * NB;
    const C *ev = Sel<R>::ev(t);
    const C *P4 = Sel<R>::P4(t);
    const R *occ = Sel<R>::occ(t);
    const R *invw = Sel<R>::invw(t);

    Acc<R> acc_g, acc_wp;
    Acc<R> acc_d[BTE ? 3 : 1];
    long long acc_n = 0, acc_items = 0, acc_ent = 0, acc_ev = 0, acc_cev = 0;
    const unsigned vm1 = t.vmask[q1];

    if (!(q0 == 0 && j0 < 3) && vm1) {
        const int4 c0 = t.qc[q0], c1 = t.qc[q1];
        const int b0 = c0.x + s1 * c1.x, b1 = c0.y + s1 * c1.y, b2 = c0.z + s1 * c1.z;
        const double w0 = t.om[m0];
        const float w0f = t.om32[m0];
        {                                                        // W of (λ, q') for every j'
            const C *src = wall + (size_t)unit * (NB * nk * 9);
            for (int k = threadIdx.x; k < NB * nk * 9; k += kTileQ) sW[k] = src[k];
        }
        float base32[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) base32[j] = w0f + (float)s1 * t.om32[q1 * NB + j];

        // The triangular domain is walked without idle lanes: ++ and -- start at q'' = q'; +- takes
        // its q'' <= q''' from a list built per chunk of kTriChunk q'' (ascending order).
        const bool pm_list = (ch == 3) && (a.tri & 1);
        const int qstart = (ch != 3 && (a.tri & 2)) ? q1 : 0;
        for (int cb = qstart; cb < N; cb += pm_list ? kTriChunk : N) {
          int cnt = N - cb;
          if (pm_list) {
            constexpr int kPer = kTriChunk / kTileQ;
            const int ce = min(N, cb + kTriChunk), lo = cb + threadIdx.x * kPer;
            unsigned fl = 0;
            int nf = 0;
#pragma unroll
            for (int i = 0; i < kPer; ++i) {
                const int q2 = lo + i;
                if (q2 < ce) {
                    const int4 c2 = t.qc[q2];
                    const int q3 = q_index_near(b0 + s2 * c2.x, b1 + s2 * c2.y, b2 + s2 * c2.z,
                                                t.mesh[0], t.mesh[1], t.mesh[2]);
                    if (q2 <= q3) { fl |= 1u << i; ++nf; }
                }
            }
            int off = block_exclusive_scan(nf, s_scan, &cnt);
#pragma unroll
            for (int i = 0; i < kPer; ++i)
                if ((fl >> i) & 1u) s_tri[off++] = (unsigned short)(threadIdx.x * kPer + i);
            __syncthreads();
          }
          for (int qb = 0; qb < cnt; qb += kTileQ * kQPT) {
            // window: this thread's q'' of the round (up to kQPT) against every partner branch j'
            int n_ent = 0;
            unsigned long long ent[NB * kQPT];
            for (int ix = qb + threadIdx.x; ix < min(cnt, qb + kTileQ * kQPT); ix += kTileQ) {
                const int q2 = cb + (pm_list ? (int)s_tri[ix] : ix);
                const int4 c2 = t.qc[q2];
                const int q3 = q_index_near(b0 + s2 * c2.x, b1 + s2 * c2.y, b2 + s2 * c2.z,
                                            t.mesh[0], t.mesh[1], t.mesh[2]);
                const unsigned v2 = t.vmask[q2], v3 = t.vmask[q3];
                float w2f[NB], w3f[NB];
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    w2f[j] = (float)s2 * t.omT32[j * N + q2];   // branch-major: lanes read consecutive q
                    w3f[j] = t.omT32[j * N + q3];
                }
                // Triangular domain (partner-swap symmetry of the summand): +- is symmetric under
                // (λ'', λ''') (q'' <-> q''' at fixed q'), ++ and -- under (λ', λ'') (q' <-> q'') when σ
                // is fixed.  One representative of each pair is evaluated with weight 2; a self-paired
                // point keeps the ordered half of its branch pairs.  The exact window test and the
                // summand are swap-symmetric, so counts and Γ equal those of the rectangular sum.
                // 0: weight 1; 1: weight 2; 2: +- with q'' = q'''; 3: ++/-- with q'' = q'; -1: the
                // swap of a pair evaluated elsewhere, or (sampling estimate) a pair outside the sample
                const int tri = tri_code_sampled(a, ch, m0, q1, q2, q3, N);
                if (tri < 0) continue;
                acc_cev += NB * NB * NB;                         // this q'' is visited
                // (j'', j''') pairs whose two partners both take part: bit NB j''' + j''
                unsigned long long okm = 0;
#pragma unroll
                for (int j3 = 0; j3 < NB; ++j3)
                    if ((v3 >> j3) & 1u) {
                        unsigned row = v2 & ((1u << NB) - 1u);
                        if (tri == 2) row &= (2u << j3) - 1u;    // j'' <= j'''
                        okm |= (unsigned long long)row << (NB * j3);
                    }
                // Adaptive σ: the width of a pair (λ'', λ''') does not depend on j', so the 36 widths
                // of this q'' are formed once, kept in this thread's column of s_g, and tested below
                // against every j' (branch-free masks as for a fixed σ, rare exact decisions out of line).
                if constexpr (ADA) {
#pragma unroll 1
                    for (int j3 = 0; j3 < NB; ++j3) {
                        const float4 h3 = t.vpT32[j3 * N + q3], l3 = t.vpTlo[j3 * N + q3];
#pragma unroll
                        for (int j2 = 0; j2 < NB; ++j2)
                            s_g[(j3 * NB + j2) * kTileQ + threadIdx.x] =
                                a.ad_c32 * vel_diff_norm32(t.vpT32[j2 * N + q2], t.vpTlo[j2 * N + q2], h3, l3);
                    }
                }
                // Adaptive ++, --: most (q'', j') have no pair near its window at all.  The necessary
                // condition min over (j'', j''') of |Δ32| - (r_hi 2σ32 + e0) <= 0 is evaluated for all
                // j' at once, so each width is read and scaled once per q'' instead of once per j'.
                unsigned j1_near = vm1;
                if constexpr (ADA) {
                    if (ch != 3) {
                        float mn[NB];
#pragma unroll
                        for (int j1 = 0; j1 < NB; ++j1) mn[j1] = 1.0f;
#pragma unroll
                        for (int j2 = 0; j2 < NB; ++j2) {
                            float th[NB];
#pragma unroll
                            for (int j3 = 0; j3 < NB; ++j3)
                                th[j3] = fmaf(a.ad_rhi, s_g[(j3 * NB + j2) * kTileQ + threadIdx.x], a.ad_e0);
#pragma unroll
                            for (int j1 = 0; j1 < NB; ++j1) {
                                const float t2 = base32[j1] + w2f[j2];
#pragma unroll
                                for (int j3 = 0; j3 < NB; ++j3) mn[j1] = fminf(mn[j1], fabsf(t2 - w3f[j3]) - th[j3]);
                            }
                        }
#pragma unroll
                        for (int j1 = 0; j1 < NB; ++j1)
                            if (!(mn[j1] <= 0.0f)) j1_near &= ~(1u << j1);
                    }
                }
#pragma unroll 1
                for (int j1 = 0; j1 < NB; ++j1) {
                    if (!((j1_near >> j1) & 1u)) continue;
                    const float b = base32[j1];
                    unsigned long long okj = okm;                // tri 3: j'' >= j'
                    if (tri == 3) {
                        const unsigned long long row = (unsigned long long)(((1u << NB) - 1u) & ~((1u << j1) - 1u));
                        unsigned long long cm = 0;
#pragma unroll
                        for (int j3 = 0; j3 < NB; ++j3) cm |= row << (NB * j3);
                        okj &= cm;
                    }
                    const unsigned long long tri_bits = (unsigned long long)tri << 36;
                    if constexpr (ADA) {
                        unsigned long long sure = 0, amb = 0;
#pragma unroll
                        for (int j3 = 0; j3 < NB; ++j3)
#pragma unroll
                            for (int j2 = 0; j2 < NB; ++j2) {
                                const float g = s_g[(j3 * NB + j2) * kTileQ + threadIdx.x];
                                const float ad = fabsf((b + w2f[j2]) - w3f[j3]);
                                const int k = NB * j3 + j2;
                                sure |= (unsigned long long)(ad <= fmaf(a.ad_rlo, g, -a.ad_e0) && g > a.ad_gmin) << k;
                                amb |= (unsigned long long)(ad <= fmaf(a.ad_rhi, g, a.ad_e0)) << k;
                            }
                        sure &= okj;
                        amb &= okj & ~sure;
                        while (amb) {                            // rare: exact FP64 σ and Δ
                            const int k = __ffsll(amb) - 1;
                            amb &= amb - 1;
                            const int j3 = k / NB, j2 = k - j3 * NB;
                            if (window_exact_adaptive(t, a, ch, m0, q1 * NB + j1, q2 * NB + j2, q3 * NB + j3,
                                                      q2 * NB + j2, q3 * NB + j3))
                                sure |= 1ull << k;
                        }
                        if (sure)
                            ent[n_ent++] = ((unsigned long long)(ix - qb) << 48) |
                                           ((unsigned long long)j1 << 40) | tri_bits | sure;
                        continue;
                    }
                    float t2[NB];
#pragma unroll
                    for (int j2 = 0; j2 < NB; ++j2) t2[j2] = b + w2f[j2];
                    if (ch != 3) {       // ++, --: most (q'', j') have no pair near the window at all
                        float mn = fabsf(t2[0] - w3f[0]);
#pragma unroll
                        for (int j3 = 0; j3 < NB; ++j3)
#pragma unroll
                            for (int j2 = 0; j2 < NB; ++j2) mn = fminf(mn, fabsf(t2[j2] - w3f[j3]));
                        if (!(mn <= a.hi32)) continue;          // nothing kept, nothing ambiguous
                    }
                    unsigned long long le_lo = 0, le_hi = 0;    // |Δ32| <= lo32, |Δ32| <= hi32
#pragma unroll
                    for (int j3 = 0; j3 < NB; ++j3)
#pragma unroll
                        for (int j2 = 0; j2 < NB; ++j2) {
                            const float ad = fabsf(t2[j2] - w3f[j3]);
                            le_lo |= (unsigned long long)(ad <= a.lo32) << (NB * j3 + j2);
                            le_hi |= (unsigned long long)(ad <= a.hi32) << (NB * j3 + j2);
                        }
                    unsigned long long sure = le_lo & okj, amb = le_hi & ~le_lo & okj;
                    while (amb) {                                // rare: exact FP64 decision
                        const int k = __ffsll(amb) - 1;
                        amb &= amb - 1;
                        const int j3 = k / NB, j2 = k - j3 * NB;
                        if (window_exact4(ch, w0, t.om[q1 * NB + j1], t.om[q2 * NB + j2], t.om[q3 * NB + j3],
                                          a.two_sigma))
                            sure |= 1ull << k;
                    }
                    if (sure)
                        ent[n_ent++] = ((unsigned long long)(ix - qb) << 48) |
                                       ((unsigned long long)j1 << 40) | tri_bits | sure;
                }
            }
            int total;
            const int off = block_exclusive_scan(n_ent, s_scan, &total);
            for (int k = 0; k < n_ent; ++k) sQ[off + k] = ent[k];
            __syncthreads();

            // Compacted: the block's entries are dealt out to the threads in order.  The ablation
            // instantiation (NOCOMP, fc4_set_ablation) instead has each thread evaluate the entries
            // its own window found, as an uncompacted GPU-only loop would, so warps diverge on
            // their counts.
            const int it_end = NOCOMP ? off + n_ent : total;
            for (int it = NOCOMP ? off : (int)threadIdx.x; it < it_end; it += NOCOMP ? 1 : kTileQ) {
                ++acc_ent;
                const unsigned long long e = sQ[it];
                const int ixe = qb + (int)(e >> 48), j1 = (int)((e >> 40) & 0xff);
                const int iq2 = cb + (pm_list ? (int)s_tri[ixe] : ixe);
                const int tri = (int)((e >> 36) & 3u);
                const int4 cc2 = t.qc[iq2];
                const int iq3 = q_index_near(b0 + s2 * cc2.x, b1 + s2 * cc2.y, b2 + s2 * cc2.z,
                                             t.mesh[0], t.mesh[1], t.mesh[2]);
                const int m1 = q1 * NB + j1;
                // per-entry constants of the mixed weight: TwoSum of ω + s1 ω', the sum of their lo
                // parts, n', 1/(ω ω')
                float ex1 = 0.0f, ee1 = 0.0f, el01 = 0.0f, iw01 = 0.0f, n1f = 0.0f;
                if constexpr (sizeof(R) == 4) {
                    ex1 = two_sum(t.om32[m0], (float)s1 * t.om32[m1], ee1);
                    el01 = t.om32lo[m0] + (float)s1 * t.om32lo[m1];
                    iw01 = invw[m0] * invw[m1];
                    n1f = occ[m1];
                }
                const C *Prow = P4 + (size_t)iq2 * nk;
                const C *Wj = sW + j1 * nk * 9;
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
                                const C ph = cconj_if(Prow[r], s2 < 0);
                                const C *Wr = Wj + 9 * r;
#pragma unroll
                                for (int k = 0; k < 9; ++k) X[c][d][k] = cfma(ph, Wr[k], X[c][d][k]);
                            }
                        }
                }
#pragma unroll 1
                for (int j3 = 0; j3 < NB; ++j3) {
                    unsigned m = (unsigned)(e >> (NB * j3)) & ((1u << NB) - 1u);
                    if (!m) continue;
                    ++acc_items;
                    C Y[NA][3];
#pragma unroll
                    for (int c = 0; c < NA; ++c)
#pragma unroll
                        for (int g = 0; g < 3; ++g) Y[c][g] = czero<C>();
#pragma unroll
                    for (int d = 0; d < NA; ++d) {
                        C e3[3];
#pragma unroll
                        for (int dl = 0; dl < 3; ++dl) e3[dl] = cconj(ev[(iq3 * NB + 3 * d + dl) * NB + j3]);
                        if constexpr (XROUTE) {
#pragma unroll
                            for (int c = 0; c < NA; ++c)
#pragma unroll
                                for (int g = 0; g < 3; ++g)
#pragma unroll
                                    for (int dl = 0; dl < 3; ++dl) Y[c][g] = cfma(X[c][d][3 * g + dl], e3[dl], Y[c][g]);
                        } else {
#pragma unroll
                            for (int c = 0; c < NA; ++c) {
                                const int r0 = t.grp_start[c * NA + d], r1 = t.grp_start[c * NA + d + 1];
                                for (int r = r0; r < r1; ++r) {
                                    const C ph = cconj_if(Prow[r], s2 < 0);
                                    const C *Wr = Wj + 9 * r;
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
                    const int m3 = iq3 * NB + j3;
                    const R n3 = occ[m3], iw3 = invw[m3];
                    float h3 = 0.0f, l3 = 0.0f;
                    if constexpr (sizeof(R) == 4) {
                        h3 = t.om32[m3];
                        l3 = t.om32lo[m3];
                    }
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
                            const double d = delta_exact(ch, w0, t.om[m1], t.om[m2], t.om[m3]);
                            double g;
                            if constexpr (ADA) g = gauss_adaptive(t, a, d, m2, m3);
                            else g = exp(-(d * d) * a.inv_sigma2) * a.gnorm;
                            w = sym4<double>(ch) * occupation_factor<double>(ch, occ[m1], occ[m2], n3) *
                                g * invw[m0] * invw[m1] * invw[m2] * iw3;
                        } else {
                            // Δ from the entry's TwoSum (ex1, ee1) and the hi/lo splits of the last two ω
                            float e2s, e3s;
                            const float x2 = two_sum(ex1, (float)s2 * t.om32[m2], e2s);
                            const float x3 = two_sum(x2, -h3, e3s);
                            const float lo = (el01 + (float)s2 * t.om32lo[m2]) - l3;
                            const float df = x3 + ((ee1 + e2s) + (e3s + lo));
                            float gs;
                            if constexpr (ADA) gs = gauss_adaptive32(t, a, df, m2, m3);
                            else gs = __expf(-(df * df) * a.inv_sigma2_32) * a.gnorm32;
                            w = sym4<float>(ch) * occupation_factor<float>(ch, n1f, occ[m2], n3) * gs *
                                iw01 * (invw[m2] * iw3);
                        }
                        // weight of the representative: 2 for a swapped pair, 1 on the diagonal
                        const int wt = tri == 0 ? 1 : tri == 1 ? 2 : tri == 2 ? (j2 < j3 ? 2 : 1) : (j2 > j1 ? 2 : 1);
                        w *= (R)wt;
                        acc_wp.add(w);
                        acc_g.add(w * (V.x * V.x + V.y * V.y));
                        acc_n += wt;
                        acc_ev += 1;
                        if constexpr (BTE) {
                            const R *F = Sel<R>::bteF(a);
                            const R g = w * (V.x * V.x + V.y * V.y);
                            const R o1 = (R)(ch == 4 ? 1 : -1) * Sel<R>::om(t)[m1];
                            const R o2 = (R)(ch == 2 ? -1 : 1) * Sel<R>::om(t)[m2];
                            const R o3 = Sel<R>::om(t)[m3];
#pragma unroll
                            for (int x = 0; x < 3; ++x)
                                acc_d[x].add(g * ((o1 * F[3 * m1 + x] + o2 * F[3 * m2 + x]) + o3 * F[3 * m3 + x]));
                        }
                    }
                }
            }
            __syncthreads();                                     // sQ reused by the next round
          }
        }
    }
    double sums[BTE ? 5 : 2];
    sums[0] = acc_g.value();
    sums[1] = acc_wp.value();
    if constexpr (BTE) {
#pragma unroll
        for (int x = 0; x < 3; ++x) sums[2 + x] = acc_d[x].value();
    }
    long long cnts[5] = {acc_n, acc_items, acc_ent, acc_ev, acc_cev};
    block_sum_multi<BTE ? 5 : 2, 5>(sums, cnts, s_red, s_redn);
    if (threadIdx.x == 0) {
        const size_t o = ((size_t)ch * a.n_modes + ms) * N + q1;
        if constexpr (BTE) {
            const double iw0 = t.invw[m0];                      // ξ_k = ω_k / ω_λ
#pragma unroll
            for (int x = 0; x < 3; ++x) a.part_d[3 * o + x] = sums[2 + x] * iw0;
        }
        a.part_g[o] = sums[0];
        a.part_wp[o] = sums[1];
        a.part_n[o] = cnts[0];
        a.part_items[o] = cnts[1];
        a.part_ent[o] = cnts[2];
        if (a.part_ev) a.part_ev[o] = cnts[3];
        if (a.part_cev) a.part_cev[o] = cnts[4];
    }
}

template <typename R, int NA>
size_t tile_smem_bytes(const Tables &t, int qpt = kQPTSparse, bool adaptive = true) {
    using C = Cplx<R>;
    constexpr int NB = 3 * NA;
    size_t b = sizeof(C) * ((size_t)NB * t.n_keys * 9) + sizeof(unsigned long long) * (size_t)kTileQ * NB * qpt +
               (adaptive ? sizeof(float) * (size_t)NB * NB * kTileQ : 0);
    return (b + 15) & ~size_t(15);
}

// W bytes per mode (all q' and j') for the tiled path
template <typename R, int NA>
size_t tile_w_bytes_per_mode(const Tables &t) {
    return sizeof(Cplx<R>) * (size_t)t.N * 3 * NA * t.n_keys * 9;
}

// Launch W (global) then the tiled kernel, over mode chunks that fit in the W buffer.
template <typename R, int NA, bool ADA, bool BTE = false>
cudaError_t launch4_tile(const Tables &t, const RateArgs &a, int ch, cudaStream_t s) {
    using C = Cplx<R>;
    constexpr int NB = 3 * NA;
    const bool dense = ch == 3;
    const size_t smem = tile_smem_bytes<R, NA>(t, qpt_of<ADA>(dense), ADA);
    auto kern = dense ? rates4_tile_kernel<R, NA, ADA, qpt_of<ADA>(true), BTE>
                      : rates4_tile_kernel<R, NA, ADA, qpt_of<ADA>(false), BTE>;
    if constexpr (sizeof(R) == 4 && !BTE)       // ablation switch: mixed precision only
        if (a.no_compact)
            kern = dense ? rates4_tile_kernel<R, NA, ADA, qpt_of<ADA>(true), false, true>
                         : rates4_tile_kernel<R, NA, ADA, qpt_of<ADA>(false), false, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const size_t wsmem = sizeof(C) * ((size_t)t.nc4 * 28 + NB * NB + NB + (size_t)t.n_keys * NA * 27);
    e = cudaFuncSetAttribute(w4_kernel<R, NA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsmem);
    if (e != cudaSuccess) return e;
    const size_t per_mode = tile_w_bytes_per_mode<R, NA>(t);
    const int chunk = (int)(a.wbuf_bytes / per_mode);
    if (chunk < 1) return cudaErrorInvalidValue;
    for (int m = 0; m < a.n_modes; m += chunk) {
        const int nm = min(chunk, a.n_modes - m);
        const long long ngrp = (t.N + kW4Group - 1) / kW4Group;
        if (!(a.w_reuse && nm == a.n_modes)) {           // W of the previous channel with the same s1
            w4_kernel<R, NA><<<(unsigned)((long long)nm * ngrp), kW4Threads, wsmem, s>>>(t, a, ch, m,
                                                                                  reinterpret_cast<C *>(a.wbuf));
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            if (a.n_kernels) ++*a.n_kernels;
        }
        if constexpr (sizeof(R) == 4 && !BTE) {
            if (ch == 3 && a.use_tc) {                  // +-: cluster contraction on the tensor cores
                e = launch_rates4_tc(t, a, ch, m, nm, reinterpret_cast<const float2 *>(a.wbuf), s);
                if (e != cudaSuccess) return e;
                if (a.n_kernels) ++*a.n_kernels;
                continue;
            }
        }
        kern<<<(unsigned)((long long)nm * t.N), kTileQ, smem, s>>>(t, a, ch, m, reinterpret_cast<const C *>(a.wbuf));
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (a.n_kernels) ++*a.n_kernels;
    }
    return cudaSuccess;
}

}  // namespace fc4
