// k_adjoint.cu - adjoint of the scattering rates with respect to the cubic and quartic force
// constants, at fixed modes and fixed σ, FP64, deterministic.
//
// L = Σ_{ch,λ} dL/dΓ_ch(λ) Γ_ch(λ) and Γ = C/N^k Σ_p w_p |V_p|², so with G_p = dL/dΓ(λ) C/N^k w_p
//   dL/dΦ_c[..] = Σ_p G_p 2 Re(conj(V_p) dV_p/dΦ_c[..]),   dV_p/dΦ_c = phase_c e e e (e) / sqrt(m),
// and V is recomputed (never stored).
//
// Four-phonon: one block per mode λ loops over (q', j').  With W_r, P_r and the keys of the forward
// kernel, V = Σ_r P_r^s2 Σ_γδ W_r[γδ] e^s2''(cγ) e*'''(dδ), and the gradient factorises through
//   Ȳ[cγ] = Σ_j'' G conj(V) e^s2''(cγ)          (per (q'', j''') item)
//   H_r[γδ] = Σ_items P_r^s2 Ȳ[c_r γ] e*'''(d_r δ) (per (λ, q', j'), owner threads, fixed order)
//   dL/dΦ_c[αβγδ] += 2 Re(phase_c / sqrt(m) e_λ(aα) e^s1'(bβ) H_{r(c)}[γδ]).
// Items of each q'' round are compacted into shared memory one per thread at a time, and every
// H entry is summed by the thread that owns it, in item order.  Each block writes its gradient
// into its own slice; a final kernel sums the slices over λ in order.
//
// Three-phonon: one block per mode λ; processes are compacted per round in the same way and
// the owner of each Φ3 entry adds 2 Re(G conj(V) phase_c e_λ e^s' e*'' / sqrt(m)) in order.
#include "k_rates4.cuh"

namespace fc4 {

constexpr int kAdjThreads = 128;

// Kahan-compensated FP32 accumulation in a (sum, compensation) pair (mixed-precision slices)
__device__ __forceinline__ void kahan_add(float2 &acc, float x) {
    const float y = x - acc.y;
    const float t = acc.x + y;
    acc.y = (t - acc.x) - y;
    acc.x = t;
}

// ------------------------------------------------------------------------------ four-phonon

template <typename R, int NA>
struct Item4 {
    int q2, q3;
    Cplx<R> ybar[3 * NA];
    Cplx<R> e3c[3 * NA];
};

template <typename R, int NA>
__global__ void __launch_bounds__(kAdjThreads)
adj4_kernel(const __grid_constant__ Tables t, const __grid_constant__ RateArgs a, int ch,
            const double *__restrict__ dLdG, double cst, double *dphi_part) {
    constexpr int NB = 3 * NA;
    using C = Cplx<R>;
    const C *ev = Sel<R>::ev(t);
    const C *rt = Sel<R>::rt(t);
    const C *P4 = Sel<R>::P4(t);
    const R *phi4 = Sel<R>::phi4(t);
    const R *ism4 = Sel<R>::ism4(t);
    const int s1 = (ch == 4) ? -1 : 1;
    const int s2 = (ch == 2) ? 1 : -1;
    const int N = t.N, nk = t.n_keys, nc4 = t.nc4;
    extern __shared__ __align__(16) unsigned char smem[];
    C *sW = reinterpret_cast<C *>(smem);                        // [nk][9]
    C *sH = sW + nk * 9;                                        // [nk][9]
    C *sCon = sH + nk * 9;                                      // [nc4][9] per-cluster terms of W
    C *sPh = sCon + nc4 * 9;                                    // [nc4] phase / sqrt(m) at (q, q')
    C *sE = sPh + nc4;                                          // [NA*NA][9]
    C *se0 = sE + NA * NA * 9;                                  // [NB]
    Item4<R, NA> *sIt = reinterpret_cast<Item4<R, NA> *>(se0 + NB);   // [kAdjThreads]
    __shared__ int s_scan[32];
    __shared__ int s_max;

    const int ms = blockIdx.x;
    const int m0 = a.modes[ms];
    const int q0 = m0 / NB, j0 = m0 - q0 * NB;
    // per-mode gradient slice: FP64, or (mixed) FP32 Kahan pairs (sum, compensation) in the same bytes
    double *dphi = dphi_part + (size_t)ms * nc4 * 81;
    float2 *dphk = reinterpret_cast<float2 *>(dphi);
    for (int k = threadIdx.x; k < nc4 * 81; k += kAdjThreads) {
        if constexpr (sizeof(R) == 8) dphi[k] = 0.0;
        else dphk[k] = make_float2(0.0f, 0.0f);
    }
    const double gl = dLdG[(size_t)ch * a.n_modes + ms] * cst;
    if ((q0 == 0 && j0 < 3) || gl == 0.0) return;
    const int4 c0 = t.qc[q0];
    const double w0 = t.om[m0];
    const float w0f = t.om32[m0];
    for (int k = threadIdx.x; k < NB; k += kAdjThreads) se0[k] = ev[(q0 * NB + k) * NB + j0];

    for (int q1 = 0; q1 < N; ++q1) {
        const int4 c1 = t.qc[q1];
        const int b0 = c0.x + s1 * c1.x, b1 = c0.y + s1 * c1.y, b2 = c0.z + s1 * c1.z;
        const unsigned vm1 = t.vmask[q1];
        for (int j1 = 0; j1 < NB; ++j1) {
            if (!((vm1 >> j1) & 1u)) continue;
            const int m1 = q1 * NB + j1;
            const double w1 = t.om[m1];
            __syncthreads();
            for (int k = threadIdx.x; k < NA * NA * 9; k += kAdjThreads) {
                const int ab = k / 9, ij = k - ab * 9;
                const int at = ab / NA, bt = ab - at * NA;
                const int al = ij / 3, be = ij - al * 3;
                sE[k] = cmul(se0[3 * at + al], cconj_if(ev[(q1 * NB + 3 * bt + be) * NB + j1], s1 < 0));
            }
            for (int c = threadIdx.x; c < nc4; c += kAdjThreads) {
                const C p = rt[mod_pos(s1 * phase_index(c1, t.c4_r13[c], t.L) - phase_index(c0, t.c4_r3[c], t.L), t.L)];
                sPh[c] = cmake(p.x * ism4[c], p.y * ism4[c]);
            }
            for (int k = threadIdx.x; k < nk * 9; k += kAdjThreads) sH[k] = czero<C>();
            __syncthreads();
            for (int k = threadIdx.x; k < nc4 * 9; k += kAdjThreads) {
                const int c = k / 9, gd = k - c * 9;
                const int4 at = t.c4_at[c];
                const R *ph4 = phi4 + 81 * c + gd;
                const C *E = sE + (at.x * NA + at.y) * 9;
                C v = czero<C>();
#pragma unroll
                for (int ab = 0; ab < 9; ++ab) v = crfma(ph4[9 * ab], E[ab], v);
                sCon[k] = cmul(sPh[c], v);
            }
            __syncthreads();
            for (int k = threadIdx.x; k < nk * 9; k += kAdjThreads) {
                const int r = k / 9, gd = k - r * 9;
                C acc = czero<C>();
                for (int c = t.key_start[r]; c < t.key_start[r + 1]; ++c) acc = cadd(acc, sCon[c * 9 + gd]);
                sW[k] = acc;
            }
            __syncthreads();
            const float base32 = w0f + (float)s1 * t.om32[m1];
            for (int qb = 0; qb < N; qb += kAdjThreads) {
                const int q2 = qb + threadIdx.x;
                unsigned mask[NB];
                int q3 = 0, n_it = 0;
                if (q2 < N) {
                    const int4 c2 = t.qc[q2];
                    q3 = q_index(b0 + s2 * c2.x, b1 + s2 * c2.y, b2 + s2 * c2.z, t.mesh[0], t.mesh[1], t.mesh[2]);
                    const unsigned v2 = t.vmask[q2], v3 = t.vmask[q3];
                    for (int j3 = 0; j3 < NB; ++j3) {
                        unsigned m = 0;
                        if ((v3 >> j3) & 1u)
                            for (int j2 = 0; j2 < NB; ++j2) {
                                if (!((v2 >> j2) & 1u)) continue;
                                const float ad = fabsf((base32 + (float)s2 * t.om32[q2 * NB + j2]) - t.om32[q3 * NB + j3]);
                                bool keep;
                                if (a.adaptive) {
                                    const int mm2 = q2 * NB + j2, mm3 = q3 * NB + j3;
                                    const int w = window_adaptive32(a, ad, two_sigma32(t, a, mm2, mm3));
                                    keep = w == 2 || (w == 1 && window_exact_adaptive(t, a, ch, m0, m1, mm2, mm3, mm2, mm3));
                                } else if (ad <= a.lo32) keep = true;
                                else if (ad > a.hi32) keep = false;
                                else keep = fabs(delta_exact(ch, w0, w1, t.om[q2 * NB + j2], t.om[q3 * NB + j3])) <= a.two_sigma;
                                m |= (unsigned)keep << j2;
                            }
                        mask[j3] = m;
                        n_it += (m != 0);
                    }
                } else {
                    for (int j3 = 0; j3 < NB; ++j3) mask[j3] = 0;
                }
                if (threadIdx.x == 0) s_max = 0;
                __syncthreads();
                atomicMax(&s_max, n_it);
                __syncthreads();
                const int rounds = s_max;
                int next_j3 = 0;
                for (int sr = 0; sr < rounds; ++sr) {
                    // this thread's next item (q'', j''')
                    int j3 = -1;
                    while (next_j3 < NB && j3 < 0) {
                        if (mask[next_j3]) j3 = next_j3;
                        ++next_j3;
                    }
                    Item4<R, NA> it;
                    if (j3 >= 0) {
                        C Y[NA][3];
                        for (int c = 0; c < NA; ++c)
                            for (int g = 0; g < 3; ++g) Y[c][g] = czero<C>();
                        const C *P = P4 + (size_t)q2 * nk;
                        for (int c = 0; c < NA; ++c)
                            for (int d = 0; d < NA; ++d) {
                                C e3[3];
                                for (int dl = 0; dl < 3; ++dl) e3[dl] = cconj(ev[(q3 * NB + 3 * d + dl) * NB + j3]);
                                for (int r = t.grp_start[c * NA + d]; r < t.grp_start[c * NA + d + 1]; ++r) {
                                    const C ph = cconj_if(P[r], s2 < 0);
                                    const C *Wr = sW + 9 * r;
                                    for (int g = 0; g < 3; ++g) {
                                        C u = cmul(Wr[3 * g], e3[0]);
                                        u = cfma(Wr[3 * g + 1], e3[1], u);
                                        u = cfma(Wr[3 * g + 2], e3[2], u);
                                        Y[c][g] = cfma(ph, u, Y[c][g]);
                                    }
                                }
                            }
                        for (int k = 0; k < NB; ++k) it.ybar[k] = czero<C>();
                        const int m3 = q3 * NB + j3;
                        unsigned m = mask[j3];
                        while (m) {
                            const int j2 = __ffs(m) - 1;
                            m &= m - 1;
                            const int m2 = q2 * NB + j2;
                            C e2[NB];
                            for (int k = 0; k < NB; ++k) e2[k] = cconj_if(ev[(q2 * NB + k) * NB + j2], s2 < 0);
                            C V = czero<C>();
                            for (int c = 0; c < NA; ++c)
                                for (int g = 0; g < 3; ++g) V = cfma(e2[3 * c + g], Y[c][g], V);
                            const double d = delta_exact(ch, w0, w1, t.om[m2], t.om[m3]);
                            const double gs = a.adaptive ? gauss_adaptive(t, a, d, m2, m3)
                                                         : exp(-(d * d) * a.inv_sigma2) * a.gnorm;
                            const double w = (ch == 4 ? 1.0 / 6.0 : 0.5) *
                                             occupation_factor<double>(ch, t.occ[m1], t.occ[m2], t.occ[m3]) * gs *
                                             t.invw[m0] * t.invw[m1] * t.invw[m2] * t.invw[m3];
                            const C f = cmake((R)(gl * w * (double)V.x), (R)(-gl * w * (double)V.y));      // G conj(V)
                            for (int k = 0; k < NB; ++k) it.ybar[k] = cfma(f, e2[k], it.ybar[k]);
                        }
                        it.q2 = q2;
                        it.q3 = q3;
                        for (int k = 0; k < NB; ++k) it.e3c[k] = cconj(ev[(q3 * NB + k) * NB + j3]);
                    }
                    int total;
                    const int off = block_exclusive_scan(j3 >= 0 ? 1 : 0, s_scan, &total);
                    if (j3 >= 0) sIt[off] = it;
                    __syncthreads();
                    // owners accumulate H_r[γδ] += P_r^s2 Ȳ[c_r γ] e*'''(d_r δ) over the items, in order
                    for (int k = threadIdx.x; k < nk * 9; k += kAdjThreads) {
                        const int r = k / 9, gd = k - r * 9, g = gd / 3, dl = gd - 3 * g;
                        int grp = 0;
                        while (t.grp_start[grp + 1] <= r) ++grp;
                        const int cc = grp / NA, dd = grp - cc * NA;
                        C h = sH[k];
                        for (int i = 0; i < total; ++i) {
                            const C ph = cconj_if(P4[(size_t)sIt[i].q2 * nk + r], s2 < 0);
                            h = cfma(cmul(ph, sIt[i].ybar[3 * cc + g]), sIt[i].e3c[3 * dd + dl], h);
                        }
                        sH[k] = h;
                    }
                    __syncthreads();
                }
            }
            // fold H into the gradient: dΦ_c[αβγδ] += 2 Re(phase_c/sqrt(m) E[a,b][αβ] H_{r(c)}[γδ])
            __syncthreads();
            for (int r = 0; r < nk; ++r)
                for (int c = t.key_start[r]; c < t.key_start[r + 1]; ++c) {
                    const int4 at = t.c4_at[c];
                    for (int k = threadIdx.x; k < 81; k += kAdjThreads) {
                        const int ab = k / 9, gd = k - ab * 9;
                        const C z = cmul(cmul(sPh[c], sE[(at.x * NA + at.y) * 9 + ab]), sH[r * 9 + gd]);
                        if constexpr (sizeof(R) == 8) dphi[(size_t)c * 81 + k] += 2.0 * z.x;
                        else kahan_add(dphk[(size_t)c * 81 + k], 2.0f * z.x);
                    }
                }
        }
    }
}

// ------------------------------------------------------------------------------ three-phonon

struct Item3 {
    int m1, m2;
    double2 f;       // G conj(V)
};

template <int NA>
__global__ void __launch_bounds__(kAdjThreads)
adj3_kernel(const __grid_constant__ Tables t, const __grid_constant__ RateArgs a, int ch,
            const double *__restrict__ dLdG, double cst, double *dphi_part) {
    constexpr int NB = 3 * NA;
    using C = double2;
    const int s = (ch == 0) ? 1 : -1;
    const double sym = (ch == 0) ? 1.0 : 0.5;
    const int N = t.N, nc3 = t.nc3;
    __shared__ Item3 sIt[kAdjThreads];
    __shared__ int s_scan[32];
    __shared__ int s_max;
    const int ms = blockIdx.x;
    const int m0 = a.modes[ms];
    const int q0 = m0 / NB, j0 = m0 - q0 * NB;
    double *dphi = dphi_part + (size_t)ms * nc3 * 27;
    for (int k = threadIdx.x; k < nc3 * 27; k += kAdjThreads) dphi[k] = 0.0;
    const double gl = dLdG[(size_t)ch * a.n_modes + ms] * cst;
    if ((q0 == 0 && j0 < 3) || gl == 0.0) return;
    const int4 c0 = t.qc[q0];
    const double w0 = t.om[m0];
    __syncthreads();
    for (int qb = 0; qb < N; qb += kAdjThreads)
      for (int j1 = 0; j1 < NB; ++j1) {           // one partner branch j' at a time (NB <= 24 bits)
        const int q1 = qb + threadIdx.x;
        // this thread's kept processes (j'', ascending) at (q', j')
        unsigned kept = 0;
        int q2 = 0;
        if (q1 < N) {
            const int4 c1 = t.qc[q1];
            q2 = q_index(c0.x + s * c1.x, c0.y + s * c1.y, c0.z + s * c1.z, t.mesh[0], t.mesh[1], t.mesh[2]);
            const unsigned v1 = t.vmask[q1], v2 = t.vmask[q2];
            for (int j2 = 0; j2 < NB; ++j2)
                if (((v1 >> j1) & (v2 >> j2) & 1u) &&
                    (a.adaptive ? window_exact_adaptive(t, a, ch, m0, q1 * NB + j1, q2 * NB + j2, -1,
                                                        q1 * NB + j1, q2 * NB + j2)
                                : fabs(delta_exact(ch, w0, t.om[q1 * NB + j1], t.om[q2 * NB + j2], 0.0)) <= a.two_sigma))
                    kept |= 1u << j2;
        }
        if (threadIdx.x == 0) s_max = 0;
        __syncthreads();
        atomicMax(&s_max, __popc(kept));
        __syncthreads();
        const int rounds = s_max;
        for (int sr = 0; sr < rounds; ++sr) {
            Item3 it;
            const bool has = kept != 0;
            if (has) {
                const int j2 = __ffs(kept) - 1;
                kept &= kept - 1;
                const int m1 = q1 * NB + j1, m2 = q2 * NB + j2;
                const int4 c1 = t.qc[q1];
                C V = czero<C>();
                for (int c = 0; c < nc3; ++c) {
                    const int4 at = t.c3_at[c];
                    const int idx = mod_pos(s * phase_index(c1, t.c3_r12[c], t.L) - phase_index(c0, t.c3_r2[c], t.L), t.L);
                    const double *phi = t.phi3 + 27 * c;
                    C acc = czero<C>();
                    for (int al = 0; al < 3; ++al) {
                        C sa = czero<C>();
                        for (int be = 0; be < 3; ++be) {
                            C sb = czero<C>();
                            for (int g = 0; g < 3; ++g)
                                sb = crfma(phi[(al * 3 + be) * 3 + g], cconj(t.ev[(q2 * NB + 3 * at.z + g) * NB + j2]), sb);
                            sa = cfma(cconj_if(t.ev[(q1 * NB + 3 * at.y + be) * NB + j1], s < 0), sb, sa);
                        }
                        acc = cfma(t.ev[(q0 * NB + 3 * at.x + al) * NB + j0], sa, acc);
                    }
                    V = crfma(t.c3_ism[c], cmul(t.rt[idx], acc), V);
                }
                const double d = delta_exact(ch, w0, t.om[m1], t.om[m2], 0.0);
                const double gs = a.adaptive ? gauss_adaptive(t, a, d, m1, m2) : exp(-(d * d) * a.inv_sigma2) * a.gnorm;
                const double w = sym * occupation_factor<double>(ch, t.occ[m1], t.occ[m2], 0.0) * gs *
                                 t.invw[m0] * t.invw[m1] * t.invw[m2];
                it.m1 = m1;
                it.m2 = m2;
                it.f = cmake(gl * w * V.x, -gl * w * V.y);
            }
            int total;
            const int off = block_exclusive_scan(has ? 1 : 0, s_scan, &total);
            if (has) sIt[off] = it;
            __syncthreads();
            for (int k = threadIdx.x; k < nc3 * 27; k += kAdjThreads) {
                const int c = k / 27, abg = k - c * 27;
                const int al = abg / 9, be = (abg / 3) % 3, g = abg % 3;
                const int4 at = t.c3_at[c];
                double acc = dphi[k];
                for (int i = 0; i < total; ++i) {
                    const int m1 = sIt[i].m1, m2 = sIt[i].m2;
                    const int q1i = m1 / NB, j1 = m1 - q1i * NB, q2i = m2 / NB, j2 = m2 - q2i * NB;
                    const int idx = mod_pos(s * phase_index(t.qc[q1i], t.c3_r12[c], t.L) - phase_index(c0, t.c3_r2[c], t.L), t.L);
                    C z = cmul(t.ev[(q0 * NB + 3 * at.x + al) * NB + j0],
                               cconj_if(t.ev[(q1i * NB + 3 * at.y + be) * NB + j1], s < 0));
                    z = cmul(z, cconj(t.ev[(q2i * NB + 3 * at.z + g) * NB + j2]));
                    z = cmul(cmul(z, t.rt[idx]), sIt[i].f);
                    acc += 2.0 * t.c3_ism[c] * z.x;
                }
                dphi[k] = acc;
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------------------ slices -> gradient

__global__ void sum_slices_kernel(int n_slices, int n, const double *part, double *out, int accumulate,
                                  int kahan32) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double s = accumulate ? out[k] : 0.0;
    if (kahan32) {                                       // FP32 (sum, compensation) pairs
        const float2 *p = reinterpret_cast<const float2 *>(part);
        for (int i = 0; i < n_slices; ++i) {
            const float2 v = p[(size_t)i * n + k];
            s += (double)v.x - (double)v.y;
        }
    } else {
        for (int i = 0; i < n_slices; ++i) s += part[(size_t)i * n + k];
    }
    out[k] = s;
}

template <int NA>
static cudaError_t launch_adj_na(const Tables &t, const RateArgs &a, int ch, const double *dLdG, double cst,
                                 double *part, int fp64, cudaStream_t s) {
    if (a.n_modes == 0) return cudaSuccess;
    if (ch < 2) {
        adj3_kernel<NA><<<a.n_modes, kAdjThreads, 0, s>>>(t, a, ch, dLdG, cst, part);
        return cudaGetLastError();
    }
    auto run = [&](auto zero) -> cudaError_t {
        using R = decltype(zero);
        using C = Cplx<R>;
        constexpr int NB = 3 * NA;
        const size_t smem = sizeof(C) * ((size_t)t.n_keys * 18 + (size_t)t.nc4 * 10 + NA * NA * 9 + NB) +
                            sizeof(Item4<R, NA>) * kAdjThreads + 16;
        cudaError_t e = cudaFuncSetAttribute(adj4_kernel<R, NA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        adj4_kernel<R, NA><<<a.n_modes, kAdjThreads, smem, s>>>(t, a, ch, dLdG, cst, part);
        return cudaGetLastError();
    };
    return fp64 ? run(0.0) : run(0.0f);
}

cudaError_t launch_adjoint(const Tables &t, const RateArgs &a, int ch, const double *dLdG, double cst,
                           double *part, int fp64, cudaStream_t s) {
    switch (t.n_atoms) {
    case 1: return launch_adj_na<1>(t, a, ch, dLdG, cst, part, fp64, s);
    case 2: return launch_adj_na<2>(t, a, ch, dLdG, cst, part, fp64, s);
    case 3: return launch_adj_na<3>(t, a, ch, dLdG, cst, part, fp64, s);
    case 4: return launch_adj_na<4>(t, a, ch, dLdG, cst, part, fp64, s);
    default: return cudaErrorInvalidValue;       // cells of more than 4 atoms: not instantiated
    }
}

cudaError_t launch_sum_slices(int n_slices, int n, const double *part, double *out, int accumulate,
                              int kahan32, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    sum_slices_kernel<<<(n + 255) / 256, 256, 0, s>>>(n_slices, n, part, out, accumulate, kahan32);
    return cudaGetLastError();
}

}  // namespace fc4
