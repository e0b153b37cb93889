// k_rates3.cu - three-phonon kernel (channels 3ph+ and 3ph-), FP64 in both precision modes.
//
// One block per mode λ.  Φ3 contracted with e_λ and the mass factor,
//   Φ~_c[β][γ] = Σ_α Φ_c[αβγ] e_λ(aα) / sqrt(m_a m_b m_c),
// is built once in shared memory.  The block sweeps q' in rounds of 128 (one per thread) and the
// partner branch j' one at a time: the partner q'' = q ± q' is closed on the integer mesh, the
// window over j'' is tested with the FP32 prefilter of proven bound (exact FP64 Δ inside the
// ambiguity band), kept (q', j'') processes are compacted in order by a block scan, and each
// thread then evaluates one process:
//   V3^s = Σ_c exp(-i q.R2) exp(i s q'.(R1 - R2)) Σ_βγ Φ~_c[β][γ] e^s_λ'(bβ) e*_λ''(cγ)
// (the phase of exp(i(s q'.R1 - q''.R2)) with q'' = q + s q'), its weight, and w |V3|².
// Compaction keeps the rare kept processes from serialising warps.  With adaptive broadening the
// width of a process comes from v' - v'' (prefiltered in FP32 the same way, exact FP64 otherwise).
#include "fc4_window.cuh"

namespace fc4 {

constexpr int kR3Threads = 128;

template <int NA, bool ADA>
__global__ void __launch_bounds__(kR3Threads)
rates3_kernel(const __grid_constant__ Tables t, const __grid_constant__ RateArgs a, int ch) {
    constexpr int NB = 3 * NA;
    const int s = (ch == 0) ? 1 : -1;
    const double sym = (ch == 0) ? 1.0 : 0.5;
    const int N = t.N, nc3 = t.nc3;
    extern __shared__ __align__(16) unsigned char smem[];
    double2 *sPt = reinterpret_cast<double2 *>(smem);           // [nc3][9]
    int *sR2 = reinterpret_cast<int *>(sPt + nc3 * 9);           // [nc3] phase index of q.R2
    unsigned *sList = reinterpret_cast<unsigned *>(sR2 + nc3);   // [kR3Threads * NB] kept (q', j'')
    __shared__ double2 se0[NB];
    __shared__ int s_scan[32];
    __shared__ double s_red[32];
    __shared__ long long s_redn[32];

    const int ms = blockIdx.x;
    const int m0 = a.modes[ms];
    const int q0 = m0 / NB, j0 = m0 - q0 * NB;
    double acc_g = 0.0, acc_wp = 0.0;
    double acc_d[3] = {0.0, 0.0, 0.0};         // iterative BTE (a.part_d set): Σ γ Σ_k s_k ω_k F_k
    long long acc_n = 0;
    if (!(q0 == 0 && j0 < 3)) {
        const int4 c0 = t.qc[q0];
        const double w0 = t.om[m0];
        const float w0f = t.om32[m0];
        for (int k = threadIdx.x; k < NB; k += kR3Threads) se0[k] = t.ev[(q0 * NB + k) * NB + j0];
        __syncthreads();
        for (int k = threadIdx.x; k < nc3 * 9; k += kR3Threads) {
            const int c = k / 9, bg = k - 9 * c;
            const int a0 = t.c3_at[c].x;
            const double *phi = t.phi3 + 27 * c + bg;
            double2 v = czero<double2>();
            for (int al = 0; al < 3; ++al) v = crfma(phi[9 * al], se0[3 * a0 + al], v);
            sPt[k] = cmake(v.x * t.c3_ism[c], v.y * t.c3_ism[c]);
        }
        for (int c = threadIdx.x; c < nc3; c += kR3Threads) sR2[c] = phase_index(c0, t.c3_r2[c], t.L);
        for (int qb = 0; qb < N; qb += kR3Threads) {
            const int q1 = qb + threadIdx.x;
            int q2 = 0;
            unsigned v1 = 0, v2 = 0;
            int4 c1 = make_int4(0, 0, 0, 0);
            if (q1 < N) {
                c1 = t.qc[q1];
                q2 = q_index(c0.x + s * c1.x, c0.y + s * c1.y, c0.z + s * c1.z, t.mesh[0], t.mesh[1], t.mesh[2]);
                v1 = t.vmask[q1];
                v2 = t.vmask[q2];
            }
            for (int j1 = 0; j1 < NB; ++j1) {
                // window: this thread's (q', j') against every j''
                unsigned kept = 0;
                if ((v1 >> j1) & 1u) {
                    const float base32 = w0f + (float)s * t.om32[q1 * NB + j1];
                    const int m1 = q1 * NB + j1;
                    for (int j2 = 0; j2 < NB; ++j2) {
                        if (!((v2 >> j2) & 1u)) continue;
                        const int m2 = q2 * NB + j2;
                        const float ad = fabsf(base32 - t.om32[m2]);
                        bool keep;
                        if constexpr (ADA) {
                            const int w = window_adaptive32(a, ad, two_sigma32(t, a, m1, m2));
                            keep = w == 2 || (w == 1 && window_exact_adaptive(t, a, ch, m0, m1, m2, -1, m1, m2));
                        } else {
                            if (ad <= a.lo32) keep = true;
                            else if (ad > a.hi32) keep = false;
                            else keep = fabs(delta_exact(ch, w0, t.om[m1], t.om[m2], 0.0)) <= a.two_sigma;
                        }
                        kept |= (unsigned)keep << j2;
                    }
                }
                int total;
                int off = block_exclusive_scan(__popc(kept), s_scan, &total);   // also orders sPt / sR2
                while (kept) {
                    const int j2 = __ffs(kept) - 1;
                    kept &= kept - 1;
                    sList[off++] = ((unsigned)threadIdx.x << 8) | (unsigned)j2;
                }
                __syncthreads();
                for (int it = threadIdx.x; it < total; it += kR3Threads) {
                    const unsigned e = sList[it];
                    const int iq1 = qb + (int)(e >> 8), j2 = (int)(e & 0xff);
                    const int4 cc1 = t.qc[iq1];
                    const int iq2 = q_index(c0.x + s * cc1.x, c0.y + s * cc1.y, c0.z + s * cc1.z,
                                            t.mesh[0], t.mesh[1], t.mesh[2]);
                    const int m1 = iq1 * NB + j1, m2 = iq2 * NB + j2;
                    double2 V = czero<double2>();
                    for (int c = 0; c < nc3; ++c) {
                        const int4 at = t.c3_at[c];
                        const double2 *pt = sPt + 9 * c;
                        double2 e2[3];
#pragma unroll
                        for (int g = 0; g < 3; ++g) e2[g] = cconj(t.ev[(iq2 * NB + 3 * at.z + g) * NB + j2]);
                        double2 u = czero<double2>();
#pragma unroll
                        for (int be = 0; be < 3; ++be) {
                            double2 sb = cmul(pt[3 * be], e2[0]);
                            sb = cfma(pt[3 * be + 1], e2[1], sb);
                            sb = cfma(pt[3 * be + 2], e2[2], sb);
                            u = cfma(cconj_if(t.ev[(iq1 * NB + 3 * at.y + be) * NB + j1], s < 0), sb, u);
                        }
                        const int idx = mod_pos(s * phase_index(cc1, t.c3_r12[c], t.L) - sR2[c], t.L);
                        V = cfma(t.rt[idx], u, V);
                    }
                    const double d = delta_exact(ch, w0, t.om[m1], t.om[m2], 0.0);
                    double g;
                    if constexpr (ADA) g = gauss_adaptive(t, a, d, m1, m2);
                    else g = exp(-(d * d) * a.inv_sigma2) * a.gnorm;
                    const double w = sym * occupation_factor<double>(ch, t.occ[m1], t.occ[m2], 0.0) * g *
                                     t.invw[m0] * t.invw[m1] * t.invw[m2];
                    acc_wp += w;
                    acc_g += w * (V.x * V.x + V.y * V.y);
                    acc_n += 1;
                    if (a.part_d) {                    // partner signs: 3ph+ (-, +), 3ph- (+, +)
                        const double gp = w * (V.x * V.x + V.y * V.y);
                        const double o1 = (ch == 0 ? -1.0 : 1.0) * t.om[m1], o2 = t.om[m2];
                        for (int x = 0; x < 3; ++x)
                            acc_d[x] += gp * (o1 * a.bte_F[3 * m1 + x] + o2 * a.bte_F[3 * m2 + x]);
                    }
                }
                __syncthreads();                               // sList reused next
            }
        }
    }
    const double g = block_sum(acc_g, s_red);
    const double wp = block_sum(acc_wp, s_red);
    const long long n = block_sum(acc_n, s_redn);
    double dsum[3] = {0.0, 0.0, 0.0};
    if (a.part_d)
        for (int x = 0; x < 3; ++x) dsum[x] = block_sum(acc_d[x], s_red);
    if (threadIdx.x == 0) {
        const size_t o = ((size_t)ch * a.n_modes + ms) * N;   // one partial slot per mode
        if (a.part_d)
            for (int x = 0; x < 3; ++x) a.part_d[3 * o + x] = dsum[x] * t.invw[m0];
        a.part_g[o] = g;
        a.part_wp[o] = wp;
        a.part_n[o] = n;
        a.part_items[o] = 0;
        a.part_ent[o] = 0;
        if (a.part_ev) a.part_ev[o] = n;
        if (a.part_cev) a.part_cev[o] = (long long)N * NB * NB;
    }
}

template <int NA>
static cudaError_t launch3(const Tables &t, RateArgs &a, int ch, cudaStream_t s) {
    constexpr int NB = 3 * NA;
    a.n_part[ch] = 1;
    if (a.n_modes == 0) return cudaSuccess;
    const size_t smem = sizeof(double2) * (size_t)t.nc3 * 9 + sizeof(int) * (size_t)t.nc3 +
                        sizeof(unsigned) * (size_t)kR3Threads * NB + 16;
    auto kern = a.adaptive ? rates3_kernel<NA, true> : rates3_kernel<NA, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<a.n_modes, kR3Threads, smem, s>>>(t, a, ch);
    e = cudaGetLastError();
    if (e == cudaSuccess && a.n_kernels) ++*a.n_kernels;
    return e;
}

cudaError_t launch_rates3(const Tables &t, RateArgs &a, int ch, int fp64, cudaStream_t s) {
    (void)fp64;
    switch (t.n_atoms) {
    case 1: return launch3<1>(t, a, ch, s);
    case 2: return launch3<2>(t, a, ch, s);
    case 3: return launch3<3>(t, a, ch, s);
    case 4: return launch3<4>(t, a, ch, s);
    case 5: return launch3<5>(t, a, ch, s);
    case 6: return launch3<6>(t, a, ch, s);
    case 7: return launch3<7>(t, a, ch, s);
    case 8: return launch3<8>(t, a, ch, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace fc4
