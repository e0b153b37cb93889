// k_misc.cu - the harmonic prelude (batched FP64 Jacobi eigensolver of D(q), Hellmann-Feynman
// group velocities), per-mode tables, occupations, key phase tables, the deterministic reduction
// of per-(λ, q') partials into Γ / WP / counts, the RTA conductivity, and process lists.
#include "fc4_window.cuh"

namespace fc4 {

// ------------------------------------------------------------------------------ harmonic

// One warp per q point; D and the accumulated rotations U live in shared memory.
// D(q) = Σ_c Φ2_c exp(i q.R_c) / sqrt(m_a m_b) (Hermitised), one lane per matrix entry (clusters
// summed in order); cyclic complex Jacobi: every lane derives the same rotation from shared
// values, lanes k < nb update row/column k; sweeps stop when the off-diagonal mass is below
// (1e-16 |D|_F)².  Eigenpairs sorted ascending, ω = sqrt(λ * eig_to_w2) (rad/ps), and
// v_x = Re(e^H dD/dq_x e) eig_to_w2 / (2ω) (Hellmann-Feynman), one lane per branch.
template <int NA>
__global__ void __launch_bounds__(32)
harmonic_kernel(const __grid_constant__ Tables t, int nc2, const int4 *__restrict__ c2_at,
                const int4 *__restrict__ c2_r, const double *__restrict__ c2_R,
                const double *__restrict__ c2_phi, const double *__restrict__ c2_ism,
                double eig_to_w2, double *om, double *vel, double2 *ev, double *eig, int *err) {
    constexpr int NB = 3 * NA;
    constexpr int LD = NB + 1;
    __shared__ double2 sA[NB * LD], sU[NB * LD];
    __shared__ int s_ord[NB];
    const int q = blockIdx.x, lane = threadIdx.x;
    const int4 qc = t.qc[q];
    for (int k = lane; k < NB * NB; k += 32) {
        const int i = k / NB, j = k - i * NB;
        const int a = i / 3, al = i - 3 * a, b = j / 3, be = j - 3 * b;
        double2 x = czero<double2>();
        for (int c = 0; c < nc2; ++c) {
            const int4 at = c2_at[c];
            if (at.x != a || at.y != b) continue;
            const double2 ph = t.rt[phase_index(qc, c2_r[c], t.L)];
            const double pv = c2_phi[9 * c + 3 * al + be] * c2_ism[c];
            x.x += pv * ph.x;
            x.y += pv * ph.y;
        }
        sA[i * LD + j] = x;
        sU[i * LD + j] = cmake(i == j ? 1.0 : 0.0, 0.0);
    }
    __syncwarp();
    double2 h[(NB * NB + 31) / 32];
    for (int k = lane, n = 0; k < NB * NB; k += 32, ++n) {      // (A + A^H) / 2
        const int i = k / NB, j = k - i * NB;
        const double2 x = sA[i * LD + j], y = sA[j * LD + i];
        h[n] = cmake(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
    }
    __syncwarp();
    double fro = 0.0;
    for (int k = lane, n = 0; k < NB * NB; k += 32, ++n) {
        sA[(k / NB) * LD + (k % NB)] = h[n];
        fro += cabs2(h[n]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(kFull, fro, o);
    __syncwarp();
    const double tol = 1e-32 * fro;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int k = lane; k < NB * NB; k += 32) {
            const int i = k / NB, j = k - i * NB;
            if (j > i) off += cabs2(sA[i * LD + j]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(kFull, off, o);
        if (off <= tol) break;
        for (int p = 0; p < NB - 1; ++p)
            for (int r = p + 1; r < NB; ++r) {
                const double2 apr = sA[p * LD + r];
                const double b = sqrt(cabs2(apr));
                if (b <= 1e-300) continue;                            // uniform across the warp
                const double2 e = cmake(apr.x / b, apr.y / b);        // e^{iφ}
                const double th = (sA[r * LD + r].x - sA[p * LD + p].x) / (2.0 * b);
                const double tt = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = tt * cs;
                const double2 me = cmake(-sn * e.x, sn * e.y);       // -s e^{-iφ}
                const double2 ce = cmake(cs * e.x, -cs * e.y);       //  c e^{-iφ}
                __syncwarp();
                if (lane < NB) {                                      // A <- A U, U_acc <- U_acc U
                    const int k = lane;
                    const double2 ap = sA[k * LD + p], ar = sA[k * LD + r];
                    sA[k * LD + p] = cfma(ar, me, cmake(cs * ap.x, cs * ap.y));
                    sA[k * LD + r] = cfma(ar, ce, cmake(sn * ap.x, sn * ap.y));
                    const double2 up = sU[k * LD + p], ur = sU[k * LD + r];
                    sU[k * LD + p] = cfma(ur, me, cmake(cs * up.x, cs * up.y));
                    sU[k * LD + r] = cfma(ur, ce, cmake(sn * up.x, sn * up.y));
                }
                __syncwarp();
                if (lane < NB) {                                      // A <- U^H A
                    const int k = lane;
                    const double2 ap = sA[p * LD + k], ar = sA[r * LD + k];
                    sA[p * LD + k] = cfma(cconj(me), ar, cmake(cs * ap.x, cs * ap.y));
                    sA[r * LD + k] = cfma(cconj(ce), ar, cmake(sn * ap.x, sn * ap.y));
                }
                __syncwarp();
                if (lane == 0) {
                    sA[p * LD + r] = czero<double2>();
                    sA[r * LD + p] = czero<double2>();
                    sA[p * LD + p].y = 0.0;
                    sA[r * LD + r].y = 0.0;
                }
                __syncwarp();
            }
    }
    if (lane == 0) {                                                  // ascending order
        int ord[NB];
        for (int i = 0; i < NB; ++i) ord[i] = i;
        for (int i = 0; i < NB; ++i)
            for (int j = i + 1; j < NB; ++j)
                if (sA[ord[j] * LD + ord[j]].x < sA[ord[i] * LD + ord[i]].x) {
                    const int x = ord[i];
                    ord[i] = ord[j];
                    ord[j] = x;
                }
        for (int i = 0; i < NB; ++i) s_ord[i] = ord[i];
    }
    __syncwarp();
    for (int k = lane; k < NB * NB; k += 32) {
        const int comp = k / NB, j = k - comp * NB;
        ev[((size_t)q * NB + comp) * NB + j] = sU[comp * LD + s_ord[j]];
    }
    if (lane < NB) {
        const int j = lane, o = s_ord[j];
        const double l = sA[o * LD + o].x;
        eig[q * NB + j] = l;
        const bool excl = (q == 0 && j < 3);
        if (!excl && l < -1e-8) atomicOr(err, 1);
        double w = 0.0;
        if (!excl) w = (l >= 0.0 ? 1.0 : -1.0) * sqrt(fabs(l) * eig_to_w2);
        if (!excl && !(w > 0.0)) atomicOr(err, 1);
        om[q * NB + j] = (excl || !(w > 0.0)) ? 0.0 : w;       // imaginary modes take no part
        double v[3] = {0.0, 0.0, 0.0};
        if (!excl && w > 0.0) {
            for (int c = 0; c < nc2; ++c) {
                const int4 at = c2_at[c];
                const double2 ph = t.rt[phase_index(qc, c2_r[c], t.L)];
                double2 s = czero<double2>();
                for (int al = 0; al < 3; ++al) {
                    double2 sb = czero<double2>();
                    for (int be = 0; be < 3; ++be)
                        sb = crfma(c2_phi[9 * c + 3 * al + be], sU[(3 * at.y + be) * LD + o], sb);
                    s = cfma(cconj(sU[(3 * at.x + al) * LD + o]), sb, s);
                }
                s = cmul(s, ph);                                      // e^H Φ e exp(iqR)
                // dD/dq_x contributes i R_x (...): Re(i z) = -Im z
                for (int x = 0; x < 3; ++x) v[x] += -c2_R[3 * c + x] * c2_ism[c] * s.y;
            }
            for (int x = 0; x < 3; ++x) v[x] = v[x] * eig_to_w2 / (2.0 * w);
        }
        for (int x = 0; x < 3; ++x) vel[((size_t)q * NB + j) * 3 + x] = v[x];
    }
}

cudaError_t launch_harmonic(const Tables &t, int nc2, const int4 *c2_at, const int4 *c2_r,
                            const double *c2_R, const double *c2_phi, const double *c2_ism,
                            double eig_to_w2, double *om, double *vel, double2 *ev, double *eig,
                            int *err, cudaStream_t s) {
    const int threads = 32, blocks = t.N;
#define FC4_H(NA_)                                                                           \
    case NA_:                                                                                \
        harmonic_kernel<NA_><<<blocks, threads, 0, s>>>(t, nc2, c2_at, c2_r, c2_R, c2_phi,   \
                                                        c2_ism, eig_to_w2, om, vel, ev, eig, err); \
        break;
    switch (t.n_atoms) {
        FC4_H(1) FC4_H(2) FC4_H(3) FC4_H(4) FC4_H(5) FC4_H(6) FC4_H(7) FC4_H(8)
    default: return cudaErrorInvalidValue;
    }
#undef FC4_H
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ tables

// Per-mode tables derived from ω, e and v: FP32 hi/lo splits of ω, 1/ω, FP32 eigenvectors, the
// participation mask, and the velocity projections P_k = (v . b_k) / n_k (hi/lo FP32) of the
// adaptive width.
__global__ void mode_tables_kernel(const __grid_constant__ Tables t, double *om, float *om32, float *om32lo,
                                   float2 *ev32, const double2 *ev, unsigned *vmask, double *invw,
                                   float *invw32, float4 *vp32, float4 *vp32lo, float *omT32, float4 *vpT32,
                                   float4 *vpTlo) {
    const int N = t.N, nb = t.nb;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nm = (long long)N * nb;
    if (i < nm) {
        const int q = (int)(i / nb), j = (int)(i - (long long)q * nb);
        if (q == 0 && j < 3) om[i] = 0.0;
        const double w = om[i];
        om32[i] = (float)w;
        om32lo[i] = (float)(w - (double)(float)w);
        invw[i] = w > 0.0 ? 1.0 / w : 0.0;
        invw32[i] = w > 0.0 ? (float)(1.0 / w) : 0.0f;
        const double *v = t.vel + 3 * i;
        float h[3], l[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double p = (v[0] * t.recip[3 * k] + v[1] * t.recip[3 * k + 1] + v[2] * t.recip[3 * k + 2]) / t.mesh[k];
            h[k] = (float)p;
            l[k] = (float)(p - (double)h[k]);
        }
        vp32[i] = make_float4(h[0], h[1], h[2], 0.0f);
        vp32lo[i] = make_float4(l[0], l[1], l[2], 0.0f);
        const size_t it = (size_t)j * N + q;                 // branch-major copies
        omT32[it] = (float)w;
        vpT32[it] = make_float4(h[0], h[1], h[2], 0.0f);
        vpTlo[it] = make_float4(l[0], l[1], l[2], 0.0f);
    }
    if (i < nm * nb) {
        const double2 e = ev[i];
        ev32[i] = make_float2((float)e.x, (float)e.y);
    }
    if (i < N) {
        unsigned m = 0;
        for (int j = 0; j < nb; ++j)
            if (!(i == 0 && j < 3) && om[i * nb + j] > 0.0) m |= 1u << j;
        vmask[i] = m;
    }
}

cudaError_t launch_mode_tables(const Tables &t, double *om, float *om32, float *om32lo,
                               float2 *ev32, const double2 *ev, unsigned *vmask, double *invw,
                               float *invw32, float4 *vp32, float4 *vp32lo, float *omT32, float4 *vpT32,
                               float4 *vpTlo, cudaStream_t s) {
    const long long n = (long long)t.N * t.nb * t.nb;
    mode_tables_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(t, om, om32, om32lo, ev32, ev, vmask, invw,
                                                                    invw32, vp32, vp32lo, omT32, vpT32, vpTlo);
    return cudaGetLastError();
}

__global__ void occupations_kernel(int nm, const double *om, double x_per_w, double *occ,
                                   float *occ32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nm) return;
    const double w = om[i];
    const double n = w > 0.0 ? 1.0 / expm1(w * x_per_w) : 0.0;
    occ[i] = n;
    occ32[i] = (float)n;
}

cudaError_t launch_occupations(const Tables &t, double hbar_over_kT, double *occ, float *occ32,
                               cudaStream_t s) {
    const int nm = t.N * t.nb;
    occupations_kernel<<<(nm + 255) / 256, 256, 0, s>>>(nm, t.om, hbar_over_kT, occ, occ32);
    return cudaGetLastError();
}

__global__ void phase_tables_kernel(const __grid_constant__ Tables t, const int4 *key_r,
                                    double2 *P4, float2 *P4_32) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)t.N * t.n_keys) return;
    const int q = (int)(i / t.n_keys), r = (int)(i - (long long)q * t.n_keys);
    const double2 p = t.rt[phase_index(t.qc[q], key_r[r], t.L)];
    P4[i] = p;
    P4_32[i] = make_float2((float)p.x, (float)p.y);
}

cudaError_t launch_phase_tables(const Tables &t, const int4 *key_r, double2 *P4, float2 *P4_32,
                                cudaStream_t s) {
    const long long n = (long long)t.N * t.n_keys;
    if (n == 0) return cudaSuccess;
    phase_tables_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(t, key_r, P4, P4_32);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ reduction

struct int5 { int a, b, c, d, e; };

// One warp per (channel, mode): lane l sums q' = l, l + 32, ... in order, then a fixed
// butterfly; Γ = C / N^k * Σ, WP = Σ / N^k (k = 1 for 3ph, 2 for 4ph).
__global__ void reduce_kernel(int n_modes, int ld, int N, int5 n_part, int channel_mask, double c3, double c4,
                              double scale4,
                              const double *part_g, const double *part_wp, const long long *part_n,
                              const long long *part_items, const long long *part_ent, const long long *part_ev,
                              const long long *part_cev, double *gamma, double *wp, long long *counts,
                              unsigned long long *stats, const int *err) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= 5 * n_modes) return;
    const int ch = w / n_modes, ms = w - ch * n_modes;
    double g = 0.0, p = 0.0;
    long long n = 0, it = 0, en = 0, ev = 0, cv = 0;
    if ((channel_mask >> ch) & 1) {
        const size_t base = ((size_t)ch * n_modes + ms) * N;
        const int np = ch == 0 ? n_part.a : ch == 1 ? n_part.b : ch == 2 ? n_part.c : ch == 3 ? n_part.d : n_part.e;
        for (int q = lane; q < np; q += 32) {
            g += part_g[base + q];
            p += part_wp[base + q];
            n += part_n[base + q];
            it += part_items[base + q];
            en += part_ent[base + q];
            if (part_ev) ev += part_ev[base + q];
            if (part_cev) cv += part_cev[base + q];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            g += __shfl_xor_sync(kFull, g, o);
            p += __shfl_xor_sync(kFull, p, o);
            n += __shfl_xor_sync(kFull, n, o);
            it += __shfl_xor_sync(kFull, it, o);
            en += __shfl_xor_sync(kFull, en, o);
            ev += __shfl_xor_sync(kFull, ev, o);
            cv += __shfl_xor_sync(kFull, cv, o);
        }
    }
    if (lane == 0 && stats) {
        atomicAdd(stats + 5 * ch, (unsigned long long)n);       // integer sums: order-independent
        atomicAdd(stats + 5 * ch + 1, (unsigned long long)it);
        atomicAdd(stats + 5 * ch + 2, (unsigned long long)en);
        atomicAdd(stats + 5 * ch + 3, (unsigned long long)ev);
        atomicAdd(stats + 5 * ch + 4, (unsigned long long)cv);
    }
    if (lane == 0) {
        const double norm = ch < 2 ? (double)N : (double)N * (double)N;
        const double cst = ch < 2 ? c3 : c4;
        if (ch >= 2 && scale4 != 1.0) {              // sampling estimate: inverse inclusion probability
            g *= scale4;
            p *= scale4;
        }
        // a rate kernel whose bounded wait expired leaves incomplete partials: poison Γ
        if (err && *err) g = __longlong_as_double(0x7ff8000000000000ll);
        gamma[(size_t)ch * ld + ms] = g * cst / norm;
        if (wp) wp[(size_t)ch * ld + ms] = p / norm;
        if (counts) counts[(size_t)ch * ld + ms] = n;
    }
}

cudaError_t launch_reduce(const Tables &t, const RateArgs &a, int channel_mask, double c3,
                          double c4, double *gamma, double *wp, long long *counts,
                          unsigned long long *stats, cudaStream_t s) {
    const long long threads = 32LL * 5 * a.n_modes;
    if (threads == 0) return cudaSuccess;
    int5 np;
    np.a = a.n_part[0]; np.b = a.n_part[1]; np.c = a.n_part[2]; np.d = a.n_part[3]; np.e = a.n_part[4];
    reduce_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        a.n_modes, a.out_ld > 0 ? a.out_ld : a.n_modes, t.N, np, channel_mask, c3, c4,
        a.sample_all ? 1.0 : a.sample_scale, a.part_g, a.part_wp, a.part_n, a.part_items, a.part_ent,
        a.part_ev, a.part_cev, gamma, wp, counts, stats, a.err);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ kappa

// Γ_tot(λ) = Σ over the channels in mask of gamma[ch][λ]
__device__ __forceinline__ double gamma_total(const double *gamma, int nm, int mask, int i) {
    double g = 0.0;
    for (int ch = 0; ch < 5; ++ch)
        if ((mask >> ch) & 1) g += gamma[(size_t)ch * nm + i];
    return g;
}

// κ_ab = scale Σ_λ C_λ v_a v_b / Γ_λ, C = k_B x² n (n + 1), over modes with ω > 0 and Γ > 0.
// One block; thread i sums modes i, i + 256, ... in order; fixed-order block sums.
__global__ void __launch_bounds__(256)
kappa_kernel(int nm, const double *om, const double *vel, double x_per_w, double kB,
             const double *gamma, int mask, double scale, double *kappa) {
    __shared__ double s_red[32];
    double acc[9];
    for (int k = 0; k < 9; ++k) acc[k] = 0.0;
    for (int i = threadIdx.x; i < nm; i += blockDim.x) {
        const double w = om[i], g = gamma_total(gamma, nm, mask, i);
        if (!(w > 0.0) || !(g > 0.0)) continue;
        const double x = w * x_per_w;
        const double n = 1.0 / expm1(x);
        const double c = kB * x * x * n * (n + 1.0) / g;
        const double *v = vel + 3 * (size_t)i;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) acc[3 * a + b] += c * v[a] * v[b];
    }
    for (int k = 0; k < 9; ++k) {
        const double r = block_sum(acc[k], s_red);
        if (threadIdx.x == 0) kappa[k] = r * scale;
    }
}

cudaError_t launch_kappa(const Tables &t, double hbar_over_kT, double kB, const double *gamma,
                         int mask, double scale, double *kappa, cudaStream_t s) {
    kappa_kernel<<<1, 256, 0, s>>>(t.N * t.nb, t.om, t.vel, hbar_over_kT, kB, gamma, mask, scale, kappa);
    return cudaGetLastError();
}

// dL/dΓ_ch(λ) = Σ_ab dL/dκ_ab dκ_ab/dΓ_tot(λ) = -scale C_λ (v . G v) / Γ_tot² for every channel in
// mask (Γ_tot depends on each of them with weight 1); 0 for skipped modes and other channels.
__global__ void kappa_backward_kernel(int nm, const double *om, const double *vel, double x_per_w, double kB,
                                      const double *gamma, int mask, double scale, const double *dLdk,
                                      double *dLdg) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nm) return;
    const double w = om[i], g = gamma_total(gamma, nm, mask, i);
    double d = 0.0;
    if (w > 0.0 && g > 0.0) {
        const double x = w * x_per_w;
        const double n = 1.0 / expm1(x);
        const double c = kB * x * x * n * (n + 1.0);
        const double *v = vel + 3 * (size_t)i;
        double q = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) q += dLdk[3 * a + b] * v[a] * v[b];
        d = -scale * c * q / (g * g);
    }
    for (int ch = 0; ch < 5; ++ch) dLdg[(size_t)ch * nm + i] = ((mask >> ch) & 1) ? d : 0.0;
}

cudaError_t launch_kappa_backward(const Tables &t, double hbar_over_kT, double kB, const double *gamma,
                                  int mask, double scale, const double *dLdk, double *dLdg, cudaStream_t s) {
    const int nm = t.N * t.nb;
    kappa_backward_kernel<<<(nm + 255) / 256, 256, 0, s>>>(nm, t.om, t.vel, hbar_over_kT, kB, gamma, mask,
                                                            scale, dLdk, dLdg);
    return cudaGetLastError();
}

// out[perm[s]][k] = in[s][k]: device cluster order back to the caller's order
__global__ void unpermute_kernel(int nc, int width, const int *perm, const double *in, double *out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nc * width) return;
    const int s = (int)(i / width), k = (int)(i - (long long)s * width);
    out[(size_t)perm[s] * width + k] = in[i];
}

cudaError_t launch_unpermute(int nc, int width, const int *perm, const double *in, double *out, cudaStream_t s) {
    const long long n = (long long)nc * width;
    if (n == 0) return cudaSuccess;
    unpermute_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(nc, width, perm, in, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ process lists

// The same window decision as the rate kernels: exact FP64 for 3ph; FP32 prefilter with a proven
// bound plus exact FP64 for the ambiguous band for 4ph (fixed or adaptive σ).  One thread per
// (q', j') (3ph) or (q', j', q'') (4ph), in canonical order; counts first, then words at scanned
// offsets.
__device__ __forceinline__ bool keep3(const Tables &t, const RateArgs &a, int ch, int m0, int m1, int m2) {
    if (a.adaptive) return window_exact_adaptive(t, a, ch, m0, m1, m2, -1, m1, m2);
    return fabs(delta_exact(ch, t.om[m0], t.om[m1], t.om[m2], 0.0)) <= a.two_sigma;
}

__device__ __forceinline__ bool keep4(const Tables &t, const RateArgs &a, int ch, int m0, int m1, int m2, int m3) {
    const int s1 = (ch == 4) ? -1 : 1, s2 = (ch == 2) ? 1 : -1;
    const float base = t.om32[m0] + (float)s1 * t.om32[m1];
    const float ad = fabsf((base + (float)s2 * t.om32[m2]) - t.om32[m3]);
    if (a.adaptive) {
        const int w = window_adaptive32(a, ad, two_sigma32(t, a, m2, m3));
        return w == 2 || (w == 1 && window_exact_adaptive(t, a, ch, m0, m1, m2, m3, m2, m3));
    }
    if (ad <= a.lo32) return true;
    if (ad > a.hi32) return false;
    return fabs(delta_exact(ch, t.om[m0], t.om[m1], t.om[m2], t.om[m3])) <= a.two_sigma;
}

template <bool WRITE>
__global__ void processes_kernel(const __grid_constant__ Tables t, const __grid_constant__ RateArgs a, int ch,
                                 int m0, int *counts, const long long *offsets, unsigned long long *words) {
    const int nb = t.nb, N = t.N;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int q0 = m0 / nb;
    const int4 c0 = t.qc[q0];
    if (ch < 2) {
        if (i >= (long long)N * nb) return;
        const int m1 = (int)i, q1 = m1 / nb, j1 = m1 - q1 * nb;
        const int s = ch == 0 ? 1 : -1;
        const int4 c1 = t.qc[q1];
        const int q2 = q_index(c0.x + s * c1.x, c0.y + s * c1.y, c0.z + s * c1.z,
                               t.mesh[0], t.mesh[1], t.mesh[2]);
        long long n = 0, o = WRITE ? offsets[i] : 0;
        if (((t.vmask[q0] >> (m0 - q0 * nb)) & 1u) && ((t.vmask[q1] >> j1) & 1u))
            for (int j2 = 0; j2 < nb; ++j2) {
                if (!((t.vmask[q2] >> j2) & 1u)) continue;
                if (keep3(t, a, ch, m0, m1, q2 * nb + j2)) {
                    if (WRITE) words[o + n] = (unsigned long long)m1 * nb + j2;
                    ++n;
                }
            }
        if (!WRITE) counts[i] = (int)n;
    } else {
        if (i >= (long long)N * nb * N) return;
        const int q2 = (int)(i % N);
        const int m1 = (int)(i / N), q1 = m1 / nb, j1 = m1 - q1 * nb;
        const int s1 = (ch == 4) ? -1 : 1, s2 = (ch == 2) ? 1 : -1;
        const int4 c1 = t.qc[q1], c2 = t.qc[q2];
        const int q3 = q_index(c0.x + s1 * c1.x + s2 * c2.x, c0.y + s1 * c1.y + s2 * c2.y,
                               c0.z + s1 * c1.z + s2 * c2.z, t.mesh[0], t.mesh[1], t.mesh[2]);
        long long n = 0, o = WRITE ? offsets[i] : 0;
        // sampling estimate: only the pairs (λ, q', q'') in the sample have processes
        const bool in_sample = a.sample_all || pair_sampled(a, m0, q1, q2, N);
        if (in_sample && ((t.vmask[q0] >> (m0 - q0 * nb)) & 1u) && ((t.vmask[q1] >> j1) & 1u))
            for (int j2 = 0; j2 < nb; ++j2) {
                if (!((t.vmask[q2] >> j2) & 1u)) continue;
                for (int j3 = 0; j3 < nb; ++j3) {
                    if (!((t.vmask[q3] >> j3) & 1u)) continue;
                    if (keep4(t, a, ch, m0, m1, q2 * nb + j2, q3 * nb + j3)) {
                        if (WRITE)
                            words[o + n] = (((unsigned long long)m1 * N + q2) * nb + j2) * nb + j3;
                        ++n;
                    }
                }
            }
        if (!WRITE) counts[i] = (int)n;
    }
}

static long long process_threads(const Tables &t, int ch) {
    return ch < 2 ? (long long)t.N * t.nb : (long long)t.N * t.nb * t.N;
}

cudaError_t launch_count_processes(const Tables &t, const RateArgs &a, int ch, int mode, int *counts,
                                   cudaStream_t s) {
    const long long n = process_threads(t, ch);
    processes_kernel<false><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(t, a, ch, mode, counts, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_write_processes(const Tables &t, const RateArgs &a, int ch, int mode,
                                   const long long *offsets, unsigned long long *words, cudaStream_t s) {
    const long long n = process_threads(t, ch);
    processes_kernel<true><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(t, a, ch, mode, nullptr, offsets, words);
    return cudaGetLastError();
}

}  // namespace fc4

// ------------------------------------------------------------------------------ iterative BTE

namespace fc4 {

// Δ[ms][x] = Σ_ch (C_ch / N^k_ch) s_ch Σ_q' part_d[ch][ms][q'][x], one warp per (mode, x); the
// partial slots are summed in a fixed order (lane stride, then a fixed shuffle tree).
__global__ void bte_reduce_kernel(int n_modes, int N, int5 n_part, int channel_mask, double c3, double c4,
                                  double scale4, const double *part_d, double *delta) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= 3 * n_modes) return;
    const int ms = w / 3, x = w - 3 * ms;
    double tot = 0.0;
    for (int ch = 0; ch < 5; ++ch) {
        if (!((channel_mask >> ch) & 1)) continue;
        const int np = ch == 0 ? n_part.a : ch == 1 ? n_part.b : ch == 2 ? n_part.c : ch == 3 ? n_part.d : n_part.e;
        const size_t base = ((size_t)ch * n_modes + ms) * N;
        double d = 0.0;
        for (int q = lane; q < np; q += 32) d += part_d[3 * (base + q) + x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(kFull, d, o);
        const double norm = ch < 2 ? (double)N : (double)N * (double)N;
        const double cst = ch < 2 ? c3 : c4;
        if (ch >= 2) d *= scale4;
        tot += d * cst / norm;
    }
    if (lane == 0) delta[3 * (size_t)ms + x] = tot;
}

cudaError_t launch_bte_reduce(const Tables &t, const RateArgs &a, int channel_mask, double c3, double c4,
                              double *delta, cudaStream_t s) {
    const long long threads = 32LL * 3 * a.n_modes;
    if (threads == 0) return cudaSuccess;
    int5 np;
    np.a = a.n_part[0]; np.b = a.n_part[1]; np.c = a.n_part[2]; np.d = a.n_part[3]; np.e = a.n_part[4];
    bte_reduce_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        a.n_modes, t.N, np, channel_mask, c3, c4, a.sample_all ? 1.0 : a.sample_scale, a.part_d, delta);
    return cudaGetLastError();
}

// F = (v + Δ) / Γ_tot for modes with ω > 0 and Γ_tot > 0, else 0 (Δ = NULL: the RTA start v / Γ);
// F32 receives the FP32 copy the mixed-precision kernels read.
__global__ void bte_update_kernel(int nm, const double *om, const double *vel, const double *gamma, int mask,
                                  const double *delta, double *F, float *F32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nm) return;
    const double g = gamma_total(gamma, nm, mask, i);
    const bool ok = om[i] > 0.0 && g > 0.0;
    for (int x = 0; x < 3; ++x) {
        const double f = ok ? (vel[3 * (size_t)i + x] + (delta ? delta[3 * (size_t)i + x] : 0.0)) / g : 0.0;
        F[3 * (size_t)i + x] = f;
        F32[3 * (size_t)i + x] = (float)f;
    }
}

cudaError_t launch_bte_update(const Tables &t, const double *gamma, int mask, const double *delta, double *F,
                              float *F32, cudaStream_t s) {
    const int nm = t.N * t.nb;
    bte_update_kernel<<<(nm + 255) / 256, 256, 0, s>>>(nm, t.om, t.vel, gamma, mask, delta, F, F32);
    return cudaGetLastError();
}

__global__ void to_f32_kernel(const double *in, float *out, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

cudaError_t launch_to_f32(const double *in, float *out, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    to_f32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

// κ_ab = scale Σ_λ C_λ v_a F_b over modes with ω > 0 (one block, fixed-order sums).
__global__ void __launch_bounds__(256)
kappa_F_kernel(int nm, const double *om, const double *vel, double x_per_w, double kB, const double *F,
               double scale, double *kappa) {
    __shared__ double s_red[32];
    double acc[9];
    for (int k = 0; k < 9; ++k) acc[k] = 0.0;
    for (int i = threadIdx.x; i < nm; i += blockDim.x) {
        const double w = om[i];
        if (!(w > 0.0)) continue;
        const double x = w * x_per_w;
        const double n = 1.0 / expm1(x);
        const double c = kB * x * x * n * (n + 1.0);
        const double *v = vel + 3 * (size_t)i;
        const double *f = F + 3 * (size_t)i;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) acc[3 * a + b] += c * v[a] * f[b];
    }
    for (int k = 0; k < 9; ++k) {
        const double r = block_sum(acc[k], s_red);
        if (threadIdx.x == 0) kappa[k] = r * scale;
    }
}

cudaError_t launch_kappa_F(const Tables &t, double hbar_over_kT, double kB, const double *F, double scale,
                           double *kappa, cudaStream_t s) {
    kappa_F_kernel<<<1, 256, 0, s>>>(t.N * t.nb, t.om, t.vel, hbar_over_kT, kB, F, scale, kappa);
    return cudaGetLastError();
}

}  // namespace fc4
