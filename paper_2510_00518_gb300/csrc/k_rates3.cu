// k_rates3.cu - three-phonon kernel (channels 3ph+ and 3ph-): one thread per (λ, q'), the
// partner q'' = q ± q' closed on the integer mesh, the exact FP64 window over (j', j''), and
// for each kept process V3 summed over the clusters (the paper's Algorithm 1 body, one thread
// per outer iteration); partial sums per (λ, q') are reduced deterministically afterwards.
//
// V3^s(λ, λ', λ'') = Σ_c exp(-i q.R2) exp(i s q'.(R1 - R2)) / sqrt(m) Σ_αβγ Φ[αβγ] e_λ(aα) e^s_λ'(bβ) e*_λ''(cγ)
// (the phase of exp(i(s q'.R1 - q''.R2)) with q'' = q + s q').  Three-phonon work is a few
// percent of the four-phonon work, so this kernel stays FP64 in both precision modes.
#include "fc4_device.cuh"
#include "fc4_kernels.h"

namespace fc4 {

template <int NA>
__global__ void __launch_bounds__(128)
rates3_kernel(const __grid_constant__ Tables t, const __grid_constant__ RateArgs a, int ch) {
    constexpr int NB = 3 * NA;
    const int s = (ch == 0) ? 1 : -1;
    const double sym = (ch == 0) ? 1.0 : 0.5;
    const int N = t.N;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)a.n_modes * N) return;
    const int ms = (int)(tid / N), q1 = (int)(tid - (long long)ms * N);
    const int m0 = a.modes[ms];
    const int q0 = m0 / NB, j0 = m0 - q0 * NB;
    double acc_g = 0.0, acc_wp = 0.0;
    long long acc_n = 0;
    if (!(q0 == 0 && j0 < 3)) {
        const int4 c0 = t.qc[q0], c1 = t.qc[q1];
        const int q2 = q_index(c0.x + s * c1.x, c0.y + s * c1.y, c0.z + s * c1.z,
                               t.mesh[0], t.mesh[1], t.mesh[2]);
        const unsigned v1 = t.vmask[q1], v2 = t.vmask[q2];
        const double w0 = t.om[m0];
        for (int j1 = 0; j1 < NB; ++j1) {
            if (!((v1 >> j1) & 1u)) continue;
            const int m1 = q1 * NB + j1;
            const double w1 = t.om[m1];
            for (int j2 = 0; j2 < NB; ++j2) {
                if (!((v2 >> j2) & 1u)) continue;
                const int m2 = q2 * NB + j2;
                const double d = delta_exact(ch, w0, w1, t.om[m2], 0.0);
                if (!(fabs(d) <= a.two_sigma)) continue;
                double2 V = czero<double2>();
                for (int c = 0; c < t.nc3; ++c) {
                    const int4 at = t.c3_at[c];
                    const int idx = mod_pos(s * phase_index(c1, t.c3_r12[c], t.L) -
                                                phase_index(c0, t.c3_r2[c], t.L), t.L);
                    const double *phi = t.phi3 + 27 * c;
                    double2 e2[3];
#pragma unroll
                    for (int g = 0; g < 3; ++g) e2[g] = cconj(t.ev[(q2 * NB + 3 * at.z + g) * NB + j2]);
                    double2 acc = czero<double2>();
#pragma unroll
                    for (int al = 0; al < 3; ++al) {
                        double2 sa = czero<double2>();
#pragma unroll
                        for (int be = 0; be < 3; ++be) {
                            double2 sb = czero<double2>();
#pragma unroll
                            for (int g = 0; g < 3; ++g) sb = crfma(phi[(al * 3 + be) * 3 + g], e2[g], sb);
                            sa = cfma(cconj_if(t.ev[(q1 * NB + 3 * at.y + be) * NB + j1], s < 0), sb, sa);
                        }
                        acc = cfma(t.ev[(q0 * NB + 3 * at.x + al) * NB + j0], sa, acc);
                    }
                    V = crfma(t.c3_ism[c], cmul(t.rt[idx], acc), V);
                }
                const double g = exp(-(d * d) * a.inv_sigma2) * a.gnorm;
                const double w = sym * occupation_factor<double>(ch, t.occ[m1], t.occ[m2], 0.0) * g *
                                 t.invw[m0] * t.invw[m1] * t.invw[m2];
                acc_wp += w;
                acc_g += w * (V.x * V.x + V.y * V.y);
                acc_n += 1;
            }
        }
    }
    const size_t o = ((size_t)ch * a.n_modes + ms) * N + q1;
    a.part_g[o] = acc_g;
    a.part_wp[o] = acc_wp;
    a.part_n[o] = acc_n;
    a.part_items[o] = 0;
}

template <int NA>
static cudaError_t launch3(const Tables &t, const RateArgs &a, int ch, cudaStream_t s) {
    const long long n = (long long)a.n_modes * t.N;
    if (n == 0) return cudaSuccess;
    const long long blocks = (n + 127) / 128;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    rates3_kernel<NA><<<(unsigned)blocks, 128, 0, s>>>(t, a, ch);
    return cudaGetLastError();
}

cudaError_t launch_rates3(const Tables &t, RateArgs &a, int ch, int fp64, cudaStream_t s) {
    (void)fp64;
    a.n_part[ch] = t.N;
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
