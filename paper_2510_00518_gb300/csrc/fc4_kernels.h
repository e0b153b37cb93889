// fc4_kernels.h - launch interfaces of libfc4's kernels (host side), shared between the C-ABI
// translation unit and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fc4 {

constexpr int kMaxAtoms = 8;      // nb <= 24: branch masks fit in 32 bits
constexpr int kGroups = kMaxAtoms * kMaxAtoms + 1;   // (leg-2 atom, leg-3 atom) groups + 1
constexpr double kAdaptiveSigmaMin = 1e-9;           // rad/ps: adaptive widths at or below are noise

// Device tables of one context (all pointers are device memory).
struct Tables {
    int n_atoms, nb, N, L;
    int mesh[3];
    // mesh
    const int4 *qc;              // [N] integer coordinates (i1, i2, i3, 0)
    const double2 *rt;           // [L] exp(2πi k / L)
    const float2 *rt32;          // [L]
    // modes
    const double *om;            // [N*nb] rad/ps (0 for excluded)
    const float *om32;           // [N*nb] ω rounded to FP32 (hi part)
    const float *om32lo;         // [N*nb] ω - hi rounded to FP32 (lo part)
    const double *vel;           // [N*nb][3] Å/ps
    const double2 *ev;           // [N][nb comp][nb branch]
    const float2 *ev32;          // [N][nb][nb]
    const unsigned *vmask;       // [N] bit j set iff mode (q, j) takes part
    const float4 *vp32;          // [N*nb] P_k = (v . b_k) / n_k, k = 1..3 (rad/ps), FP32 hi parts
    const float4 *vp32lo;        // [N*nb] P_k - hi, FP32 (lo parts)
    // branch-major copies for the window, whose lanes read consecutive q: [nb][N]
    const float *omT32;          // ω hi
    const float4 *vpT32;         // P hi
    const float4 *vpTlo;         // P lo
    double recip[9];             // reciprocal vectors b_k (rows, 1/Å), a_i . b_k = 2π δ_ik
    // occupations at the current T
    const double *occ;           // [N*nb]
    const float *occ32;          // [N*nb]
    const double *invw;          // [N*nb] 1/ω (0 for excluded)
    const float *invw32;         // [N*nb]
    // third order
    int nc3;
    const int4 *c3_at;           // [nc3] (a, b, c, 0)
    const int4 *c3_r2;           // [nc3] R2 (L/n) mod L
    const int4 *c3_r12;          // [nc3] (R1 - R2)(L/n) mod L
    const double *c3_ism;        // [nc3] 1/sqrt(m_a m_b m_c)
    const double *phi3;          // [nc3][27]
    // fourth order: clusters sorted by key; keys sorted by (leg-2 atom, leg-3 atom) group
    int nc4, n_keys;
    const int4 *c4_at;           // [nc4] (a, b, c, d)
    const int4 *c4_r3;           // [nc4] R3 (L/n) mod L
    const int4 *c4_r13;          // [nc4] (R1 - R3)(L/n) mod L
    const double *c4_ism;        // [nc4] 1/sqrt(m_a m_b m_c m_d)
    const float *c4_ism32;
    const double *phi4;          // [nc4][81]
    const float *phi4_32;
    const int *key_start;        // [n_keys + 1] cluster range of each key
    const int *kb_start;         // [n_keys * n_atoms + 1] range in kb_idx of (key r, leg-1 atom b)
    const int *kb_idx;           // [nc4] clusters grouped by (r, b), ascending within a group
    const double2 *P4;           // [N][n_keys] exp(i q.(R2 - R3)) of each key
    const float2 *P4_32;
    int grp_start[kGroups];      // key range of group g = c * n_atoms + d
};

// Per-call parameters of the rate kernels.
struct RateArgs {
    int n_modes;                 // modes in the subset (n_q * nb)
    const int *modes;            // [n_modes] device
    double two_sigma;            // 2σ (rad/ps)
    double inv_sigma2;           // 1/σ²
    double gnorm;                // 1/(σ sqrt(π))
    float lo32, hi32;            // prefilter: |Δ32| <= lo keep, > hi reject, else exact
    float inv_sigma2_32, gnorm32;  // FP32 copies of 1/σ² and 1/(σ sqrt(π)) (mixed weights)
    double *part_g;              // [5][n_modes][N] per-(mode, q') partial sums
    double *part_wp;
    long long *part_n;           // kept processes
    long long *part_items;       // 4ph: (q'', j''') items evaluated; 3ph: 0
    long long *part_ent;         // 4ph: (q'', j') entries whose X or Y was contracted; 3ph: 0
    long long *part_ev;          // processes evaluated (kept counts a swap pair twice); may be NULL
    long long *part_cev;         // candidates visited by the window; may be NULL
    int n_part[5];               // partial slots written per mode for each channel (<= N)
    void *wbuf;                  // optional scratch for the tiled 4ph path (W per (λ, q')); may be NULL
    size_t wbuf_bytes;
    int w_reuse;                 // 1: wbuf already holds W of every mode for this channel's sign s1
    // adaptive broadening: σ of a process from the velocities of the two legs its free partner
    // sum moves together (3ph: λ', λ''; 4ph: λ'', λ'''), σ = s |ΔP| / sqrt(6)
    int adaptive;
    double ad_scale;             // s
    float ad_c32;                // 2 s / sqrt(6): 2σ ≈ ad_c32 |ΔP| (FP32)
    float ad_s32;                // s / sqrt(6)
    float ad_rlo, ad_rhi;        // prefilter: keep if |Δ32| <= ad_rlo 2σ32 - ad_e0,
    float ad_e0;                 //   reject if |Δ32| > ad_rhi 2σ32 + ad_e0, else exact FP64
    float ad_gmin;               // sure keep also needs 2σ32 > ad_gmin (σ above the noise floor)
    int use_tc;                  // tensor-core contraction of 4ph +- (two atoms): 0 off, 1 FP16 x3,
                                 // 2 BF16 x3, 3 BF16, 4 TF32 x3
    long long spin_limit;        // bound (SM clocks) of device-side waits; 0 = default
    int *err;                    // device flag set by a kernel whose wait expired (may be NULL)
    long long *n_kernels;        // host counter of kernels launched (may be NULL; never read on device)
    int out_ld;                  // row stride of the reduction's outputs [5][out_ld] (0: n_modes)
    // sampling estimate of the 4ph sums: pair (mode, q', q'') taken iff its SplitMix64 hash <
    // sample_threshold (sample_all: every pair); the reduction scales the 4ph sums by sample_scale
    int sample_all;
    unsigned long long sample_threshold, sample_seed;
    double sample_scale;
    // iterative BTE: with part_d set, the kernels also accumulate Σ_p γ_p Σ_k s_k ω_k F_k / ω_λ
    // into part_d [5][n_modes][N][3] for the deviation vectors F [N nb][3]
    int no_compact;              // ablation: evaluate each thread's own window entries (no compaction)
    const double *bte_F;
    const float *bte_F32;
    double *part_d;
    int tri;                     // triangular 4ph domain allowed: bit 0 +- (Φ4 symmetric in legs 2, 3),
                                 // bit 1 ++ and -- (legs 1, 2; fixed σ only)
};

// launchers (stream-ordered; return cudaGetLastError())
// each rate launcher records in a.n_part[ch] how many partial slots per mode it writes
cudaError_t launch_rates3(const Tables &t, RateArgs &a, int ch, int fp64, cudaStream_t s);
cudaError_t launch_rates4(const Tables &t, RateArgs &a, int ch, int fp64, int threads,
                          cudaStream_t s);
// tensor-core +- path (k_rates4_tc.cu): availability for a context, and its launch over a mode chunk
bool tc_supported(const Tables &t);
cudaError_t launch_rates4_tc(const Tables &t, const RateArgs &a, int ch, int mode0, int nm, const float2 *w,
                             cudaStream_t s);
// batched persistent 4ph launch over many contexts of one cell size (FP32, fixed σ): work items
// (context, channel, unit); the contexts' tables and arguments are uploaded first into the constant
// memory of both translation units (atoms 1-4 and 5-8), at most kMaxBatch contexts
constexpr int kMaxBatch = 40;
cudaError_t launch4_batch_f_1_4(int na, const int4 *items, int n_items, int *counter, size_t smem, cudaStream_t s);
cudaError_t launch4_batch_f_5_8(int na, const int4 *items, int n_items, int *counter, size_t smem, cudaStream_t s);
cudaError_t batch_upload_f_1_4(const Tables *tabs, const RateArgs *args, int n, cudaStream_t s);
cudaError_t batch_upload_f_5_8(const Tables *tabs, const RateArgs *args, int n, cudaStream_t s);
size_t general_smem_f(int na, const Tables &t);
// bytes of W scratch the tiled 4ph path needs per mode (0 if the general kernel is used)
size_t rates4_wbuf_per_mode(const Tables &t, int fp64);
// iterative BTE: Δ [n_modes][3] from part_d (fixed order), F = v / Γ, F = (v + Δ) / Γ, κ from F
cudaError_t launch_bte_reduce(const Tables &t, const RateArgs &a, int channel_mask, double c3, double c4,
                              double *delta, cudaStream_t s);
cudaError_t launch_bte_update(const Tables &t, const double *gamma, int mask, const double *delta, double *F,
                              float *F32, cudaStream_t s);
cudaError_t launch_to_f32(const double *in, float *out, size_t n, cudaStream_t s);
cudaError_t launch_kappa_F(const Tables &t, double hbar_over_kT, double kB, const double *F, double scale,
                           double *kappa, cudaStream_t s);
cudaError_t launch_reduce(const Tables &t, const RateArgs &a, int channel_mask, double c3,
                          double c4, double *gamma, double *wp, long long *counts,
                          unsigned long long *stats, cudaStream_t s);
cudaError_t launch_harmonic(const Tables &t, int nc2, const int4 *c2_at, const int4 *c2_r,
                            const double *c2_R, const double *c2_phi, const double *c2_ism,
                            double eig_to_w2, double *om, double *vel, double2 *ev, double *eig,
                            int *err, cudaStream_t s);
cudaError_t launch_mode_tables(const Tables &t, double *om, float *om32, float *om32lo,
                               float2 *ev32, const double2 *ev, unsigned *vmask, double *invw,
                               float *invw32, float4 *vp32, float4 *vp32lo, float *omT32, float4 *vpT32,
                               float4 *vpTlo, cudaStream_t s);
cudaError_t launch_occupations(const Tables &t, double hbar_over_kT, double *occ, float *occ32,
                               cudaStream_t s);
// message returned by fc4_last_error(NULL) (errors of calls without a context)
void set_host_error(const char *msg);

cudaError_t launch_phase_tables(const Tables &t, const int4 *key_r, double2 *P4, float2 *P4_32,
                                cudaStream_t s);
cudaError_t launch_kappa(const Tables &t, double hbar_over_kT, double kB, const double *gamma,
                         int mask, double scale, double *kappa, cudaStream_t s);
cudaError_t launch_kappa_backward(const Tables &t, double hbar_over_kT, double kB, const double *gamma,
                                  int mask, double scale, const double *dLdk, double *dLdg, cudaStream_t s);
cudaError_t launch_unpermute(int nc, int width, const int *perm, const double *in, double *out, cudaStream_t s);
// fp64 = 0: the 4ph adjoint in FP32 (slices of FP32 Kahan pairs; sum them with kahan32 = 1)
cudaError_t launch_adjoint(const Tables &t, const RateArgs &a, int ch, const double *dLdG, double cst,
                           double *part, int fp64, cudaStream_t s);
cudaError_t launch_sum_slices(int n_slices, int n, const double *part, double *out, int accumulate,
                              int kahan32, cudaStream_t s);
cudaError_t launch_count_processes(const Tables &t, const RateArgs &a, int ch, int mode, int *counts,
                                   cudaStream_t s);
cudaError_t launch_write_processes(const Tables &t, const RateArgs &a, int ch, int mode,
                                   const long long *offsets, unsigned long long *words, cudaStream_t s);

}  // namespace fc4
