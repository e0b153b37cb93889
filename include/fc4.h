/*
 * fc4.h - C interface of libfc4: three- and four-phonon scattering rates Γ(q,j), weighted phase
 * space, process lists, RTA thermal conductivity and the adjoint with respect to the cubic and
 * quartic force constants, computed on one GB300 GPU (sm_103a).
 *
 * Method: arxiv 2510.00518 (FourPhonon_GPU).  The paper states the problem as: for every mode
 * (q, j), enumerate the momentum-conserving partners, keep those inside the energy window
 * |Δ| <= 2σ, and accumulate the weighted phase space and WP * |V|² into Γ (Algorithms 1-4,
 * Methodology section); κ follows in the relaxation-time approximation (Results section).
 * The channel conventions, matrix elements, weights and unit constants that the paper leaves
 * as black boxes are spelled out at each entry point below.
 *
 * Conventions shared by every call
 *   - Units: Å, amu, eV; ω in rad/ps; Γ in ps^-1; κ in W/(m K); T in K.
 *   - Mesh: Γ-centred n1 x n2 x n3, q index = i1 + n1 (i2 + n2 i3) (first axis fastest),
 *     q = Σ_k (i_k / n_k) b_k with a_i . b_j = 2π δ_ij.  Mode index = q * nb + j, nb = 3 n_atoms.
 *   - Channels (bit k of a channel mask selects channel k):
 *       0 3ph+  q'' = q + q'          Δ = (ω + ω') - ω''
 *       1 3ph-  q'' = q - q'          Δ = ω - (ω' + ω'')
 *       2 4ph++ q''' = q + q' + q''   Δ = (ω - ω''') + (ω' + ω'')
 *       3 4ph+- q''' = q + q' - q''   Δ = (ω + ω') - (ω'' + ω''')
 *       4 4ph-- q''' = q - q' - q''   Δ = ω - ((s0 + s1) + s2), partner ω in ascending order
 *     A process is kept iff |Δ| <= 2σ evaluated in IEEE FP64 with exactly these parentheses.
 *   - The three acoustic modes at Γ (q index 0, branches 0..2) are excluded as the mode and as
 *     partners (ω = 0).
 *   - Ownership: the caller owns every buffer it passes.  fc4_init copies its inputs.  Output
 *     buffers named "device" must be device memory of the current CUDA device, allocated by the
 *     caller; results are ready when the given stream (cudaStream_t, NULL = legacy default
 *     stream) reaches the point of the call.  Host pointers are read or written before return.
 *   - Errors: no call throws.  On any status other than FC4_OK the outputs are unspecified and
 *     fc4_last_error(ctx) holds a one-line message.  Calls on one context must not overlap.
 */
#ifndef FC4_H
#define FC4_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fc4_ctx fc4_ctx;

typedef enum {
    FC4_OK = 0,
    FC4_ERR_INVALID = 1,   /* bad argument (size, index, pointer, channel, mesh) */
    FC4_ERR_CUDA = 2,      /* a CUDA runtime call failed */
    FC4_ERR_OOM = 3,       /* device allocation failed */
    FC4_ERR_TIMEOUT = 4,   /* a bounded device wait expired */
    FC4_ERR_UNSTABLE = 5,  /* harmonic eigenvalue below -1e-8 eV/(Å² amu) (imaginary mode) */
    FC4_ERR_STATE = 6      /* call order violated (e.g. backward before rates) */
} fc4_status;

/* Arithmetic of the matrix-element contraction.  The energy window, the process counts and the
 * final reduction into Γ are FP64 in every mode (the window decided exactly, the sums
 * accumulated per thread in Kahan FP32 or FP64 and across threads in FP64).
 *   FC4_FP64    every channel: FP64 contraction and FP64 weights (reference-accurate)
 *   FC4_MIXED   four-phonon channels: FP32 contraction and FP32 weights on the CUDA cores;
 *               three-phonon channels: FP64 (their acoustic-sum-rule cancellations need it)
 * The tensor-core modes are FC4_MIXED with the cluster contraction X = Σ_r P_r W_r of the 4ph +-
 * channel (the dense one) run by tcgen05.mma with FP32 accumulation in tensor memory, for cells
 * of two atoms (other cells, and the sparse ++ and -- channels, stay on the CUDA cores):
 *   FC4_TF32X3  TF32 hi/lo operand splits, three products (hi.hi + hi.lo + lo.hi): ~2^-21 relative
 *   FC4_BF16    BF16 operands, one product: ~2^-8 relative (single pass; Γ off by ~1e-3)
 *   FC4_BF16X3  BF16 hi/lo splits, three products: ~2^-16 relative
 *   FC4_FP16X3  FP16 hi/lo splits of W scaled by a power of two per unit, three products: ~2^-21
 * Mixed-precision arithmetic is the paper's named direction for further speed (Results, end). */
typedef enum {
    FC4_FP64 = 0,
    FC4_MIXED = 1,
    FC4_TF32X3 = 2,
    FC4_BF16 = 3,
    FC4_BF16X3 = 4,
    FC4_FP16X3 = 5
} fc4_precision;

typedef struct {
    int n_atoms;
    double lattice[9];        /* rows a1, a2, a3 (Å) */
    const double *positions;  /* [n_atoms][3] Cartesian Å (host) */
    const double *masses;     /* [n_atoms] amu (host) */
} fc4_crystal;

/* Force-constant clusters of one order (2, 3 or 4); leg 0 sits in the home cell. */
typedef struct {
    int order;
    int n_clusters;
    const int *atoms;         /* [n_clusters][order] basis-atom index per leg (host) */
    const int *cells;         /* [n_clusters][order-1][3] lattice coordinates of legs 1.. (host) */
    const double *phi;        /* [n_clusters][3^order] eV/Å^order, last Cartesian index fastest (host) */
} fc4_ifc;

typedef struct {
    int precision;            /* fc4_precision */
    int block_threads;        /* threads per block of the 4ph kernel: 64, 96 or 128; 0 = 128 */
    long long timeout_cycles; /* bound (SM clocks) of device-side waits; 0 = default (2e9, ~1 s) */
    int timing;               /* 1: record CUDA events around every kernel launch (fc4_timings) */
    int allow_unstable;       /* 1: fc4_init keeps a crystal with imaginary modes (ω set to 0 for them) */
    int tensor_cores;         /* 1: 4ph +- cluster contraction on the tensor cores where available
                                 (see fc4_set_tensor_cores); 0 = default: CUDA cores */
    int reserved;
} fc4_options;

/* fc4_init - build a context: copy the crystal, the clusters and the mesh to the device, solve
 * the harmonic problem on the device (batched FP64 Jacobi eigensolver of the dynamical matrix
 * D(q) = Σ_R Φ2(0a, Rb) exp(i q.R) / sqrt(m_a m_b), Hermitised; ω = sqrt(λ); group velocities
 * by Hellmann-Feynman), and build the phase tables exp(i q.R) of every cluster cell vector.
 * phi2 is required; phi3 / phi4 may have n_clusters = 0.  opt may be NULL (FP64 defaults).
 * Paper: harmonic properties are an input of Algorithm 1 (ω, v, e of every mode).
 * Returns FC4_ERR_UNSTABLE if an eigenvalue other than the Γ acoustic ones is below -1e-8. */
fc4_status fc4_init(const fc4_crystal *crystal, const fc4_ifc *phi2, const fc4_ifc *phi3,
                    const fc4_ifc *phi4, const int mesh[3], const fc4_options *opt,
                    fc4_ctx **out);

/* fc4_set_modes - replace the harmonic modes (host arrays): omega [N*nb] rad/ps, vel [N*nb][3]
 * Å/ps, evec [N][nb component][nb branch][2] (re, im).  Used to evaluate the rates for modes
 * computed elsewhere (e.g. to compare against a reference with the same eigenvector gauge). */
fc4_status fc4_set_modes(fc4_ctx *ctx, const double *omega, const double *vel, const double *evec);

/* fc4_get_modes - copy the current modes to host arrays (same layouts; any pointer may be NULL). */
fc4_status fc4_get_modes(fc4_ctx *ctx, double *omega, double *vel, double *evec);

/* fc4_rates - Γ, WP and kept-process counts of every mode (q, j) of the q points in q_subset.
 *
 *   Γ3(λ) = C3/N  Σ w |V3|²,  Γ4(λ) = C4/N² Σ w |V4|²,  WP3 = Σ w / N,  WP4 = Σ w / N²
 *   w = sym * F * exp(-Δ²/σ²) / (σ sqrt(π)) / (ω ω' ω'' [ω'''])          (Algorithm 1, WP)
 *   sym = 1, 1/2, 1/2, 1/2, 1/6 for channels 0..4;  F = n' - n'', 1 + n' + n'',
 *   n'n''(1+n''') - (1+n')(1+n'')n''', n'(1+n'')(1+n''') - (1+n')n''n''',
 *   (1+n')(1+n'')(1+n''') - n'n''n''' (n = Bose-Einstein occupation at T);
 *   V3 = Σ_c Σ Φ_c e_λ e^±_λ' e*_λ'' exp(i(±q'.R1 - q''.R2)) / sqrt(m m m)
 *   V4 = Σ_c Σ Φ_c e_λ e^s1_λ' e^s2_λ'' e*_λ''' exp(i(s1 q'.R1 + s2 q''.R2 - q'''.R3)) / sqrt(m m m m)
 *   (e^+ = e, e^- = conj(e); C3 = ħπ/4, C4 = ħ²π/8 converted to ps^-1.)
 *
 * Four-phonon sums use the triangular partner domain where the summand is swap-symmetric: the
 * +- channel under (λ'', λ''') when Φ4 is invariant under exchanging cluster legs 2 and 3, the ++
 * and -- channels under (λ', λ'') when Φ4 is invariant under exchanging legs 1 and 2 and σ is
 * fixed (checked on the host to 1e-12 of max |Φ4| at fc4_init and fc4_update_anharmonic).  One
 * process of each swapped pair is evaluated with weight 2; counts and Γ are those of the
 * rectangular sum (Γ to rounding).
 *
 * T_K > 0.  sigma_adaptive = 0: fixed Gaussian width sigma_value in THz (σ = 2π sigma_value
 * rad/ps).  sigma_adaptive = 1: adaptive width per process from the group velocities of the two
 * legs that the free partner sum moves together (3ph: λ', λ''; 4ph: λ'', λ'''),
 *   σ = s sqrt(Σ_k ((Δv . b_k) / n_k)² / 6),  s = sigma_value (the scale factor, > 0),
 * b_k the reciprocal vectors and n_k the mesh; a process is kept iff σ > 1e-9 rad/ps and
 * |Δ| <= 2σ, both in FP64 (legs of equal velocity, or velocities equal by symmetry up to rounding
 * noise, give no usable width and the process is dropped).  Any other sigma_adaptive value,
 * or sigma_value <= 0 or not finite, returns FC4_ERR_INVALID.
 * q_subset: host array of n_q distinct q indices (NULL = all N q points, n_q ignored).
 * gamma_out, wp_out: device [5][n_q*nb] doubles; counts_out: device [5][n_q*nb] long long;
 * wp_out and counts_out may be NULL.  Channels outside channel_mask are written as 0.
 * The call records (T, σ, mask, subset) for fc4_rates_backward.  After a first call with the same
 * subset, size and T (which sizes every buffer), a call performs only stream-ordered kernel
 * launches and memsets, so it can be captured in a CUDA graph (relaxed or thread-local mode). */
fc4_status fc4_rates(fc4_ctx *ctx, double T_K, int sigma_adaptive, double sigma_value,
                     int channel_mask, const int *q_subset, int n_q, double *gamma_out,
                     double *wp_out, long long *counts_out, void *stream);

/* fc4_rates_static - fc4_rates for callers that cannot allocate device memory during the call.
 * The paper has no counterpart.  Some host programs own every byte of device memory through
 * their own pooled allocator and do not let a library call cudaMalloc or cudaFree (a direct
 * allocation escapes the pool's accounting, and cudaFree synchronises the whole device); others
 * run latency-bound loops in which an allocation, with its implicit synchronisation, is not
 * acceptable.  Such callers create the context once with fc4_init (which does allocate) during
 * set-up, then call this entry point, which allocates nothing.
 *
 * Fixed σ only, q_subset required, no work counters (fc4_stats).  The three-phonon channels run
 * the same kernels as fc4_rates.  The four-phonon channels run the general kernel, which builds
 * W per block in shared memory, not the tiled path that fc4_rates takes for cells of up to two
 * atoms (that path needs the large W buffer) and never the tensor-core contraction; kept counts
 * are identical, Γ and WP agree with fc4_rates to rounding in FP64 and to the mixed tolerance
 * (1e-4 relative) in mixed precision.
 * Its per-call scratch (q list, mode list, per-(channel, mode, q') partials) is one file-scope
 * device array of 13 MB, created when the library is loaded and held by every GPU that loads it
 * until the process exits.  Limit: n_q * nb * N <= 65536 (e.g. all 27 q of a 3x3x3 mesh, or up
 * to 21 q of an 8x8x8 two-atom mesh); larger requests return FC4_ERR_INVALID and write nothing.
 * No cudaMalloc, cudaFree or other allocating routine is called.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) and caches it, so make that first
 * call before any stream capture.  q_subset (host) is copied into the array on the given stream
 * at every call; if it is page-locked memory, keep it unchanged until the stream has passed the
 * call.  Every call reuses the same array, so calls that overlap on the GPU (different streams,
 * different contexts, different threads) race and give wrong results; serialise them.  Nothing
 * in the array is read before the same call has written it.  Does not change the state that
 * fc4_rates_backward and fc4_processes read. */
fc4_status fc4_rates_static(fc4_ctx *ctx, double T_K, double sigma_value, int channel_mask,
                            const int *q_subset, int n_q, double *gamma_out, double *wp_out,
                            long long *counts_out, void *stream);

/* ---------------------------------------------------------------- iterative Boltzmann equation
 * The paper names the solution of the linearised BTE beyond the RTA as future work (Results,
 * end) without a scheme.  These calls implement the ShengBTE / FourPhonon iterative scheme on the
 * rates' own per-process terms γ_p (Γ_λ = Σ_p γ_p, symmetry factors included): with the deviation
 * vectors F_λ (Å; n_λ = n0_λ - F_λ . ∇T dn0_λ/dT),
 *   F_λ = (v_λ + Δ_λ) / Γ_λ,   Δ_λ = Σ_p γ_p Σ_k s_k (ω_k / ω_λ) F_k,
 * k over the partners of the process, s_k = +1 for a partner on the other side of the process
 * from λ and -1 for one on the same side: 3ph+ (-λ', +λ''), 3ph- (+λ', +λ''), 4ph++ (-λ', -λ'',
 * +λ'''), 4ph+- (-λ', +λ'', +λ'''), 4ph-- (+λ', +λ'', +λ''').  κ_αβ = 1/(N V_cell) Σ_λ C_λ v_λα
 * F_λβ (W/(m K)); F = v / Γ gives the RTA κ of fc4_kappa.  The matrix elements are recomputed at
 * every application (no stored scattering matrix), with the same window, triangular domain,
 * precision and sampling as fc4_rates.  Cells of at most two atoms. */

/* fc4_bte_offdiag - Δ of the modes of q_subset (NULL: all) for deviation vectors F (device
 * [N nb][3], Å), channels in channel_mask, σ as in fc4_rates: delta_out device [n_q nb][3]
 * (Å/ps).  It counts as the last rates call for fc4_rates_backward and fc4_processes
 * (T, σ, mask, subset). */
fc4_status fc4_bte_offdiag(fc4_ctx *ctx, double T_K, int sigma_adaptive, double sigma_value,
                           int channel_mask, const int *q_subset, int n_q, const double *F,
                           double *delta_out, void *stream);

/* fc4_kappa_iterative - iterate F^0 = v / Γ, F^{n+1} = (v + Δ(F^n)) / Γ (Γ_λ = Σ of gamma[ch][λ]
 * over channel_mask; modes with ω = 0 or Γ <= 0 keep F = 0) until the largest change of a κ
 * component is at most tol x max |κ| or max_iter applications of Δ were made.  gamma: device
 * [5][N nb] from fc4_rates over the whole mesh with the same T, σ and mask; kappa_out: device [9]
 * of the last iterate (W/(m K)); F_out: device [N nb][3] or NULL; *iters_out (host, may be
 * NULL): the number of Δ applications.  Synchronises the stream once per iteration. */
fc4_status fc4_kappa_iterative(fc4_ctx *ctx, double T_K, int sigma_adaptive, double sigma_value,
                               int channel_mask, const double *gamma, int max_iter, double tol,
                               double *kappa_out, double *F_out, int *iters_out, void *stream);

/* fc4_processes - the kept processes of one mode and channel, as canonical 64-bit words in
 * ascending order (the paper's loop order q', j', then the remaining branches; Algorithm 3):
 *   3ph: word = (q' nb + j') nb + j''
 *   4ph: word = (((q' nb + j') N + q'') nb + j'') nb + j'''
 * words: host array of capacity cap (may be NULL when cap = 0); *n_out receives the count even
 * when it exceeds cap (then only the first cap words are written).  Uses the (T, σ) of the last
 * fc4_rates call (fixed or adaptive), or 300 K and a fixed 0.1 THz before any. */
fc4_status fc4_processes(fc4_ctx *ctx, int channel, int mode, unsigned long long *words,
                         long long cap, long long *n_out);

/* fc4_kappa - RTA thermal conductivity κ_αβ = 1/(N V_cell) Σ_λ C_λ v_α v_β / Γ_λ (W/(m K)),
 * C_λ = k_B x² n (n + 1), x = ħω / k_B T, Γ_λ = Σ of gamma[ch][λ] over the channels in
 * channel_mask, over every mode of the mesh with ω > 0 and Γ_λ > 0 (Results section: RTA κ).
 * gamma: device [5][N*nb] in ps^-1 (the layout fc4_rates writes for the whole mesh);
 * kappa_out: device [9], row-major. */
fc4_status fc4_kappa(fc4_ctx *ctx, double T_K, const double *gamma, int channel_mask,
                     double *kappa_out, void *stream);

/* fc4_kappa_backward - dL/dΓ_ch(λ) = Σ_αβ dL/dκ_αβ dκ_αβ/dΓ_λ = -C_λ (v_λ . G v_λ) / (N V_cell Γ_λ²)
 * (G = dL/dκ, units as fc4_kappa) for every channel in channel_mask, 0 elsewhere and for
 * skipped modes.  gamma: device [5][N*nb]; dL_dkappa: device [9]; dL_dgamma: device [5][N*nb]. */
fc4_status fc4_kappa_backward(fc4_ctx *ctx, double T_K, const double *gamma, int channel_mask,
                              const double *dL_dkappa, double *dL_dgamma, void *stream);

/* fc4_rates_backward - gradient of L = Σ_{ch,i} dL_dgamma[ch][i] Γ_ch(i) with respect to every
 * stored Φ3 and Φ4 entry (entries independent), at fixed modes and σ (fixed or adaptive: both
 * depend on the modes only), for the (T, σ, mask, subset) of the last fc4_rates call.  FP64 in
 * an FC4_FP64 context; otherwise the 4ph terms run in FP32 (V recomputed in FP32, per-mode slices
 * accumulated as FP32 Kahan pairs, summed in FP64) and the 3ph terms in FP64:
 *   dL/dΦ_c = Σ_processes dL/dΓ C/N^k w 2 Re(conj(V) dV/dΦ_c),  V recomputed (not stored).
 * Deterministic (fixed summation order).  dL_dgamma: device [5][n_q*nb]; dphi3: device
 * [nc3][27]; dphi4: device [nc4][81], in the cluster order given to fc4_init (overwritten;
 * either may be NULL to skip that order).  Cells of at most 4 atoms.  Returns FC4_ERR_STATE
 * before any fc4_rates call.  Scratch: n_q*nb*max(27 nc3, 81 nc4) doubles (grown on demand). */
fc4_status fc4_rates_backward(fc4_ctx *ctx, const double *dL_dgamma, double *dphi3,
                              double *dphi4, void *stream);

/* fc4_update_anharmonic - replace the Φ3 and/or Φ4 values (host, same cluster lists and layout
 * as fc4_init; NULL keeps the current values).  Modes and phase tables are unchanged. */
fc4_status fc4_update_anharmonic(fc4_ctx *ctx, const double *phi3, const double *phi4);

/* fc4_stats - work counters of the last fc4_rates call (synchronises the device), for channels
 * ch = 0..4:
 *   out[6*ch + 0] kept processes of the rectangular partner domain (the counts of fc4_rates);
 *   out[6*ch + 1] four-phonon (q'', j''') items evaluated;
 *   out[6*ch + 2] candidate tuples of the rectangular domain before the window;
 *   out[6*ch + 3] four-phonon (q'', j') entries whose cluster sum was contracted;
 *   out[6*ch + 4] processes actually evaluated: where a partner-swap symmetry of the summand
 *                 holds (see fc4_rates), one process of each swapped pair is evaluated and
 *                 counted twice in out[6*ch + 0];
 *   out[6*ch + 5] candidate tuples the energy-window test visited.
 * Items and entries are 0 for 3ph. */
fc4_status fc4_stats(fc4_ctx *ctx, long long out[30]);

/* fc4_timings - device time in ms of the kernels launched by the last fc4_rates / fc4_kappa
 * calls, measured with CUDA events recorded on the launching stream around each launch (needs
 * fc4_options.timing = 1; synchronises on those events): out[0..4] the rate kernel of channel
 * 0..4 (0 if not launched), out[5] the reduction, out[6] the conductivity, out[7] the occupation
 * table, out[8] the number of kernels libfc4 launched since the context was created. */
fc4_status fc4_timings(fc4_ctx *ctx, double out[9]);

/* fc4_set_block_threads - threads per block of the general four-phonon kernel (cells of more
 * than 2 atoms): 64, 96 or 128 (0 = 128).  A tuning knob; results do not depend on it. */
fc4_status fc4_set_block_threads(fc4_ctx *ctx, int block_threads);

/* fc4_set_mode_chunk - how many modes one fc4_rates call processes at a time (the paper's
 * all-modes and mode-by-mode strategies, Results and Algorithm 5).  A call splits its modes into
 * chunks of at most modes_per_chunk modes (0: no bound) and of at most w_limit_bytes of W scratch
 * for the tiled 4ph path (0: max(4 GiB, a quarter of the device memory)); each chunk runs every
 * channel and its reduction before the next.  The per-call device memory (partials of 56 bytes
 * per (channel, mode, q'), and W of fc4_memory's out[1] bytes per mode) grows with the chunk, not
 * with the subset.  modes_per_chunk = 1 is mode by mode.  Results do not depend on the chunking. */
fc4_status fc4_set_mode_chunk(fc4_ctx *ctx, int modes_per_chunk, long long w_limit_bytes);

/* fc4_memory - device memory of a context: out[0] bytes allocated by the context in total,
 * out[1] W bytes per mode of the tiled 4ph path in the current precision (0: general kernel),
 * out[2] bytes of the current W buffer, out[3] bytes of the current partials, out[4] modes per
 * chunk of the last fc4_rates call. */
fc4_status fc4_memory(const fc4_ctx *ctx, long long out[5]);

/* fc4_set_sampling - sampling estimate of the four-phonon sums for later fc4_rates and
 * fc4_processes calls (the paper names combining the GPU path with sampling estimation as future
 * work, Introduction and end of Results, without a scheme; this is the reading implemented).
 * Each partner pair (λ, q', q'') enters the 4ph sums independently with probability `fraction`:
 * it is taken iff SplitMix64's output function (Steele, Lea and Flood, OOPSLA 2014) of
 * seed + (key + 1) * 0x9e3779b97f4a7c15, key = (mode * N + q') * N + q'' (64-bit wrap-around), is
 * below floor(fraction * 2^64).  Γ and WP of the 4ph channels are multiplied by 2^64 / that
 * threshold, the inverse inclusion probability (an unbiased estimate of the full sums); counts
 * report the kept processes of the sampled pairs.  Skipped pairs cost no evaluation.  fraction
 * >= 1 (the default) takes every pair; fraction in (0, 1) samples; other values return
 * FC4_ERR_INVALID.  Three-phonon channels are never sampled.  fc4_rates_backward refuses
 * (FC4_ERR_STATE) while sampling is on. */
fc4_status fc4_set_sampling(fc4_ctx *ctx, double fraction, unsigned long long seed);

/* fc4_set_ablation - measurement switches of the tiled 4ph kernels (results do not change):
 * bit 0: no compaction - each thread evaluates the (q'', j') entries its own window test found, as
 * an uncompacted GPU-only loop does (the paper's Algorithm 2 and its warp divergence, Results),
 * instead of the block's entries being dealt out to all threads in order.  0 (the default)
 * restores compaction.  Mixed-precision tiled kernels only (others ignore it).  Other bits return
 * FC4_ERR_INVALID. */
fc4_status fc4_set_ablation(fc4_ctx *ctx, int flags);

/* fc4_set_precision - change the arithmetic of later fc4_rates calls (any fc4_precision; the
 * tables of every mode are built at fc4_init).  Kept sets do not depend on it. */
fc4_status fc4_set_precision(fc4_ctx *ctx, int precision);

/* fc4_set_tensor_cores - shorthand for the FP16 x3 tensor-core format in an FC4_MIXED context:
 * on = 1 runs the 4ph +- cluster contraction X = Σ_r P_r W_r on the tensor cores (tcgen05, FP16
 * hi/lo operands, three products, FP32 accumulation) for two-atom cells; on = 0 (the default,
 * faster on the measured workloads) keeps the CUDA cores.  Kept sets are identical either way; Γ
 * agrees to rounding.  fc4_set_precision selects every format.  FC4_ERR_INVALID for other values. */
fc4_status fc4_set_tensor_cores(fc4_ctx *ctx, int on);

/* fc4_check_device - FC4_ERR_TIMEOUT if a kernel of this context gave up a bounded device-side
 * wait since the last check (the Γ of that call were written as NaN), else FC4_OK; clears the
 * flag.  Synchronises the device. */
fc4_status fc4_check_device(fc4_ctx *ctx);

/* fc4_info - sizes of a context: out[0..7] = n_atoms, nb, N, nc2, nc3, nc4, n_keys, precision. */
fc4_status fc4_info(const fc4_ctx *ctx, long long out[8]);

/* ---------------------------------------------------------------- irreducible q-points
 * The mode loops of Algorithms 1 and 3-5 run over N_bands x N_list modes, N_list being the
 * irreducible q-points of the mesh.  A space-group operation of the crystal that also maps its
 * force constants onto themselves permutes the partner q-points of the mesh and keeps
 * frequencies, occupations and |V|², so Γ(S q, j) = Γ(q, j) in every channel; q -> -q (real
 * force constants) does the same.  These three host-only calls (no context, no GPU; errors in
 * fc4_last_error(NULL)) find the operations, the irreducible points, and spread the rates that
 * fc4_rates computes on those points (q_subset) over the whole mesh for fc4_kappa.  Exact for
 * a fixed σ only: the adaptive width σ = s sqrt(Σ_k ((Δv . b_k) / n_k)² / 6) takes its Δv from
 * Hellmann-Feynman velocities, which inside a degenerate subspace depend on the eigenvector basis
 * chosen at each q, so Γ with that width is not constant on a star. */

/* fc4_symmetry_ops - the space-group operations {W | w} of a primitive cell, in fractional
 * coordinates f -> W f + w (W integer with entries in {-1, 0, 1}, det W = ±1, W^T G W = G for the
 * metric G_ij = a_i . a_j; w in [0, 1)).  An operation is returned when it maps every atom onto
 * an atom of the same mass (within 1e-6 of the longest lattice vector) and every cluster of
 * phi2, phi3 and phi4 (each may be NULL or empty) onto a stored cluster with the tensor rotated,
 * Φ'[α'β'..] = Σ S_α'α S_β'β .. Φ[αβ..] with S = A^T W A^-T, within tol x max |Φ| of that order
 * (tol <= 0: 1e-8); a cluster whose image is not stored must rotate to below that bound.
 * Layouts as for fc4_init.  rot: host [max_ops][3][3] row-major W; trans: host [max_ops][3] w;
 * *n_ops receives the number of operations.  max_ops = 0 (rot and trans may be NULL) only
 * counts them; with max_ops > 0, finding more than max_ops returns FC4_ERR_INVALID (with *n_ops
 * set and the first max_ops written). */
fc4_status fc4_symmetry_ops(const fc4_crystal *crystal, const fc4_ifc *phi2, const fc4_ifc *phi3,
                            const fc4_ifc *phi4, double tol, int max_ops, int *rot, double *trans,
                            int *n_ops);

/* fc4_irreducible_q - orbits of the mesh q-points under the group generated by the operations
 * W (rot: host [n_ops][3][3], as from fc4_symmetry_ops) and, with flags bit 0, time reversal
 * q -> -q.  A q in reciprocal fractional coordinates maps as k' = W^-T k; an operation that
 * does not map the mesh onto itself is ignored.  rep: host [N] receives for every q the
 * smallest q index of its orbit (rep[q] == q marks an irreducible point); *n_irr the number of
 * orbits.  FC4_ERR_INVALID for det W != ±1 or any other flag bit. */
fc4_status fc4_irreducible_q(const int mesh[3], int n_ops, const int *rot, int flags, int *rep,
                             int *n_irr);

/* fc4_expand_irreducible - per-mode values of the whole mesh from those of its irreducible
 * points: full[s][q nb + j] = the mean of sub[s][p nb + j'] over the branches j' degenerate with
 * j at the representative r = rep[q] (|ω difference| <= deg_tol between neighbours in ascending
 * ω), p = the position of r among the irreducible points in ascending order.  Averaging over a
 * degenerate group makes the result independent of the eigenvector basis chosen inside it (the
 * group's sum is invariant; its members are not).  rep: host [N] as from fc4_irreducible_q;
 * omega: host [N nb] rad/ps; sub: host [n_sets][n_irr nb] (e.g. Γ, WP of fc4_rates on the
 * irreducible points, copied to the host); full: host [n_sets][N nb]. */
fc4_status fc4_expand_irreducible(const int mesh[3], int nb, const int *rep, const double *omega,
                                  double deg_tol, int n_sets, const double *sub, double *full);

/* ---------------------------------------------------------------- batches of crystals
 * Many contexts (crystals of different cell sizes, meshes and clusters) evaluated together.
 * fc4_batch_rates runs the four-phonon units (λ, q') of every context of more than two atoms with
 * the same cell size as ONE persistent launch of the general kernel: a work list of (context,
 * channel, unit) from the largest meshes down, each 128-thread block taking the next item from a
 * global counter, so that the uneven per-crystal and per-q work balances across the whole GPU;
 * their three-phonon kernels and reductions run per context, FP32 contractions, no tensor cores,
 * and their Γ, WP and counts equal fc4_rates_static's (the same kernel arithmetic).  Contexts of up
 * to two atoms run their own fc4_rates (the tiled kernels, several times faster than the general
 * one on such cells).  Contexts of any precision but FC4_FP64; fixed σ; at most 40 contexts.  The
 * contexts' tables and call arguments go to the kernel's constant memory, one copy per process and
 * device: calls of different batches that overlap on the GPU race.  After a first call with the
 * same arguments (which sizes every buffer), a call performs only stream-ordered launches and
 * memsets, so it can be captured in a CUDA graph. */

typedef struct fc4_batch fc4_batch;

/* fc4_batch_create - a batch over n contexts (the contexts must outlive it; not copied). */
fc4_status fc4_batch_create(fc4_ctx *const *ctxs, int n, fc4_batch **out);

/* fc4_batch_rates - rates of every context: q_subsets[i] (host, n_q[i] q points; q_subsets or
 * q_subsets[i] NULL = all q), fixed σ sigma_value THz, T_K > 0, channel_mask as for fc4_rates;
 * gamma_out[i] (and wp_out[i], counts_out[i] if the arrays are not NULL): device [5][n_q nb] of
 * context i.  fc4_stats of each context reports its part. */
fc4_status fc4_batch_rates(fc4_batch *b, double T_K, double sigma_value, int channel_mask,
                           const int *const *q_subsets, const int *n_q, double *const *gamma_out,
                           double *const *wp_out, long long *const *counts_out, void *stream);

/* fc4_batch_last_error - message of the last failed call on b. */
const char *fc4_batch_last_error(const fc4_batch *b);

/* fc4_batch_destroy - free the batch (not its contexts; NULL is a no-op). */
void fc4_batch_destroy(fc4_batch *b);

/* fc4_device_peaks - calibration of the current device's CUDA cores (no context): out[0] the FP32
 * and out[1] the FP64 fused multiply-add rate in TFLOP/s (2 flops per FMA), each timed with CUDA
 * events on `stream` over one launch of 8 x 256-thread blocks per SM running 8 independent FMA
 * chains per thread, after a warm-up launch.  The rate kernels' arithmetic runs on these units,
 * so these are the denominators of their roofline.  Synchronises the stream. */
fc4_status fc4_device_peaks(double out[2], void *stream);

/* fc4_last_error - message of the last failed call on ctx (or, when ctx is NULL, of the last
 * failed fc4_init or host-only call).  The string lives until the next call on ctx. */
const char *fc4_last_error(const fc4_ctx *ctx);

/* fc4_destroy - free every device and host resource of ctx (NULL is a no-op). */
void fc4_destroy(fc4_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* FC4_H */
