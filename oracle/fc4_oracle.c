/*
 * fc4_oracle.c - plain, slow FP64 reference of the three- and four-phonon scattering rates.
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the package smoke check and the CPU-baseline leg of the
 * bench call it; the CUDA library never does, and the two share no code, header or table.
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (oracle/build.py).
 *
 * It follows the paper's Algorithm 1 (original CPU computation, absorption process): for each
 * mode, loop over partner q-points and branches, close momentum on the integer mesh, test the
 * energy window |Δ| <= 2σ, add the weighted phase space WP and WP * |V|^2, then divide by the
 * number of q-points and multiply by the unit constant.  The paper spells out only the 3ph
 * absorption case; the emission and the three four-phonon channels repeat the same pattern
 * with the conventions below (the formulas the paper treats as black boxes, restated from the
 * Maradudin / Feng-Ruan theory the paper builds on):
 *
 *   channel 0  3ph +  : q'' = q + q'          Δ = (ω + ω') - ω''
 *   channel 1  3ph -  : q'' = q - q'          Δ = ω - (ω' + ω'')
 *   channel 2  4ph ++ : q''' = q + q' + q''   Δ = (ω - ω''') + (ω' + ω'')
 *   channel 3  4ph +- : q''' = q + q' - q''   Δ = (ω + ω') - (ω'' + ω''')
 *   channel 4  4ph -- : q''' = q - q' - q''   Δ = ω - ((s0 + s1) + s2), s = partner ω ascending
 *
 *   V3(s)     = Σ_c Σ_αβγ  Φ_c e_λ(aα) e^s_λ'(bβ) e*_λ''(cγ) exp(i(s q'·R1 - q''·R2)) / sqrt(m_a m_b m_c)
 *   V4(s1,s2) = Σ_c Σ_αβγδ Φ_c e_λ(aα) e^s1_λ'(bβ) e^s2_λ''(cγ) e*_λ'''(dδ)
 *                          exp(i(s1 q'·R1 + s2 q''·R2 - q'''·R3)) / sqrt(m_a m_b m_c m_d)
 *   with e^+ = e and e^- = conj(e); R are the cell vectors of the cluster legs.
 *
 *   weight w = sym * F * δ(Δ) / (ω ω' ω'' [ω''']),   δ(Δ) = exp(-Δ²/σ²) / (σ sqrt(π))
 *     3ph +: F = n' - n''                            sym = 1
 *     3ph -: F = 1 + n' + n''                        sym = 1/2
 *     4ph ++: F = n'n''(1+n''') - (1+n')(1+n'')n'''  sym = 1/2
 *     4ph +-: F = n'(1+n'')(1+n''') - (1+n')n''n'''  sym = 1/2
 *     4ph --: F = (1+n')(1+n'')(1+n''') - n'n''n''' sym = 1/6
 *   Γ3 = C3 / N  Σ w |V3|²,  Γ4 = C4 / N² Σ w |V4|²;  WP3 = Σ w / N,  WP4 = Σ w / N².
 *
 * Broadening: fixed σ, or adaptive σ = s sqrt(Σ_k ((Δv . b_k) / n_k)² / 6) from the velocity
 * difference of the two legs the free partner sum moves together (3ph: v' - v''; 4ph: v'' - v''');
 * with adaptive widths a process is kept only if σ > 1e-9 rad/ps: equal velocities give σ = 0, and
 * velocities equal by symmetry give a σ of rounding noise (~1e-15) whose 1/σ weight is meaningless.
 * Acoustic modes at Γ (q index 0, branches 0..2) are excluded as the mode and as partners.
 * Units: ω rad/ps, e dimensionless, Φ eV/Å^k, masses amu, Γ ps^-1 (C3, C4 come from Python).
 *
 * Sampling estimate (the paper's Results section names combining the GPU with sampling estimation
 * as future work; it does not state the scheme, so this is a reading): for the four-phonon
 * channels each partner pair (λ, q', q'') enters the sums independently with probability f, decided
 * by a counter-based hash, and the sums of Γ and WP are multiplied by 2^64 / threshold (1/f up to
 * the rounding of the threshold), an unbiased Monte-Carlo estimate of the full sums.  The hash is
 * SplitMix64's output function (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014) applied to seed + (key + 1) * 0x9e3779b97f4a7c15 with
 * key = (mode * nq + q') * nq + q''; the pair is taken iff the hash is below threshold =
 * floor(f 2^64) (threshold = 2^64 - 1 with every pair taken when f = 1).  Counts report the
 * processes of the sampled pairs (not rescaled).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int n_atoms, nb;
    int mesh[3];
    int nq;
    double lattice[9];        /* rows a1, a2, a3 (Å) */
    double recip[9];          /* rows b1, b2, b3 (rad/Å), a_i . b_j = 2π δ_ij */
    const double *mass;       /* [n_atoms] amu */
    const double *omega;      /* [nq*nb] rad/ps */
    const double *vel;        /* [nq*nb][3] Å/ps */
    const double *evec;       /* [nq][nb comp][nb branch][re,im] */
    const double *occ;        /* [nq*nb] Bose-Einstein occupation at T */
    int nc3;
    const int *atoms3;        /* [nc3][3] */
    const int *cells3;        /* [nc3][2][3] */
    const double *phi3;       /* [nc3][27] */
    int nc4;
    const int *atoms4;        /* [nc4][4] */
    const int *cells4;        /* [nc4][3][3] */
    const double *phi4;       /* [nc4][81] */
    int sigma_adaptive;       /* 0: fixed σ, 1: adaptive */
    double sigma;             /* fixed: σ in rad/ps; adaptive: scale factor */
    double c3, c4;            /* unit constants of Γ3, Γ4 (ps^-1 per unit sum) */
    int sample_all;           /* 1: every four-phonon partner pair (no sampling) */
    unsigned long long sample_threshold, sample_seed;   /* sampling estimate (see above) */
} fc4o_problem;

typedef struct { double re, im; } cplx;

static inline cplx cadd(cplx a, cplx b) { cplx r = {a.re + b.re, a.im + b.im}; return r; }
static inline cplx cmul(cplx a, cplx b) {
    cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
    return r;
}
static inline cplx cscale(double s, cplx a) { cplx r = {s * a.re, s * a.im}; return r; }
static inline cplx cconj(cplx a) { cplx r = {a.re, -a.im}; return r; }

/* ------------------------------------------------------------------ mesh and mode tables */

static void q_coords(const fc4o_problem *p, int iq, int c[3]) {
    c[0] = iq % p->mesh[0];
    c[1] = (iq / p->mesh[0]) % p->mesh[1];
    c[2] = iq / (p->mesh[0] * p->mesh[1]);
}

static int q_index(const fc4o_problem *p, const int c[3]) {
    int i0 = ((c[0] % p->mesh[0]) + p->mesh[0]) % p->mesh[0];
    int i1 = ((c[1] % p->mesh[1]) + p->mesh[1]) % p->mesh[1];
    int i2 = ((c[2] % p->mesh[2]) + p->mesh[2]) % p->mesh[2];
    return i0 + p->mesh[0] * (i1 + p->mesh[1] * i2);
}

/* q-point index of sa*qa + sb*qb + sc*qc on the integer mesh (modulo per axis) */
static int q_combine(const fc4o_problem *p, int sa, int qa, int sb, int qb, int sc, int qc) {
    int a[3], b[3], c[3], r[3];
    q_coords(p, qa, a);
    q_coords(p, qb, b);
    q_coords(p, qc, c);
    for (int k = 0; k < 3; k++) r[k] = sa * a[k] + sb * b[k] + sc * c[k];
    return q_index(p, r);
}

/* Cartesian q of mesh point iq: q = Σ_k (i_k / n_k) b_k */
static void q_cart(const fc4o_problem *p, int iq, double q[3]) {
    int c[3];
    q_coords(p, iq, c);
    for (int x = 0; x < 3; x++) {
        q[x] = 0.0;
        for (int k = 0; k < 3; k++) q[x] += ((double)c[k] / (double)p->mesh[k]) * p->recip[3 * k + x];
    }
}

/* q . R for a cell vector given in lattice coordinates */
static double q_dot_R(const fc4o_problem *p, const double q[3], const int n[3]) {
    double R[3];
    for (int x = 0; x < 3; x++)
        R[x] = n[0] * p->lattice[x] + n[1] * p->lattice[3 + x] + n[2] * p->lattice[6 + x];
    return q[0] * R[0] + q[1] * R[1] + q[2] * R[2];
}

static int excluded(int iq, int j) { return iq == 0 && j < 3; }

/* SplitMix64's output function (the mixing of the state into one 64-bit output) */
unsigned long long fc4o_splitmix64_mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

/* 1 iff the four-phonon partner pair (mode m0, q1, q2) belongs to the sample */
static int pair_sampled(const fc4o_problem *p, int m0, int q1, int q2) {
    if (p->sample_all) return 1;
    unsigned long long key = ((unsigned long long)m0 * p->nq + q1) * p->nq + q2;
    unsigned long long z = p->sample_seed + (key + 1ull) * 0x9e3779b97f4a7c15ull;
    return fc4o_splitmix64_mix(z) < p->sample_threshold;
}

/* eigenvector component (3*atom + cart) of branch j at q, conjugated when conj != 0 */
static cplx evec(const fc4o_problem *p, int iq, int comp, int j, int conj) {
    const double *e = p->evec + 2 * (((size_t)iq * p->nb + comp) * p->nb + j);
    cplx r = {e[0], conj ? -e[1] : e[1]};
    return r;
}

/* ------------------------------------------------------------------ broadening */

/* adaptive σ from the difference of two group velocities: s * sqrt(Σ_k ((Δv . b_k) / n_k)² / 6) */
static double sigma_of(const fc4o_problem *p, int ma, int mb) {
    if (!p->sigma_adaptive) return p->sigma;
    const double *va = p->vel + 3 * (size_t)ma, *vb = p->vel + 3 * (size_t)mb;
    double dv[3] = {va[0] - vb[0], va[1] - vb[1], va[2] - vb[2]};
    double s = 0.0;
    for (int k = 0; k < 3; k++) {
        double t = dv[0] * p->recip[3 * k] + dv[1] * p->recip[3 * k + 1] + dv[2] * p->recip[3 * k + 2];
        t = t / (double)p->mesh[k];
        s = s + t * t;
    }
    return p->sigma * sqrt(s / 6.0);
}

/* σ usable as a Gaussian width: any fixed σ > 0; an adaptive σ above the noise floor */
#define ADAPTIVE_SIGMA_MIN 1e-9
static int width_ok(const fc4o_problem *p, double sg) {
    return p->sigma_adaptive ? sg > ADAPTIVE_SIGMA_MIN : sg > 0.0;
}

static double gaussian(double delta, double sigma) {
    return exp(-(delta * delta) / (sigma * sigma)) / (sigma * sqrt(M_PI));
}

/* ------------------------------------------------------------------ energy mismatch */

static double delta_of(int ch, double w, double w1, double w2, double w3) {
    switch (ch) {
    case 0: return (w + w1) - w2;
    case 1: return w - (w1 + w2);
    case 2: return (w - w3) + (w1 + w2);
    case 3: return (w + w1) - (w2 + w3);
    default: {
        double s[3] = {w1, w2, w3}, t;
        if (s[0] > s[1]) { t = s[0]; s[0] = s[1]; s[1] = t; }
        if (s[1] > s[2]) { t = s[1]; s[1] = s[2]; s[2] = t; }
        if (s[0] > s[1]) { t = s[0]; s[0] = s[1]; s[1] = t; }
        return w - ((s[0] + s[1]) + s[2]);
    }
    }
}

static double occupation_factor(int ch, double n1, double n2, double n3) {
    switch (ch) {
    case 0: return n1 - n2;
    case 1: return 1.0 + n1 + n2;
    case 2: return n1 * n2 * (1.0 + n3) - (1.0 + n1) * (1.0 + n2) * n3;
    case 3: return n1 * (1.0 + n2) * (1.0 + n3) - (1.0 + n1) * n2 * n3;
    default: return (1.0 + n1) * (1.0 + n2) * (1.0 + n3) - n1 * n2 * n3;
    }
}

static double symmetry_factor(int ch) {
    switch (ch) {
    case 0: return 1.0;
    case 1: return 0.5;
    case 2: return 0.5;
    case 3: return 0.5;
    default: return 1.0 / 6.0;
    }
}

/* ------------------------------------------------------------------ matrix elements */

/* V3^s(λ, λ', λ'') for modes m0 = (q, j), m1 = (q', j'), m2 = (q'', j'') (any q's). */
cplx fc4o_v3_c(const fc4o_problem *p, int s, int m0, int m1, int m2) {
    int nb = p->nb;
    int q0 = m0 / nb, j0 = m0 % nb, q1 = m1 / nb, j1 = m1 % nb, q2 = m2 / nb, j2 = m2 % nb;
    double qc1[3], qc2[3];
    q_cart(p, q1, qc1);
    q_cart(p, q2, qc2);
    cplx V = {0.0, 0.0};
    for (int c = 0; c < p->nc3; c++) {
        const int *at = p->atoms3 + 3 * c;
        const int *R1 = p->cells3 + 6 * c, *R2 = p->cells3 + 6 * c + 3;
        const double *phi = p->phi3 + 27 * c;
        double arg = s * q_dot_R(p, qc1, R1) - q_dot_R(p, qc2, R2);
        cplx ph = {cos(arg), sin(arg)};
        double inv_m = 1.0 / sqrt(p->mass[at[0]] * p->mass[at[1]] * p->mass[at[2]]);
        cplx acc = {0.0, 0.0};
        for (int a = 0; a < 3; a++) {
            cplx sa = {0.0, 0.0};
            for (int b = 0; b < 3; b++) {
                cplx sb = {0.0, 0.0};
                for (int g = 0; g < 3; g++)
                    sb = cadd(sb, cscale(phi[(a * 3 + b) * 3 + g], evec(p, q2, 3 * at[2] + g, j2, 1)));
                sa = cadd(sa, cmul(evec(p, q1, 3 * at[1] + b, j1, s < 0), sb));
            }
            acc = cadd(acc, cmul(evec(p, q0, 3 * at[0] + a, j0, 0), sa));
        }
        V = cadd(V, cscale(inv_m, cmul(ph, acc)));
    }
    return V;
}

/* V4^(s1,s2)(λ, λ', λ'', λ''') for modes m0..m3 (any q's). */
cplx fc4o_v4_c(const fc4o_problem *p, int s1, int s2, int m0, int m1, int m2, int m3) {
    int nb = p->nb;
    int q0 = m0 / nb, j0 = m0 % nb, q1 = m1 / nb, j1 = m1 % nb;
    int q2 = m2 / nb, j2 = m2 % nb, q3 = m3 / nb, j3 = m3 % nb;
    double qc1[3], qc2[3], qc3[3];
    q_cart(p, q1, qc1);
    q_cart(p, q2, qc2);
    q_cart(p, q3, qc3);
    cplx V = {0.0, 0.0};
    for (int c = 0; c < p->nc4; c++) {
        const int *at = p->atoms4 + 4 * c;
        const int *R1 = p->cells4 + 9 * c, *R2 = R1 + 3, *R3 = R1 + 6;
        const double *phi = p->phi4 + 81 * c;
        double arg = s1 * q_dot_R(p, qc1, R1) + s2 * q_dot_R(p, qc2, R2) - q_dot_R(p, qc3, R3);
        cplx ph = {cos(arg), sin(arg)};
        double inv_m = 1.0 / sqrt(p->mass[at[0]] * p->mass[at[1]] * p->mass[at[2]] * p->mass[at[3]]);
        cplx acc = {0.0, 0.0};
        for (int a = 0; a < 3; a++) {
            cplx sa = {0.0, 0.0};
            for (int b = 0; b < 3; b++) {
                cplx sb = {0.0, 0.0};
                for (int g = 0; g < 3; g++) {
                    cplx sg = {0.0, 0.0};
                    for (int d = 0; d < 3; d++)
                        sg = cadd(sg, cscale(phi[((a * 3 + b) * 3 + g) * 3 + d],
                                             evec(p, q3, 3 * at[3] + d, j3, 1)));
                    sb = cadd(sb, cmul(evec(p, q2, 3 * at[2] + g, j2, s2 < 0), sg));
                }
                sa = cadd(sa, cmul(evec(p, q1, 3 * at[1] + b, j1, s1 < 0), sb));
            }
            acc = cadd(acc, cmul(evec(p, q0, 3 * at[0] + a, j0, 0), sa));
        }
        V = cadd(V, cscale(inv_m, cmul(ph, acc)));
    }
    return V;
}

void fc4o_v3(const fc4o_problem *p, int s, int m0, int m1, int m2, double *out) {
    cplx v = fc4o_v3_c(p, s, m0, m1, m2);
    out[0] = v.re;
    out[1] = v.im;
}

void fc4o_v4(const fc4o_problem *p, int s1, int s2, int m0, int m1, int m2, int m3, double *out) {
    cplx v = fc4o_v4_c(p, s1, s2, m0, m1, m2, m3);
    out[0] = v.re;
    out[1] = v.im;
}

/* ------------------------------------------------------------------ process visitor */

/* One kept process: partner modes (m1, m2, m3 = -1 for 3ph), its Δ, σ and canonical word. */
typedef void (*visit_fn)(void *ctx, const fc4o_problem *p, int ch, int m0, int m1, int m2, int m3,
                         double delta, double sigma, unsigned long long word);

static const int ch_s1[5] = {+1, -1, +1, +1, -1};
static const int ch_s2[5] = {0, 0, +1, -1, -1};

/* Enumerate the kept processes of mode m0 in channel ch in canonical order:
 * 3ph: (q', j', j'') ascending;  4ph: (q', j', q'', j'', j''') ascending. */
static void enumerate(const fc4o_problem *p, int ch, int m0, int qp_limit, visit_fn f, void *ctx) {
    int nb = p->nb, N = p->nq;
    int q0 = m0 / nb, j0 = m0 % nb;
    if (excluded(q0, j0)) return;
    double w0 = p->omega[m0];
    int nq1 = (qp_limit > 0 && qp_limit < N) ? qp_limit : N;
    if (ch < 2) {
        int s = ch_s1[ch];
        for (int q1 = 0; q1 < nq1; q1++) {
            int q2 = q_combine(p, 1, q0, s, q1, 0, 0);
            for (int j1 = 0; j1 < nb; j1++) {
                if (excluded(q1, j1)) continue;
                int m1 = q1 * nb + j1;
                for (int j2 = 0; j2 < nb; j2++) {
                    if (excluded(q2, j2)) continue;
                    int m2 = q2 * nb + j2;
                    double sg = sigma_of(p, m1, m2);
                    double d = delta_of(ch, w0, p->omega[m1], p->omega[m2], 0.0);
                    if (width_ok(p, sg) && fabs(d) <= 2.0 * sg) {
                        unsigned long long word = ((unsigned long long)m1) * nb + j2;
                        f(ctx, p, ch, m0, m1, m2, -1, d, sg, word);
                    }
                }
            }
        }
    } else {
        int s1 = ch_s1[ch], s2 = ch_s2[ch];
        for (int q1 = 0; q1 < nq1; q1++) {
            for (int j1 = 0; j1 < nb; j1++) {
                if (excluded(q1, j1)) continue;
                int m1 = q1 * nb + j1;
                for (int q2 = 0; q2 < N; q2++) {
                    if (!pair_sampled(p, m0, q1, q2)) continue;
                    int q3 = q_combine(p, 1, q0, s1, q1, s2, q2);
                    for (int j2 = 0; j2 < nb; j2++) {
                        if (excluded(q2, j2)) continue;
                        int m2 = q2 * nb + j2;
                        for (int j3 = 0; j3 < nb; j3++) {
                            if (excluded(q3, j3)) continue;
                            int m3 = q3 * nb + j3;
                            double sg = sigma_of(p, m2, m3);
                            double d = delta_of(ch, w0, p->omega[m1], p->omega[m2], p->omega[m3]);
                            if (width_ok(p, sg) && fabs(d) <= 2.0 * sg) {
                                unsigned long long word =
                                    (((unsigned long long)m1 * N + q2) * nb + j2) * nb + j3;
                                f(ctx, p, ch, m0, m1, m2, m3, d, sg, word);
                            }
                        }
                    }
                }
            }
        }
    }
}

static double weight_of(const fc4o_problem *p, int ch, int m0, int m1, int m2, int m3,
                        double delta, double sigma) {
    double n1 = p->occ[m1], n2 = p->occ[m2], n3 = (m3 >= 0) ? p->occ[m3] : 0.0;
    double wprod = p->omega[m0] * p->omega[m1] * p->omega[m2];
    if (m3 >= 0) wprod = wprod * p->omega[m3];
    return symmetry_factor(ch) * occupation_factor(ch, n1, n2, n3) * gaussian(delta, sigma) / wprod;
}

static cplx v_of(const fc4o_problem *p, int ch, int m0, int m1, int m2, int m3) {
    if (ch < 2) return fc4o_v3_c(p, ch_s1[ch], m0, m1, m2);
    return fc4o_v4_c(p, ch_s1[ch], ch_s2[ch], m0, m1, m2, m3);
}

/* ------------------------------------------------------------------ rates */

typedef struct { double gamma, wp; long long count; } rate_acc;

static void rate_visit(void *ctx, const fc4o_problem *p, int ch, int m0, int m1, int m2, int m3,
                       double delta, double sigma, unsigned long long word) {
    (void)word;
    rate_acc *a = (rate_acc *)ctx;
    double w = weight_of(p, ch, m0, m1, m2, m3, delta, sigma);
    cplx V = v_of(p, ch, m0, m1, m2, m3);
    a->wp += w;
    a->gamma += w * (V.re * V.re + V.im * V.im);
    a->count += 1;
}

/* Γ, WP and kept-process counts of the listed modes, channels in channel_mask (bit ch).
 * Outputs are [5][n_modes].  qp_limit > 0 restricts q' to [0, qp_limit) (a bounded sample). */
int fc4o_rates(const fc4o_problem *p, int n_modes, const int *modes, int channel_mask, int qp_limit,
               double *gamma, double *wp, long long *counts) {
    double N = (double)p->nq;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < n_modes; i++) {
        for (int ch = 0; ch < 5; ch++) {
            rate_acc a = {0.0, 0.0, 0};
            if (channel_mask & (1 << ch)) enumerate(p, ch, modes[i], qp_limit, rate_visit, &a);
            double norm = (ch < 2) ? N : N * N;
            double cst = (ch < 2) ? p->c3 : p->c4;
            /* sampled four-phonon sums scaled by the inverse inclusion probability 2^64 / threshold */
            double scale = (ch < 2 || p->sample_all) ? 1.0 : ldexp(1.0, 64) / (double)p->sample_threshold;
            gamma[(size_t)ch * n_modes + i] = a.gamma * scale * cst / norm;
            wp[(size_t)ch * n_modes + i] = a.wp * scale / norm;
            counts[(size_t)ch * n_modes + i] = a.count;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ process lists */

typedef struct { unsigned long long *words; long long cap, n; } list_acc;

static void list_visit(void *ctx, const fc4o_problem *p, int ch, int m0, int m1, int m2, int m3,
                       double delta, double sigma, unsigned long long word) {
    (void)p; (void)ch; (void)m0; (void)m1; (void)m2; (void)m3; (void)delta; (void)sigma;
    list_acc *a = (list_acc *)ctx;
    if (a->n < a->cap) a->words[a->n] = word;
    a->n += 1;
}

/* Canonical process words of one mode and channel; returns the count (writes at most cap). */
long long fc4o_processes(const fc4o_problem *p, int ch, int mode, unsigned long long *words,
                         long long cap) {
    list_acc a = {words, cap, 0};
    enumerate(p, ch, mode, 0, list_visit, &a);
    return a.n;
}

/* ------------------------------------------------------------------ gradient */

typedef struct { double coef; double *g3, *g4; } grad_acc;

/* d/dΦ_c[...] of coef * w |V|² = coef * w * 2 Re(conj(V) dV/dΦ_c[...]) for every cluster entry */
static void grad_visit(void *ctx, const fc4o_problem *p, int ch, int m0, int m1, int m2, int m3,
                       double delta, double sigma, unsigned long long word) {
    (void)word;
    grad_acc *a = (grad_acc *)ctx;
    int nb = p->nb;
    double w = weight_of(p, ch, m0, m1, m2, m3, delta, sigma);
    cplx V = v_of(p, ch, m0, m1, m2, m3);
    double f = 2.0 * a->coef * w;
    int q0 = m0 / nb, j0 = m0 % nb, q1 = m1 / nb, j1 = m1 % nb, q2 = m2 / nb, j2 = m2 % nb;
    int s1 = ch_s1[ch], s2 = ch_s2[ch];
    if (ch < 2) {
        double qc1[3], qc2[3];
        q_cart(p, q1, qc1);
        q_cart(p, q2, qc2);
        for (int c = 0; c < p->nc3; c++) {
            const int *at = p->atoms3 + 3 * c;
            const int *R1 = p->cells3 + 6 * c, *R2 = R1 + 3;
            double arg = s1 * q_dot_R(p, qc1, R1) - q_dot_R(p, qc2, R2);
            cplx ph = {cos(arg), sin(arg)};
            double inv_m = 1.0 / sqrt(p->mass[at[0]] * p->mass[at[1]] * p->mass[at[2]]);
            cplx cv = cconj(V);
            for (int a_ = 0; a_ < 3; a_++)
                for (int b = 0; b < 3; b++)
                    for (int g = 0; g < 3; g++) {
                        cplx t = cmul(evec(p, q0, 3 * at[0] + a_, j0, 0), evec(p, q1, 3 * at[1] + b, j1, s1 < 0));
                        t = cmul(t, evec(p, q2, 3 * at[2] + g, j2, 1));
                        t = cmul(cv, cmul(ph, t));
                        a->g3[27 * (size_t)c + (a_ * 3 + b) * 3 + g] += f * inv_m * t.re;
                    }
        }
    } else {
        int q3 = m3 / nb, j3 = m3 % nb;
        double qc1[3], qc2[3], qc3[3];
        q_cart(p, q1, qc1);
        q_cart(p, q2, qc2);
        q_cart(p, q3, qc3);
        for (int c = 0; c < p->nc4; c++) {
            const int *at = p->atoms4 + 4 * c;
            const int *R1 = p->cells4 + 9 * c, *R2 = R1 + 3, *R3 = R1 + 6;
            double arg = s1 * q_dot_R(p, qc1, R1) + s2 * q_dot_R(p, qc2, R2) - q_dot_R(p, qc3, R3);
            cplx ph = {cos(arg), sin(arg)};
            double inv_m = 1.0 / sqrt(p->mass[at[0]] * p->mass[at[1]] * p->mass[at[2]] * p->mass[at[3]]);
            cplx cv = cconj(V);
            for (int a_ = 0; a_ < 3; a_++)
                for (int b = 0; b < 3; b++)
                    for (int g = 0; g < 3; g++)
                        for (int d = 0; d < 3; d++) {
                            cplx t = cmul(evec(p, q0, 3 * at[0] + a_, j0, 0), evec(p, q1, 3 * at[1] + b, j1, s1 < 0));
                            t = cmul(t, evec(p, q2, 3 * at[2] + g, j2, s2 < 0));
                            t = cmul(t, evec(p, q3, 3 * at[3] + d, j3, 1));
                            t = cmul(cv, cmul(ph, t));
                            a->g4[81 * (size_t)c + ((a_ * 3 + b) * 3 + g) * 3 + d] += f * inv_m * t.re;
                        }
        }
    }
}

/* Gradient of L = Σ_{ch,i} dL_dgamma[ch][i] * Γ_ch(modes[i]) with respect to every stored Φ3
 * and Φ4 entry (entries treated as independent), at fixed modes and σ. */
int fc4o_grad(const fc4o_problem *p, int n_modes, const int *modes, int channel_mask,
              const double *dL_dgamma, double *dphi3, double *dphi4) {
    size_t n3 = 27 * (size_t)p->nc3, n4 = 81 * (size_t)p->nc4;
    memset(dphi3, 0, n3 * sizeof(double));
    memset(dphi4, 0, n4 * sizeof(double));
    double N = (double)p->nq;
    for (int i = 0; i < n_modes; i++) {
        for (int ch = 0; ch < 5; ch++) {
            if (!(channel_mask & (1 << ch))) continue;
            double g = dL_dgamma[(size_t)ch * n_modes + i];
            if (g == 0.0) continue;
            double norm = (ch < 2) ? N : N * N;
            double cst = (ch < 2) ? p->c3 : p->c4;
            grad_acc a = {g * cst / norm, dphi3, dphi4};
            enumerate(p, ch, modes[i], 0, grad_visit, &a);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ scalar helpers (pins) */

double fc4o_delta(int ch, double w, double w1, double w2, double w3) {
    return delta_of(ch, w, w1, w2, w3);
}

double fc4o_occupation_factor(int ch, double n1, double n2, double n3) {
    return occupation_factor(ch, n1, n2, n3);
}

double fc4o_sigma(const fc4o_problem *p, int ma, int mb) { return sigma_of(p, ma, mb); }

/* ------------------------------------------------------------------ iterative BTE
 * The paper names solving the linearised Boltzmann equation beyond the RTA as future work
 * (Results, end); it gives no scheme.  Reading: the ShengBTE / FourPhonon iterative scheme, whose
 * collision operator reuses the rates' per-process terms.  With F_λ the deviation vector
 * (n_λ = n0_λ - F_λ . ∇T dn0_λ/dT),
 *   F_λ = (v_λ + Δ_λ) / Γ_λ,    Δ_λ = Σ_processes γ_p Σ_k s_k (ω_k / ω_λ) F_k,
 * where γ_p = (C/N^k) w_p |V_p|² is the process's term of Γ_λ (symmetry factor included, so that
 * Γ_λ = Σ_p γ_p), k runs over the partners of the process, s_k = +1 for a partner on the other
 * side of the process from λ and -1 for one on the same side:
 *   3ph+  λ + λ' -> λ''           s = (-1, +1)
 *   3ph-  λ -> λ' + λ''           s = (+1, +1)
 *   4ph++ λ + λ' + λ'' -> λ'''    s = (-1, -1, +1)
 *   4ph+- λ + λ' -> λ'' + λ'''    s = (-1, +1, +1)
 *   4ph-- λ -> λ' + λ'' + λ'''    s = (+1, +1, +1)
 * On shell Σ_k s_k ω_k = ω_λ (energy conservation), so a uniform F = u gives Δ_λ = Γ_λ u; with
 * Gaussian broadening the process's mismatch enters as Σ_k s_k ω_k = ω_λ - Δ_p. */
static const int bte_sign[5][3] = {{-1, +1, 0}, {+1, +1, 0}, {-1, -1, +1}, {-1, +1, +1}, {+1, +1, +1}};

typedef struct { const double *F; double d[3]; } bte_acc;

static void bte_visit(void *ctx, const fc4o_problem *p, int ch, int m0, int m1, int m2, int m3,
                      double delta, double sigma, unsigned long long word) {
    (void)word;
    bte_acc *a = (bte_acc *)ctx;
    double w = weight_of(p, ch, m0, m1, m2, m3, delta, sigma);
    cplx V = v_of(p, ch, m0, m1, m2, m3);
    double g = w * (V.re * V.re + V.im * V.im);          /* γ_p without C / N^k (applied per mode) */
    int mk[3] = {m1, m2, m3};
    int np = (ch < 2) ? 2 : 3;
    for (int k = 0; k < np; k++) {
        double xi = p->omega[mk[k]] / p->omega[m0];
        double c = g * ((double)bte_sign[ch][k] * xi);
        for (int x = 0; x < 3; x++) a->d[x] += c * a->F[3 * (size_t)mk[k] + x];
    }
}

/* Δ_λ [n_modes][3] of the listed modes for the deviation vectors F [nq * nb][3] over the channels
 * in channel_mask (units of F times ps^-1; the sampling estimate's scale applies as for Γ). */
int fc4o_bte_offdiag(const fc4o_problem *p, int n_modes, const int *modes, int channel_mask,
                     const double *F, double *delta) {
    double N = (double)p->nq;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < n_modes; i++) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int ch = 0; ch < 5; ch++) {
            if (!(channel_mask & (1 << ch))) continue;
            bte_acc a = {F, {0.0, 0.0, 0.0}};
            enumerate(p, ch, modes[i], 0, bte_visit, &a);
            double norm = (ch < 2) ? N : N * N;
            double cst = (ch < 2) ? p->c3 : p->c4;
            double scale = (ch < 2 || p->sample_all) ? 1.0 : ldexp(1.0, 64) / (double)p->sample_threshold;
            for (int x = 0; x < 3; x++) acc[x] += a.d[x] * scale * cst / norm;
        }
        for (int x = 0; x < 3; x++) delta[3 * (size_t)i + x] = acc[x];
    }
    return 0;
}
