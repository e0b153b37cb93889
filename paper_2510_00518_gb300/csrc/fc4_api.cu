// fc4_api.cu - the C interface of libfc4 (declared in include/fc4.h): argument checks, host-side
// layout of the clusters (keys, phase indices, mass factors), device tables, and the
// stream-ordered launch sequence of each call.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "fc4.h"
#include "fc4_kernels.h"

namespace {

// CODATA 2018 (SI)
constexpr double kHbar = 1.054571817e-34;   // J s
constexpr double kEv = 1.602176634e-19;     // J
constexpr double kAmu = 1.66053906660e-27;  // kg
constexpr double kKb = 1.380649e-23;        // J/K
constexpr double kPi = 3.14159265358979323846;

// eigenvalue of D in eV/(Å² amu) -> ω² in (rad/ps)²
constexpr double kEigToW2 = kEv / (1e-20 * kAmu) * 1e-24;

// Γ3 = C3/N Σ w|V3|², Γ4 = C4/N² Σ w|V4|² in ps^-1 for V in eV/Å^k/amu^(k/2), ω in rad/ps, δ in ps
double unit_c3() {
    const double fv = kEv / 1e-30 / std::pow(kAmu, 1.5);
    return kHbar * kPi / 4.0 * fv * fv * 1e-48 * 1e-12;
}
double unit_c4() {
    const double fv = kEv / 1e-40 / (kAmu * kAmu);
    return kHbar * kHbar * kPi / 8.0 * fv * fv * 1e-60 * 1e-12;
}

thread_local std::string g_init_error;

}  // namespace

void fc4::set_host_error(const char *msg) { g_init_error = msg; }

struct fc4_ctx {
    fc4::Tables t{};
    int nc2 = 0, nc3 = 0, nc4 = 0;
    int precision = FC4_FP64, block_threads = 128;
    bool use_tc = false;                    // tensor-core contraction of the 4ph +- channel (mixed)
    long long timeout_cycles = 0;           // bound of device-side waits (0: kernel default)
    int *dev_err = nullptr;                 // set by a kernel whose bounded wait expired
    bool timing = false;
    bool allow_unstable = false;
    cudaEvent_t ev_a[8] = {}, ev_b[8] = {};
    bool ev_used[8] = {};
    long long n_launches = 0;
    double volume = 0.0;
    std::vector<void *> owned;
    std::map<void *, size_t> alloc_bytes;  // size of each allocation (entries of freed ones are stale)
    std::vector<int> perm4;                 // device cluster slot -> input cluster index
    std::vector<int> swap12, swap23;        // input cluster -> the cluster with legs 1,2 (2,3) swapped
    bool sym12 = false, sym23 = false;      // Φ4 invariant under those swaps (triangular domains)
    std::vector<double> om_host;            // current ω (for the prefilter bound)
    double vmax = 0.0;                      // max |v| over modes (adaptive prefilter bound)
    // writable views of the tables
    double *om = nullptr, *vel = nullptr, *eig = nullptr, *invw = nullptr, *occ = nullptr;
    double *phi3 = nullptr, *phi4 = nullptr;
    float *om32 = nullptr, *om32lo = nullptr, *invw32 = nullptr, *occ32 = nullptr, *phi4_32 = nullptr;
    double2 *ev = nullptr;
    float2 *ev32 = nullptr;
    float4 *vp32 = nullptr, *vp32lo = nullptr;
    float *omT32 = nullptr;                 // branch-major window copies [nb][N]
    float4 *vpT32 = nullptr, *vpTlo = nullptr;
    unsigned *vmask = nullptr;
    int *err = nullptr;
    double occ_T = -1.0;
    // scratch
    double *part_g = nullptr, *part_wp = nullptr;
    long long *part_n = nullptr, *part_items = nullptr, *part_ent = nullptr;
    long long *part_ev = nullptr, *part_cev = nullptr;
    size_t part_cap = 0;
    unsigned long long *stats = nullptr;    // [25] kept, items, entries, evaluated, visited per channel
    long long cand[5] = {0, 0, 0, 0, 0};    // candidates per channel of the last call
    int *modes = nullptr;
    size_t modes_cap = 0;
    void *wbuf = nullptr;                  // W scratch of the tiled 4ph path
    size_t wbuf_bytes = 0;
    int w_s1 = 0;                          // sign s1 of the W held for w_modes (0: none)
    int mode_chunk = 0;                    // modes per chunk of a rates call (0: as many as W allows)
    size_t w_limit = 0;                    // cap of the W buffer in bytes (0: max(4 GiB, HBM / 4))
    int last_chunk = 0;                    // modes per chunk of the last rates call
    // sampling estimate of the 4ph sums (fc4_set_sampling); every pair by default
    int sample_all = 1;
    unsigned long long sample_threshold = ~0ull, sample_seed = 0;
    int no_compact = 0;                    // ablation of the entry compaction (fc4_set_ablation)
    // iterative BTE scratch
    double *part_d = nullptr, *bte_F = nullptr, *bte_delta = nullptr, *bte_kappa = nullptr;
    float *bte_F32 = nullptr;
    size_t part_d_cap = 0;
    std::vector<int> w_modes;
    int *perm4_dev = nullptr;              // device cluster slot -> input index (gradients)
    double *adj_part = nullptr;            // per-mode gradient slices of fc4_rates_backward
    size_t adj_cap = 0;
    double *adj_tmp = nullptr;             // Φ4 gradient in device cluster order
    std::vector<int> modes_on_device;      // content of `modes` (skip re-uploading an unchanged list)
    // last rates call
    bool have_last = false;
    double last_T = 300.0, last_sigma = 0.1;   // σ in THz, or the scale s if adaptive
    bool last_adaptive = false;
    int last_mask = 0;
    std::vector<int> last_modes;
    std::string last_error;
};

namespace {

fc4_status fail(fc4_ctx *ctx, fc4_status s, const std::string &msg) {
    if (ctx) ctx->last_error = msg;
    else g_init_error = msg;
    return s;
}

fc4_status cuda_fail(fc4_ctx *ctx, cudaError_t e, const char *where) {
    return fail(ctx, e == cudaErrorMemoryAllocation ? FC4_ERR_OOM : FC4_ERR_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

#define FC4_CUDA(ctx, call)                                             \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);      \
    } while (0)

template <typename T>
cudaError_t dalloc(fc4_ctx *c, T **p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
    if (e == cudaSuccess) {
        c->owned.push_back(*p);
        c->alloc_bytes[(void *)*p] = n * sizeof(T);
    }
    return e;
}

template <typename T>
cudaError_t upload(fc4_ctx *c, T **p, const std::vector<T> &h) {
    cudaError_t e = dalloc(c, p, h.size());
    if (e != cudaSuccess) return e;
    if (!h.empty()) e = cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

int gcd_i(int a, int b) { return b ? gcd_i(b, a % b) : a; }
int lcm_i(int a, int b) { return a / gcd_i(a, b) * b; }
int mod_i(long long x, int n) { long long r = x % n; return (int)(r < 0 ? r + n : r); }

int4 phase_vec(const int R[3], const int mesh[3], int L) {
    return make_int4(mod_i((long long)R[0] * (L / mesh[0]), L), mod_i((long long)R[1] * (L / mesh[1]), L),
                     mod_i((long long)R[2] * (L / mesh[2]), L), 0);
}

fc4_status check_ifc(const fc4_ifc *f, int order, int n_atoms, bool required, const char *name) {
    if (!f) {
        if (required) return fail(nullptr, FC4_ERR_INVALID, std::string(name) + " is NULL");
        return FC4_OK;
    }
    if (f->order != order) return fail(nullptr, FC4_ERR_INVALID, std::string(name) + ": wrong order");
    if (f->n_clusters < 0 || (f->n_clusters > 0 && (!f->atoms || !f->cells || !f->phi)))
        return fail(nullptr, FC4_ERR_INVALID, std::string(name) + ": bad cluster arrays");
    if (required && f->n_clusters == 0)
        return fail(nullptr, FC4_ERR_INVALID, std::string(name) + ": no clusters");
    for (long long i = 0; i < (long long)f->n_clusters * order; ++i)
        if (f->atoms[i] < 0 || f->atoms[i] >= n_atoms)
            return fail(nullptr, FC4_ERR_INVALID, std::string(name) + ": atom index out of range");
    for (long long i = 0; i < (long long)f->n_clusters * (order - 1) * 3; ++i)
        if (std::abs(f->cells[i]) > 1000000)
            return fail(nullptr, FC4_ERR_INVALID, std::string(name) + ": cell vector out of range");
    return FC4_OK;
}

// Rebuild the derived mode tables after ω / e changed (also zeroes the excluded ω).
fc4_status refresh_modes(fc4_ctx *c) {
    FC4_CUDA(c, fc4::launch_mode_tables(c->t, c->om, c->om32, c->om32lo, c->ev32, c->ev, c->vmask,
                                        c->invw, c->invw32, c->vp32, c->vp32lo, c->omT32, c->vpT32, c->vpTlo, 0));
    const size_t nm = (size_t)c->t.N * c->t.nb;
    c->om_host.assign(nm, 0.0);
    FC4_CUDA(c, cudaMemcpy(c->om_host.data(), c->om, nm * sizeof(double), cudaMemcpyDeviceToHost));
    std::vector<double> v(3 * nm);
    FC4_CUDA(c, cudaMemcpy(v.data(), c->vel, v.size() * sizeof(double), cudaMemcpyDeviceToHost));
    c->vmax = 0.0;
    for (size_t i = 0; i < nm; ++i)
        c->vmax = std::max(c->vmax, std::sqrt(v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] +
                                              v[3 * i + 2] * v[3 * i + 2]));
    c->occ_T = -1.0;
    return FC4_OK;
}

// Launch bracket: events on the launching stream around kernel slot k (when timing is on).
struct Timed {
    fc4_ctx *c;
    int k;
    cudaStream_t s;
    Timed(fc4_ctx *c_, int k_, cudaStream_t s_) : c(c_), k(k_), s(s_) {
        if (c->timing) cudaEventRecord(c->ev_a[k], s);
    }
    ~Timed() {
        if (c->timing) {
            cudaEventRecord(c->ev_b[k], s);
            c->ev_used[k] = true;
        }
        if (k >= 5) c->n_launches += 1;      // rate launchers count their own kernels
    }
};

fc4_status ensure_occupations(fc4_ctx *c, double T, cudaStream_t s) {
    if (c->occ_T == T) return FC4_OK;
    {
        Timed tm(c, 7, s);
        FC4_CUDA(c, fc4::launch_occupations(c->t, kHbar * 1e12 / (kKb * T), c->occ, c->occ32, s));
    }
    c->occ_T = T;
    return FC4_OK;
}

// Leg-swap invariance of Φ4 (input cluster order): every cluster has its partner with legs 1, 2
// (resp. 2, 3) exchanged, with the correspondingly transposed tensor, to 1e-12 of max |Φ4|.  The
// triangular domains of the 4ph sums are used only then (a single perturbed entry, as in a
// finite-difference check of the gradient, falls back to the rectangular sum).
void check_sym4(fc4_ctx *c, const double *phi) {
    double mx = 0.0;
    for (size_t k = 0; k < 81 * (size_t)c->nc4; ++k) mx = std::max(mx, std::fabs(phi[k]));
    const double tol = 1e-12 * mx;
    auto ok = [&](const std::vector<int> &sw, bool twelve) {
        for (int i = 0; i < c->nc4; ++i) {
            const int j = sw[i];
            if (j < 0) return false;
            const double *p = phi + 81 * (size_t)i, *q = phi + 81 * (size_t)j;
            for (int al = 0; al < 3; ++al)
                for (int x = 0; x < 3; ++x)
                    for (int y = 0; y < 3; ++y)
                        for (int z = 0; z < 3; ++z) {
                            const double v = p[((al * 3 + x) * 3 + y) * 3 + z];
                            const double w = twelve ? q[((al * 3 + y) * 3 + x) * 3 + z] : q[((al * 3 + x) * 3 + z) * 3 + y];
                            if (std::fabs(v - w) > tol) return false;
                        }
        }
        return true;
    };
    c->sym12 = ok(c->swap12, true);
    c->sym23 = ok(c->swap23, false);
}

// Prefilter thresholds: |Δ32 - Δ64| <= 13 u ω_max (u = 2^-24; three roundings of the inputs'
// partial sums plus four input roundings); margin 32 u ω_max, doubled to cover the rounding of
// the thresholds themselves.
double prefilter_eps(const fc4_ctx *c) {
    double wmax = 0.0;
    for (double w : c->om_host) wmax = std::max(wmax, std::fabs(w));
    return 32.0 * std::ldexp(1.0, -24) * wmax;
}

void prefilter(const fc4_ctx *c, double two_sigma, float *lo, float *hi) {
    const double eps = prefilter_eps(c);
    *lo = std::nextafter((float)(two_sigma - 2.0 * eps), 0.0f);
    *hi = std::nextafter((float)(two_sigma + 2.0 * eps), 1e30f);
}

// Operand format of the tensor-core +- contraction for a context (the launcher's a.use_tc):
// 0 none (CUDA cores), 1 FP16 x3, 2 BF16 x3, 3 BF16, 4 TF32 x3.
int tc_op(const fc4_ctx *c) {
    switch (c->precision) {
        case FC4_MIXED: return c->use_tc ? 1 : 0;
        case FC4_FP16X3: return 1;
        case FC4_BF16X3: return 2;
        case FC4_BF16: return 3;
        case FC4_TF32X3: return 4;
        default: return 0;
    }
}

// Window and Gaussian parameters of a rates call: fixed σ = 2π sigma_value rad/ps, or adaptive
// σ = s |ΔP| / sqrt(6) with s = sigma_value.  For the adaptive prefilter, Q = max|v| max_k |b_k| / n_k
// bounds every |P_k| and the FP64 rounding of the exact σ (<= 2^-50 Q per component); the margins
// are those stated with the kernels' window test.
void set_window(const fc4_ctx *c, fc4::RateArgs &a, bool adaptive, double sigma_value) {
    a.adaptive = adaptive ? 1 : 0;
    a.use_tc = fc4::tc_supported(c->t) ? tc_op(c) : 0;
    a.spin_limit = c->timeout_cycles;
    a.err = c->dev_err;
    a.n_kernels = const_cast<long long *>(&c->n_launches);
    a.tri = (c->sym23 ? 1 : 0) | (c->sym12 && !adaptive ? 2 : 0);
    a.no_compact = c->no_compact;
    a.sample_all = c->sample_all;
    a.sample_threshold = c->sample_threshold;
    a.sample_seed = c->sample_seed;
    a.sample_scale = c->sample_all ? 1.0 : std::ldexp(1.0, 64) / (double)c->sample_threshold;
    if (!adaptive) {
        const double sigma = 2.0 * kPi * sigma_value;
        a.two_sigma = 2.0 * sigma;
        a.inv_sigma2 = 1.0 / (sigma * sigma);
        a.gnorm = 1.0 / (sigma * std::sqrt(kPi));
        a.inv_sigma2_32 = (float)a.inv_sigma2;
        a.gnorm32 = (float)a.gnorm;
        prefilter(c, a.two_sigma, &a.lo32, &a.hi32);
        return;
    }
    const double u = std::ldexp(1.0, -24);
    double bmax = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double *b = c->t.recip + 3 * k;
        bmax = std::max(bmax, std::sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]) / c->t.mesh[k]);
    }
    const double Q = c->vmax * bmax;
    const double c2 = 2.0 * sigma_value / std::sqrt(6.0);
    a.ad_scale = sigma_value;
    a.ad_c32 = (float)c2;
    a.ad_s32 = (float)(sigma_value / std::sqrt(6.0));
    a.ad_rlo = (float)(1.0 - 32.0 * u);
    a.ad_rhi = (float)(1.0 + 32.0 * u);
    a.ad_e0 = std::nextafter((float)(2.0 * prefilter_eps(c) + std::ldexp(c2 * Q, -40)), 1e30f);
    a.ad_gmin = std::nextafter((float)((2.0 * fc4::kAdaptiveSigmaMin + std::ldexp(c2 * Q, -40)) * (1.0 + 64.0 * u)), 1e30f);
    a.two_sigma = 0.0;                  // unused with adaptive σ; thresholds that keep nothing
    a.lo32 = -1.0f;
    a.hi32 = -1.0f;
}

}  // namespace

extern "C" {

fc4_status fc4_init(const fc4_crystal *crystal, const fc4_ifc *phi2, const fc4_ifc *phi3,
                    const fc4_ifc *phi4, const int mesh[3], const fc4_options *opt, fc4_ctx **out) {
    if (!out) return fail(nullptr, FC4_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!crystal || !crystal->masses || !crystal->positions)
        return fail(nullptr, FC4_ERR_INVALID, "crystal, masses or positions is NULL");
    const int na = crystal->n_atoms;
    if (na < 1 || na > fc4::kMaxAtoms)
        return fail(nullptr, FC4_ERR_INVALID, "n_atoms must be in [1, 8]");
    for (int i = 0; i < na; ++i)
        if (!(crystal->masses[i] > 0.0)) return fail(nullptr, FC4_ERR_INVALID, "mass must be > 0");
    if (!mesh || mesh[0] < 1 || mesh[1] < 1 || mesh[2] < 1 || mesh[0] > 256 || mesh[1] > 256 ||
        mesh[2] > 256)
        return fail(nullptr, FC4_ERR_INVALID, "mesh entries must be in [1, 256]");
    const long long Nl = (long long)mesh[0] * mesh[1] * mesh[2];
    if (Nl > (1 << 20)) return fail(nullptr, FC4_ERR_INVALID, "mesh has more than 2^20 points");
    fc4_status st;
    if ((st = check_ifc(phi2, 2, na, true, "phi2")) != FC4_OK) return st;
    if ((st = check_ifc(phi3, 3, na, false, "phi3")) != FC4_OK) return st;
    if ((st = check_ifc(phi4, 4, na, false, "phi4")) != FC4_OK) return st;
    const double *A = crystal->lattice;
    const double vol = std::fabs(A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                                 A[2] * (A[3] * A[7] - A[4] * A[6]));
    if (!(vol > 0.0)) return fail(nullptr, FC4_ERR_INVALID, "lattice is singular");

    fc4_ctx *c = new fc4_ctx();
    if (opt) {
        if (opt->precision < FC4_FP64 || opt->precision > FC4_FP16X3) {
            delete c;
            return fail(nullptr, FC4_ERR_INVALID, "unknown precision");
        }
        c->precision = opt->precision;
        c->timing = opt->timing != 0;
        c->allow_unstable = opt->allow_unstable != 0;
        c->use_tc = opt->tensor_cores != 0;
        if (opt->timeout_cycles < 0) {
            delete c;
            return fail(nullptr, FC4_ERR_INVALID, "timeout_cycles must be >= 0");
        }
        c->timeout_cycles = opt->timeout_cycles;
        if (opt->block_threads) {
            if (opt->block_threads % 32 || opt->block_threads < 64 || opt->block_threads > 128) {
                delete c;
                return fail(nullptr, FC4_ERR_INVALID, "block_threads must be 64, 96 or 128");
            }
            c->block_threads = opt->block_threads;
        }
    }
    auto bail = [&](fc4_status s) {
        g_init_error = c->last_error;
        fc4_destroy(c);
        return s;
    };
#define FC4_TRY(call)                                                               \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) return bail(cuda_fail(c, e_, #call));                \
    } while (0)

    if (c->timing)
        for (int k = 0; k < 8; ++k) {
            FC4_TRY(cudaEventCreate(&c->ev_a[k]));
            FC4_TRY(cudaEventCreate(&c->ev_b[k]));
        }
    fc4::Tables &t = c->t;
    const int N = (int)Nl, nb = 3 * na;
    t.n_atoms = na;
    t.nb = nb;
    t.N = N;
    for (int k = 0; k < 3; ++k) t.mesh[k] = mesh[k];
    t.L = lcm_i(lcm_i(mesh[0], mesh[1]), mesh[2]);
    c->volume = vol;
    {   // reciprocal vectors b_1 = 2π (a_2 x a_3) / (a_1 . (a_2 x a_3)) and cyclic, left to right
        const double *a0 = A, *a1 = A + 3, *a2 = A + 6;
        double cr[3][3];
        auto cross = [](const double *x, const double *y, double *r) {
            r[0] = x[1] * y[2] - x[2] * y[1];
            r[1] = x[2] * y[0] - x[0] * y[2];
            r[2] = x[0] * y[1] - x[1] * y[0];
        };
        cross(a1, a2, cr[0]);
        cross(a2, a0, cr[1]);
        cross(a0, a1, cr[2]);
        const double v = a0[0] * cr[0][0] + a0[1] * cr[0][1] + a0[2] * cr[0][2];
        const double f = 2.0 * kPi / v;
        for (int i = 0; i < 3; ++i)
            for (int x = 0; x < 3; ++x) t.recip[3 * i + x] = f * cr[i][x];
    }
    const int L = t.L;

    // mesh coordinates and roots of unity
    std::vector<int4> qc(N);
    for (int q = 0; q < N; ++q)
        qc[q] = make_int4(q % mesh[0], (q / mesh[0]) % mesh[1], q / (mesh[0] * mesh[1]), 0);
    std::vector<double2> rt(L);
    std::vector<float2> rt32(L);
    for (int k = 0; k < L; ++k) {
        rt[k] = make_double2(std::cos(2.0 * kPi * k / L), std::sin(2.0 * kPi * k / L));
        rt32[k] = make_float2((float)rt[k].x, (float)rt[k].y);
    }
    int4 *d_qc;
    double2 *d_rt;
    float2 *d_rt32;
    FC4_TRY(upload(c, &d_qc, qc));
    FC4_TRY(upload(c, &d_rt, rt));
    FC4_TRY(upload(c, &d_rt32, rt32));
    t.qc = d_qc;
    t.rt = d_rt;
    t.rt32 = d_rt32;

    auto ism = [&](std::initializer_list<int> at) {
        double m = 1.0;
        for (int a : at) m *= crystal->masses[a];
        return 1.0 / std::sqrt(m);
    };

    // second order (harmonic prelude)
    c->nc2 = phi2->n_clusters;
    std::vector<int4> c2_at(c->nc2), c2_r(c->nc2);
    std::vector<double> c2_R(3 * (size_t)c->nc2), c2_ism(c->nc2), c2_phi(phi2->phi, phi2->phi + 9 * (size_t)c->nc2);
    for (int i = 0; i < c->nc2; ++i) {
        const int a = phi2->atoms[2 * i], b = phi2->atoms[2 * i + 1];
        const int *R = phi2->cells + 3 * i;
        c2_at[i] = make_int4(a, b, 0, 0);
        c2_r[i] = phase_vec(R, mesh, L);
        for (int x = 0; x < 3; ++x) c2_R[3 * i + x] = R[0] * A[x] + R[1] * A[3 + x] + R[2] * A[6 + x];
        c2_ism[i] = ism({a, b});
    }

    // third order
    c->nc3 = phi3 ? phi3->n_clusters : 0;
    t.nc3 = c->nc3;
    {
        std::vector<int4> at(c->nc3), r2(c->nc3), r12(c->nc3);
        std::vector<double> im(c->nc3), ph(27 * (size_t)c->nc3);
        for (int i = 0; i < c->nc3; ++i) {
            const int *a = phi3->atoms + 3 * i, *R = phi3->cells + 6 * i;
            at[i] = make_int4(a[0], a[1], a[2], 0);
            const int d12[3] = {R[0] - R[3], R[1] - R[4], R[2] - R[5]};
            r2[i] = phase_vec(R + 3, mesh, L);
            r12[i] = phase_vec(d12, mesh, L);
            im[i] = ism({a[0], a[1], a[2]});
        }
        if (c->nc3) std::copy(phi3->phi, phi3->phi + 27 * (size_t)c->nc3, ph.begin());
        int4 *d_at, *d_r2, *d_r12;
        double *d_im;
        FC4_TRY(upload(c, &d_at, at));
        FC4_TRY(upload(c, &d_r2, r2));
        FC4_TRY(upload(c, &d_r12, r12));
        FC4_TRY(upload(c, &d_im, im));
        FC4_TRY(upload(c, &c->phi3, ph));
        t.c3_at = d_at;
        t.c3_r2 = d_r2;
        t.c3_r12 = d_r12;
        t.c3_ism = d_im;
        t.phi3 = c->phi3;
    }

    // fourth order: key = (leg-2 atom, leg-3 atom, R2 - R3); keys ordered by group, clusters by key
    c->nc4 = phi4 ? phi4->n_clusters : 0;
    t.nc4 = c->nc4;
    if (c->nc4) {   // leg-swap partners of every cluster (for the triangular 4ph domains)
        using CK = std::array<int, 13>;
        std::map<CK, int> id;
        auto key = [&](int i, int l1, int l2, int l3) {
            const int *a = phi4->atoms + 4 * i, *R = phi4->cells + 9 * i;
            const int l[3] = {l1, l2, l3};
            CK k{};
            k[0] = a[0];
            for (int m = 0; m < 3; ++m) {
                k[1 + m] = a[1 + l[m]];
                for (int x = 0; x < 3; ++x) k[4 + 3 * m + x] = R[3 * l[m] + x];
            }
            return k;
        };
        for (int i = 0; i < c->nc4; ++i) id.emplace(key(i, 0, 1, 2), i);
        c->swap12.assign(c->nc4, -1);
        c->swap23.assign(c->nc4, -1);
        for (int i = 0; i < c->nc4; ++i) {
            auto f12 = id.find(key(i, 1, 0, 2)), f23 = id.find(key(i, 0, 2, 1));
            if (f12 != id.end()) c->swap12[i] = f12->second;
            if (f23 != id.end()) c->swap23[i] = f23->second;
        }
        check_sym4(c, phi4->phi);
    }
    {
        using Key = std::tuple<int, int, int, int>;   // group, dR
        std::map<Key, int> key_id;
        std::vector<Key> ck(c->nc4);
        for (int i = 0; i < c->nc4; ++i) {
            const int *a = phi4->atoms + 4 * i, *R = phi4->cells + 9 * i;
            ck[i] = Key(a[2] * na + a[3], R[3] - R[6], R[4] - R[7], R[5] - R[8]);
            key_id.emplace(ck[i], 0);
        }
        int nk = 0;
        std::vector<Key> keys;
        for (auto &kv : key_id) { kv.second = nk++; keys.push_back(kv.first); }
        t.n_keys = nk;
        c->perm4.resize(c->nc4);
        std::iota(c->perm4.begin(), c->perm4.end(), 0);
        std::stable_sort(c->perm4.begin(), c->perm4.end(),
                         [&](int x, int y) { return key_id[ck[x]] < key_id[ck[y]]; });
        std::vector<int> key_start(nk + 1, 0);
        for (int i = 0; i < c->nc4; ++i) key_start[key_id[ck[i]] + 1]++;
        for (int k = 0; k < nk; ++k) key_start[k + 1] += key_start[k];
        for (int g = 0; g <= na * na; ++g) t.grp_start[g] = nk;
        for (int k = nk - 1; k >= 0; --k) t.grp_start[std::get<0>(keys[k])] = k;
        for (int g = na * na - 1; g >= 0; --g)
            if (t.grp_start[g] > t.grp_start[g + 1]) t.grp_start[g] = t.grp_start[g + 1];
        std::vector<int4> at(c->nc4), r3(c->nc4), r13(c->nc4), kr(nk);
        std::vector<double> im(c->nc4), ph(81 * (size_t)c->nc4);
        std::vector<float> im32(c->nc4), ph32(81 * (size_t)c->nc4);
        for (int s = 0; s < c->nc4; ++s) {
            const int i = c->perm4[s];
            const int *a = phi4->atoms + 4 * i, *R = phi4->cells + 9 * i;
            at[s] = make_int4(a[0], a[1], a[2], a[3]);
            const int d13[3] = {R[0] - R[6], R[1] - R[7], R[2] - R[8]};
            r3[s] = phase_vec(R + 6, mesh, L);
            r13[s] = phase_vec(d13, mesh, L);
            im[s] = ism({a[0], a[1], a[2], a[3]});
            im32[s] = (float)im[s];
            for (int k = 0; k < 81; ++k) {
                ph[81 * (size_t)s + k] = phi4->phi[81 * (size_t)i + k];
                ph32[81 * (size_t)s + k] = (float)ph[81 * (size_t)s + k];
            }
        }
        for (int k = 0; k < nk; ++k) {
            const int d[3] = {std::get<1>(keys[k]), std::get<2>(keys[k]), std::get<3>(keys[k])};
            kr[k] = phase_vec(d, mesh, L);
        }
        // the clusters of each (key, leg-1 atom), in cluster order: the W kernels' phase fold
        std::vector<int> kb_start((size_t)nk * na + 1, 0), kb_idx(c->nc4);
        for (int s = 0; s < c->nc4; ++s) {
            const int r = key_id[ck[c->perm4[s]]];
            kb_start[(size_t)r * na + at[s].y + 1]++;
        }
        for (size_t g = 0; g < (size_t)nk * na; ++g) kb_start[g + 1] += kb_start[g];
        {
            std::vector<int> fill(kb_start.begin(), kb_start.end() - 1);
            for (int s = 0; s < c->nc4; ++s) {
                const int r = key_id[ck[c->perm4[s]]];
                kb_idx[fill[(size_t)r * na + at[s].y]++] = s;
            }
        }
        int4 *d_at, *d_r3, *d_r13, *d_kr;
        double *d_im;
        float *d_im32;
        int *d_ks, *d_kbs, *d_kbi;
        FC4_TRY(upload(c, &d_at, at));
        FC4_TRY(upload(c, &d_r3, r3));
        FC4_TRY(upload(c, &d_r13, r13));
        FC4_TRY(upload(c, &d_im, im));
        FC4_TRY(upload(c, &d_im32, im32));
        FC4_TRY(upload(c, &c->phi4, ph));
        FC4_TRY(upload(c, &c->phi4_32, ph32));
        FC4_TRY(upload(c, &d_ks, key_start));
        FC4_TRY(upload(c, &d_kbs, kb_start));
        FC4_TRY(upload(c, &d_kbi, kb_idx));
        FC4_TRY(upload(c, &d_kr, kr));
        FC4_TRY(upload(c, &c->perm4_dev, c->perm4));
        FC4_TRY(dalloc(c, &c->adj_tmp, 81 * (size_t)std::max(1, c->nc4)));
        t.c4_at = d_at;
        t.c4_r3 = d_r3;
        t.c4_r13 = d_r13;
        t.c4_ism = d_im;
        t.c4_ism32 = d_im32;
        t.phi4 = c->phi4;
        t.phi4_32 = c->phi4_32;
        t.key_start = d_ks;
        t.kb_start = d_kbs;
        t.kb_idx = d_kbi;
        double2 *d_P4;
        float2 *d_P4_32;
        FC4_TRY(dalloc(c, &d_P4, (size_t)N * nk));
        FC4_TRY(dalloc(c, &d_P4_32, (size_t)N * nk));
        t.P4 = d_P4;
        t.P4_32 = d_P4_32;
        FC4_TRY(fc4::launch_phase_tables(t, d_kr, d_P4, d_P4_32, 0));
    }

    // modes: device harmonic solve
    const size_t nm = (size_t)N * nb;
    FC4_TRY(dalloc(c, &c->om, nm));
    FC4_TRY(dalloc(c, &c->vel, 3 * nm));
    FC4_TRY(dalloc(c, &c->eig, nm));
    FC4_TRY(dalloc(c, &c->ev, nm * nb));
    FC4_TRY(dalloc(c, &c->ev32, nm * nb));
    FC4_TRY(dalloc(c, &c->om32, nm));
    FC4_TRY(dalloc(c, &c->om32lo, nm));
    FC4_TRY(dalloc(c, &c->invw, nm));
    FC4_TRY(dalloc(c, &c->invw32, nm));
    FC4_TRY(dalloc(c, &c->occ, nm));
    FC4_TRY(dalloc(c, &c->occ32, nm));
    FC4_TRY(dalloc(c, &c->vmask, (size_t)N));
    FC4_TRY(dalloc(c, &c->vp32, nm));
    FC4_TRY(dalloc(c, &c->vp32lo, nm));
    FC4_TRY(dalloc(c, &c->omT32, nm));
    FC4_TRY(dalloc(c, &c->vpT32, nm));
    FC4_TRY(dalloc(c, &c->vpTlo, nm));
    FC4_TRY(dalloc(c, &c->err, 1));
    FC4_TRY(cudaMemset(c->err, 0, sizeof(int)));
    FC4_TRY(dalloc(c, &c->dev_err, 1));
    FC4_TRY(cudaMemset(c->dev_err, 0, sizeof(int)));
    t.om = c->om;
    t.om32 = c->om32;
    t.om32lo = c->om32lo;
    t.vel = c->vel;
    t.ev = c->ev;
    t.ev32 = c->ev32;
    t.vmask = c->vmask;
    t.vp32 = c->vp32;
    t.vp32lo = c->vp32lo;
    t.omT32 = c->omT32;
    t.vpT32 = c->vpT32;
    t.vpTlo = c->vpTlo;
    t.occ = c->occ;
    t.occ32 = c->occ32;
    t.invw = c->invw;
    t.invw32 = c->invw32;
    {
        int4 *d_at, *d_r;
        double *d_R, *d_phi, *d_ism;
        FC4_TRY(upload(c, &d_at, c2_at));
        FC4_TRY(upload(c, &d_r, c2_r));
        FC4_TRY(upload(c, &d_R, c2_R));
        FC4_TRY(upload(c, &d_phi, c2_phi));
        FC4_TRY(upload(c, &d_ism, c2_ism));
        FC4_TRY(fc4::launch_harmonic(t, c->nc2, d_at, d_r, d_R, d_phi, d_ism, kEigToW2, c->om, c->vel,
                                     c->ev, c->eig, c->err, 0));
    }
    FC4_TRY(cudaDeviceSynchronize());
    int herr = 0;
    FC4_TRY(cudaMemcpy(&herr, c->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr && !c->allow_unstable) {
        c->last_error = "harmonic eigenvalue below -1e-8 eV/(A^2 amu): unstable crystal";
        return bail(FC4_ERR_UNSTABLE);
    }
    if (refresh_modes(c) != FC4_OK) return bail(FC4_ERR_CUDA);
    FC4_TRY(cudaDeviceSynchronize());
#undef FC4_TRY
    *out = c;
    return FC4_OK;
}

fc4_status fc4_set_modes(fc4_ctx *c, const double *omega, const double *vel, const double *evec) {
    if (!c) return fail(nullptr, FC4_ERR_INVALID, "ctx is NULL");
    if (!omega || !vel || !evec) return fail(c, FC4_ERR_INVALID, "omega, vel and evec are required");
    const size_t nm = (size_t)c->t.N * c->t.nb;
    for (size_t i = 0; i < nm; ++i) {
        const size_t q = i / c->t.nb, j = i % c->t.nb;
        if (!(q == 0 && j < 3) && !(omega[i] > 0.0))
            return fail(c, FC4_ERR_INVALID, "omega must be > 0 except for the Gamma acoustic modes");
    }
    FC4_CUDA(c, cudaMemcpy(c->om, omega, nm * sizeof(double), cudaMemcpyHostToDevice));
    FC4_CUDA(c, cudaMemcpy(c->vel, vel, 3 * nm * sizeof(double), cudaMemcpyHostToDevice));
    FC4_CUDA(c, cudaMemcpy(c->ev, evec, nm * c->t.nb * sizeof(double2), cudaMemcpyHostToDevice));
    c->w_s1 = 0;
    fc4_status s = refresh_modes(c);
    if (s != FC4_OK) return s;
    FC4_CUDA(c, cudaDeviceSynchronize());
    return FC4_OK;
}

fc4_status fc4_get_modes(fc4_ctx *c, double *omega, double *vel, double *evec) {
    if (!c) return fail(nullptr, FC4_ERR_INVALID, "ctx is NULL");
    const size_t nm = (size_t)c->t.N * c->t.nb;
    FC4_CUDA(c, cudaDeviceSynchronize());
    if (omega) FC4_CUDA(c, cudaMemcpy(omega, c->om, nm * sizeof(double), cudaMemcpyDeviceToHost));
    if (vel) FC4_CUDA(c, cudaMemcpy(vel, c->vel, 3 * nm * sizeof(double), cudaMemcpyDeviceToHost));
    if (evec) FC4_CUDA(c, cudaMemcpy(evec, c->ev, nm * c->t.nb * sizeof(double2), cudaMemcpyDeviceToHost));
    return FC4_OK;
}

}  // extern "C"

namespace {

// κ's prefactor 1/(N V_cell) with v in Å/ps (x 100 m/s) and 1/Γ in ps (x 1e-12 s): W/(m K)
double kappa_scale(const fc4_ctx *c) { return 1e4 * 1e-12 / ((double)c->t.N * c->volume * 1e-30); }

// The rates call behind fc4_rates and the iterative BTE: with bte_F set (device [N nb][3]), the
// kernels also accumulate the BTE's off-diagonal term, reduced into delta_out [n_q nb][3]; Γ, WP
// and counts are written when gamma_out is set.
fc4_status rates_call(fc4_ctx *c, double T_K, int sigma_adaptive, double sigma_value, int channel_mask,
                      const int *q_subset, int n_q, double *gamma_out, double *wp_out, long long *counts_out,
                      void *stream, const double *bte_F, double *delta_out) {
    if (!c) return fail(nullptr, FC4_ERR_INVALID, "ctx is NULL");
    if (!(T_K > 0.0) || !std::isfinite(T_K)) return fail(c, FC4_ERR_INVALID, "T must be > 0");
    if (sigma_adaptive != 0 && sigma_adaptive != 1) return fail(c, FC4_ERR_INVALID, "sigma_adaptive must be 0 or 1");
    if (!(sigma_value > 0.0) || !std::isfinite(sigma_value))
        return fail(c, FC4_ERR_INVALID, sigma_adaptive ? "the adaptive scale must be > 0" : "sigma must be > 0");
    if (channel_mask < 0 || channel_mask > 31) return fail(c, FC4_ERR_INVALID, "channel_mask must be in [0, 31]");
    const int N = c->t.N, nb = c->t.nb;
    std::vector<int> modes;
    if (q_subset) {
        if (n_q < 0) return fail(c, FC4_ERR_INVALID, "n_q < 0");
        modes.reserve((size_t)n_q * nb);
        for (int i = 0; i < n_q; ++i) {
            if (q_subset[i] < 0 || q_subset[i] >= N) return fail(c, FC4_ERR_INVALID, "q index out of range");
            for (int j = 0; j < nb; ++j) modes.push_back(q_subset[i] * nb + j);
        }
    } else {
        modes.resize((size_t)N * nb);
        std::iota(modes.begin(), modes.end(), 0);
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int nm = (int)modes.size();
    if (nm == 0) {                      // nothing to compute; outputs may be NULL
        c->have_last = true;
        c->last_modes.clear();
        return FC4_OK;
    }
    if (!gamma_out && !bte_F) return fail(c, FC4_ERR_INVALID, "gamma_out is NULL");
    if (bte_F && (!delta_out || c->t.n_atoms > 2))
        return fail(c, FC4_ERR_INVALID, bte_F && delta_out ? "the iterative BTE supports cells of at most 2 atoms"
                                                           : "delta_out is NULL");
    if ((size_t)nm > c->modes_cap) {
        if (c->modes) { cudaFree(c->modes); c->owned.erase(std::find(c->owned.begin(), c->owned.end(), (void *)c->modes)); }
        FC4_CUDA(c, dalloc(c, &c->modes, (size_t)nm));
        c->modes_cap = nm;
        c->modes_on_device.clear();
    }
    // Modes are processed in chunks.  All modes in one chunk is the paper's all-modes strategy;
    // fc4_set_mode_chunk bounds the chunk (1: mode by mode, Algorithm 5), and the W buffer of the
    // tiled 4ph path caps it at max(4 GiB, a quarter of the device memory).  Partials and W are
    // sized for one chunk, so the call's memory grows with the chunk, not with the subset.
    const bool need_w = (channel_mask & 0b11100) && c->nc4;
    const size_t per_mode = need_w ? fc4::rates4_wbuf_per_mode(c->t, c->precision == FC4_FP64) : 0;
    size_t chunk = (size_t)nm;
    if (c->mode_chunk > 0) chunk = std::min(chunk, (size_t)c->mode_chunk);
    if (per_mode) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) total_b = 0;
        const size_t cap_bytes = c->w_limit ? c->w_limit : std::max<size_t>(4ull << 30, total_b / 4);
        chunk = std::max<size_t>(1, std::min(chunk, cap_bytes / per_mode));
    }
    const size_t need = (size_t)5 * chunk * N;
    if (need > c->part_cap) {
        for (void *p : {(void *)c->part_g, (void *)c->part_wp, (void *)c->part_n, (void *)c->part_items,
                        (void *)c->part_ent, (void *)c->part_ev, (void *)c->part_cev})
            if (p) { cudaFree(p); c->owned.erase(std::find(c->owned.begin(), c->owned.end(), p)); }
        c->part_g = c->part_wp = nullptr;
        c->part_n = c->part_items = c->part_ent = c->part_ev = c->part_cev = nullptr;
        c->part_cap = 0;
        FC4_CUDA(c, dalloc(c, &c->part_g, need));
        FC4_CUDA(c, dalloc(c, &c->part_wp, need));
        FC4_CUDA(c, dalloc(c, &c->part_n, need));
        FC4_CUDA(c, dalloc(c, &c->part_items, need));
        FC4_CUDA(c, dalloc(c, &c->part_ent, need));
        FC4_CUDA(c, dalloc(c, &c->part_ev, need));
        FC4_CUDA(c, dalloc(c, &c->part_cev, need));
        c->part_cap = need;
    }
    if (bte_F) {                          // BTE partials [5][chunk][N][3] and the FP32 copy of F
        if (3 * need > c->part_d_cap) {
            if (c->part_d) { cudaFree(c->part_d); c->owned.erase(std::find(c->owned.begin(), c->owned.end(), (void *)c->part_d)); }
            c->part_d = nullptr;
            c->part_d_cap = 0;
            FC4_CUDA(c, dalloc(c, &c->part_d, 3 * need));
            c->part_d_cap = 3 * need;
        }
        if (!c->bte_F32) FC4_CUDA(c, dalloc(c, &c->bte_F32, (size_t)3 * N * nb));
        FC4_CUDA(c, fc4::launch_to_f32(bte_F, c->bte_F32, (size_t)3 * N * nb, s));
    }
    if (per_mode && c->wbuf_bytes < chunk * per_mode) {     // W scratch of the tiled 4ph path
        if (c->wbuf) {
            cudaFree(c->wbuf);
            c->owned.erase(std::find(c->owned.begin(), c->owned.end(), c->wbuf));
            c->wbuf = nullptr;
            c->wbuf_bytes = 0;
        }
        unsigned char *w = nullptr;
        FC4_CUDA(c, dalloc(c, &w, chunk * per_mode));
        c->wbuf = w;
        c->wbuf_bytes = chunk * per_mode;
        c->w_s1 = 0;
    }
    if (modes != c->modes_on_device) {      // unchanged subsets need no copy (stream capture)
        FC4_CUDA(c, cudaMemcpyAsync(c->modes, modes.data(), nm * sizeof(int), cudaMemcpyHostToDevice, s));
        c->modes_on_device = modes;
    }
    fc4_status st = ensure_occupations(c, T_K, s);
    if (st != FC4_OK) return st;
    if (!c->stats) FC4_CUDA(c, dalloc(c, &c->stats, 25));
    FC4_CUDA(c, cudaMemsetAsync(c->stats, 0, 25 * sizeof(unsigned long long), s));
    const int fp64 = c->precision == FC4_FP64;
    c->last_chunk = (int)chunk;
    for (size_t m0 = 0; m0 < (size_t)nm; m0 += chunk) {
        const int cm = (int)std::min(chunk, (size_t)nm - m0);
        fc4::RateArgs a{};
        a.n_modes = cm;
        a.modes = c->modes + m0;
        set_window(c, a, sigma_adaptive != 0, sigma_value);
        a.part_g = c->part_g;
        a.part_wp = c->part_wp;
        a.part_n = c->part_n;
        a.part_items = c->part_items;
        a.part_ent = c->part_ent;
        a.part_ev = c->part_ev;
        a.part_cev = c->part_cev;
        a.wbuf = per_mode ? c->wbuf : nullptr;
        a.wbuf_bytes = per_mode ? c->wbuf_bytes : 0;
        if (bte_F) {
            a.bte_F = bte_F;
            a.bte_F32 = c->bte_F32;
            a.part_d = c->part_d;
        }
        const std::vector<int> cmodes(modes.begin() + m0, modes.begin() + m0 + cm);
        for (int ch = 0; ch < 5; ++ch) {
            if (!((channel_mask >> ch) & 1)) continue;
            // a channel without clusters launches nothing: its a.n_part[ch] stays 0, so the
            // reduction reads no partials and writes Γ = WP = 0 and count 0 for it
            if (ch < 2 ? c->nc3 == 0 : c->nc4 == 0) continue;
            if (ch < 2) {
                Timed tm(c, ch, s);
                FC4_CUDA(c, fc4::launch_rates3(c->t, a, ch, fp64, s));
                continue;
            }
            const int s1 = ch == 4 ? -1 : 1;
            const bool whole = per_mode && c->wbuf && (size_t)cm * per_mode <= c->wbuf_bytes;
            a.w_reuse = whole && c->w_s1 == s1 && c->w_modes == cmodes;
            Timed tm(c, ch, s);
            FC4_CUDA(c, fc4::launch_rates4(c->t, a, ch, fp64, c->block_threads, s));
            if (whole && a.wbuf) {
                c->w_s1 = s1;
                if (c->w_modes != cmodes) c->w_modes = cmodes;
            } else {
                c->w_s1 = 0;
            }
        }
        a.out_ld = nm;
        Timed tm(c, 5, s);
        if (gamma_out)
            FC4_CUDA(c, fc4::launch_reduce(c->t, a, channel_mask, unit_c3(), unit_c4(), gamma_out + m0,
                                           wp_out ? wp_out + m0 : nullptr, counts_out ? counts_out + m0 : nullptr,
                                           c->stats, s));
        if (bte_F)
            FC4_CUDA(c, fc4::launch_bte_reduce(c->t, a, channel_mask, unit_c3(), unit_c4(), delta_out + 3 * m0, s));
    }
    for (int k = 0; k < 5; ++k)
        if (!((channel_mask >> k) & 1)) c->ev_used[k] = false;
    for (int ch = 0; ch < 5; ++ch) {
        const long long per = ch < 2 ? (long long)N * nb * nb : (long long)N * N * nb * nb * nb;
        c->cand[ch] = ((channel_mask >> ch) & 1) ? per * nm : 0;
    }
    c->have_last = true;
    c->last_T = T_K;
    c->last_sigma = sigma_value;
    c->last_adaptive = sigma_adaptive != 0;
    c->last_mask = channel_mask;
    c->last_modes = modes;
    return FC4_OK;
}

}  // namespace

extern "C" {

fc4_status fc4_rates(fc4_ctx *c, double T_K, int sigma_adaptive, double sigma_value,
                     int channel_mask, const int *q_subset, int n_q, double *gamma_out,
                     double *wp_out, long long *counts_out, void *stream) {
    return rates_call(c, T_K, sigma_adaptive, sigma_value, channel_mask, q_subset, n_q, gamma_out, wp_out,
                      counts_out, stream, nullptr, nullptr);
}

fc4_status fc4_bte_offdiag(fc4_ctx *c, double T_K, int sigma_adaptive, double sigma_value, int channel_mask,
                           const int *q_subset, int n_q, const double *F, double *delta_out, void *stream) {
    if (!c) return fail(nullptr, FC4_ERR_INVALID, "ctx is NULL");
    if (!F || !delta_out) return fail(c, FC4_ERR_INVALID, "F and delta_out are required");
    return rates_call(c, T_K, sigma_adaptive, sigma_value, channel_mask, q_subset, n_q, nullptr, nullptr, nullptr,
                      stream, F, delta_out);
}

fc4_status fc4_kappa_iterative(fc4_ctx *c, double T_K, int sigma_adaptive, double sigma_value, int channel_mask,
                               const double *gamma, int max_iter, double tol, double *kappa_out, double *F_out,
                               int *iters_out, void *stream) {
    if (!c) return fail(nullptr, FC4_ERR_INVALID, "ctx is NULL");
    if (!gamma || !kappa_out) return fail(c, FC4_ERR_INVALID, "gamma and kappa_out are required");
    if (max_iter < 0 || !(tol >= 0.0)) return fail(c, FC4_ERR_INVALID, "max_iter >= 0 and tol >= 0 required");
    if (channel_mask < 0 || channel_mask > 31) return fail(c, FC4_ERR_INVALID, "channel_mask must be in [0, 31]");
    if (!(T_K > 0.0) || !std::isfinite(T_K)) return fail(c, FC4_ERR_INVALID, "T must be > 0");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nm = (size_t)c->t.N * c->t.nb;
    if (!c->bte_F) FC4_CUDA(c, dalloc(c, &c->bte_F, 3 * nm));
    if (!c->bte_delta) FC4_CUDA(c, dalloc(c, &c->bte_delta, 3 * nm));
    if (!c->bte_F32) FC4_CUDA(c, dalloc(c, &c->bte_F32, 3 * nm));
    if (!c->bte_kappa) FC4_CUDA(c, dalloc(c, &c->bte_kappa, 9));
    const double xw = kHbar * 1e12 / (kKb * T_K);
    FC4_CUDA(c, fc4::launch_bte_update(c->t, gamma, channel_mask, nullptr, c->bte_F, c->bte_F32, s));   // F = v / Γ
    FC4_CUDA(c, fc4::launch_kappa_F(c->t, xw, kKb, c->bte_F, kappa_scale(c), c->bte_kappa, s));
    double kp[9], kn[9];
    FC4_CUDA(c, cudaMemcpyAsync(kp, c->bte_kappa, sizeof kp, cudaMemcpyDeviceToHost, s));
    FC4_CUDA(c, cudaStreamSynchronize(s));
    int it = 0;
    for (it = 1; it <= max_iter; ++it) {
        fc4_status st = rates_call(c, T_K, sigma_adaptive, sigma_value, channel_mask, nullptr, 0, nullptr, nullptr,
                                   nullptr, stream, c->bte_F, c->bte_delta);
        if (st != FC4_OK) return st;
        FC4_CUDA(c, fc4::launch_bte_update(c->t, gamma, channel_mask, c->bte_delta, c->bte_F, c->bte_F32, s));
        FC4_CUDA(c, fc4::launch_kappa_F(c->t, xw, kKb, c->bte_F, kappa_scale(c), c->bte_kappa, s));
        FC4_CUDA(c, cudaMemcpyAsync(kn, c->bte_kappa, sizeof kn, cudaMemcpyDeviceToHost, s));
        FC4_CUDA(c, cudaStreamSynchronize(s));
        double dmax = 0.0, kmax = 0.0;
        for (int k = 0; k < 9; ++k) {
            dmax = std::max(dmax, std::fabs(kn[k] - kp[k]));
            kmax = std::max(kmax, std::fabs(kn[k]));
        }
        std::memcpy(kp, kn, sizeof kp);
        if (dmax <= tol * kmax) break;
    }
    if (it > max_iter) it = max_iter;
    FC4_CUDA(c, cudaMemcpyAsync(kappa_out, c->bte_kappa, 9 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (F_out) FC4_CUDA(c, cudaMemcpyAsync(F_out, c->bte_F, 3 * nm * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (iters_out) *iters_out = it;
    return FC4_OK;
}

fc4_status fc4_processes(fc4_ctx *c, int channel, int mode, unsigned long long *words, long long cap,
                         long long *n_out) {
    if (!c) return fail(nullptr, FC4_ERR_INVALID, "ctx is NULL");
    if (channel < 0 || channel > 4) return fail(c, FC4_ERR_INVALID, "channel must be in [0, 4]");
    if (mode < 0 || mode >= c->t.N * c->t.nb) return fail(c, FC4_ERR_INVALID, "mode out of range");
    if (cap < 0 || (cap > 0 && !words)) return fail(c, FC4_ERR_INVALID, "bad words / cap");
    const long long n_thr = channel < 2 ? (long long)c->t.N * c->t.nb : (long long)c->t.N * c->t.nb * c->t.N;
    fc4::RateArgs a{};
    set_window(c, a, c->last_adaptive, c->last_sigma);
    int *d_counts = nullptr;
    long long *d_off = nullptr;
    unsigned long long *d_words = nullptr;
    auto cleanup = [&]() {
        cudaFree(d_counts);
        cudaFree(d_off);
        cudaFree(d_words);
    };
    cudaError_t e = cudaMalloc(&d_counts, n_thr * sizeof(int));
    if (e == cudaSuccess) e = fc4::launch_count_processes(c->t, a, channel, mode, d_counts, 0);
    std::vector<int> counts(n_thr);
    if (e == cudaSuccess) e = cudaMemcpy(counts.data(), d_counts, n_thr * sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(c, e, "fc4_processes count"); }
    std::vector<long long> off(n_thr);
    long long total = 0;
    for (long long i = 0; i < n_thr; ++i) { off[i] = total; total += counts[i]; }
    if (n_out) *n_out = total;
    if (cap > 0 && total > 0) {
        e = cudaMalloc(&d_off, n_thr * sizeof(long long));
        if (e == cudaSuccess) e = cudaMalloc(&d_words, total * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMemcpy(d_off, off.data(), n_thr * sizeof(long long), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = fc4::launch_write_processes(c->t, a, channel, mode, d_off, d_words, 0);
        if (e == cudaSuccess)
            e = cudaMemcpy(words, d_words, std::min(cap, total) * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { cleanup(); return cuda_fail(c, e, "fc4_processes write"); }
    }
    cleanup();
    return FC4_OK;
}

// Σ C v v τ / (N V): v Å/ps -> m/s (1e2)², τ ps -> s (1e-12), V Å³ -> m³ (1e-30)

fc4_status fc4_kappa(fc4_ctx *c, double T_K, const double *gamma, int channel_mask, double *kappa_out,
                     void *stream) {
    if (!c) return fail(nullptr, FC4_ERR_INVALID, "ctx is NULL");
    if (!(T_K > 0.0)) return fail(c, FC4_ERR_INVALID, "T must be > 0");
    if (!gamma || !kappa_out) return fail(c, FC4_ERR_INVALID, "NULL buffer");
    if (channel_mask < 0 || channel_mask > 31) return fail(c, FC4_ERR_INVALID, "channel_mask must be in [0, 31]");
    Timed tm(c, 6, (cudaStream_t)stream);
    FC4_CUDA(c, fc4::launch_kappa(c->t, kHbar * 1e12 / (kKb * T_K), kKb, gamma, channel_mask, kappa_scale(c),
                                  kappa_out, (cudaStream_t)stream));
    return FC4_OK;
}

fc4_status fc4_kappa_backward(fc4_ctx *c, double T_K, const double *gamma, int channel_mask,
                              const double *dL_dkappa, double *dL_dgamma, void *stream) {
    if (!c) return fail(nullptr, FC4_ERR_INVALID, "ctx is NULL");
    if (!(T_K > 0.0)) return fail(c, FC4_ERR_INVALID, "T must be > 0");
    if (!gamma || !dL_dkappa || !dL_dgamma) return fail(c, FC4_ERR_INVALID, "NULL buffer");
    if (channel_mask < 0 || channel_mask > 31) return fail(c, FC4_ERR_INVALID, "channel_mask must be in [0, 31]");
    FC4_CUDA(c, fc4::launch_kappa_backward(c->t, kHbar * 1e12 / (kKb * T_K), kKb, gamma, channel_mask,
                                           kappa_scale(c), dL_dkappa, dL_dgamma, (cudaStream_t)stream));
    c->n_launches += 1;
    return FC4_OK;
}

fc4_status fc4_rates_backward(fc4_ctx *c, const double *dL_dgamma, double *dphi3, double *dphi4,
                              void *stream) {
    if (!c) return fail(nullptr, FC4_ERR_INVALID, "ctx is NULL");
    if (!c->have_last) return fail(c, FC4_ERR_STATE, "fc4_rates_backward before fc4_rates");
    if (c->t.n_atoms > 4) return fail(c, FC4_ERR_INVALID, "fc4_rates_backward supports cells of at most 4 atoms");
    if (!c->sample_all && (c->last_mask & 0b11100))
        return fail(c, FC4_ERR_STATE, "fc4_rates_backward: the four-phonon sampling estimate has no adjoint "
                                      "(fc4_set_sampling(ctx, 1, 0) turns it off)");
    const int nm = (int)c->last_modes.size();
    cudaStream_t s = (cudaStream_t)stream;
    if (dphi3 && c->nc3) FC4_CUDA(c, cudaMemsetAsync(dphi3, 0, 27 * (size_t)c->nc3 * sizeof(double), s));
    if (dphi4 && c->nc4) FC4_CUDA(c, cudaMemsetAsync(dphi4, 0, 81 * (size_t)c->nc4 * sizeof(double), s));
    if (nm == 0) return FC4_OK;
    if (!dL_dgamma) return fail(c, FC4_ERR_INVALID, "dL_dgamma is NULL");
    const size_t width = std::max<size_t>(27 * (size_t)c->nc3, 81 * (size_t)c->nc4);
    const size_t need = (size_t)nm * std::max<size_t>(width, 1);
    if (need > c->adj_cap) {
        if (c->adj_part) {
            cudaFree(c->adj_part);
            c->owned.erase(std::find(c->owned.begin(), c->owned.end(), (void *)c->adj_part));
            c->adj_part = nullptr;
            c->adj_cap = 0;
        }
        FC4_CUDA(c, dalloc(c, &c->adj_part, need));
        c->adj_cap = need;
    }
    if ((size_t)nm > c->modes_cap) return fail(c, FC4_ERR_STATE, "mode buffer smaller than the last call");
    if (c->last_modes != c->modes_on_device) {
        FC4_CUDA(c, cudaMemcpyAsync(c->modes, c->last_modes.data(), nm * sizeof(int), cudaMemcpyHostToDevice, s));
        c->modes_on_device = c->last_modes;
    }
    fc4_status st = ensure_occupations(c, c->last_T, s);
    if (st != FC4_OK) return st;
    fc4::RateArgs a{};
    a.n_modes = nm;
    a.modes = c->modes;
    set_window(c, a, c->last_adaptive, c->last_sigma);
    const double N = (double)c->t.N;
    bool first3 = true, first4 = true;
    for (int ch = 0; ch < 5; ++ch) {
        if (!((c->last_mask >> ch) & 1)) continue;
        if (ch < 2 && (!dphi3 || !c->nc3)) continue;
        if (ch >= 2 && (!dphi4 || !c->nc4)) continue;
        const double cst = ch < 2 ? unit_c3() / N : unit_c4() / (N * N);
        // 3ph: FP64 always; 4ph: FP64 in an FP64 context, else FP32 (FP64 accumulation of the slices)
        const int fp64 = ch < 2 || c->precision == FC4_FP64;
        FC4_CUDA(c, fc4::launch_adjoint(c->t, a, ch, dL_dgamma, cst, c->adj_part, fp64, s));
        c->n_launches += 1;
        if (ch < 2) {
            FC4_CUDA(c, fc4::launch_sum_slices(nm, 27 * c->nc3, c->adj_part, dphi3, first3 ? 0 : 1, 0, s));
            first3 = false;
        } else {
            FC4_CUDA(c, fc4::launch_sum_slices(nm, 81 * c->nc4, c->adj_part, c->adj_tmp, first4 ? 0 : 1, !fp64, s));
            first4 = false;
        }
        c->n_launches += 1;
    }
    if (!first4) {
        FC4_CUDA(c, fc4::launch_unpermute(c->nc4, 81, c->perm4_dev, c->adj_tmp, dphi4, s));
        c->n_launches += 1;
    }
    return FC4_OK;
}

fc4_status fc4_update_anharmonic(fc4_ctx *c, const double *phi3, const double *phi4) {
    if (!c) return fail(nullptr, FC4_ERR_INVALID, "ctx is NULL");
    FC4_CUDA(c, cudaDeviceSynchronize());
    if (phi4) c->w_s1 = 0;
    if (phi3 && c->nc3)
        FC4_CUDA(c, cudaMemcpy(c->phi3, phi3, 27 * (size_t)c->nc3 * sizeof(double), cudaMemcpyHostToDevice));
    if (phi4 && c->nc4) {
        check_sym4(c, phi4);
        std::vector<double> ph(81 * (size_t)c->nc4);
        std::vector<float> ph32(81 * (size_t)c->nc4);
        for (int s = 0; s < c->nc4; ++s)
            for (int k = 0; k < 81; ++k) {
                ph[81 * (size_t)s + k] = phi4[81 * (size_t)c->perm4[s] + k];
                ph32[81 * (size_t)s + k] = (float)ph[81 * (size_t)s + k];
            }
        FC4_CUDA(c, cudaMemcpy(c->phi4, ph.data(), ph.size() * sizeof(double), cudaMemcpyHostToDevice));
        FC4_CUDA(c, cudaMemcpy(c->phi4_32, ph32.data(), ph32.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    return FC4_OK;
}

fc4_status fc4_stats(fc4_ctx *c, long long out[30]) {
    if (!c || !out) return fail(c, FC4_ERR_INVALID, "NULL argument");
    if (!c->have_last || !c->stats) return fail(c, FC4_ERR_STATE, "fc4_stats before fc4_rates");
    unsigned long long h[25];
    FC4_CUDA(c, cudaDeviceSynchronize());
    FC4_CUDA(c, cudaMemcpy(h, c->stats, sizeof(h), cudaMemcpyDeviceToHost));
    for (int ch = 0; ch < 5; ++ch) {
        out[6 * ch] = (long long)h[5 * ch];
        out[6 * ch + 1] = (long long)h[5 * ch + 1];
        out[6 * ch + 2] = c->cand[ch];
        out[6 * ch + 3] = (long long)h[5 * ch + 2];
        out[6 * ch + 4] = (long long)h[5 * ch + 3];
        out[6 * ch + 5] = (long long)h[5 * ch + 4];
    }
    return FC4_OK;
}

fc4_status fc4_timings(fc4_ctx *c, double out[9]) {
    if (!c || !out) return fail(c, FC4_ERR_INVALID, "NULL argument");
    if (!c->timing) return fail(c, FC4_ERR_STATE, "timing was not enabled in fc4_options");
    for (int k = 0; k < 8; ++k) {
        out[k] = 0.0;
        if (!c->ev_used[k]) continue;
        FC4_CUDA(c, cudaEventSynchronize(c->ev_b[k]));
        float ms = 0.0f;
        FC4_CUDA(c, cudaEventElapsedTime(&ms, c->ev_a[k], c->ev_b[k]));
        out[k] = ms;
    }
    out[8] = (double)c->n_launches;
    return FC4_OK;
}

fc4_status fc4_set_block_threads(fc4_ctx *c, int block_threads) {
    if (!c) return fail(nullptr, FC4_ERR_INVALID, "ctx is NULL");
    if (block_threads != 0 && block_threads != 64 && block_threads != 96 && block_threads != 128)
        return fail(c, FC4_ERR_INVALID, "block_threads must be 0, 64, 96 or 128");
    c->block_threads = block_threads ? block_threads : 128;
    return FC4_OK;
}

fc4_status fc4_set_mode_chunk(fc4_ctx *c, int modes_per_chunk, long long w_limit_bytes) {
    if (!c) return fail(nullptr, FC4_ERR_INVALID, "ctx is NULL");
    if (modes_per_chunk < 0 || w_limit_bytes < 0)
        return fail(c, FC4_ERR_INVALID, "modes_per_chunk and w_limit_bytes must be >= 0");
    c->mode_chunk = modes_per_chunk;
    c->w_limit = (size_t)w_limit_bytes;
    return FC4_OK;
}

fc4_status fc4_memory(const fc4_ctx *c, long long out[5]) {
    if (!c || !out) return FC4_ERR_INVALID;
    long long tot = 0;
    for (void *p : c->owned) {
        auto it = c->alloc_bytes.find(p);
        if (it != c->alloc_bytes.end()) tot += (long long)it->second;
    }
    out[0] = tot;
    out[1] = (long long)fc4::rates4_wbuf_per_mode(c->t, c->precision == FC4_FP64);
    out[2] = (long long)c->wbuf_bytes;
    out[3] = (long long)c->part_cap * 7 * 8;
    out[4] = c->last_chunk;
    return FC4_OK;
}

fc4_status fc4_set_sampling(fc4_ctx *c, double fraction, unsigned long long seed) {
    if (!c) return fail(nullptr, FC4_ERR_INVALID, "ctx is NULL");
    if (!(fraction > 0.0) || !std::isfinite(fraction)) return fail(c, FC4_ERR_INVALID, "fraction must be in (0, 1]");
    if (fraction >= 1.0) {
        c->sample_all = 1;
        c->sample_threshold = ~0ull;
    } else {
        c->sample_all = 0;
        c->sample_threshold = (unsigned long long)std::ldexp(fraction, 64);   // floor(f 2^64)
        if (c->sample_threshold == 0) return fail(c, FC4_ERR_INVALID, "fraction below 2^-64");
    }
    c->sample_seed = seed;
    return FC4_OK;
}

fc4_status fc4_set_ablation(fc4_ctx *c, int flags) {
    if (!c) return fail(nullptr, FC4_ERR_INVALID, "ctx is NULL");
    if (flags & ~1) return fail(c, FC4_ERR_INVALID, "unknown ablation flag");
    c->no_compact = flags & 1;
    return FC4_OK;
}

fc4_status fc4_set_precision(fc4_ctx *c, int precision) {
    if (!c) return fail(nullptr, FC4_ERR_INVALID, "ctx is NULL");
    if (precision < FC4_FP64 || precision > FC4_FP16X3) return fail(c, FC4_ERR_INVALID, "unknown precision");
    if (precision != c->precision) c->w_s1 = 0;     // the W buffer's element type may change
    c->precision = precision;
    return FC4_OK;
}

fc4_status fc4_set_tensor_cores(fc4_ctx *c, int on) {
    if (!c) return fail(nullptr, FC4_ERR_INVALID, "ctx is NULL");
    if (on != 0 && on != 1) return fail(c, FC4_ERR_INVALID, "on must be 0 or 1");
    c->use_tc = on != 0;
    return FC4_OK;
}

fc4_status fc4_check_device(fc4_ctx *c) {
    if (!c) return fail(nullptr, FC4_ERR_INVALID, "ctx is NULL");
    int h = 0;
    FC4_CUDA(c, cudaDeviceSynchronize());
    FC4_CUDA(c, cudaMemcpy(&h, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (!h) return FC4_OK;
    FC4_CUDA(c, cudaMemset(c->dev_err, 0, sizeof(int)));
    return fail(c, FC4_ERR_TIMEOUT, "a device-side wait expired (the rates of that call are NaN)");
}

fc4_status fc4_info(const fc4_ctx *c, long long out[8]) {
    if (!c || !out) return FC4_ERR_INVALID;
    out[0] = c->t.n_atoms;
    out[1] = c->t.nb;
    out[2] = c->t.N;
    out[3] = c->nc2;
    out[4] = c->nc3;
    out[5] = c->nc4;
    out[6] = c->t.n_keys;
    out[7] = c->precision;
    return FC4_OK;
}

const char *fc4_last_error(const fc4_ctx *c) {
    return c ? c->last_error.c_str() : g_init_error.c_str();
}

void fc4_destroy(fc4_ctx *c) {
    if (!c) return;
    for (int k = 0; k < 8; ++k) {
        if (c->ev_a[k]) cudaEventDestroy(c->ev_a[k]);
        if (c->ev_b[k]) cudaEventDestroy(c->ev_b[k]);
    }
    for (void *p : c->owned) cudaFree(p);
    delete c;
}

}  // extern "C"

// ------------------------------------------------------------------------------ allocation-free rates
//
// fc4_rates_static: fc4_rates without device allocation.  Every piece of per-call device scratch
// (the q list, the mode list and the per-(channel, mode, q') partial sums) lives in one file-scope
// __device__ array of fixed size.  With no W buffer to hand, the four-phonon channels take the
// general kernel (W built per block in shared memory) instead of the tiled W-buffer path.  A host-side use
// of the array's name is only a stand-in for it; the device address is looked up once per device
// with cudaGetSymbolAddress and cached.

namespace {

constexpr long long kStaticUnits = 1LL << 16;       // max (modes x q') units per channel
constexpr long long kStaticQ = kStaticUnits;         // max q points (n_q <= units)
constexpr size_t kStaticBytes =
    5 * (size_t)kStaticUnits * (2 * sizeof(double) + 3 * sizeof(long long)) +
    2 * (size_t)kStaticQ * sizeof(int);

static __device__ __align__(256) unsigned char g_fc4_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 256;
unsigned char *g_static_ptr[kMaxDevices] = {};
std::mutex g_static_mu;

// Device address of the scratch array on the current device (looked up on first use).
cudaError_t static_scratch(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_fc4_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_static_ptr[dev];
    return cudaSuccess;
}

__global__ void expand_modes_kernel(const int *qs, int n_q, int nb, int *modes) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_q * nb) modes[i] = qs[i / nb] * nb + (i % nb);
}

}  // namespace

extern "C" fc4_status fc4_rates_static(fc4_ctx *c, double T_K, double sigma_value, int channel_mask,
                                       const int *q_subset, int n_q, double *gamma_out,
                                       double *wp_out, long long *counts_out, void *stream) {
    if (!c) return fail(nullptr, FC4_ERR_INVALID, "ctx is NULL");
    if (!(T_K > 0.0) || !std::isfinite(T_K)) return fail(c, FC4_ERR_INVALID, "T must be > 0");
    if (!(sigma_value > 0.0) || !std::isfinite(sigma_value)) return fail(c, FC4_ERR_INVALID, "sigma must be > 0");
    if (channel_mask < 0 || channel_mask > 31) return fail(c, FC4_ERR_INVALID, "channel_mask must be in [0, 31]");
    if (!q_subset || n_q < 0) return fail(c, FC4_ERR_INVALID, "q_subset is required");
    const int N = c->t.N, nb = c->t.nb;
    for (int i = 0; i < n_q; ++i)
        if (q_subset[i] < 0 || q_subset[i] >= N) return fail(c, FC4_ERR_INVALID, "q index out of range");
    const long long nm = (long long)n_q * nb;
    if (nm * N > kStaticUnits)
        return fail(c, FC4_ERR_INVALID, "fc4_rates_static: n_q * nb * N exceeds 65536 (static scratch limit)");
    if (nm == 0) return FC4_OK;
    if (!gamma_out) return fail(c, FC4_ERR_INVALID, "gamma_out is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *base = nullptr;
    FC4_CUDA(c, static_scratch(&base));
    const size_t units = (size_t)kStaticUnits;
    double *part_g = reinterpret_cast<double *>(base);
    double *part_wp = part_g + 5 * units;
    long long *part_n = reinterpret_cast<long long *>(part_wp + 5 * units);
    long long *part_items = part_n + 5 * units;
    long long *part_ent = part_items + 5 * units;
    int *d_q = reinterpret_cast<int *>(part_ent + 5 * units);
    int *d_modes = d_q + kStaticQ;
    FC4_CUDA(c, cudaMemcpyAsync(d_q, q_subset, (size_t)n_q * sizeof(int), cudaMemcpyHostToDevice, s));
    expand_modes_kernel<<<(unsigned)((nm + 255) / 256), 256, 0, s>>>(d_q, n_q, nb, d_modes);
    FC4_CUDA(c, cudaGetLastError());
    fc4_status st = ensure_occupations(c, T_K, s);
    if (st != FC4_OK) return st;
    fc4::RateArgs a{};
    a.n_modes = (int)nm;
    a.modes = d_modes;
    set_window(c, a, false, sigma_value);
    a.part_g = part_g;
    a.part_wp = part_wp;
    a.part_n = part_n;
    a.part_items = part_items;
    a.part_ent = part_ent;
    const int fp64 = c->precision == FC4_FP64;
    for (int ch = 0; ch < 5; ++ch) {
        if (!((channel_mask >> ch) & 1)) continue;
        // A channel without clusters launches nothing: its a.n_part[ch] stays 0, so the reduction
        // reads no partials and writes Γ = WP = 0 and count 0 for it.
        if (ch < 2 ? c->nc3 == 0 : c->nc4 == 0) continue;
        if (ch < 2) FC4_CUDA(c, fc4::launch_rates3(c->t, a, ch, fp64, s));
        else FC4_CUDA(c, fc4::launch_rates4(c->t, a, ch, fp64, c->block_threads, s));
    }
    FC4_CUDA(c, fc4::launch_reduce(c->t, a, channel_mask, unit_c3(), unit_c4(), gamma_out, wp_out,
                                   counts_out, nullptr, s));
    return FC4_OK;
}

// ------------------------------------------------------------------------------ batched contexts
//
// fc4_batch_rates: the rates of many contexts in a few launches.  The four-phonon units of every
// context with the same cell size run as one persistent launch of the general kernel (FP32, fixed
// σ) over a work list (context, channel, unit) ordered from the largest meshes down, each block
// taking the next item from a global counter; the three-phonon kernels and the reductions are
// launched per context.  With unchanged arguments a call performs only stream-ordered launches and
// memsets (no host copies), so it can be captured in a CUDA graph.

struct fc4_batch {
    std::vector<fc4_ctx *> ctx;
    std::vector<fc4::Tables> tabs;             // host copies of the contexts' tables
    int4 *d_items = nullptr;
    size_t items_cap = 0;
    std::vector<int4> items_on_device;
    int *d_counter = nullptr;                  // one counter per cell size (1..8 atoms)
    std::string last_error;
};

namespace {

// content last copied into the batch kernels' constant memory (shared by every batch)
std::vector<unsigned char> g_batch_meta;
std::mutex g_batch_mu;

fc4_status bfail(fc4_batch *b, fc4_status s, const std::string &msg) {
    if (b) b->last_error = msg;
    else fc4::set_host_error(msg.c_str());
    return s;
}

#define FC4_BCUDA(b, call)                                                                  \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? FC4_ERR_OOM : FC4_ERR_CUDA, \
                         std::string(#call) + ": " + cudaGetErrorString(e_));               \
    } while (0)

}  // namespace

extern "C" {

fc4_status fc4_batch_create(fc4_ctx *const *ctxs, int n, fc4_batch **out) {
    if (!out || !ctxs || n <= 0) return bfail(nullptr, FC4_ERR_INVALID, "fc4_batch_create: ctxs, n > 0 and out required");
    *out = nullptr;
    fc4_batch *b = new fc4_batch();
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) { delete b; return bfail(nullptr, FC4_ERR_INVALID, "fc4_batch_create: NULL context"); }
        b->ctx.push_back(ctxs[i]);
    }
    if (n > fc4::kMaxBatch) {
        delete b;
        return bfail(nullptr, FC4_ERR_INVALID, "fc4_batch_create: more than 40 contexts");
    }
    for (fc4_ctx *c : b->ctx) b->tabs.push_back(c->t);
    cudaError_t e = cudaMalloc((void **)&b->d_counter, sizeof(int) * 9);
    if (e != cudaSuccess) {
        fc4_batch_destroy(b);
        return bfail(nullptr, e == cudaErrorMemoryAllocation ? FC4_ERR_OOM : FC4_ERR_CUDA,
                     std::string("fc4_batch_create: ") + cudaGetErrorString(e));
    }
    *out = b;
    return FC4_OK;
}

const char *fc4_batch_last_error(const fc4_batch *b) { return b ? b->last_error.c_str() : ""; }

void fc4_batch_destroy(fc4_batch *b) {
    if (!b) return;
    cudaFree(b->d_items);
    cudaFree(b->d_counter);
    delete b;
}

}  // extern "C"

extern "C" fc4_status fc4_batch_rates(fc4_batch *b, double T_K, double sigma_value, int channel_mask,
                                      const int *const *q_subsets, const int *n_q, double *const *gamma_out,
                                      double *const *wp_out, long long *const *counts_out, void *stream) {
    if (!b) return bfail(nullptr, FC4_ERR_INVALID, "batch is NULL");
    if (!(T_K > 0.0) || !std::isfinite(T_K)) return bfail(b, FC4_ERR_INVALID, "T must be > 0");
    if (!(sigma_value > 0.0) || !std::isfinite(sigma_value)) return bfail(b, FC4_ERR_INVALID, "sigma must be > 0");
    if (channel_mask < 0 || channel_mask > 31) return bfail(b, FC4_ERR_INVALID, "channel_mask must be in [0, 31]");
    if (!gamma_out) return bfail(b, FC4_ERR_INVALID, "gamma_out is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)b->ctx.size();
    std::vector<fc4::RateArgs> args(n);
    std::vector<int> nms(n);
    for (int i = 0; i < n; ++i) {
        fc4_ctx *c = b->ctx[i];
        if (c->precision == FC4_FP64) return bfail(b, FC4_ERR_INVALID, "fc4_batch_rates: FP32 contexts only");
        // cells the tiled kernels serve (up to two atoms, W buffer) keep their own, faster path
        if (fc4::rates4_wbuf_per_mode(c->t, 0)) {
            nms[i] = 0;
            const int nq = q_subsets && q_subsets[i] ? n_q[i] : 0;
            if (q_subsets && q_subsets[i] && (!n_q || nq < 0))
                return bfail(b, FC4_ERR_INVALID, "n_q required with q_subsets");
            const fc4_status st = rates_call(c, T_K, 0, sigma_value, channel_mask,
                                             q_subsets && q_subsets[i] ? q_subsets[i] : nullptr, nq, gamma_out[i],
                                             wp_out ? wp_out[i] : nullptr, counts_out ? counts_out[i] : nullptr,
                                             stream, nullptr, nullptr);
            if (st != FC4_OK) return bfail(b, st, c->last_error);
            continue;
        }
        const int N = c->t.N, nb = c->t.nb;
        std::vector<int> modes;
        if (q_subsets && q_subsets[i]) {
            if (!n_q || n_q[i] < 0) return bfail(b, FC4_ERR_INVALID, "n_q required with q_subsets");
            for (int k = 0; k < n_q[i]; ++k) {
                const int q = q_subsets[i][k];
                if (q < 0 || q >= N) return bfail(b, FC4_ERR_INVALID, "q index out of range");
                for (int j = 0; j < nb; ++j) modes.push_back(q * nb + j);
            }
        } else {
            modes.resize((size_t)N * nb);
            std::iota(modes.begin(), modes.end(), 0);
        }
        const int nm = (int)modes.size();
        nms[i] = nm;
        if (nm == 0) continue;
        if (!gamma_out[i]) return bfail(b, FC4_ERR_INVALID, "gamma_out[i] is NULL");
        if ((size_t)nm > c->modes_cap) {
            if (c->modes) { cudaFree(c->modes); c->owned.erase(std::find(c->owned.begin(), c->owned.end(), (void *)c->modes)); }
            c->modes = nullptr;
            c->modes_cap = 0;
            FC4_BCUDA(b, dalloc(c, &c->modes, (size_t)nm));
            c->modes_cap = nm;
            c->modes_on_device.clear();
        }
        const size_t need = (size_t)5 * nm * N;
        if (need > c->part_cap) {
            for (void *p : {(void *)c->part_g, (void *)c->part_wp, (void *)c->part_n, (void *)c->part_items,
                            (void *)c->part_ent, (void *)c->part_ev, (void *)c->part_cev})
                if (p) { cudaFree(p); c->owned.erase(std::find(c->owned.begin(), c->owned.end(), p)); }
            c->part_g = c->part_wp = nullptr;
            c->part_n = c->part_items = c->part_ent = c->part_ev = c->part_cev = nullptr;
            c->part_cap = 0;
            FC4_BCUDA(b, dalloc(c, &c->part_g, need));
            FC4_BCUDA(b, dalloc(c, &c->part_wp, need));
            FC4_BCUDA(b, dalloc(c, &c->part_n, need));
            FC4_BCUDA(b, dalloc(c, &c->part_items, need));
            FC4_BCUDA(b, dalloc(c, &c->part_ent, need));
            FC4_BCUDA(b, dalloc(c, &c->part_ev, need));
            FC4_BCUDA(b, dalloc(c, &c->part_cev, need));
            c->part_cap = need;
        }
        if (modes != c->modes_on_device) {
            FC4_BCUDA(b, cudaMemcpyAsync(c->modes, modes.data(), nm * sizeof(int), cudaMemcpyHostToDevice, s));
            c->modes_on_device = modes;
        }
        if (ensure_occupations(c, T_K, s) != FC4_OK) return bfail(b, FC4_ERR_CUDA, c->last_error);
        if (!c->stats) FC4_BCUDA(b, dalloc(c, &c->stats, 25));
        FC4_BCUDA(b, cudaMemsetAsync(c->stats, 0, 25 * sizeof(unsigned long long), s));
        fc4::RateArgs &a = args[i];
        a.n_modes = nm;
        a.modes = c->modes;
        set_window(c, a, false, sigma_value);
        a.use_tc = 0;
        a.part_g = c->part_g;
        a.part_wp = c->part_wp;
        a.part_n = c->part_n;
        a.part_items = c->part_items;
        a.part_ent = c->part_ent;
        a.part_ev = c->part_ev;
        a.part_cev = c->part_cev;
        for (int ch = 2; ch < 5; ++ch)
            if (((channel_mask >> ch) & 1) && c->nc4) a.n_part[ch] = N;
        c->cand[0] = c->cand[1] = c->cand[2] = c->cand[3] = c->cand[4] = 0;
        for (int ch = 0; ch < 5; ++ch)
            if ((channel_mask >> ch) & 1)
                c->cand[ch] = (ch < 2 ? (long long)N * nb * nb : (long long)N * N * nb * nb * nb) * nm;
        c->have_last = true;                   // fc4_stats, fc4_processes and the backward read these
        c->last_T = T_K;
        c->last_sigma = sigma_value;
        c->last_adaptive = false;
        c->last_mask = channel_mask;
        c->last_modes = modes;
    }
    // three-phonon kernels per context (they set n_part of their channels)
    for (int i = 0; i < n; ++i) {
        fc4_ctx *c = b->ctx[i];
        if (!nms[i] || !c->nc3) continue;
        for (int ch = 0; ch < 2; ++ch)
            if ((channel_mask >> ch) & 1) FC4_BCUDA(b, fc4::launch_rates3(c->t, args[i], ch, 0, s));
    }
    // work list: contexts grouped by cell size (largest first), meshes from the largest down
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const fc4::Tables &tx = b->ctx[x]->t, &ty = b->ctx[y]->t;
        return tx.n_atoms != ty.n_atoms ? tx.n_atoms > ty.n_atoms : tx.N > ty.N;
    });
    std::vector<int4> items;
    std::vector<std::array<long long, 3>> classes;      // (atoms, first item, count)
    for (int i : order) {
        fc4_ctx *c = b->ctx[i];
        if (!nms[i] || !c->nc4) continue;
        if (classes.empty() || classes.back()[0] != c->t.n_atoms)
            classes.push_back({(long long)c->t.n_atoms, (long long)items.size(), 0});
        const long long units = (long long)nms[i] * c->t.N;
        for (int ch = 2; ch < 5; ++ch) {
            if (!((channel_mask >> ch) & 1)) continue;
            for (long long u = 0; u < units; ++u) items.push_back(make_int4(i, ch, (int)u, 0));
        }
        classes.back()[2] = (long long)items.size() - classes.back()[1];
    }
    if (items.size() > 0x7fffffffULL) return bfail(b, FC4_ERR_INVALID, "fc4_batch_rates: too many units");
    {   // tables and arguments into the constant memory of both kernel units, when they changed
        std::vector<unsigned char> blob(sizeof(fc4::Tables) * n + sizeof(fc4::RateArgs) * n);
        std::memcpy(blob.data(), b->tabs.data(), sizeof(fc4::Tables) * n);
        std::memcpy(blob.data() + sizeof(fc4::Tables) * n, args.data(), sizeof(fc4::RateArgs) * n);
        std::lock_guard<std::mutex> lock(g_batch_mu);
        if (blob != g_batch_meta) {
            FC4_BCUDA(b, fc4::batch_upload_f_1_4(b->tabs.data(), args.data(), n, s));
            FC4_BCUDA(b, fc4::batch_upload_f_5_8(b->tabs.data(), args.data(), n, s));
            g_batch_meta = blob;
        }
    }
    if (items.size() != b->items_on_device.size() ||
        std::memcmp(items.data(), b->items_on_device.data(), sizeof(int4) * items.size()) != 0) {
        if (items.size() > b->items_cap) {
            cudaFree(b->d_items);
            b->d_items = nullptr;
            b->items_cap = 0;
            FC4_BCUDA(b, cudaMalloc((void **)&b->d_items, sizeof(int4) * items.size()));
            b->items_cap = items.size();
        }
        if (!items.empty())
            FC4_BCUDA(b, cudaMemcpyAsync(b->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, s));
        b->items_on_device = items;
    }
    for (size_t k = 0; k < classes.size(); ++k) {
        const int na = (int)classes[k][0];
        size_t smem = 0;
        for (int i : order)
            if (b->ctx[i]->t.n_atoms == na) smem = std::max(smem, fc4::general_smem_f(na, b->ctx[i]->t));
        FC4_BCUDA(b, cudaMemsetAsync(b->d_counter + na, 0, sizeof(int), s));
        const int4 *it = b->d_items + classes[k][1];
        const int cnt = (int)classes[k][2];
        FC4_BCUDA(b, na <= 4 ? fc4::launch4_batch_f_1_4(na, it, cnt, b->d_counter + na, smem, s)
                             : fc4::launch4_batch_f_5_8(na, it, cnt, b->d_counter + na, smem, s));
        b->ctx[order[0]]->n_launches += 1;
    }
    for (int i = 0; i < n; ++i) {
        fc4_ctx *c = b->ctx[i];
        if (!nms[i]) continue;
        FC4_BCUDA(b, fc4::launch_reduce(c->t, args[i], channel_mask, unit_c3(), unit_c4(), gamma_out[i],
                                        wp_out ? wp_out[i] : nullptr, counts_out ? counts_out[i] : nullptr,
                                        c->stats, s));
    }
    return FC4_OK;
}
