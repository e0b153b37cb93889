// fc4_symmetry.cu - space-group operations of a crystal and its force constants, the irreducible
// q-points of a mesh under them, and the expansion of per-mode results from those points to the
// whole mesh (declared in include/fc4.h).  Host code only: no context and no device memory.
//
// The mode loops of Algorithms 1 and 3-5 run over N_bands x N_list modes, N_list being the
// irreducible q-points of the mesh.  A space-group operation {W | w} of the crystal that also maps
// every force-constant cluster onto a stored one (tensor rotated) leaves the scattering sums
// invariant: q -> S q permutes the partner q-points of the mesh, frequencies and occupations are
// unchanged and |V|² only sees the rotated eigenvectors.  q -> -q (real force constants) does the
// same.  Γ(S q, j) = Γ(q, j) then holds for every channel with a fixed width σ, so rates are
// evaluated on one q of each star (fc4_rates with a q subset) and copied to the rest of the star.
// The adaptive width is built from Hellmann-Feynman velocities, which inside a degenerate subspace
// depend on the eigenvector basis the solver picks at each q; it is not star-invariant.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "fc4.h"
#include "fc4_kernels.h"

namespace {

using Mat3 = std::array<std::array<double, 3>, 3>;
using IMat3 = std::array<std::array<int, 3>, 3>;

fc4_status fail(fc4_status s, const std::string &msg) {
    fc4::set_host_error(msg.c_str());
    return s;
}

bool inverse3(const Mat3 &a, Mat3 &inv) {
    const double c00 = a[1][1] * a[2][2] - a[1][2] * a[2][1];
    const double c01 = a[1][2] * a[2][0] - a[1][0] * a[2][2];
    const double c02 = a[1][0] * a[2][1] - a[1][1] * a[2][0];
    const double det = a[0][0] * c00 + a[0][1] * c01 + a[0][2] * c02;
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return false;
    inv[0][0] = c00 / det;
    inv[1][0] = c01 / det;
    inv[2][0] = c02 / det;
    inv[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) / det;
    inv[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) / det;
    inv[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) / det;
    inv[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) / det;
    inv[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) / det;
    inv[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) / det;
    return true;
}

int idet3(const IMat3 &w) {
    return w[0][0] * (w[1][1] * w[2][2] - w[1][2] * w[2][1]) -
           w[0][1] * (w[1][0] * w[2][2] - w[1][2] * w[2][0]) +
           w[0][2] * (w[1][0] * w[2][1] - w[1][1] * w[2][0]);
}

// inverse of an integer matrix with determinant ±1 (adjugate / det)
IMat3 iinverse3(const IMat3 &w) {
    const int d = idet3(w);
    IMat3 r;
    r[0][0] = (w[1][1] * w[2][2] - w[1][2] * w[2][1]) * d;
    r[0][1] = (w[0][2] * w[2][1] - w[0][1] * w[2][2]) * d;
    r[0][2] = (w[0][1] * w[1][2] - w[0][2] * w[1][1]) * d;
    r[1][0] = (w[1][2] * w[2][0] - w[1][0] * w[2][2]) * d;
    r[1][1] = (w[0][0] * w[2][2] - w[0][2] * w[2][0]) * d;
    r[1][2] = (w[0][2] * w[1][0] - w[0][0] * w[1][2]) * d;
    r[2][0] = (w[1][0] * w[2][1] - w[1][1] * w[2][0]) * d;
    r[2][1] = (w[0][1] * w[2][0] - w[0][0] * w[2][1]) * d;
    r[2][2] = (w[0][0] * w[1][1] - w[0][1] * w[1][0]) * d;
    return r;
}

// One structure operation: fractional f -> W f + w maps atom a onto atom perm[a] shifted by the
// lattice vector shift[a] (W f_a + w = f_perm[a] + shift[a]).
struct StructOp {
    IMat3 W;
    double w[3];
    std::vector<int> perm;
    std::vector<std::array<int, 3>> shift;
};

// Does the operation map the clusters of one order onto stored clusters with the tensor rotated
// by S (Cartesian), Φ'[α'β'..] = Σ S_α'α S_β'β .. Φ[αβ..], within tol * max |Φ|?  Legs: atom a_i in
// cell R_i (R_0 = 0); the image leg is atom perm[a_i] in cell W R_i + shift[a_i], translated so
// that leg 0 is in the home cell.
bool maps_clusters(const fc4_ifc *f, const StructOp &op, const Mat3 &S, double tol) {
    if (!f || f->n_clusters <= 0) return true;
    const int n = f->order, nc = f->n_clusters;
    int ncomp = 1;
    for (int k = 0; k < n; ++k) ncomp *= 3;
    std::map<std::vector<int>, int> index;
    double mx = 0.0;
    for (int c = 0; c < nc; ++c) {
        std::vector<int> key(f->atoms + (size_t)n * c, f->atoms + (size_t)n * (c + 1));
        key.insert(key.end(), f->cells + (size_t)3 * (n - 1) * c, f->cells + (size_t)3 * (n - 1) * (c + 1));
        index.emplace(std::move(key), c);
        for (int k = 0; k < ncomp; ++k) mx = std::max(mx, std::fabs(f->phi[(size_t)ncomp * c + k]));
    }
    if (mx == 0.0) return true;
    std::vector<double> t(ncomp), u(ncomp);
    for (int c = 0; c < nc; ++c) {
        const int *at = f->atoms + (size_t)n * c;
        const int *cl = f->cells + (size_t)3 * (n - 1) * c;
        std::vector<int> key(n + 3 * (n - 1));
        const auto &s0 = op.shift[at[0]];
        for (int i = 0; i < n; ++i) key[i] = op.perm[at[i]];
        for (int i = 1; i < n; ++i)
            for (int x = 0; x < 3; ++x) {
                int v = op.shift[at[i]][x] - s0[x];
                for (int y = 0; y < 3; ++y) v += op.W[x][y] * cl[3 * (i - 1) + y];
                key[n + 3 * (i - 1) + x] = v;
            }
        // rotate the tensor one index at a time (index k has stride 3^(n-1-k))
        std::copy(f->phi + (size_t)ncomp * c, f->phi + (size_t)ncomp * (c + 1), t.begin());
        for (int k = 0, stride = ncomp / 3; k < n; ++k, stride /= 3) {
            for (int e = 0; e < ncomp; ++e) {
                const int a = (e / stride) % 3, base = e - a * stride;
                u[e] = S[a][0] * t[base] + S[a][1] * t[base + stride] + S[a][2] * t[base + 2 * stride];
            }
            t.swap(u);
        }
        const auto it = index.find(key);
        for (int e = 0; e < ncomp; ++e) {
            const double stored = it == index.end() ? 0.0 : f->phi[(size_t)ncomp * it->second + e];
            if (std::fabs(stored - t[e]) > tol * mx) return false;
        }
    }
    return true;
}

}  // namespace

extern "C" fc4_status fc4_symmetry_ops(const fc4_crystal *crystal, const fc4_ifc *phi2,
                                       const fc4_ifc *phi3, const fc4_ifc *phi4, double tol,
                                       int max_ops, int *rot, double *trans, int *n_ops) {
    if (!crystal || crystal->n_atoms <= 0 || !crystal->positions || !crystal->masses || !n_ops)
        return fail(FC4_ERR_INVALID, "fc4_symmetry_ops: crystal and n_ops are required");
    if (max_ops < 0 || (max_ops > 0 && (!rot || !trans)))
        return fail(FC4_ERR_INVALID, "fc4_symmetry_ops: max_ops > 0 needs rot and trans");
    const fc4_ifc *ifcs[3] = {phi2, phi3, phi4};
    for (int o = 0; o < 3; ++o) {
        const fc4_ifc *f = ifcs[o];
        if (!f || f->n_clusters <= 0) continue;
        if (f->order != o + 2 || !f->atoms || !f->cells || !f->phi)
            return fail(FC4_ERR_INVALID, "fc4_symmetry_ops: cluster set of order " + std::to_string(o + 2) +
                                             " is incomplete or has the wrong order");
        for (long long k = 0; k < (long long)f->n_clusters * f->order; ++k)
            if (f->atoms[k] < 0 || f->atoms[k] >= crystal->n_atoms)
                return fail(FC4_ERR_INVALID, "fc4_symmetry_ops: cluster atom index out of range");
    }
    if (!(tol > 0.0)) tol = 1e-8;
    const int na = crystal->n_atoms;
    Mat3 A, At, AtInv, Ainv;                          // A: rows a_i
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) A[i][j] = crystal->lattice[3 * i + j];
    if (!inverse3(A, Ainv)) return fail(FC4_ERR_INVALID, "fc4_symmetry_ops: singular lattice");
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) At[i][j] = A[j][i];
    inverse3(At, AtInv);
    Mat3 G{};                                         // metric a_i . a_j
    double gmax = 0.0, amax = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            for (int k = 0; k < 3; ++k) G[i][j] += A[i][k] * A[j][k];
            gmax = std::max(gmax, std::fabs(G[i][j]));
        }
    for (int i = 0; i < 3; ++i) amax = std::max(amax, std::sqrt(G[i][i]));
    // fractional coordinates: x = Σ_i f_i a_i
    std::vector<std::array<double, 3>> fr(na);
    for (int a = 0; a < na; ++a)
        for (int i = 0; i < 3; ++i) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += crystal->positions[3 * a + k] * Ainv[k][i];
            fr[a][i] = s;
        }
    const double pos_tol = 1e-6 * amax;

    int count = 0;
    IMat3 W;
    for (int code = 0; code < 19683; ++code) {        // every W with entries in {-1, 0, 1}
        int c = code;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                W[i][j] = c % 3 - 1;
                c /= 3;
            }
        const int d = idet3(W);
        if (d != 1 && d != -1) continue;
        // the metric is preserved: W^T G W = G (S = A^T W A^-T orthogonal)
        bool metric = true;
        for (int i = 0; i < 3 && metric; ++i)
            for (int j = 0; j < 3 && metric; ++j) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) s += W[k][i] * G[k][l] * W[l][j];
                metric = std::fabs(s - G[i][j]) <= 1e-8 * gmax;
            }
        if (!metric) continue;
        // a translation taking atom 0 to an atom of the same mass
        for (int b = 0; b < na; ++b) {
            if (crystal->masses[b] != crystal->masses[0]) continue;
            StructOp op;
            op.W = W;
            for (int i = 0; i < 3; ++i) {
                double s = fr[b][i];
                for (int k = 0; k < 3; ++k) s -= W[i][k] * fr[0][k];
                op.w[i] = s - std::floor(s);
            }
            op.perm.assign(na, -1);
            op.shift.assign(na, {0, 0, 0});
            bool ok = true;
            for (int a = 0; a < na && ok; ++a) {
                double img[3];
                for (int i = 0; i < 3; ++i) {
                    img[i] = op.w[i];
                    for (int k = 0; k < 3; ++k) img[i] += W[i][k] * fr[a][k];
                }
                ok = false;
                for (int a2 = 0; a2 < na && !ok; ++a2) {
                    if (crystal->masses[a2] != crystal->masses[a]) continue;
                    double dl[3], dist = 0.0;
                    for (int i = 0; i < 3; ++i) dl[i] = std::nearbyint(img[i] - fr[a2][i]);
                    for (int x = 0; x < 3; ++x) {
                        double cx = 0.0;
                        for (int i = 0; i < 3; ++i) cx += (img[i] - fr[a2][i] - dl[i]) * A[i][x];
                        dist = std::max(dist, std::fabs(cx));
                    }
                    if (dist <= pos_tol) {
                        ok = true;
                        op.perm[a] = a2;
                        for (int i = 0; i < 3; ++i) op.shift[a][i] = (int)dl[i];
                    }
                }
            }
            if (!ok) continue;
            // Cartesian rotation S = A^T W A^-T
            Mat3 S{};
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double s = 0.0;
                    for (int k = 0; k < 3; ++k)
                        for (int l = 0; l < 3; ++l) s += At[i][k] * W[k][l] * AtInv[l][j];
                    S[i][j] = s;
                }
            bool sym = true;
            for (int o = 0; o < 3 && sym; ++o) sym = maps_clusters(ifcs[o], op, S, tol);
            if (!sym) continue;
            if (count < max_ops) {
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) rot[9 * count + 3 * i + j] = W[i][j];
                for (int i = 0; i < 3; ++i) trans[3 * count + i] = op.w[i];
            }
            ++count;
            break;                                    // one translation per W (primitive cell)
        }
    }
    *n_ops = count;
    if (max_ops > 0 && count > max_ops)
        return fail(FC4_ERR_INVALID, "fc4_symmetry_ops: " + std::to_string(count) +
                                         " operations found, max_ops = " + std::to_string(max_ops));
    return FC4_OK;
}

extern "C" fc4_status fc4_irreducible_q(const int mesh[3], int n_ops, const int *rot, int flags,
                                        int *rep, int *n_irr) {
    if (!mesh || mesh[0] <= 0 || mesh[1] <= 0 || mesh[2] <= 0 || !rep || !n_irr || n_ops < 0 ||
        (n_ops > 0 && !rot) || (flags & ~1))
        return fail(FC4_ERR_INVALID, "fc4_irreducible_q: bad mesh, pointer, n_ops or flags");
    const long long N = (long long)mesh[0] * mesh[1] * mesh[2];
    if (N > (1LL << 30)) return fail(FC4_ERR_INVALID, "fc4_irreducible_q: mesh too large");
    // each usable operation as integer coefficients on mesh indices: i'_a = Σ_b c_ab i_b mod n_a,
    // c = n_a M_ab / n_b with M = W^-T (q in reciprocal fractional coordinates maps as k' = W^-T k)
    std::vector<IMat3> gens;
    for (int o = 0; o < n_ops; ++o) {
        IMat3 W;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) W[i][j] = rot[9 * o + 3 * i + j];
        const int d = idet3(W);
        if (d != 1 && d != -1) return fail(FC4_ERR_INVALID, "fc4_irreducible_q: det W must be +-1");
        const IMat3 Wi = iinverse3(W);
        IMat3 c;
        bool fits = true;
        for (int a = 0; a < 3 && fits; ++a)
            for (int b = 0; b < 3 && fits; ++b) {
                const long long num = (long long)mesh[a] * Wi[b][a];     // M_ab = (W^-1)_ba
                fits = num % mesh[b] == 0;
                c[a][b] = (int)(num / mesh[b]);
            }
        if (fits) gens.push_back(c);
    }
    if (flags & 1) {           // time reversal: q -> -q
        IMat3 c{};
        for (int a = 0; a < 3; ++a) c[a][a] = -1;
        gens.push_back(c);
    }
    auto apply = [&](const IMat3 &c, long long q) {
        const int i[3] = {(int)(q % mesh[0]), (int)((q / mesh[0]) % mesh[1]), (int)(q / ((long long)mesh[0] * mesh[1]))};
        long long r = 0, mul = 1;
        for (int a = 0; a < 3; ++a) {
            long long s = 0;
            for (int b = 0; b < 3; ++b) s += (long long)c[a][b] * i[b];
            s %= mesh[a];
            if (s < 0) s += mesh[a];
            r += s * mul;
            mul *= mesh[a];
        }
        return r;
    };
    // orbits under the group the operations generate; the representative is the smallest index
    std::vector<int> stack;
    for (long long q = 0; q < N; ++q) rep[q] = -1;
    int count = 0;
    for (long long q = 0; q < N; ++q) {
        if (rep[q] >= 0) continue;
        ++count;
        rep[q] = (int)q;
        stack.assign(1, (int)q);
        while (!stack.empty()) {
            const int p = stack.back();
            stack.pop_back();
            for (const auto &c : gens) {
                const long long p2 = apply(c, p);
                if (rep[p2] < 0) {
                    rep[p2] = (int)q;
                    stack.push_back((int)p2);
                }
            }
        }
    }
    *n_irr = count;
    return FC4_OK;
}

extern "C" fc4_status fc4_expand_irreducible(const int mesh[3], int nb, const int *rep,
                                             const double *omega, double deg_tol, int n_sets,
                                             const double *sub, double *full) {
    if (!mesh || mesh[0] <= 0 || mesh[1] <= 0 || mesh[2] <= 0 || nb <= 0 || !rep || !omega ||
        n_sets < 0 || (n_sets > 0 && (!sub || !full)))
        return fail(FC4_ERR_INVALID, "fc4_expand_irreducible: bad mesh, nb, pointer or n_sets");
    const long long N = (long long)mesh[0] * mesh[1] * mesh[2];
    std::vector<long long> pos(N, -1);
    long long n_irr = 0;
    for (long long q = 0; q < N; ++q) {
        const int r = rep[q];
        if (r < 0 || r > q || rep[r] != r)
            return fail(FC4_ERR_INVALID, "fc4_expand_irreducible: rep is not a representative map");
        if (r == q) pos[q] = n_irr++;
    }
    if (!(deg_tol >= 0.0)) return fail(FC4_ERR_INVALID, "fc4_expand_irreducible: deg_tol < 0");
    // degenerate groups at each representative: branches sorted by ω, split where the gap > deg_tol
    std::vector<int> order(nb), group(nb), gsize(nb);
    std::vector<std::vector<int>> grp_of((size_t)n_irr * nb);
    for (long long q = 0; q < N; ++q) {
        if (pos[q] < 0) continue;
        const double *w = omega + (size_t)q * nb;
        for (int j = 0; j < nb; ++j) order[j] = j;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return w[x] < w[y]; });
        int g = 0;
        for (int k = 0; k < nb; ++k) {
            if (k > 0 && w[order[k]] - w[order[k - 1]] > deg_tol) ++g;
            group[order[k]] = g;
        }
        for (int j = 0; j < nb; ++j) {
            auto &members = grp_of[(size_t)pos[q] * nb + j];
            for (int j2 = 0; j2 < nb; ++j2)
                if (group[j2] == group[j]) members.push_back(j2);
        }
    }
    for (int s = 0; s < n_sets; ++s) {
        const double *src = sub + (size_t)s * n_irr * nb;
        double *dst = full + (size_t)s * N * nb;
        for (long long q = 0; q < N; ++q) {
            const long long p = pos[rep[q]];
            for (int j = 0; j < nb; ++j) {
                const auto &members = grp_of[(size_t)p * nb + j];
                double acc = 0.0;
                for (int j2 : members) acc += src[(size_t)p * nb + j2];
                dst[(size_t)q * nb + j] = acc / (double)members.size();
            }
        }
    }
    return FC4_OK;
}
