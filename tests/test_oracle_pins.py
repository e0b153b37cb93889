"""Pins of the FP64 oracle against closed forms, the mathematics and brute force (no GPU).

Each test checks the oracle against something other than itself: the Morse pair potential
differentiated numerically on a periodic supercell, closed-form frequencies, exact symmetries,
a brute-force enumeration, band folding, and exact identities of a quadratic form."""
import itertools
import math

import numpy as np
import pytest

import oracle
from synth import diamond_crystal, morse_ifcs, morse_system, supercell_crystal, MorseParams
from tests.fd_energy import SupercellEnergy

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


@pytest.fixture(scope="module")
def sys0():
    return morse_system(seed=0)


@pytest.fixture(scope="module")
def sys_clean():
    return morse_system(seed=0, perturb=0.0)


@pytest.fixture(scope="module")
def prob3(sys0):
    return oracle.Problem(*sys0, (3, 3, 3))


# ------------------------------------------------------------------------------ units

def test_unit_constants_two_routes():
    """Γ prefactors through SI and through amu-Å-ps natural units agree."""
    a = oracle.unit_constants_si()
    b = oracle.unit_constants_natural()
    for x, y in zip(a, b):
        assert abs(x - y) <= 1e-14 * abs(x)
    # eigenvalue conversion: 1 eV/(Å² amu) = (e / amu) * 1e-4 (rad/ps)², close to F / 10 C/g
    assert abs(oracle.EIG_TO_RADPS2 - 9648.5332) < 1e-3


# ------------------------------------------------------------------------------ harmonic

@pytest.mark.parametrize("seed,n", [(0, 8), (1, 8), (1, 16)])
def test_crystal_stable(seed, n):
    """The Morse diamond crystal (Φ2 from the first shell) has no imaginary mode."""
    c, p2, p3, p4 = morse_system(seed=seed)
    m = oracle.harmonic(c, p2, (n, n, n))
    assert m.eig[1:].min() > 0.0
    assert np.abs(m.eig[0, :3]).max() < 1e-12        # acoustic sum rule at Γ


def test_gamma_optical_closed_form(sys_clean):
    """Unperturbed first-shell central-force diamond: ω_opt(Γ)² = (2/m)(4/3 k_r + 8/3 k_t),
    k_r = φ''(r1), k_t = φ'(r1)/r1 (triply degenerate)."""
    c, p2, _, _ = sys_clean
    r1 = 5.43 * math.sqrt(3) / 4
    d1, d2, _, _ = MorseParams().radial_derivatives(r1)
    w2 = 2.0 / c.masses[0] * (4.0 / 3.0 * d2 + 8.0 / 3.0 * d1 / r1) * oracle.EIG_TO_RADPS2
    m = oracle.harmonic(c, p2, (1, 1, 1))
    assert np.allclose(m.omega[3:6] ** 2, w2, rtol=1e-12)


def test_group_velocity_finite_difference(sys0):
    """v = dω/dq (Hellmann-Feynman) vs central differences of ω along each axis (non-degenerate)."""
    c, p2, _, _ = sys0
    q0 = np.array([0.13, 0.07, 0.21])
    h = 1e-6
    D, dD = oracle.dynamical_matrix(c, p2, q0)
    lam, v = np.linalg.eigh(D)
    j = 5
    w = math.sqrt(lam[j] * oracle.EIG_TO_RADPS2)
    g = np.array([np.real(np.conj(v[:, j]) @ dD[x] @ v[:, j]) for x in range(3)])
    vel = g * oracle.EIG_TO_RADPS2 / (2 * w)
    for x in range(3):
        dq = np.zeros(3)
        dq[x] = h
        lp = np.linalg.eigh(oracle.dynamical_matrix(c, p2, q0 + dq)[0])[0][j]
        lm = np.linalg.eigh(oracle.dynamical_matrix(c, p2, q0 - dq)[0])[0][j]
        fd = (math.sqrt(lp * oracle.EIG_TO_RADPS2) - math.sqrt(lm * oracle.EIG_TO_RADPS2)) / (2 * h)
        assert abs(fd - vel[x]) < 1e-6 * max(1.0, abs(vel[x]))


# ------------------------------------------------------------------------------ matrix elements

def _fd_problem():
    c, p2, p3, p4 = morse_system(seed=0, perturb=0.0)
    P = oracle.Problem(c, p2, p3, p4, (3, 3, 3))
    return c, P, SupercellEnergy(c, 3)


def test_v3_equals_supercell_third_derivative():
    """Re and Im of V3+(λ, λ', λ'') at finite q equal (4/N_cells) ∂³E/∂t1∂t2∂t3 of the Morse energy
    of a 3x3x3 supercell displaced along Re/Im(e/sqrt(m) exp(iq.R)) of the three modes."""
    c, P, S = _fd_problem()
    nb, qs = P.nb, oracle.q_cart(c.lattice, P.mesh)
    q1, q2 = 1, 3                            # (1,0,0)/3 and (0,1,0)/3
    q3 = 1 + 3 * 1                           # q1 + q2 = (1,1,0)/3
    for (j1, j2, j3) in [(3, 4, 5), (1, 5, 2), (4, 0, 3)]:
        m1, m2, m3 = q1 * nb + j1, q2 * nb + j2, q3 * nb + j3
        V = P.v3(+1, m1, m2, m3)
        e1, e2, e3 = P.modes.evec[q1][:, j1], P.modes.evec[q2][:, j2], P.modes.evec[q3][:, j3]
        p1, p2_ = S.pattern(e1, qs[q1]), S.pattern(e2, qs[q2])
        re = S.mixed_derivative([p1, p2_, S.pattern(e3, qs[q3])], 0.05)
        im = S.mixed_derivative([p1, p2_, S.pattern(e3, qs[q3], imag=True)], 0.05)
        scale = S.ncell / 4.0
        assert abs(re - scale * V.real) < 2e-6 * scale * abs(V)
        # the Im pattern is Re(-i ũ e^{iqR}); its conjugate leg carries +i, giving -Im V
        assert abs(im + scale * V.imag) < 2e-6 * scale * abs(V)


def test_v4_equals_supercell_fourth_derivative():
    """Re V4++(λ, λ', λ'', λ''') at finite q equals (8/N_cells) ∂⁴E of the supercell energy."""
    c, P, S = _fd_problem()
    nb, qs = P.nb, oracle.q_cart(c.lattice, P.mesh)
    q1, q2, q3 = 1, 3, 9                     # unit steps along b1, b2, b3 (over 3)
    q4 = 1 + 3 * (1 + 3 * 1)                 # (1,1,1)/3
    for (j1, j2, j3, j4) in [(3, 4, 5, 3), (1, 2, 5, 4)]:
        ms = [q1 * nb + j1, q2 * nb + j2, q3 * nb + j3, q4 * nb + j4]
        V = P.v4(+1, +1, *ms)
        pats = [S.pattern(P.modes.evec[q][:, j], qs[q]) for q, j in
                [(q1, j1), (q2, j2), (q3, j3), (q4, j4)]]
        re = S.mixed_derivative(pats, 0.06)
        scale = S.ncell / 8.0
        assert abs(re - scale * V.real) < 1e-5 * scale * abs(V)


def test_v_vanishes_for_acoustic_partner_at_gamma(prob3):
    """A uniform translation (Γ acoustic partner, e ∝ sqrt(m) u) decouples under the acoustic sum
    rule: V3 = 0 and V4 = 0 for any other legs."""
    P = prob3
    nb = P.nb
    for jac in range(3):
        for (m0, m2) in [(1 * nb + 4, 1 * nb + 2), (5 * nb + 3, 5 * nb + 5)]:
            v = P.v3(+1, m0, jac, m2)
            ref = abs(P.v3(+1, m0, 4, m2))
            assert abs(v) < 1e-12 * max(ref, 1.0)
        v4 = P.v4(+1, -1, 1 * nb + 4, jac, 7 * nb + 2, 1 * nb + 3)
        assert abs(v4) < 1e-11


def test_v_time_reversal(sys0):
    """With e(-q) = conj(e(q)): V3-(λ, λ', λ'') = V3+(λ, -λ', λ'') and
    V4^(s1,s2) flips the same way leg by leg."""
    c, p2, p3, p4 = sys0
    mesh = (3, 3, 3)
    base = oracle.harmonic(c, p2, mesh)
    qc = oracle.q_coords(mesh)
    minus = [int(((-x) % 3) + 3 * (((-y) % 3) + 3 * ((-z) % 3))) for x, y, z in qc]
    ev = base.evec.copy()
    for iq in range(27):
        if minus[iq] > iq:
            ev[minus[iq]] = np.conj(ev[iq])
    modes = oracle.Modes(base.omega, base.vel, ev, base.eig)
    P = oracle.Problem(c, p2, p3, p4, mesh, modes=modes)
    nb = P.nb
    q, q1 = 4, 11
    q2 = oracle.q_coords(mesh)
    for (j, j1, j2) in [(3, 4, 5), (2, 1, 0)]:
        m0 = q * nb + j
        m1 = q1 * nb + j1
        m1m = minus[q1] * nb + j1
        m2 = 13 * nb + j2
        assert abs(P.v3(-1, m0, m1, m2) - P.v3(+1, m0, m1m, m2)) < 1e-12 * abs(P.v3(-1, m0, m1, m2)) + 1e-14
        m3 = 20 * nb + 5
        a = P.v4(-1, -1, m0, m1, 7 * nb + j2, m3)
        b = P.v4(+1, +1, m0, m1m, minus[7] * nb + j2, m3)
        assert abs(a - b) < 1e-12 * abs(a) + 1e-14


def test_v_gauge_invariance(sys0):
    """Multiplying each eigenvector by an arbitrary phase leaves |V|² unchanged."""
    c, p2, p3, p4 = sys0
    mesh = (3, 3, 3)
    base = oracle.harmonic(c, p2, mesh)
    rng = np.random.default_rng(5)
    ph = np.exp(2j * np.pi * rng.random((27, 1, 6)))
    m2 = oracle.Modes(base.omega, base.vel, base.evec * ph, base.eig)
    A = oracle.Problem(c, p2, p3, p4, mesh, modes=base)
    B = oracle.Problem(c, p2, p3, p4, mesh, modes=m2)
    nb = 6
    for ms in [(4 * nb + 3, 2 * nb + 1, 6 * nb + 4), (10 * nb + 5, 8 * nb + 3, 18 * nb + 4)]:
        assert abs(abs(A.v3(1, *ms)) ** 2 - abs(B.v3(1, *ms)) ** 2) < 1e-13 * abs(A.v3(1, *ms)) ** 2 + 1e-20
    ms4 = (4 * nb + 3, 2 * nb + 1, 6 * nb + 4, 12 * nb + 5)
    assert abs(abs(A.v4(1, -1, *ms4)) ** 2 - abs(B.v4(1, -1, *ms4)) ** 2) < 1e-12 * abs(A.v4(1, -1, *ms4)) ** 2


# ------------------------------------------------------------------------------ enumeration

def _brute_force_words(P, ch, m0):
    """Unpruned enumeration: every partner tuple; momentum closure found by searching all q
    for the one whose Cartesian vector matches q + s1 q' (+ s2 q'') modulo a reciprocal vector."""
    nb, N = P.nb, P.nq
    B = oracle.reciprocal(P.crystal.lattice)
    qs = oracle.q_cart(P.crystal.lattice, P.mesh)
    Binv = np.linalg.inv(B)

    def same_mod_G(a, b):
        f = (a - b) @ Binv
        return np.all(np.abs(f - np.round(f)) < 1e-9)

    s1 = [1, -1, 1, 1, -1][ch]
    s2 = [0, 0, 1, -1, -1][ch]
    q0, j0 = divmod(m0, nb)
    w = P.modes.omega
    sig2 = 2.0 * P.sigma * oracle.SIGMA_THZ_TO_RADPS
    excl = lambda q, j: q == 0 and j < 3
    out = []
    if excl(q0, j0):
        return np.zeros(0, np.uint64)
    for q1 in range(N):
        if ch < 2:
            target = qs[q0] + s1 * qs[q1]
            q2 = [k for k in range(N) if same_mod_G(qs[k], target)][0]
            for j1 in range(nb):
                for j2 in range(nb):
                    if excl(q1, j1) or excl(q2, j2):
                        continue
                    d = oracle.delta(ch, w[m0], w[q1 * nb + j1], w[q2 * nb + j2])
                    if abs(d) <= sig2:
                        out.append((q1 * nb + j1) * nb + j2)
        else:
            for j1 in range(nb):
                for q2 in range(N):
                    target = qs[q0] + s1 * qs[q1] + s2 * qs[q2]
                    q3 = [k for k in range(N) if same_mod_G(qs[k], target)][0]
                    for j2 in range(nb):
                        for j3 in range(nb):
                            if excl(q1, j1) or excl(q2, j2) or excl(q3, j3):
                                continue
                            d = oracle.delta(ch, w[m0], w[q1 * nb + j1], w[q2 * nb + j2], w[q3 * nb + j3])
                            if abs(d) <= sig2:
                                out.append((((q1 * nb + j1) * N + q2) * nb + j2) * nb + j3)
    return np.array(out, np.uint64)


@pytest.mark.parametrize("mesh", [(1, 1, 1), (2, 2, 2)])
def test_enumeration_matches_brute_force(sys0, mesh):
    P = oracle.Problem(*sys0, mesh)
    rng = np.random.default_rng(0)
    nm = P.nq * P.nb
    for m0 in sorted(set(rng.integers(0, nm, size=4).tolist()) | {nm - 1}):
        for ch in range(5):
            a = P.processes(ch, m0)
            b = _brute_force_words(P, ch, m0)
            assert a.dtype == np.uint64 and np.array_equal(a, b), (ch, m0)


def test_enumeration_matches_brute_force_3ph_3cubed(prob3):
    P = prob3
    for m0 in [4, 17, 40, 161]:
        for ch in (0, 1):
            assert np.array_equal(P.processes(ch, m0), _brute_force_words(P, ch, m0))


def test_partner_swap_symmetry(prob3):
    """With fixed σ and the symmetric Δ forms: the ++ list is closed under (λ' <-> λ''), +- under
    (λ'' <-> λ''') and -- under every permutation of the three partners."""
    P = prob3
    nb, N = P.nb, P.nq
    for m0 in [10, 33, 77]:
        for ch, perms in [(2, [(1, 0, 2)]), (3, [(0, 2, 1)]), (4, list(itertools.permutations(range(3))))]:
            words = P.processes(ch, m0)
            q0 = m0 // nb
            s1, s2 = [(1, 1), (1, -1), (-1, -1)][ch - 2]
            tuples = set()
            for wd in words.tolist():
                q1, j1, q2, j2, j3 = oracle.decode4(wd, nb, N)
                q3c = (oracle.q_coords(P.mesh)[q0] + s1 * oracle.q_coords(P.mesh)[q1] + s2 * oracle.q_coords(P.mesh)[q2]) % 3
                q3 = int(q3c[0] + 3 * (q3c[1] + 3 * q3c[2]))
                tuples.add(((q1, j1), (q2, j2), (q3, j3)))
            for perm in perms:
                for t in tuples:
                    assert tuple(t[i] for i in perm) in tuples


def test_occupation_factors_on_shell():
    """On shell the forward-minus-backward occupation factors equal the RTA forms
    (equilibrium forward rate)/(n (n+1)) x n: n'(1+n'')/(1+n) etc."""
    rng = np.random.default_rng(3)
    x = lambda w: 1.0 / math.expm1(w)          # ħω/kT = w
    for _ in range(50):
        a, b, c = rng.uniform(0.05, 3.0, size=3)
        # 3ph+: λ + λ' -> λ'' ; ω'' = ω + ω'
        n, n1, n2 = x(a), x(b), x(a + b)
        assert abs(oracle.occupation_factor(0, n1, n2) - n1 * (1 + n2) / (1 + n)) < 1e-12 * (1 + n1)
        # 3ph-: λ -> λ' + λ'' ; ω = ω' + ω''
        n, n1, n2 = x(b + c), x(b), x(c)
        assert abs(oracle.occupation_factor(1, n1, n2) - (1 + n1) * (1 + n2) / (1 + n)) < 1e-12 * (1 + n1 * n2)
        # 4ph++: λ + λ' + λ'' -> λ''' ; ω''' = ω + ω' + ω''
        n, n1, n2, n3 = x(a), x(b), x(c), x(a + b + c)
        ref = n1 * n2 * (1 + n3) / (1 + n)
        assert abs(oracle.occupation_factor(2, n1, n2, n3) - ref) < 1e-10 * (1 + abs(ref))
        # 4ph+-: λ + λ' -> λ'' + λ''' ; ω''' = ω + ω' - ω''
        if a + b > c:
            n, n1, n2, n3 = x(a), x(b), x(c), x(a + b - c)
            ref = n1 * (1 + n2) * (1 + n3) / (1 + n)
            assert abs(oracle.occupation_factor(3, n1, n2, n3) - ref) < 1e-10 * (1 + abs(ref))
        # 4ph--: λ -> λ' + λ'' + λ''' ; ω = ω' + ω'' + ω'''
        n, n1, n2, n3 = x(a + b + c), x(a), x(b), x(c)
        ref = (1 + n1) * (1 + n2) * (1 + n3) / (1 + n)
        assert abs(oracle.occupation_factor(4, n1, n2, n3) - ref) < 1e-10 * (1 + abs(ref))


def test_delta_swap_bit_symmetric():
    """The canonical Δ forms are bit-identical under the partner swaps they must respect."""
    rng = np.random.default_rng(1)
    for _ in range(2000):
        w, a, b, c = rng.uniform(0.1, 90.0, size=4)
        assert oracle.delta(2, w, a, b, c) == oracle.delta(2, w, b, a, c)
        assert oracle.delta(3, w, a, b, c) == oracle.delta(3, w, a, c, b)
        for p in itertools.permutations((a, b, c)):
            assert oracle.delta(4, w, *p) == oracle.delta(4, w, a, b, c)


def test_weighted_phase_space_3ph_brute_force(prob3):
    """WP3+ = (1/N) Σ (n'-n'') δ / (ω ω' ω'') over the brute-force kept set (Alg. 1)."""
    P = prob3
    nb, N = P.nb, P.nq
    occ = oracle.occupations(P.modes.omega, P.T)
    w = P.modes.omega
    sig = P.sigma * oracle.SIGMA_THZ_TO_RADPS
    modes = [8, 25, 50]
    _, wp, _ = P.rates(modes, channel_mask=1)
    for i, m0 in enumerate(modes):
        tot = 0.0
        for wd in _brute_force_words(P, 0, m0).tolist():
            q1, j1, j2 = oracle.decode3(wd, nb)
            qc = oracle.q_coords(P.mesh)
            q2c = (qc[m0 // nb] + qc[q1]) % 3
            m1, m2 = q1 * nb + j1, int(q2c[0] + 3 * (q2c[1] + 3 * q2c[2])) * nb + j2
            d = w[m0] + w[m1] - w[m2]
            tot += (occ[m1] - occ[m2]) * math.exp(-d * d / sig ** 2) / (sig * math.sqrt(math.pi) * w[m0] * w[m1] * w[m2])
        assert abs(wp[0, i] - tot / N) < 1e-12 * abs(tot / N)


@pytest.mark.parametrize("ch", [2, 3, 4])
def test_weighted_phase_space_4ph_brute_force(prob3, ch):
    """WP4 = (1/N²) Σ c_s F_s g(Δ) / (ω ω1 ω2 ω3) over every candidate (q1, j1, q2, j2, j3) of the
    rectangular partner domain with |Δ| <= 2σ, written out with numpy: c = ½, ½, ⅙ for ++, +-,
    --; F the forward-minus-backward occupation products; the three acoustic modes at Γ excluded
    as partners.  The kept counts match too."""
    P = prob3
    nb, N = P.nb, P.nq
    s1, s2 = {2: (1, 1), 3: (1, -1), 4: (-1, -1)}[ch]
    c_s = {2: 0.5, 3: 0.5, 4: 1.0 / 6.0}[ch]
    w = P.modes.omega.reshape(N, nb)
    n = oracle.occupations(P.modes.omega, P.T).reshape(N, nb)
    ok = np.ones((N, nb), bool)
    ok[0, :3] = False
    sig = P.sigma * oracle.SIGMA_THZ_TO_RADPS
    qc = oracle.q_coords(P.mesh)
    mesh = np.asarray(P.mesh)
    modes = [m for m in range(3, N * nb) if P.processes(ch, m).size > 0][:3]
    assert len(modes) == 3
    _, wp, cnt = P.rates(modes, channel_mask=1 << ch)
    for i, m0 in enumerate(modes):
        q0, j0 = divmod(m0, nb)
        w0 = w[q0, j0]
        tot, kept = 0.0, 0
        for q1 in range(N):
            for q2 in range(N):
                c3 = (qc[q0] + s1 * qc[q1] + s2 * qc[q2]) % mesh
                q3 = int(c3[0] + mesh[0] * (c3[1] + mesh[1] * c3[2]))
                a = w[q1][:, None, None]
                b = w[q2][None, :, None]
                c = w[q3][None, None, :]
                if ch == 2:
                    d = (w0 - c) + (a + b)
                elif ch == 3:
                    d = (w0 + a) - (b + c)
                else:
                    srt = np.sort(np.stack(np.broadcast_arrays(a, b, c)), axis=0)
                    d = w0 - ((srt[0] + srt[1]) + srt[2])
                m = (np.abs(d) <= 2.0 * sig) & ok[q1][:, None, None] & ok[q2][None, :, None] & ok[q3][None, None, :]
                if not m.any():
                    continue
                n1 = n[q1][:, None, None]
                n2 = n[q2][None, :, None]
                n3 = n[q3][None, None, :]
                if ch == 2:
                    F = n1 * n2 * (1 + n3) - (1 + n1) * (1 + n2) * n3
                elif ch == 3:
                    F = n1 * (1 + n2) * (1 + n3) - (1 + n1) * n2 * n3
                else:
                    F = (1 + n1) * (1 + n2) * (1 + n3) - n1 * n2 * n3
                with np.errstate(divide="ignore", invalid="ignore"):
                    term = c_s * F * np.exp(-d * d / sig ** 2) / (sig * math.sqrt(math.pi) * w0 * a * b * c)
                tot += float(term[m].sum())
                kept += int(m.sum())
        assert cnt[ch, i] == kept
        assert kept > 0
        assert abs(wp[ch, i] - tot / N ** 2) < 1e-11 * abs(tot / N ** 2)


# ------------------------------------------------------------------------------ rates

def test_band_folding_equivalence():
    """The primitive cell on a 2x2x4 mesh and its 1x1x2 supercell on a 2x2x2 mesh describe the
    same crystal: every channel's Γ, summed over degenerate groups, agrees.  This pins the 1/N and
    1/N² normalisations, the mass factors and the multi-atom cluster handling."""
    base = diamond_crystal()
    sc = supercell_crystal(base, 2)
    pp = oracle.Problem(base, *morse_ifcs(base, seed=0, perturb=0.0), (2, 2, 4))
    ps = oracle.Problem(sc, *morse_ifcs(sc, seed=0, perturb=0.0), (2, 2, 2))
    qS = [1, 5]                                       # supercell q indices checked
    for iqS in qS:
        cS = oracle.q_coords((2, 2, 2))[iqS]
        # primitive q's folding onto it: i3_P = i3_S and i3_S + 2
        prim = [int(cS[0] + 2 * (cS[1] + 2 * i3)) for i3 in (cS[2], cS[2] + 2)]
        mS = [iqS * 12 + j for j in range(12)]
        mP = [q * 6 + j for q in prim for j in range(6)]
        gS, _, _ = ps.rates(mS)
        gP, _, _ = pp.rates(mP)
        wS = ps.modes.omega[mS]
        wP = pp.modes.omega[mP]
        oS, oP = np.argsort(wS, kind="stable"), np.argsort(wP, kind="stable")
        assert np.allclose(wS[oS], wP[oP], rtol=1e-10)
        ws = wS[oS]
        groups = np.split(np.arange(12), np.where(np.diff(ws) > 1e-6 * ws.max())[0] + 1)
        for ch in range(5):
            floor = 1e-12 * np.abs(gP[ch]).max()      # channels that vanish by symmetry
            for g in groups:
                a = gS[ch][oS][g].sum()
                b = gP[ch][oP][g].sum()
                assert abs(a - b) <= 1e-9 * max(abs(a), abs(b)) + floor, (ch, g, a, b)


def test_gamma_nonnegative_for_hard_modes(prob3):
    """Γ >= 0 for every mode with ω >= 2σ (off-shell Gaussian tails can make softer modes negative)."""
    P = prob3
    modes = np.arange(3, P.nq * P.nb, 7)
    g, wp, cnt = P.rates(modes, channel_mask=0b11)
    hard = P.modes.omega[modes] >= 2 * P.sigma * oracle.SIGMA_THZ_TO_RADPS
    assert np.all(g[:2, hard] >= 0.0)
    assert np.all(cnt >= 0)


def test_excluded_modes_are_zero(prob3):
    g, wp, cnt = prob3.rates([0, 1, 2])
    assert np.all(g == 0) and np.all(wp == 0) and np.all(cnt == 0)


def test_kappa_isotropic_unperturbed(sys_clean):
    """The unperturbed crystal on a Γ-centred cubic-symmetric mesh gives κ ∝ I (3ph, RTA)."""
    P = oracle.Problem(*sys_clean, (4, 4, 4))
    g, _, _ = P.rates(channel_mask=0b11)
    k = P.kappa(g[0] + g[1])
    assert k[0, 0] > 0
    assert np.allclose(np.diag(k), k[0, 0], rtol=1e-6)
    assert np.abs(k - np.diag(np.diag(k))).max() < 1e-6 * k[0, 0]


def test_kappa_classical_limit(sys0):
    """At T = 1e8 K every mode carries k_B (x = ħω/k_B T ~ 1e-5, C/k_B = 1 - x²/12 + ...), so with
    Γ = 1 ps⁻¹ on every mode κ = k_B Σ v⊗v τ / (N V).  In Å, ps and Å³ the unit chain collapses to
    one factor, k_B [J/K] x 10⁴ (Å²/ps² -> m²/s²) x 10⁻¹² (ps) / 10⁻³⁰ (Å³) = 1.380649e-23 x 10²²."""
    c, p2, _, _ = sys0
    mesh = (3, 3, 3)
    m = oracle.harmonic(c, p2, mesh)
    g = np.ones_like(m.omega)
    k = oracle.kappa(c, m, 1e8, g, mesh)
    on = m.omega > 0
    v = m.vel[on]
    vol = abs(np.linalg.det(np.asarray(c.lattice)))
    ref = 1.380649e-23 * 1e22 * (v.T @ v) / (27 * vol)
    assert np.allclose(k, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())
    k2 = oracle.kappa(c, m, 1e8, 2.0 * g, mesh)                  # τ = 1/Γ
    assert np.allclose(k2, 0.5 * k, rtol=1e-14)


# ------------------------------------------------------------------------------ gradient

@pytest.fixture(scope="module")
def prob2(sys0):
    return oracle.Problem(*sys0, (2, 2, 2))


def test_gradient_euler_identity(prob2):
    """Γ is a quadratic form in Φ3 (3ph) and in Φ4 (4ph) at fixed modes: Σ Φ ∂Γ/∂Φ = 2Γ."""
    P = prob2
    modes = [4, 9, 23, 40]
    g, _, _ = P.rates(modes)
    rng = np.random.default_rng(0)
    dL = rng.standard_normal((5, len(modes)))
    L3 = float(np.sum(dL[:2] * g[:2]))
    L4 = float(np.sum(dL[2:] * g[2:]))
    g3, g4 = P.grad(modes, dL)
    assert abs(np.sum(P.phi3.phi * g3) - 2 * L3) < 1e-10 * abs(L3)
    assert abs(np.sum(P.phi4.phi * g4) - 2 * L4) < 1e-10 * abs(L4)


def test_gradient_central_differences(prob2):
    """Central differences of L along single cluster entries (exact for a quadratic up to rounding)."""
    P = prob2
    modes = [7, 22]
    rng = np.random.default_rng(1)
    dL = rng.standard_normal((5, len(modes)))
    g3, g4 = P.grad(modes, dL)
    for (order, c, k) in [(3, 5, 13), (3, 40, 2), (4, 3, 40), (4, 100, 7), (4, 200, 80)]:
        ifc = (P.phi3 if order == 3 else P.phi4)
        h = 1e-3 * max(abs(ifc.phi[c, k]), 1.0)
        vals = []
        for s in (+1, -1):
            mod = ifc.copy()
            mod.phi[c, k] += s * h
            Q = P.with_anharmonic(phi3=mod) if order == 3 else P.with_anharmonic(phi4=mod)
            gg, _, _ = Q.rates(modes)
            part = slice(0, 2) if order == 3 else slice(2, 5)      # Φ3 enters 3ph only, Φ4 4ph only
            vals.append(float(np.sum(dL[part] * gg[part])))
        fd = (vals[0] - vals[1]) / (2 * h)
        an = (g3 if order == 3 else g4)[c, k]
        gref = np.abs(g3 if order == 3 else g4).max()
        assert abs(fd - an) < 1e-7 * max(abs(an), 1e-3 * gref), (order, c, k, fd, an)


def _weight(ch, w0, ws, ns, sig):
    """c_s F_s g(Δ) / Π ω of one process, written out (Δ in the canonical parenthesisation)."""
    g = lambda d: math.exp(-d * d / sig ** 2) / (sig * math.sqrt(math.pi))
    if ch == 0:
        (a, b), (n1, n2) = ws, ns
        return (n1 - n2) * g((w0 + a) - b) / (w0 * a * b)
    if ch == 1:
        (a, b), (n1, n2) = ws, ns
        return 0.5 * (1 + n1 + n2) * g(w0 - (a + b)) / (w0 * a * b)
    (a, b, c), (n1, n2, n3) = ws, ns
    if ch == 2:
        return 0.5 * (n1 * n2 * (1 + n3) - (1 + n1) * (1 + n2) * n3) * g((w0 - c) + (a + b)) / (w0 * a * b * c)
    if ch == 3:
        return 0.5 * (n1 * (1 + n2) * (1 + n3) - (1 + n1) * n2 * n3) * g((w0 + a) - (b + c)) / (w0 * a * b * c)
    s = sorted((a, b, c))
    return ((1 + n1) * (1 + n2) * (1 + n3) - n1 * n2 * n3) / 6.0 * g(w0 - ((s[0] + s[1]) + s[2])) / (w0 * a * b * c)


@pytest.mark.parametrize("ch", [0, 1, 2, 3, 4])
def test_gamma_assembled_from_matrix_elements(prob3, ch):
    """Γ = C/N^k Σ_kept w |V|² rebuilt term by term from the oracle's kept list, its matrix
    elements (pinned by supercell finite differences) and the weights written out here, on the
    3x3x3 mesh; C3, C4 from the two-route unit derivation."""
    P = prob3
    nb, N = P.nb, P.nq
    qc = oracle.q_coords(P.mesh)
    mesh = np.asarray(P.mesh)
    w = P.modes.omega
    n = oracle.occupations(w, P.T)
    sig = P.sigma * oracle.SIGMA_THZ_TO_RADPS
    modes = [m for m in range(3, N * nb) if P.processes(ch, m).size > 0][:2]
    assert len(modes) == 2
    g, _, _ = P.rates(modes, channel_mask=1 << ch)
    idx = lambda c: int(c[0] + mesh[0] * (c[1] + mesh[1] * c[2]))
    for i, m0 in enumerate(modes):
        q0 = m0 // nb
        tot = 0.0
        for wd in P.processes(ch, m0).tolist():
            if ch < 2:
                q1, j1, j2 = oracle.decode3(wd, nb)
                s = 1 if ch == 0 else -1
                m1 = q1 * nb + j1
                m2 = idx((qc[q0] + s * qc[q1]) % mesh) * nb + j2
                V = P.v3(s, m0, m1, m2)
                tot += _weight(ch, w[m0], (w[m1], w[m2]), (n[m1], n[m2]), sig) * abs(V) ** 2
            else:
                q1, j1, q2, j2, j3 = oracle.decode4(wd, nb, N)
                s1, s2 = {2: (1, 1), 3: (1, -1), 4: (-1, -1)}[ch]
                m1, m2 = q1 * nb + j1, q2 * nb + j2
                m3 = idx((qc[q0] + s1 * qc[q1] + s2 * qc[q2]) % mesh) * nb + j3
                V = P.v4(s1, s2, m0, m1, m2, m3)
                tot += _weight(ch, w[m0], (w[m1], w[m2], w[m3]), (n[m1], n[m2], n[m3]), sig) * abs(V) ** 2
        ref = (oracle.C3 / N if ch < 2 else oracle.C4 / N ** 2) * tot
        assert abs(g[ch, i] - ref) <= 1e-11 * abs(ref) + 1e-300


def test_gamma_scales_quadratically(prob2):
    modes = [5, 30]
    g, _, _ = prob2.rates(modes)
    p4 = prob2.phi4.copy()
    p4.phi *= 1.7
    g2, _, _ = prob2.with_anharmonic(phi4=p4).rates(modes)
    assert np.allclose(g2[2:], 1.7 ** 2 * g[2:], rtol=1e-13)
    assert np.array_equal(g2[:2], g[:2])


# ------------------------------------------------------------------------------ adaptive broadening

def _with_velocities(P, vel):
    m = oracle.Modes(P.modes.omega.copy(), np.asarray(vel, np.float64).copy(), P.modes.evec, P.modes.eig)
    return oracle.Problem(P.crystal, P.phi2, P.phi3, P.phi4, P.mesh, P.T, P.sigma, P.sigma_adaptive, m)


@pytest.mark.parametrize("mesh", [(4, 4, 4), (2, 3, 4)])
def test_adaptive_sigma_closed_forms(sys_clean, mesh):
    """Adaptive width on the fcc lattice of the diamond cell, whose reciprocal vectors are
    (2π/a)(-1,1,1), (2π/a)(1,-1,1), (2π/a)(1,1,-1) (worked out by hand from a_i = (a/2)(0,1,1) and
    cyclic): for Δv = t x̂, each (Δv . b_k) = ±2π t/a, so σ = s (2π t / a) sqrt(Σ_k n_k^-2 / 6); for
    Δv = t (1,1,1)/√3 each (Δv . b_k) = 2π t/(a√3).  Also σ = 0 for equal velocities, symmetry in
    the pair and linearity in the scale s."""
    a = 5.43
    s = 1.7
    P0 = oracle.Problem(*sys_clean, mesh, sigma=s, sigma_adaptive=True)
    nm = P0.nq * P0.nb
    t = 3.25
    vel = np.zeros((nm, 3))
    vel[5] = (t, 0.0, 0.0)
    vel[6] = t * np.ones(3) / math.sqrt(3.0)
    vel[7] = (0.4, -1.1, 2.0)
    vel[8] = vel[7] + (0.0, 0.0, t)
    P = _with_velocities(P0, vel)
    inv_n2 = sum(1.0 / n ** 2 for n in mesh)
    k = 2.0 * math.pi * t / a
    assert P.sigma_of(5, 4) == pytest.approx(s * k * math.sqrt(inv_n2 / 6.0), rel=1e-14)
    assert P.sigma_of(6, 4) == pytest.approx(s * k / math.sqrt(3.0) * math.sqrt(inv_n2 / 6.0), rel=1e-14)
    assert P.sigma_of(8, 7) == pytest.approx(s * k * math.sqrt(inv_n2 / 6.0), rel=1e-14)   # Δv = t ẑ
    assert P.sigma_of(3, 4) == 0.0 and P.sigma_of(7, 7) == 0.0
    assert P.sigma_of(5, 6) == P.sigma_of(6, 5)
    P2 = oracle.Problem(P.crystal, P.phi2, P.phi3, P.phi4, P.mesh, P.T, 2.0 * s, True, P.modes)
    assert P2.sigma_of(5, 6) == pytest.approx(2.0 * P.sigma_of(5, 6), rel=1e-15)


def test_reciprocal_vectors_definition(sys0):
    """a_i . b_j = 2π δ_ij for the lattice of the crystal and for a skewed one."""
    for A in (sys0[0].lattice, np.array([[3.0, 0.2, -0.1], [0.5, 4.0, 0.3], [-0.2, 0.7, 5.5]])):
        B = oracle.reciprocal(A)
        assert np.abs(A @ B.T - 2.0 * math.pi * np.eye(3)).max() < 1e-13


def _brute_force_words_adaptive(P, ch, m0):
    """Unpruned enumeration with adaptive widths: momentum closure by searching all q for the
    Cartesian match modulo a reciprocal vector, σ from the quadratic form Δvᵀ Bᵀ diag(n^-2) B Δv
    (a different route to the same width).  Returns (words, borderline words whose decision is
    within 1e-9 relative of the window edge)."""
    nb, N = P.nb, P.nq
    B = oracle.reciprocal(P.crystal.lattice)
    G = B.T @ np.diag(1.0 / np.asarray(P.mesh, float) ** 2) @ B
    qs = oracle.q_cart(P.crystal.lattice, P.mesh)
    Binv = np.linalg.inv(B)
    w, v = P.modes.omega, P.modes.vel

    cache = {}

    def closure(target):
        key = tuple(np.round(target, 9))
        if key not in cache:
            for k in range(N):
                f = (qs[k] - target) @ Binv
                if np.all(np.abs(f - np.round(f)) < 1e-9):
                    cache[key] = k
                    break
        return cache[key]

    def sigma(ma, mb):
        dv = v[ma] - v[mb]
        return P.sigma * math.sqrt(max(dv @ G @ dv, 0.0) / 6.0)

    s1 = [1, -1, 1, 1, -1][ch]
    s2 = [0, 0, 1, -1, -1][ch]
    q0, j0 = divmod(m0, nb)
    excl = lambda q, j: q == 0 and j < 3
    out, border = [], set()
    if excl(q0, j0):
        return np.zeros(0, np.uint64), set()

    def decide(word, d, sg):
        if sg > 1e-9 and abs(abs(d) - 2.0 * sg) <= 1e-9 * max(abs(d), 2.0 * sg):
            border.add(word)
        if abs(sg - 1e-9) <= 1e-12:
            border.add(word)
        if sg > 1e-9 and abs(d) <= 2.0 * sg:      # adaptive widths at rounding-noise level are dropped
            out.append(word)

    for q1 in range(N):
        if ch < 2:
            q2 = closure(qs[q0] + s1 * qs[q1])
            for j1 in range(nb):
                for j2 in range(nb):
                    if excl(q1, j1) or excl(q2, j2):
                        continue
                    m1, m2 = q1 * nb + j1, q2 * nb + j2
                    d = w[m0] + s1 * w[m1] - w[m2]
                    decide((q1 * nb + j1) * nb + j2, d, sigma(m1, m2))
        else:
            for j1 in range(nb):
                for q2 in range(N):
                    q3 = closure(qs[q0] + s1 * qs[q1] + s2 * qs[q2])
                    for j2 in range(nb):
                        for j3 in range(nb):
                            if excl(q1, j1) or excl(q2, j2) or excl(q3, j3):
                                continue
                            m1, m2, m3 = q1 * nb + j1, q2 * nb + j2, q3 * nb + j3
                            d = w[m0] + s1 * w[m1] + s2 * w[m2] - w[m3]
                            decide((((q1 * nb + j1) * N + q2) * nb + j2) * nb + j3, d, sigma(m2, m3))
    return np.array(out, np.uint64), border


@pytest.mark.parametrize("mesh", [(1, 1, 1), (2, 2, 2), (3, 3, 3)])
def test_enumeration_adaptive_matches_brute_force(sys0, mesh):
    """Adaptive σ: the oracle's kept lists equal the brute-force ones up to candidates on the
    window edge.  On the 1x1x1 and 2x2x2 meshes every q equals -q modulo a reciprocal vector, so
    time reversal makes every group velocity vanish: σ is zero or rounding noise and nothing is
    kept."""
    P = oracle.Problem(*sys0, mesh, sigma=1.0, sigma_adaptive=True)
    nm = P.nq * P.nb
    rng = np.random.default_rng(2)
    total = 0
    n_pick = 4 if mesh != (3, 3, 3) else 2
    for m0 in sorted(set(rng.integers(3, nm, size=n_pick).tolist()) | {nm - 1}):
        for ch in range(5):
            a = P.processes(ch, m0)
            b, border = _brute_force_words_adaptive(P, ch, m0)
            diff = set(a.tolist()) ^ set(b.tolist())
            assert diff <= border, (ch, m0, len(diff))
            total += a.size
    if mesh != (3, 3, 3):
        assert total == 0
    else:
        assert total > 0


def test_weighted_phase_space_4ph_adaptive(sys0):
    """WP4+- with adaptive widths: (1/N²) Σ ½ F g(Δ, σ) / (ω ω1 ω2 ω3) over the oracle's kept list,
    with σ = s sqrt(Δv^T G Δv / 6), Δv = v2 - v3 (the two legs the free partner sum moves
    together), G = B^T diag(n^-2) B (the quadratic-form route), and the kept count."""
    P = oracle.Problem(*sys0, (3, 3, 3), sigma=1.0, sigma_adaptive=True)
    nb, N = P.nb, P.nq
    occ = oracle.occupations(P.modes.omega, P.T)
    w, v = P.modes.omega, P.modes.vel
    B = oracle.reciprocal(P.crystal.lattice)
    G = B.T @ np.diag(1.0 / np.asarray(P.mesh, float) ** 2) @ B
    qc = oracle.q_coords(P.mesh)
    modes = [m for m in range(3, N * nb) if P.processes(3, m).size > 0][:2]
    assert len(modes) == 2
    _, wp, cnt = P.rates(modes, channel_mask=8)
    for i, m0 in enumerate(modes):
        words = P.processes(3, m0)
        assert cnt[3, i] == words.size
        tot = 0.0
        for wd in words.tolist():
            q1, j1, q2, j2, j3 = oracle.decode4(wd, nb, N)
            c3 = (qc[m0 // nb] + qc[q1] - qc[q2]) % 3
            m1, m2 = q1 * nb + j1, q2 * nb + j2
            m3 = int(c3[0] + 3 * (c3[1] + 3 * c3[2])) * nb + j3
            dv = v[m2] - v[m3]
            sg = math.sqrt(dv @ G @ dv / 6.0)
            d = (w[m0] + w[m1]) - (w[m2] + w[m3])
            n1, n2, n3 = occ[m1], occ[m2], occ[m3]
            F = n1 * (1 + n2) * (1 + n3) - (1 + n1) * n2 * n3
            tot += 0.5 * F * math.exp(-d * d / sg ** 2) / (sg * math.sqrt(math.pi) * w[m0] * w[m1] * w[m2] * w[m3])
        assert abs(wp[3, i] - tot / N ** 2) < 1e-10 * abs(tot / N ** 2)


def test_weighted_phase_space_adaptive_brute_force(sys0):
    """WP3- with adaptive widths: (1/N) Σ ½ (1 + n' + n'') g(Δ, σ_λ'λ'') / (ω ω' ω'') (the ½ counts
    each unordered partner pair once), with σ by the quadratic-form route, over the brute-force
    kept set."""
    P = oracle.Problem(*sys0, (3, 3, 3), sigma=1.0, sigma_adaptive=True)
    nb, N = P.nb, P.nq
    occ = oracle.occupations(P.modes.omega, P.T)
    w, v = P.modes.omega, P.modes.vel
    B = oracle.reciprocal(P.crystal.lattice)
    G = B.T @ np.diag(1.0 / np.asarray(P.mesh, float) ** 2) @ B
    qc = oracle.q_coords(P.mesh)
    modes = [9, 40, 100]
    _, wp, cnt = P.rates(modes, channel_mask=2)
    for i, m0 in enumerate(modes):
        words, _ = _brute_force_words_adaptive(P, 1, m0)
        assert cnt[1, i] == words.size
        tot = 0.0
        for wd in words.tolist():
            q1, j1, j2 = oracle.decode3(wd, nb)
            q2c = (qc[m0 // nb] - qc[q1]) % 3
            m1, m2 = q1 * nb + j1, int(q2c[0] + 3 * (q2c[1] + 3 * q2c[2])) * nb + j2
            dv = v[m1] - v[m2]
            sg = math.sqrt(dv @ G @ dv / 6.0)
            d = w[m0] - w[m1] - w[m2]
            tot += 0.5 * (1 + occ[m1] + occ[m2]) * math.exp(-d * d / sg ** 2) / (sg * math.sqrt(math.pi) * w[m0] * w[m1] * w[m2])
        assert abs(wp[1, i] - tot / N) < 1e-11 * abs(tot / N)
