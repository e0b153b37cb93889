"""Irreducible q-points (host calls of libfc4, no GPU) against the oracle and brute force.

The mode loops of Algorithms 1 and 3-5 run over the irreducible q-points (N_list).  Pinned here:
- the unperturbed Morse diamond has the 48 operations of its point group (m-3m), and they form
  a group; the seeded bond perturbations leave the identity only;
- every operation is a symmetry of the harmonic problem: ω(W^-T k) = ω(k) from the oracle's own
  dynamical matrix;
- the orbits match a brute-force closure, and the fcc Γ-centred 4x4x4 and 8x8x8 meshes have the
  textbook 8 and 29 irreducible points;
- the oracle's Γ (all five channels) is constant on a star up to degenerate-branch averaging, for
  the symmetric crystal, and under q -> -q for the perturbed one;
- rates and κ of the whole mesh expanded from the irreducible points equal the oracle's full-mesh
  ones for a fixed width;
- the adaptive width is not constant on a star (degenerate modes' Hellmann-Feynman velocities
  depend on the eigenvector basis), which is why the irreducible-point path takes a fixed width.
"""
import itertools

import numpy as np
import pytest

import oracle
from synth import morse_system

S = pytest.importorskip("paper_2510_00518_gb300.symmetry")


@pytest.fixture(scope="module", autouse=True)
def _library():
    from paper_2510_00518_gb300 import build as fc4_build
    fc4_build.build()                      # host-only calls: the library must exist, no GPU needed


@pytest.fixture(scope="module")
def clean():
    return morse_system(seed=0, perturb=0.0)


@pytest.fixture(scope="module")
def ops(clean):
    return S.symmetry_ops(*clean)


def mesh_map(W, mesh):
    """Index map q -> q' of k' = W^-T k on a Γ-centred mesh (None if the mesh is not kept)."""
    M = np.rint(np.linalg.inv(W).T).astype(int)
    n = np.asarray(mesh)
    qc = oracle.q_coords(mesh)
    out = []
    for c in qc:
        num = M @ (c * (np.prod(n) // n))          # k' scaled by the product of the mesh sizes
        kp = num * n
        if np.any(kp % np.prod(n)):
            return None
        i = (kp // np.prod(n)) % n
        out.append(int(i[0] + n[0] * (i[1] + n[1] * i[2])))
    return np.array(out)


def degenerate_mean(values, omega, nb, tol=1e-5):
    """Average per-mode values over branches whose ω lie within tol of a neighbour (per q)."""
    v = np.asarray(values, float).reshape(-1, nb).copy()
    w = np.asarray(omega, float).reshape(-1, nb)
    for q in range(v.shape[0]):
        order = np.argsort(w[q], kind="stable")
        groups, cur = [], [order[0]]
        for a, b in zip(order[:-1], order[1:]):
            if w[q][b] - w[q][a] > tol:
                groups.append(cur)
                cur = []
            cur.append(b)
        groups.append(cur)
        for g in groups:
            v[q, g] = v[q, g].mean()
    return v.reshape(-1)


def test_diamond_point_group(clean, ops):
    rot, trans = ops
    assert len(rot) == 48
    assert any(np.array_equal(W, np.eye(3, dtype=int)) for W in rot)
    keys = {W.tobytes() for W in rot.astype(np.int32)}
    for A, B in itertools.product(rot, rot):                # closed under products
        assert (A @ B).astype(np.int32).tobytes() in keys
    c = clean[0]
    L = np.asarray(c.lattice)
    for W in rot:                                           # Cartesian images are rotations
        Sc = L.T @ W @ np.linalg.inv(L.T)
        assert np.allclose(Sc @ Sc.T, np.eye(3), atol=1e-12)


def test_bond_perturbations_leave_the_identity():
    rot, _ = S.symmetry_ops(*morse_system(seed=0, perturb=0.01))
    assert len(rot) == 1 and np.array_equal(rot[0], np.eye(3))


def test_structure_ops_without_force_constants_check(clean):
    """A perturbed crystal still has the diamond structure: with only Φ2 of the clean crystal the
    48 operations return; with the perturbed Φ3 they do not."""
    c, p2, p3, _ = clean
    assert len(S.symmetry_ops(c, p2)[0]) == 48
    q2, q3 = morse_system(seed=0, perturb=0.01)[1:3]
    assert len(S.symmetry_ops(c, p2, q3)[0]) == 1


def test_operations_keep_the_harmonic_frequencies(clean, ops):
    mesh = (4, 4, 4)
    modes = oracle.harmonic(clean[0], clean[1], mesh)
    w = modes.omega.reshape(-1, clean[0].nb)
    for W in ops[0]:
        m = mesh_map(W, mesh)
        assert m is not None
        assert np.allclose(w[m], w, rtol=0, atol=1e-10 * w.max())


@pytest.mark.parametrize("mesh", [(4, 4, 4), (3, 3, 3), (4, 4, 2), (5, 3, 4), (8, 8, 8)])
@pytest.mark.parametrize("tr", [True, False])
def test_orbits_match_brute_force(ops, mesh, tr):
    rep, irr = S.irreducible_q(mesh, ops[0], time_reversal=tr)
    N = int(np.prod(mesh))
    maps = [m for m in (mesh_map(W, mesh) for W in ops[0]) if m is not None]
    if tr:
        n = np.asarray(mesh)
        qc = oracle.q_coords(mesh)
        neg = (-qc) % n
        maps.append(neg[:, 0] + n[0] * (neg[:, 1] + n[1] * neg[:, 2]))
    ref = -np.ones(N, int)
    for q in range(N):
        if ref[q] >= 0:
            continue
        orbit, todo = {q}, [q]
        while todo:
            p = todo.pop()
            for m in maps:
                if m[p] not in orbit:
                    orbit.add(int(m[p]))
                    todo.append(int(m[p]))
        for p in orbit:
            ref[p] = q
    assert np.array_equal(rep, ref)
    assert np.array_equal(irr, np.flatnonzero(ref == np.arange(N)))


def test_fcc_textbook_counts(ops):
    assert S.irreducible_q((4, 4, 4), ops[0])[1].size == 8
    assert S.irreducible_q((8, 8, 8), ops[0])[1].size == 29


def test_gamma_constant_on_a_star(clean, ops):
    """Oracle Γ, all channels, on every q of the largest star of the 3x3x3 mesh."""
    mesh = (3, 3, 3)
    P = oracle.Problem(*clean, mesh)
    nb = P.nb
    rep, _ = S.irreducible_q(mesh, ops[0])
    r = np.bincount(rep).argmax()
    star = np.flatnonzero(rep == r)
    assert star.size > 1
    modes = (star[:, None] * nb + np.arange(nb)).reshape(-1)
    g, wp, cnt = P.rates(modes)
    om = P.modes.omega[modes]
    for ch in range(5):
        v = degenerate_mean(g[ch], om, nb).reshape(star.size, nb)
        assert np.allclose(v, v[0], rtol=1e-10, atol=1e-14 * max(1.0, np.abs(v).max()))
        assert np.array_equal(cnt[ch].reshape(star.size, nb).sum(1), np.full(star.size, cnt[ch][:nb].sum()))
    assert g[3].sum() > 0


def test_time_reversal_without_spatial_symmetry():
    """Perturbed crystal: Γ(-q) = Γ(q) in every channel for the pairs of the 3x3x3 mesh."""
    sysp = morse_system(seed=0, perturb=0.01)
    mesh = (3, 3, 3)
    P = oracle.Problem(*sysp, mesh)
    nb = P.nb
    rep, irr = S.irreducible_q(mesh, np.eye(3, dtype=np.int32)[None])
    assert irr.size == 14
    pairs = [(int(rep[q]), q) for q in range(27) if rep[q] != q][:3]
    for a, b in pairs:
        modes = np.r_[a * nb + np.arange(nb), b * nb + np.arange(nb)]
        g, _, cnt = P.rates(modes)
        om = P.modes.omega[modes]
        for ch in range(5):
            v = degenerate_mean(g[ch], om, nb).reshape(2, nb)
            assert np.allclose(v[1], v[0], rtol=1e-10, atol=1e-14 * max(1.0, np.abs(v).max()))


def test_expanded_rates_and_kappa_equal_the_full_mesh(clean, ops):
    """Three-phonon rates of the 4x4x4 mesh from its 8 irreducible points (library expansion)
    against the oracle on every mode; κ from both."""
    mesh = (4, 4, 4)
    P = oracle.Problem(*clean, mesh)
    nb, N = P.nb, P.nq
    rep, irr = S.irreducible_q(mesh, ops[0])
    assert irr.size == 8
    g_full, wp_full, _ = P.rates(None, channel_mask=3)
    modes = (irr[:, None] * nb + np.arange(nb)).reshape(-1)
    g_irr, wp_irr, _ = P.rates(modes, channel_mask=3)
    ex = S.expand_irreducible(mesh, nb, rep, P.modes.omega, np.stack([g_irr, wp_irr]))
    for ch in (0, 1):
        ref = degenerate_mean(g_full[ch], P.modes.omega, nb)
        assert np.allclose(ex[0][ch], ref, rtol=1e-10, atol=1e-14 * np.abs(ref).max())
        refw = degenerate_mean(wp_full[ch], P.modes.omega, nb)
        assert np.allclose(ex[1][ch], refw, rtol=1e-10, atol=1e-14 * np.abs(refw).max())
    k_full = P.kappa(g_full.sum(0))
    k_ex = P.kappa(ex[0].sum(0))
    assert np.allclose(k_ex, k_full, rtol=1e-9, atol=1e-12 * np.abs(k_full).max())


def test_host_calls_reject_bad_input(clean, ops):
    lib = S.load()
    with pytest.raises(S.FC4Error):
        S.symmetry_ops(*clean, max_ops=4)               # 48 found
    assert "48 operations found" in lib.fc4_last_error(None).decode()
    with pytest.raises(S.FC4Error):
        S.irreducible_q((4, 4, 0), ops[0])
    import ctypes
    from paper_2510_00518_gb300 import _structs
    keep = []
    c, i2, i3, i4 = _structs(*clean, keep)
    n = ctypes.c_int(-1)
    assert lib.fc4_symmetry_ops(ctypes.byref(c), ctypes.byref(i2), ctypes.byref(i3), ctypes.byref(i4),
                                0.0, 0, None, None, ctypes.cast(ctypes.pointer(n), ctypes.c_void_p)) == 0
    assert n.value == 48                                 # max_ops = 0: count only
    with pytest.raises(S.FC4Error):
        S.irreducible_q((4, 4, 4), np.array([[[2, 0, 0], [0, 1, 0], [0, 0, 1]]], np.int32))
    rep = np.arange(8, dtype=np.int32)
    rep[3] = 5                                   # not a representative map (5 > 3)
    with pytest.raises(S.FC4Error):
        S.expand_irreducible((2, 2, 2), 6, rep, np.ones(48), np.zeros((1, 48)))
    assert "rep" in lib.fc4_last_error(None).decode()


def test_adaptive_width_is_not_star_invariant(clean, ops):
    """With the adaptive width the oracle's 3ph rates differ across a star by far more than
    rounding: the reason the irreducible-point path is restricted to a fixed width."""
    mesh = (4, 4, 4)
    P = oracle.Problem(*clean, mesh, sigma=1.0, sigma_adaptive=True)
    nb = P.nb
    rep, irr = S.irreducible_q(mesh, ops[0])
    worst = 0.0
    for r in irr[1:]:
        star = np.flatnonzero(rep == r)
        modes = (star[:, None] * nb + np.arange(nb)).reshape(-1)
        g, _, _ = P.rates(modes, channel_mask=3)
        v = degenerate_mean(g.sum(0), P.modes.omega[modes], nb).reshape(star.size, nb)
        worst = max(worst, float(np.max(np.abs(v - v[0]) / np.maximum(np.abs(v[0]), 1e-12))))
    assert worst > 1e-3


def _batch_system(seed):
    from synth.morse import batch_crystal, morse_ifcs
    c, _ = batch_crystal(seed)
    return (c,) + tuple(morse_ifcs(c, None, seed=seed, perturb=0.0))


def test_zincblende_point_group():
    """Two unequal masses on the diamond sites: the 24 operations of -43m; with q -> -q the
    fcc 4x4x4 mesh again has 8 irreducible points (10 without)."""
    sysz = _batch_system(0)
    rot, trans = S.symmetry_ops(*sysz)
    assert len(rot) == 24
    assert np.allclose(trans, 0.0)                           # no operation swaps the two sites
    assert S.irreducible_q((4, 4, 4), rot)[1].size == 8
    assert S.irreducible_q((4, 4, 4), rot, time_reversal=False)[1].size == 10


@pytest.mark.parametrize("seed", [0, 1])
def test_gamma_constant_on_every_star_of_a_small_mesh(seed):
    """Zincblende (24 operations) and a four-atom 1x1x2 supercell with four masses (2
    operations): the oracle's 3ph rates on every q of the 3x3x3 mesh are constant on each star
    of the library's orbits (with q -> -q)."""
    sysb = _batch_system(seed)
    rot, _ = S.symmetry_ops(*sysb)
    mesh = (3, 3, 3)
    P = oracle.Problem(*sysb, mesh)
    nb = P.nb
    rep, irr = S.irreducible_q(mesh, rot)
    assert irr.size < 27
    g, _, _ = P.rates(None, channel_mask=3)
    for ch in (0, 1):
        v = degenerate_mean(g[ch], P.modes.omega, nb).reshape(27, nb)
        ref = v[rep]
        assert np.allclose(v, ref, rtol=1e-10, atol=1e-14 * np.abs(v).max())
