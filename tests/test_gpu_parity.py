"""GPU path vs the FP64 oracle, through the C interface (needs a GB300).

Process counts and process words must match bit for bit; Γ, WP and κ within 1e-10 relative
(FP64 path) or 1e-4 (mixed path).  Modes computed by the oracle are injected into the engine
(fc4_set_modes) so that both sides use identical ω bits and eigenvector gauges; the device's own
harmonic solution is compared with the oracle's separately."""
import numpy as np
import pytest

import oracle
from synth import morse_system, random_cluster_ifcs, supercell_crystal, diamond_crystal, morse_ifcs
from synth.sampling import sample_q
from tests.helpers import assert_close, make_engine, modes_of

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sys0():
    return morse_system(seed=0)


@pytest.fixture(scope="module")
def prob3(sys0):
    return oracle.Problem(*sys0, (3, 3, 3))


@pytest.fixture(scope="module")
def oracle3_all(prob3):
    return prob3.rates()


@pytest.fixture(scope="module")
def eng3(sys0, prob3):
    return make_engine(sys0, (3, 3, 3), precision=0, prob=prob3)


# ------------------------------------------------------------------------------ harmonic

@pytest.mark.parametrize("n", [3, 8])
def test_device_harmonic_matches_oracle(sys0, n):
    c, p2, p3, p4 = sys0
    e = make_engine(sys0, (n, n, n), inject=False)
    om, vel, ev = e.get_modes()
    ref = oracle.harmonic(c, p2, (n, n, n))
    w2max = (ref.omega ** 2).max()
    assert np.abs(om ** 2 - ref.omega ** 2).max() <= 1e-12 * w2max
    # eigenvectors up to a phase, and velocities, for modes with a non-degenerate frequency
    nb = e.nb
    for q in range(0, n ** 3, max(1, n ** 3 // 37)):
        w = ref.omega[q * nb:(q + 1) * nb]
        for j in range(nb):
            if q == 0 and j < 3:
                continue
            gap = np.min(np.abs(np.delete(w, j) - w[j]))
            if gap < 1e-6 * w.max():
                continue
            ov = abs(np.vdot(ref.evec[q][:, j], ev[q][:, j]))
            assert abs(ov - 1.0) < 1e-10
            assert np.abs(vel[q * nb + j] - ref.vel[q * nb + j]).max() < 1e-8 * max(1.0, np.abs(ref.vel).max())


def test_unstable_crystal_is_rejected():
    from paper_2510_00518_gb300 import Engine, FC4Error
    c = diamond_crystal()
    p2, p3, p4 = morse_ifcs(c, seed=0, harmonic_shells=2)      # second shell: imaginary modes
    with pytest.raises(FC4Error) as ei:
        Engine(c, p2, p3, p4, (3, 3, 3))
    assert ei.value.status == 5


# ------------------------------------------------------------------------------ processes

def test_process_words_bit_exact(eng3, prob3):
    rng = np.random.default_rng(0)
    modes = sorted(set(rng.integers(0, 162, size=14).tolist()) | {3, 161})
    eng3.rates(300.0, 0.1, 31, q_subset=[0])      # records σ for fc4_processes
    for m in modes:
        for ch in range(5):
            a = eng3.processes(ch, m)
            b = prob3.processes(ch, m)
            assert a.dtype == np.uint64
            assert np.array_equal(a, b), (m, ch, a.size, b.size)


# ------------------------------------------------------------------------------ rates

def test_rates_fp64_all_modes_3cubed(eng3, oracle3_all):
    g, wp, cnt = eng3.rates(300.0, 0.1, 31)
    torch.cuda.synchronize()
    G, WP, CNT = oracle3_all
    assert np.array_equal(cnt.cpu().numpy(), CNT)
    assert_close(g.cpu().numpy(), G, 1e-10, what="gamma")
    assert_close(wp.cpu().numpy(), WP, 1e-10, what="wp")


def test_rates_mixed_all_modes_3cubed(sys0, prob3, oracle3_all):
    e = make_engine(sys0, (3, 3, 3), precision=1, prob=prob3)
    g, wp, cnt = e.rates(300.0, 0.1, 31)
    G, WP, CNT = oracle3_all
    assert np.array_equal(cnt.cpu().numpy(), CNT)
    assert_close(g.cpu().numpy(), G, 1e-4, floor_frac=1e-6, what="gamma mixed")
    # κ with 3ph + 4ph
    k_gpu = e.kappa(300.0, g, 31).cpu().numpy()
    k_ref = prob3.kappa(G.sum(0))
    assert np.abs(k_gpu - k_ref).max() <= 1e-4 * np.abs(k_ref).max()


def test_kappa_fp64(eng3, prob3, oracle3_all):
    G = oracle3_all[0]
    gt = torch.tensor(G, device="cuda")
    k = eng3.kappa(300.0, gt, 31).cpu().numpy()
    kr = prob3.kappa(G.sum(0))
    assert np.abs(k - kr).max() <= 1e-10 * np.abs(kr).max()


def test_subset_order_and_masks(eng3, oracle3_all):
    """Γ of a mode does not depend on the subset it is computed in or on the other channels."""
    G = oracle3_all[0]
    sub = [26, 3, 14, 0]
    g, _, _ = eng3.rates(300.0, 0.1, 0b01010, q_subset=sub)
    g = g.cpu().numpy()
    ref = G[:, modes_of(sub, 6)]
    for ch in range(5):
        if (0b01010 >> ch) & 1:
            assert_close(g[ch], ref[ch], 1e-10, what=f"ch{ch}")
        else:
            assert np.all(g[ch] == 0)


def test_deterministic(eng3):
    a = eng3.rates(300.0, 0.1, 31)[0].cpu().numpy()
    b = eng3.rates(300.0, 0.1, 31)[0].cpu().numpy()
    assert np.array_equal(a, b)


def test_shards_sum_to_whole(eng3):
    """Mode-block shards computed separately equal the unsharded result bit for bit."""
    full = eng3.rates(300.0, 0.1, 31)[0].cpu().numpy()
    parts = [eng3.rates(300.0, 0.1, 31, q_subset=list(range(s, 27, 3)))[0].cpu().numpy() for s in range(3)]
    for s in range(3):
        assert np.array_equal(parts[s], full[:, modes_of(list(range(s, 27, 3)), 6)])


@pytest.mark.parametrize("mesh", [(1, 1, 1), (2, 3, 1), (2, 2, 4)])
def test_ragged_meshes(sys0, mesh):
    prob = oracle.Problem(*sys0, mesh)
    e = make_engine(sys0, mesh, prob=prob)
    g, wp, cnt = e.rates(700.0, 0.1, 31)
    G, WP, CNT = prob.with_T(700.0).rates()
    assert np.array_equal(cnt.cpu().numpy(), CNT)
    assert_close(g.cpu().numpy(), G, 1e-10, what=str(mesh))


def test_generic_clusters_four_atoms():
    """A 4-atom cell with random clusters on up to four distinct sites (no pair structure)."""
    c = supercell_crystal(diamond_crystal(), 2, masses=np.array([28.0855, 12.0, 72.6, 28.0855]))
    p2, _, _ = morse_ifcs(c, seed=3)
    p3 = random_cluster_ifcs(c, 3, 40, seed=4, scale=2.0)
    p4 = random_cluster_ifcs(c, 4, 60, seed=5, scale=5.0)
    sys = (c, p2, p3, p4)
    mesh = (2, 2, 2)
    prob = oracle.Problem(*sys, mesh)
    sub = [0, 3, 7]
    G, WP, CNT = prob.rates(modes_of(sub, 12))
    for prec, tol in ((0, 1e-10), (1, 1e-4)):
        e = make_engine(sys, mesh, precision=prec, prob=prob)
        g, wp, cnt = e.rates(300.0, 0.1, 31, q_subset=sub)
        assert np.array_equal(cnt.cpu().numpy(), CNT)
        assert_close(g.cpu().numpy(), G, tol, floor_frac=1e-6 if prec else 1e-12, what=f"prec{prec}")


def test_empty_subset_and_invalid_arguments(eng3):
    from paper_2510_00518_gb300 import FC4Error
    g = torch.zeros((5, 0), dtype=torch.float64, device="cuda")
    eng3.rates(300.0, 0.1, 31, q_subset=np.zeros(0, np.int32), out=(g, g, g.long()))
    for bad in [dict(T=-1.0), dict(sigma_thz=0.0), dict(channel_mask=64), dict(q_subset=[27])]:
        kw = dict(T=300.0, sigma_thz=0.1, channel_mask=31, q_subset=[0])
        kw.update(bad)
        with pytest.raises(FC4Error) as ei:
            eng3.rates(**kw)
        assert ei.value.status == 1


def test_config_8cubed_sampled_modes(sys0):
    """Full 8x8x8 mesh, all modes on the GPU (the bench's launch configuration); sampled modes
    against the oracle computed one by one."""
    mesh = (8, 8, 8)
    prob = oracle.Problem(*sys0, mesh)
    for prec, tol in ((1, 1e-4),):
        e = make_engine(sys0, mesh, precision=prec, prob=prob)
        g, wp, cnt = e.rates(300.0, 0.1, 31)
        g, cnt = g.cpu().numpy(), cnt.cpu().numpy()
        qs = sample_q(512, 1, seed=0)
        ms = modes_of(qs, 6)[[1, 4]]
        G, WP, CNT = prob.rates(ms)
        assert np.array_equal(cnt[:, ms], CNT)
        assert_close(g[:, ms], G, tol, floor_frac=1e-6, what="8^3")


def test_sharded_rates_kappa_single_process(eng3, oracle3_all, prob3):
    """The sharding helper on one process (no process group): its q block is the whole mesh and
    κ equals the oracle's."""
    from paper_2510_00518_gb300.dist import sharded_rates_kappa
    qs, g, k = sharded_rates_kappa(eng3, 300.0, 0.1, 31)
    assert np.array_equal(qs, np.arange(27))
    kr = prob3.kappa(oracle3_all[0].sum(0))
    assert np.abs(k.cpu().numpy() - kr).max() <= 1e-10 * np.abs(kr).max()


def test_triangular_domain_matches_rectangle(sys0, prob3):
    """Partner-swap symmetric Φ4: one process per swapped pair is evaluated (stats), with the
    rectangular kept counts and Γ.  Breaking the leg-exchange symmetry of one cluster entry by
    1e-9 turns the triangle off (every kept process evaluated) and moves Γ by that much only."""
    G = prob3.rates()[0]
    for prec, tol in ((0, 1e-10), (1, 1e-4)):
        e = make_engine(sys0, (3, 3, 3), precision=prec, prob=prob3)
        g_tri, _, c_tri = e.rates(300.0, 0.1, 0b11100)
        st = e.stats()
        assert np.array_equal(c_tri.cpu().numpy()[2:], prob3.rates(channel_mask=0b11100)[2][2:])
        assert all(st["evaluated"][ch] < st["kept"][ch] for ch in (2, 3, 4))
        assert_close(g_tri.cpu().numpy()[2:], G[2:], tol, floor_frac=1e-6 if prec else 1e-12, what="triangle")
        # an entry with distinct Cartesian indices on legs 1, 2 and on legs 2, 3, so that both
        # leg exchanges map it to another entry (the on-site Φ[αααα] terms map to themselves)
        p4 = sys0[3].phi.copy()
        k = np.arange(81)
        be, ga, de = (k // 9) % 3, (k // 3) % 3, k % 3
        cand = np.where((be != ga) & (ga != de), np.abs(p4), 0.0)
        i, k = np.unravel_index(cand.argmax(), cand.shape)
        p4[i, k] *= 1.0 + 1e-9                        # well above the 1e-12 symmetry tolerance
        e.update_anharmonic(None, p4)
        g_rect, _, c_rect = e.rates(300.0, 0.1, 0b11100)
        st = e.stats()
        assert all(st["evaluated"][ch] == st["kept"][ch] for ch in (2, 3, 4))
        assert np.array_equal(c_rect.cpu().numpy(), c_tri.cpu().numpy())
        assert_close(g_rect.cpu().numpy()[2:], g_tri.cpu().numpy()[2:], 1e-5 if prec else 1e-8,
                     floor_frac=1e-6 if prec else 1e-12, what="rectangle vs triangle")
