"""Adaptive broadening on the GPU against the FP64 oracle, through the C interface (needs a GB300).

σ of each process comes from the group velocities of the two legs that the free partner sum
moves together; the FP32 prefilter on the velocity projections decides the clear cases and the
exact FP64 test the rest, so kept counts and process words must match the oracle bit for bit;
Γ within 1e-10 (FP64 path) or 1e-4 (mixed path)."""
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
def prob3a(sys0):
    return oracle.Problem(*sys0, (3, 3, 3), sigma=1.0, sigma_adaptive=True)


@pytest.fixture(scope="module")
def oracle3a(prob3a):
    return prob3a.rates()


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
def test_rates_adaptive_all_modes_3cubed(sys0, prob3a, oracle3a, prec, tol):
    e = make_engine(sys0, (3, 3, 3), precision=prec, prob=prob3a)
    g, wp, cnt = e.rates(300.0, 1.0, 31, adaptive=True)
    G, WP, CNT = oracle3a
    assert CNT[2:].sum() > 0
    assert np.array_equal(cnt.cpu().numpy(), CNT)
    assert_close(g.cpu().numpy(), G, tol, floor_frac=1e-6 if prec else 1e-12, what="gamma adaptive")
    assert_close(wp.cpu().numpy(), WP, tol, floor_frac=1e-6 if prec else 1e-12, what="wp adaptive")


def test_process_words_adaptive_bit_exact(sys0, prob3a):
    e = make_engine(sys0, (3, 3, 3), precision=1, prob=prob3a)
    e.rates(300.0, 1.0, 31, q_subset=[0], adaptive=True)       # records the adaptive σ
    for m in [3, 29, 77, 118, 161]:
        for ch in range(5):
            assert np.array_equal(e.processes(ch, m), prob3a.processes(ch, m)), (m, ch)


def test_adaptive_and_fixed_calls_interleave(sys0, prob3a, oracle3a):
    """A fixed-σ call between adaptive calls leaves neither result changed."""
    prob = oracle.Problem(*sys0, (3, 3, 3), modes=prob3a.modes)
    e = make_engine(sys0, (3, 3, 3), precision=1, prob=prob3a)
    sub = [4, 17]
    a1 = e.rates(300.0, 1.0, 31, q_subset=sub, adaptive=True)[0].cpu().numpy()
    f = e.rates(300.0, 0.1, 31, q_subset=sub)[0].cpu().numpy()
    a2 = e.rates(300.0, 1.0, 31, q_subset=sub, adaptive=True)[0].cpu().numpy()
    assert np.array_equal(a1, a2)
    assert_close(a1, oracle3a[0][:, modes_of(sub, 6)], 1e-4, floor_frac=1e-6, what="adaptive")
    assert_close(f, prob.rates(modes_of(sub, 6))[0], 1e-4, floor_frac=1e-6, what="fixed")


@pytest.mark.parametrize("mesh", [(3, 4, 2), (5, 3, 3)])
def test_adaptive_ragged_meshes(sys0, mesh):
    prob = oracle.Problem(*sys0, mesh, sigma=0.7, sigma_adaptive=True)
    rng = np.random.default_rng(sum(mesh))
    sub = sorted(set(rng.integers(0, prob.nq, size=3).tolist()))
    G, WP, CNT = prob.with_T(700.0).rates(modes_of(sub, 6))
    for prec, tol in ((0, 1e-10), (1, 1e-4)):
        e = make_engine(sys0, mesh, precision=prec, prob=prob)
        g, wp, cnt = e.rates(700.0, 0.7, 31, q_subset=sub, adaptive=True)
        assert np.array_equal(cnt.cpu().numpy(), CNT)
        assert_close(g.cpu().numpy(), G, tol, floor_frac=1e-6 if prec else 1e-12, what=f"{mesh} prec{prec}")


def test_adaptive_generic_clusters_four_atoms():
    """The general (untiled) kernels with adaptive σ: 4-atom cell, random clusters, 3x3x2 mesh."""
    c = supercell_crystal(diamond_crystal(), 2, masses=np.array([28.0855, 12.0, 72.6, 28.0855]))
    p2, _, _ = morse_ifcs(c, seed=3)
    p3 = random_cluster_ifcs(c, 3, 40, seed=4, scale=2.0)
    p4 = random_cluster_ifcs(c, 4, 60, seed=5, scale=5.0)
    sys = (c, p2, p3, p4)
    mesh = (3, 3, 2)
    prob = oracle.Problem(*sys, mesh, sigma=1.0, sigma_adaptive=True)
    sub = [1, 7]
    G, WP, CNT = prob.rates(modes_of(sub, 12))
    assert CNT[2:].sum() > 0
    for prec, tol in ((0, 1e-10), (1, 1e-4)):
        e = make_engine(sys, mesh, precision=prec, prob=prob)
        g, wp, cnt = e.rates(300.0, 1.0, 31, q_subset=sub, adaptive=True)
        assert np.array_equal(cnt.cpu().numpy(), CNT)
        assert_close(g.cpu().numpy(), G, tol, floor_frac=1e-6 if prec else 1e-12, what=f"prec{prec}")


def test_adaptive_backward_matches_oracle_gradient(sys0, prob3a):
    e = make_engine(sys0, (3, 3, 3), precision=0, prob=prob3a)
    sub = [13]
    modes = modes_of(sub, 6)
    dL = np.random.default_rng(7).standard_normal((5, modes.size))
    e.rates(300.0, 1.0, 31, q_subset=sub, adaptive=True)
    d3, d4 = e.backward(torch.tensor(dL, device="cuda"))
    g3, g4 = prob3a.grad(modes, dL)
    assert_close(d3.cpu().numpy().reshape(-1), g3.reshape(-1), 1e-8, floor_frac=1e-9, what="dphi3")
    assert_close(d4.cpu().numpy().reshape(-1), g4.reshape(-1), 1e-8, floor_frac=1e-9, what="dphi4")


def test_time_reversal_mesh_keeps_nothing(sys0):
    """On a 2x2x2 mesh every q equals -q modulo a reciprocal vector, so time reversal makes every
    group velocity vanish: each adaptive σ is zero or rounding noise, and nothing is kept."""
    prob = oracle.Problem(*sys0, (2, 2, 2), sigma=1.0, sigma_adaptive=True)
    e = make_engine(sys0, (2, 2, 2), precision=1, prob=prob)
    g, wp, cnt = e.rates(300.0, 1.0, 31, adaptive=True)
    assert int(cnt.sum()) == 0 and float(g.abs().sum()) == 0.0


def test_precision_form_16cubed_mixed_vs_fp64():
    """The 16x16x16 seed-1 crystal with adaptive σ (s = 1), device harmonic modes: sampled q of the
    145-point sample, mixed path against the FP64 GPU path (kept counts identical, Γ within 1e-4)."""
    sys1 = morse_system(seed=1)
    mesh = (16, 16, 16)
    qs = sample_q(4096, 145, seed=1)[:1].tolist()
    e64 = make_engine(sys1, mesh, precision=0, inject=False)
    om, vel, ev = e64.get_modes()
    e32 = make_engine(sys1, mesh, precision=1, inject=False)
    e32.set_modes(om, vel, ev)
    g64, _, c64 = e64.rates(300.0, 1.0, 31, q_subset=qs, adaptive=True)
    g32, _, c32 = e32.rates(300.0, 1.0, 31, q_subset=qs, adaptive=True)
    c64, c32 = c64.cpu().numpy(), c32.cpu().numpy()
    assert c64[2:].sum() > 0
    assert np.array_equal(c64, c32)
    assert_close(g32.cpu().numpy(), g64.cpu().numpy(), 1e-4, floor_frac=1e-6, what="16^3 adaptive")
