"""Adjoint kernels (fc4_rates_backward, fc4_kappa_backward) against the oracle's analytic gradient
and against central finite differences of the GPU forward pass (needs a GB300).

Γ is an exact quadratic form in Φ3 (3ph) and in Φ4 (4ph) at fixed modes and σ, so central
differences are exact up to rounding; the bar is 1e-6 relative."""
import numpy as np
import pytest

import oracle
from synth import morse_system
from tests.helpers import assert_close, make_engine, modes_of

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sysm():
    return morse_system(seed=0)


@pytest.mark.parametrize("mesh,sub", [((3, 3, 3), [13]), ((4, 4, 4), [22])])
def test_rates_backward_matches_oracle_gradient(sysm, mesh, sub):
    """3x3x3, and the 4x4x4 mesh of the differentiation workload's oracle comparison."""
    prob = oracle.Problem(*sysm, mesh)
    e = make_engine(sysm, mesh, precision=0, prob=prob)
    modes = modes_of(sub, 6)
    rng = np.random.default_rng(2)
    dL = rng.standard_normal((5, modes.size))
    e.rates(300.0, 0.1, 31, q_subset=sub)
    d3, d4 = e.backward(torch.tensor(dL, device="cuda"))
    g3, g4 = prob.grad(modes, dL)
    # different FP64 summation orders over sums with cancellation: 1e-8 relative, floor 1e-9 max
    assert_close(d3.cpu().numpy().reshape(-1), g3.reshape(-1), 1e-8, floor_frac=1e-9, what="dphi3")
    assert_close(d4.cpu().numpy().reshape(-1), g4.reshape(-1), 1e-8, floor_frac=1e-9, what="dphi4")


def test_rates_backward_four_atom_cell():
    """A 4-atom cell with random clusters on up to four distinct sites (no pair structure)."""
    from synth import diamond_crystal, supercell_crystal, morse_ifcs, random_cluster_ifcs
    c = supercell_crystal(diamond_crystal(), 2, masses=np.array([28.0855, 12.0, 72.6, 28.0855]))
    p2, _, _ = morse_ifcs(c, seed=3)
    p3 = random_cluster_ifcs(c, 3, 40, seed=4, scale=2.0)
    p4 = random_cluster_ifcs(c, 4, 60, seed=5, scale=5.0)
    sys4 = (c, p2, p3, p4)
    mesh = (2, 2, 2)
    prob = oracle.Problem(*sys4, mesh)
    e = make_engine(sys4, mesh, precision=0, prob=prob)
    sub = [3]
    modes = modes_of(sub, 12)
    dL = np.random.default_rng(7).standard_normal((5, modes.size))
    e.rates(300.0, 0.1, 31, q_subset=sub)
    d3, d4 = e.backward(torch.tensor(dL, device="cuda"))
    g3, g4 = prob.grad(modes, dL)
    assert_close(d3.cpu().numpy().reshape(-1), g3.reshape(-1), 1e-8, floor_frac=1e-9, what="dphi3 (4 atoms)")
    assert_close(d4.cpu().numpy().reshape(-1), g4.reshape(-1), 1e-8, floor_frac=1e-9, what="dphi4 (4 atoms)")


def test_rates_backward_deterministic_and_euler(sysm):
    mesh = (4, 4, 4)
    prob = oracle.Problem(*sysm, mesh)
    e = make_engine(sysm, mesh, precision=0, prob=prob)
    sub = [5, 21, 42]
    g, _, _ = e.rates(300.0, 0.1, 31, q_subset=sub)
    dL = torch.tensor(np.random.default_rng(4).standard_normal(tuple(g.shape)), device="cuda")
    a3, a4 = e.backward(dL)
    b3, b4 = e.backward(dL)
    assert torch.equal(a3, b3) and torch.equal(a4, b4)
    # Euler: Σ Φ dL/dΦ = 2 L per order
    L3 = float((dL[:2] * g[:2]).sum())
    L4 = float((dL[2:] * g[2:]).sum())
    p3 = torch.tensor(sysm[2].phi, device="cuda")
    p4 = torch.tensor(sysm[3].phi, device="cuda")
    assert abs(float((p3 * a3).sum()) - 2 * L3) < 1e-9 * abs(L3)
    assert abs(float((p4 * a4).sum()) - 2 * L4) < 1e-9 * abs(L4)


def test_kappa_gradient_autograd_vs_finite_differences(sysm):
    """dκ_xx/dΦ through torch.autograd (Rates + Kappa functions) vs central differences of the
    GPU forward pass on seeded cluster entries (3x3x3 mesh, all modes, FP64)."""
    from paper_2510_00518_gb300 import rates_fn, kappa_fn
    mesh = (3, 3, 3)
    prob = oracle.Problem(*sysm, mesh)
    e = make_engine(sysm, mesh, precision=0, prob=prob)
    p3 = torch.tensor(sysm[2].phi, dtype=torch.float64, requires_grad=True)
    p4 = torch.tensor(sysm[3].phi, dtype=torch.float64, requires_grad=True)

    def kxx(a3, a4):
        g = rates_fn(a3, a4, e, 300.0, 0.1, 31)
        return kappa_fn(g, e, 300.0, 31)[0, 0]

    k = kxx(p3, p4)
    k.backward()
    rng = np.random.default_rng(16)
    picks = [(3, int(c), int(x)) for c, x in zip(rng.integers(0, p3.shape[0], 8), rng.integers(0, 27, 8))] + \
            [(4, int(c), int(x)) for c, x in zip(rng.integers(0, p4.shape[0], 8), rng.integers(0, 81, 8))]
    for order, c, x in picks:
        base = (p3 if order == 3 else p4).detach().clone()
        h = 1e-5 * max(abs(float(base[c, x])), 1.0)
        vals = []
        for sgn in (1, -1):
            mod = base.clone()
            mod[c, x] += sgn * h
            a3 = mod if order == 3 else p3.detach()
            a4 = mod if order == 4 else p4.detach()
            with torch.no_grad():
                vals.append(float(kxx(a3, a4)))
        fd = (vals[0] - vals[1]) / (2 * h)
        an = float((p3.grad if order == 3 else p4.grad)[c, x])
        noise = 1e-15 * abs(float(k.detach())) / h            # rounding of κ, amplified by the difference
        assert abs(fd - an) <= 1e-6 * abs(an) + noise, (order, c, x, fd, an, noise)
    e.update_anharmonic(sysm[2].phi, sysm[3].phi)


def test_rates_gradient_8cubed_finite_differences(sysm):
    """The differentiation workload on the 8x8x8 mesh: dL/dΦ of L = Σ_ch,λ G Γ_ch(λ) over the six
    modes of one seeded q point (FP64), against central differences of the GPU forward pass on 16
    seeded cluster entries (8 of Φ3, 8 of Φ4; h = 1e-5 relative)."""
    from synth.sampling import sample_q
    mesh = (8, 8, 8)
    e = make_engine(sysm, mesh, precision=0, inject=False)
    sub = sample_q(512, 1, seed=5).tolist()
    G = torch.tensor(np.random.default_rng(8).standard_normal((5, 6)), device="cuda")
    g0, _, _ = e.rates(300.0, 0.1, 31, q_subset=sub)
    d3, d4 = e.backward(G)
    d3, d4 = d3.cpu().numpy(), d4.cpu().numpy()
    p3, p4 = sysm[2].phi.copy(), sysm[3].phi.copy()
    L0 = float((G * g0).sum())
    rng = np.random.default_rng(21)
    picks = [(3, int(c), int(x)) for c, x in zip(rng.integers(0, p3.shape[0], 8), rng.integers(0, 27, 8))] + \
            [(4, int(c), int(x)) for c, x in zip(rng.integers(0, p4.shape[0], 8), rng.integers(0, 81, 8))]
    try:
        for order, c, x in picks:
            base = p3 if order == 3 else p4
            h = 1e-5 * max(abs(float(base[c, x])), 1.0)
            vals = []
            for sgn in (1, -1):
                mod = base.copy()
                mod[c, x] += sgn * h
                e.update_anharmonic(mod if order == 3 else None, mod if order == 4 else None)
                g, _, _ = e.rates(300.0, 0.1, 31, q_subset=sub)
                vals.append(float((G * g).sum()))
            e.update_anharmonic(p3 if order == 3 else None, p4 if order == 4 else None)
            fd = (vals[0] - vals[1]) / (2 * h)
            an = float((d3 if order == 3 else d4)[c, x])
            noise = 1e-14 * abs(L0) / h
            assert abs(fd - an) <= 1e-6 * abs(an) + noise, (order, c, x, fd, an, noise)
    finally:
        e.update_anharmonic(p3, p4)


@pytest.mark.parametrize("mesh,sub", [((3, 3, 3), [13]), ((4, 4, 4), [22])])
def test_rates_backward_mixed_precision(sysm, mesh, sub):
    """The mixed-precision adjoint (4ph terms in FP32 with FP32 Kahan slices summed in FP64; 3ph in
    FP64) against the oracle's FP64 gradient: 3ph to 1e-8 elementwise, 4ph to 1e-4 of the largest
    gradient entry (normwise: single entries are sums with cancellation)."""
    prob = oracle.Problem(*sysm, mesh)
    e = make_engine(sysm, mesh, precision=1, prob=prob)
    modes = modes_of(sub, 6)
    dL = np.random.default_rng(11).standard_normal((5, modes.size))
    e.rates(300.0, 0.1, 31, q_subset=sub)
    d3, d4 = e.backward(torch.tensor(dL, device="cuda"))
    g3, g4 = prob.grad(modes, dL)
    assert_close(d3.cpu().numpy().reshape(-1), g3.reshape(-1), 1e-8, floor_frac=1e-9, what="dphi3 (mixed context)")
    err = np.abs(d4.cpu().numpy() - g4).max() / np.abs(g4).max()
    assert err <= 1e-4, err
