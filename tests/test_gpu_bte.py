"""Iterative Boltzmann equation on the GPU against the oracle (needs a GB300).

The off-diagonal operator Δ(F) = Σ_p γ_p Σ_k s_k (ω_k / ω_λ) F_k is recomputed by the rate kernels
for a given field F; its values, the iteration F = (v + Δ(F)) / Γ and κ of every iterate must match
the oracle's: within 1e-10 (FP64), 1e-4 (mixed) of max(|ref|, 1e-6 x the largest |ref|)."""
import os

import numpy as np
import pytest

import oracle
from synth import morse_system
from tests.helpers import assert_close, make_engine, modes_of

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def sys0():
    return morse_system(seed=0)


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-4)])
@pytest.mark.parametrize("adaptive", [False, True])
def test_offdiag_matches_oracle(sys0, precision, tol, adaptive):
    mesh = (3, 3, 3)
    sigma = 1.0 if adaptive else 0.1
    prob = oracle.Problem(*sys0, mesh, sigma=sigma, sigma_adaptive=adaptive)
    e = make_engine(sys0, mesh, precision=precision, prob=prob)
    F = np.random.default_rng(3).normal(size=(27 * 6, 3))
    sub = [1, 8, 26]
    for mask in (31, 0b00011, 0b01000):
        D = e.bte_offdiag(300.0, sigma, torch.tensor(F, device="cuda"), mask, q_subset=sub,
                          adaptive=adaptive).cpu().numpy()
        ref = prob.bte_offdiag(F, modes_of(sub, 6), channel_mask=mask)
        assert_close(D.T, ref.T, tol, floor_frac=1e-12 if precision == 0 else 1e-6, what=f"mask {mask}")


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-4)])
def test_kappa_iterative_small_mesh(sys0, precision, tol):
    mesh = (4, 1, 1)
    prob = oracle.Problem(*sys0, mesh)
    e = make_engine(sys0, mesh, precision=precision, prob=prob)
    g = e.rates(300.0, 0.1, 31)[0]
    G = prob.rates()[0]
    k_ref, F_ref, it_ref, _ = prob.kappa_iterative(G.sum(0), tol=1e-12, max_iter=200)
    # FP32 noise stops the mixed iterate's κ from settling below ~1e-7 relative
    k, F, it = e.kappa_iterative(300.0, 0.1, g, 31, max_iter=200, tol=1e-12 if precision == 0 else 1e-7)
    assert it == it_ref if precision == 0 else it < 200
    assert np.abs(k.cpu().numpy() - k_ref).max() <= tol * np.abs(k_ref).max()
    assert np.abs(F.cpu().numpy() - F_ref).max() <= tol * np.abs(F_ref).max()
    # no iteration: the RTA κ of fc4_kappa
    k0, _, it0 = e.kappa_iterative(300.0, 0.1, g, 31, max_iter=0)
    assert it0 == 0
    kr = e.kappa(300.0, g, 31)
    assert torch.allclose(k0, kr, rtol=1e-12, atol=0)


def test_kappa_iterative_3cubed_golden(sys0):
    """Every iterate's κ on the full 3x3x3 mesh against the oracle's stored iteration."""
    g = np.load(os.path.join(GOLDEN, "bte_3cubed.npz"))
    from paper_2510_00518_gb300 import Engine
    e = Engine(*sys0, (3, 3, 3), precision=0)
    e.set_modes(g["omega"], g["vel"], g["evec"])
    gam = torch.tensor(g["gamma"], device="cuda")
    ks = g["kappa"]
    for n in (1, 2, 5, len(ks) - 1):
        k, F, it = e.kappa_iterative(300.0, float(g["sigma"]), gam, 31, max_iter=n, tol=0.0)
        assert it == n
        assert np.abs(k.cpu().numpy() - ks[n]).max() <= 1e-10 * np.abs(ks[n]).max(), n
    assert np.abs(F.cpu().numpy() - g["F"]).max() <= 1e-10 * np.abs(g["F"]).max()
