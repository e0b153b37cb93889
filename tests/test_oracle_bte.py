"""Pins of the oracle's iterative Boltzmann-equation operator (no GPU).

Δ_λ = Σ_p γ_p Σ_k s_k (ω_k / ω_λ) F_k reuses the rates' per-process terms γ_p (Γ_λ = Σ_p γ_p).
Energy conservation fixes it for a uniform field F ≡ u: Σ_k s_k ω_k = ω_λ - Δ_p for every process,
so Δ_λ(u) = Γ_λ u - u Σ_p γ_p Δ_p / ω_λ, and |Δ_p| <= 2σ bounds the second term by
(2σ / ω_λ) Σ_p |γ_p|.  For ω_λ > 2σ every weight is positive (each occupation factor has the sign
of ω_λ - Δ_p), so |Δ_λ(u) / (Γ_λ u) - 1| <= 2σ / ω_λ per channel: a dropped partner, a wrong sign
s_k or a missing ω ratio moves the ratio by O(1)."""
import numpy as np
import pytest

import oracle
from synth import morse_system

SIGMA_RADPS = 2 * np.pi * 0.1


@pytest.fixture(scope="module")
def prob3():
    return oracle.Problem(*morse_system(seed=0), (3, 3, 3))


@pytest.mark.parametrize("ch", range(5))
def test_uniform_field_energy_conservation(prob3, ch):
    P = prob3
    modes = np.arange(3, 162, dtype=np.int32) if ch < 2 else np.arange(3, 162, 4, dtype=np.int32)
    G = P.rates(modes, channel_mask=1 << ch)[0][ch]
    u = np.array([1.0, -2.0, 0.5])
    D = P.bte_offdiag(np.tile(u, (P.nq * P.nb, 1)), modes, channel_mask=1 << ch)
    w = P.modes.omega[modes]
    checked = 0
    for i in range(modes.size):
        if G[i] == 0.0 or w[i] <= 2 * SIGMA_RADPS:
            continue
        bound = 2 * SIGMA_RADPS / w[i]
        r = D[i] / (G[i] * u)
        assert np.all(np.abs(r - 1.0) <= bound * (1 + 1e-12)), (ch, modes[i], r, bound)
        assert np.allclose(r, r[0], rtol=1e-12)                  # one scalar per mode
        checked += 1
    assert checked >= 3


def test_operator_is_linear_and_vanishes_at_zero(prob3):
    P = prob3
    rng = np.random.default_rng(5)
    n = P.nq * P.nb
    F1, F2 = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
    modes = [20, 77, 140]
    assert np.array_equal(P.bte_offdiag(np.zeros((n, 3)), modes), np.zeros((3, 3)))
    a = P.bte_offdiag(2.0 * F1 - 3.0 * F2, modes)
    b = 2.0 * P.bte_offdiag(F1, modes) - 3.0 * P.bte_offdiag(F2, modes)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_rta_limit_and_fixed_point():
    """F⁰ = v / Γ reproduces the RTA κ; the converged iterate is a fixed point of the update."""
    P = oracle.Problem(*morse_system(seed=0), (4, 1, 1))
    G = P.rates()[0].sum(0)
    k_rta = P.kappa(G)
    F0 = oracle.rta_F(P.modes, G)
    assert np.abs(oracle.kappa_of_F(P.crystal, P.modes, P.T, F0, P.mesh) - k_rta).max() <= 1e-14 * np.abs(k_rta).max()
    k, F, it, ks = P.kappa_iterative(G, tol=1e-13, max_iter=200)
    assert it < 200 and np.array_equal(ks[0], oracle.kappa_of_F(P.crystal, P.modes, P.T, F0, P.mesh))
    ok = (P.modes.omega > 0) & (G > 0)
    Fn = np.zeros_like(F)
    Fn[ok] = (P.modes.vel[ok] + P.bte_offdiag(F)[ok]) / G[ok, None]
    assert np.abs(Fn - F).max() <= 1e-10 * np.abs(F).max()
    assert np.all(np.diag(k) > np.diag(k_rta))          # the off-diagonal terms add back heat flow
