"""Rates of the whole mesh from the irreducible q-points (fc4_rates on a q subset, host
expansion) against fc4_rates on every q point (needs a GB300).

The mode loops of Algorithms 1 and 3-5 run over the irreducible q-points.  On the unperturbed
Morse diamond (48 operations, 8 irreducible points of the 4x4x4 mesh) every channel's Γ and WP,
averaged over degenerate branches, and κ agree with the full-mesh evaluation to rounding."""
import numpy as np
import pytest

from synth import morse_system

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_irreducible_rates_and_kappa_match_full_mesh():
    from paper_2510_00518_gb300 import FP64, Engine
    from paper_2510_00518_gb300.symmetry import expand_irreducible, rates_irreducible, symmetry_ops

    sysm = morse_system(seed=0, perturb=0.0)
    mesh = (4, 4, 4)
    rot, _ = symmetry_ops(*sysm)
    e = Engine(*sysm, mesh, precision=FP64)
    g_irr, wp_irr, n_irr = rates_irreducible(e, 300.0, 0.1, 31, rot)
    assert n_irr == 8
    g, wp, _ = e.rates(300.0, 0.1, 31)
    omega = e.get_modes()[0]
    nb, N = e.nb, e.nq
    rep_id = np.arange(N, dtype=np.int32)                 # degenerate averaging of the full mesh
    ref = expand_irreducible(mesh, nb, rep_id, omega, np.stack([g.cpu().numpy(), wp.cpu().numpy()]))
    for got, want in ((g_irr.cpu().numpy(), ref[0]), (wp_irr.cpu().numpy(), ref[1])):
        floor = 1e-12 * np.abs(want).max()
        assert np.max(np.abs(got - want) / np.maximum(np.abs(want), floor)) < 1e-9
    k_irr = e.kappa(300.0, g_irr).cpu().numpy()
    k_full = e.kappa(300.0, g).cpu().numpy()
    assert np.allclose(k_irr, k_full, rtol=1e-9, atol=1e-12 * np.abs(k_full).max())
