"""Sampling estimate of the four-phonon sums on the GPU against the oracle's (needs a GB300).

Both sides take a partner pair (λ, q', q'') iff the same counter-based hash (SplitMix64's output
function of seed + (key + 1) x 0x9e3779b97f4a7c15) is below floor(f 2^64), and scale the sums by
2^64 / threshold.  So the sampled counts and process lists must match bit for bit, and Γ, WP within
the usual bars, in every kernel: the tiled CUDA-core kernel (where the triangular domain lets one
representative stand for two pairs, each with its own draw), the tensor-core kernel and the
general kernel of larger cells."""
import numpy as np
import pytest

import oracle
from synth import morse_system, diamond_crystal, supercell_crystal, morse_ifcs, random_cluster_ifcs
from tests.helpers import assert_close, make_engine, modes_of

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sys0():
    return morse_system(seed=0)


def test_fraction_one_is_the_full_sum(sys0):
    e = make_engine(sys0, (4, 4, 4), precision=0)
    a = [x.cpu().numpy() for x in e.rates(300.0, 0.1, 31, q_subset=[1, 9])]
    e.set_sampling(1.0, 123)
    b = [x.cpu().numpy() for x in e.rates(300.0, 0.1, 31, q_subset=[1, 9])]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-4), (2, 1e-4)])
@pytest.mark.parametrize("adaptive", [False, True])
def test_sampled_rates_match_oracle(sys0, precision, tol, adaptive):
    mesh = (4, 4, 4)
    sigma = 1.0 if adaptive else 0.1
    prob = oracle.Problem(*sys0, mesh, sigma=sigma, sigma_adaptive=adaptive).with_sampling(0.3, 7)
    e = make_engine(sys0, mesh, precision=precision, prob=prob)
    e.set_sampling(0.3, 7)
    sub = [1, 22, 63]
    g, wp, c = (x.cpu().numpy() for x in e.rates(300.0, sigma, 31, q_subset=sub, adaptive=adaptive))
    e.check_device()
    G, WP, CNT = prob.rates(modes_of(sub, 6))
    full = oracle.Problem(*sys0, mesh, sigma=sigma, sigma_adaptive=adaptive, modes=prob.modes).rates(modes_of(sub, 6))[2]
    assert CNT[2:].sum() < 0.5 * full[2:].sum()                # the sample is a true subset
    assert np.array_equal(c, CNT)
    floor = 1e-12 if precision == 0 else 1e-6
    assert_close(g, G, tol, floor_frac=floor, what="gamma")
    assert_close(wp, WP, tol, floor_frac=floor, what="wp")


def test_sampled_process_lists_match_oracle(sys0):
    mesh = (3, 3, 3)
    prob = oracle.Problem(*sys0, mesh).with_sampling(0.5, 99)
    e = make_engine(sys0, mesh, precision=0, prob=prob)
    e.set_sampling(0.5, 99)
    e.rates(300.0, 0.1, 31, q_subset=[0])
    for m in (4, 40, 131):
        for ch in (2, 3, 4):
            assert np.array_equal(e.processes(ch, m), prob.processes(ch, m)), (m, ch)


def test_sampled_general_kernel_four_atoms():
    c = supercell_crystal(diamond_crystal(), 2, masses=np.array([28.0855, 12.0, 72.6, 28.0855]))
    p2, _, _ = morse_ifcs(c, seed=3)
    p3 = random_cluster_ifcs(c, 3, 40, seed=4, scale=2.0)
    p4 = random_cluster_ifcs(c, 4, 60, seed=5, scale=5.0)
    sysm = (c, p2, p3, p4)
    mesh = (2, 2, 2)
    prob = oracle.Problem(*sysm, mesh).with_sampling(0.4, 3)
    e = make_engine(sysm, mesh, precision=0, prob=prob)
    e.set_sampling(0.4, 3)
    sub = [0, 5]
    g, _, cnt = (x.cpu().numpy() for x in e.rates(300.0, 0.1, 31, q_subset=sub))
    G, _, CNT = prob.rates(modes_of(sub, 12))
    assert np.array_equal(cnt, CNT)
    assert_close(g, G, 1e-10, what="4-atom sampled")


def test_backward_refused_while_sampling(sys0):
    from paper_2510_00518_gb300 import FC4Error
    e = make_engine(sys0, (3, 3, 3), precision=0)
    e.set_sampling(0.5, 1)
    g, _, _ = e.rates(300.0, 0.1, 31, q_subset=[2])
    with pytest.raises(FC4Error) as ei:
        e.backward(torch.ones_like(g))
    assert ei.value.status == 6
    e.set_sampling(1.0, 0)
    e.rates(300.0, 0.1, 31, q_subset=[2])
    e.backward(torch.ones_like(g))
