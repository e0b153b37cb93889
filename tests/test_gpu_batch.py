"""Many crystals in one CUDA-graph launch (needs a GB300).

The crystals are the synthetic batch of Morse solids (1x1xk diamond supercells, k = 1..4: 6 to
24 branches; site masses U(10, 120) amu).  The test uses the first 8 of them (two of each size)
on meshes half the batch's linear size and one seeded q point each, mixed precision; the full
24-crystal batch is timed by ``bench.py --batch``.  Replaying the captured graph must reproduce
the eager results bit for bit (deterministic kernels); cells of 6 and 8 atoms are checked
against the oracle on tiny meshes."""
import numpy as np
import pytest

import oracle
from synth import batch_crystal, morse_ifcs
from synth.sampling import sample_q
from tests.helpers import assert_close, make_engine, modes_of

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_graph_batch_matches_eager(tmp_path):
    from paper_2510_00518_gb300 import Engine, MIXED
    from paper_2510_00518_gb300.batch import BatchRunner, autotune
    jobs = []
    for seed in range(8):
        c, mesh = batch_crystal(seed)
        mesh = tuple(max(2, n // 2) for n in mesh)
        p2, p3, p4 = morse_ifcs(c, seed=seed)
        e = Engine(c, p2, p3, p4, mesh, precision=MIXED)
        qs = sample_q(int(np.prod(mesh)), 1, seed=seed)
        jobs.append((e, qs))
    cache = str(tmp_path / "tune.json")
    bt = autotune(jobs[3][0], 300.0, 0.1, 31, jobs[3][1], cache=cache)     # an 8-atom cell
    assert bt in (64, 96, 128)
    assert autotune(jobs[3][0], 300.0, 0.1, 31, jobs[3][1], cache=cache) == bt   # cached
    eager = [e.rates(300.0, 0.1, 31, q_subset=qs)[0].clone() for e, qs in jobs]
    runner = BatchRunner(jobs, 300.0, 0.1, 31, persistent=False)      # a graph of per-crystal calls
    for _ in range(2):
        out = runner.run()
        torch.cuda.synchronize()
        for a, b in zip(out, eager):
            assert torch.equal(a, b)


@pytest.mark.parametrize("seed,mesh", [(2, (1, 1, 2)), (3, (1, 1, 1))])
def test_large_cells_against_oracle(seed, mesh):
    c, _ = batch_crystal(seed)
    sysm = (c,) + morse_ifcs(c, seed=seed)
    prob = oracle.Problem(*sysm, mesh)
    nb = c.nb
    sub = [mesh[2] - 1]
    G, WP, CNT = prob.rates(modes_of(sub, nb))
    for prec, tol in ((0, 1e-10), (1, 1e-4)):
        e = make_engine(sysm, mesh, precision=prec, prob=prob)
        g, wp, cnt = e.rates(300.0, 0.1, 31, q_subset=sub)
        assert np.array_equal(cnt.cpu().numpy(), CNT)
        assert_close(g.cpu().numpy(), G, tol, floor_frac=1e-6 if prec else 1e-12, what=f"na{c.n_atoms} p{prec}")


def _jobs(n, scale=2):
    from paper_2510_00518_gb300 import Engine, MIXED
    jobs = []
    for seed in range(n):
        c, mesh = batch_crystal(seed)
        mesh = tuple(max(2, m // scale) for m in mesh)
        e = Engine(c, *morse_ifcs(c, seed=seed), mesh, precision=MIXED)
        jobs.append((e, sample_q(int(np.prod(mesh)), 1, seed=seed)))
    return jobs


def test_persistent_batch_equals_per_context_kernels():
    """One persistent launch per cell size over the units of all crystals of more than two atoms
    gives, for each, the Γ, WP and counts of its own general-kernel call (fc4_rates_static, same
    arithmetic) bit for bit; two-atom crystals give their fc4_rates result; the captured graph
    replays it exactly."""
    from paper_2510_00518_gb300 import Batch
    from paper_2510_00518_gb300.batch import BatchRunner
    jobs = _jobs(8)
    ref = []
    for e, qs in jobs:                  # cells of up to two atoms keep their own fc4_rates path
        e.set_block_threads(128)
        r = e.rates(300.0, 0.1, 31, q_subset=qs) if e.n_atoms <= 2 else e.rates_static(300.0, 0.1, 31, qs)
        ref.append([x.clone() for x in r])
    outs = Batch([e for e, _ in jobs]).rates(300.0, 0.1, 31, q_subsets=[q for _, q in jobs])
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        for a, b in zip(o, r):
            assert torch.equal(a, b)
    runner = BatchRunner(jobs, 300.0, 0.1, 31, persistent=True)
    for _ in range(2):
        out = runner.run()
        torch.cuda.synchronize()
        for a, r in zip(out, ref):
            assert torch.equal(a, r[0])


def test_persistent_batch_against_oracle():
    """Cells of 2, 6 and 8 atoms in one batch against the oracle (mixed bar)."""
    from paper_2510_00518_gb300 import Batch, Engine, MIXED
    cases = [(0, (3, 3, 3), [4]), (2, (1, 1, 2), [1]), (3, (1, 1, 1), [0])]
    engines, qsets, refs = [], [], []
    for seed, mesh, sub in cases:
        c, _ = batch_crystal(seed)
        sysm = (c,) + morse_ifcs(c, seed=seed)
        prob = oracle.Problem(*sysm, mesh)
        e = Engine(*sysm, mesh, precision=MIXED)
        e.set_modes(prob.modes.omega, prob.modes.vel, prob.modes.evec)
        engines.append(e)
        qsets.append(sub)
        refs.append(prob.rates(modes_of(sub, c.nb)))
    outs = Batch(engines).rates(300.0, 0.1, 31, q_subsets=qsets)
    for (g, wp, cnt), (G, WP, CNT) in zip(outs, refs):
        assert np.array_equal(cnt.cpu().numpy(), CNT)
        assert_close(g.cpu().numpy(), G, 1e-4, floor_frac=1e-6, what="batch")
