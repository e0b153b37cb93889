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
    runner = BatchRunner(jobs, 300.0, 0.1, 31)
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
