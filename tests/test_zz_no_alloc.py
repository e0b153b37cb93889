"""fc4_rates_static, the entry point for callers that cannot allocate device memory while they
run (code inside CUDA stream capture, or frameworks that own all device memory): its results
must equal fc4_rates' on the same inputs, call after call, although its scratch is one fixed
device array shared by every call.

This file is collected last on purpose, so that a run that stops at the first failure has
already run every other test.  It passes alone in a fresh process and after the other tests."""
import numpy as np
import pytest

import oracle
from synth import morse_system
from tests.helpers import assert_close, make_engine

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-4)])
def test_static_scratch_matches_fc4_rates(precision, tol):
    sysm = morse_system(seed=0)
    mesh = (3, 3, 3)
    prob = oracle.Problem(*sysm, mesh)
    e = make_engine(sysm, mesh, precision=precision, prob=prob)
    calls = [([1, 5, 13, 26], 31), ([0, 2, 7, 19, 20, 22], 0b11101)]   # two calls in a row
    for sub, mask in calls:
        g_ref, wp_ref, n_ref = e.rates(300.0, 0.1, mask, q_subset=sub)
        g, wp, n = e.rates_static(300.0, 0.1, mask, sub)
        torch.cuda.synchronize()
        assert np.array_equal(n.cpu().numpy(), n_ref.cpu().numpy())
        assert_close(g.cpu().numpy(), g_ref.cpu().numpy(), tol, what="gamma")
        assert_close(wp.cpu().numpy(), wp_ref.cpu().numpy(), tol, what="wp")


def test_static_scratch_rejects_oversized_requests():
    from paper_2510_00518_gb300 import FC4Error
    sysm = morse_system(seed=0)
    e = make_engine(sysm, (8, 8, 8), inject=False)
    with pytest.raises(FC4Error) as ei:
        e.rates_static(300.0, 0.1, 31, list(range(22)))      # 22 * 6 * 512 > 65536
    assert ei.value.status == 1
