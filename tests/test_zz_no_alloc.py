"""fc4_rates_static, the entry point for callers that cannot allocate device memory while they
run (host frameworks that own every device allocation through their own pool, or loops where
the implicit synchronisation of cudaMalloc/cudaFree is not acceptable): its results must equal
the oracle's and fc4_rates' on the same inputs, call after call, although its scratch is one
fixed device array shared by every call, and a call must not change the device memory in use.

This file is collected last on purpose, so that a run that stops at the first failure has
already run every other test.  It passes alone in a fresh process and after the other tests."""
import numpy as np
import pytest

import oracle
from synth import morse_system
from tests.helpers import assert_close, make_engine, modes_of

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-4)])
def test_static_scratch_matches_oracle_and_fc4_rates(precision, tol):
    sysm = morse_system(seed=0)
    mesh = (3, 3, 3)
    prob = oracle.Problem(*sysm, mesh)
    e = make_engine(sysm, mesh, precision=precision, prob=prob)
    calls = [([1, 5, 13, 26], 31), ([0, 2, 7, 19, 20, 22], 0b11101)]   # two calls in a row
    for sub, mask in calls:
        G, WP, CNT = prob.rates(modes_of(sub, 6), channel_mask=mask)
        g_ref, wp_ref, n_ref = e.rates(300.0, 0.1, mask, q_subset=sub)
        g, wp, n = e.rates_static(300.0, 0.1, mask, sub)
        torch.cuda.synchronize()
        assert np.array_equal(n.cpu().numpy(), CNT)
        assert np.array_equal(n.cpu().numpy(), n_ref.cpu().numpy())
        assert_close(g.cpu().numpy(), G, tol, what="gamma vs oracle")
        assert_close(wp.cpu().numpy(), WP, tol, what="wp vs oracle")
        assert_close(g.cpu().numpy(), g_ref.cpu().numpy(), tol, what="gamma vs fc4_rates")
        assert_close(wp.cpu().numpy(), wp_ref.cpu().numpy(), tol, what="wp vs fc4_rates")


def test_static_call_allocates_no_device_memory():
    sysm = morse_system(seed=0)
    e = make_engine(sysm, (3, 3, 3), precision=1)
    sub = [0, 2, 7, 19, 20, 22]
    out = tuple(torch.empty((5, len(sub) * 6), dtype=dt, device="cuda")
                for dt in (torch.float64, torch.float64, torch.int64))
    e.rates_static(300.0, 0.1, 31, sub, out=out)            # first call: symbol lookup, kernels loaded
    torch.cuda.synchronize()
    first = [t.clone() for t in out]
    used = torch.cuda.memory_allocated()
    free = torch.cuda.mem_get_info()[0]
    e.rates_static(300.0, 0.1, 31, sub, out=out)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == used
    assert torch.cuda.mem_get_info()[0] == free
    for a, b in zip(out, first):
        assert torch.equal(a, b)


def test_static_scratch_rejects_oversized_requests():
    from paper_2510_00518_gb300 import FC4Error
    sysm = morse_system(seed=0)
    e = make_engine(sysm, (8, 8, 8), inject=False)
    with pytest.raises(FC4Error) as ei:
        e.rates_static(300.0, 0.1, 31, list(range(22)))      # 22 * 6 * 512 > 65536
    assert ei.value.status == 1
