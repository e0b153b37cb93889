"""Tensor-core cluster contraction of the 4ph +- channel (tcgen05, mixed precision, two-atom
cells) against the CUDA-core contraction and the FP64 oracle, and its bounded wait (needs a GB300).

Every operand format feeds the same window decision, so kept counts are identical.  Γ agrees with
the FP32 CUDA-core contraction to the level of its operands: 1e-5 for the 22-bit splits (FP16 x3,
TF32 x3), 1e-4 for BF16 x3 (16 bits); all three match the oracle within the mixed-path tolerance
(1e-4).  Single-pass BF16 (8 bits) is held to 2e-2 against the oracle; bench.py states its
measured error."""
import numpy as np
import pytest

import oracle
from synth import morse_system
from synth.sampling import sample_q
from tests.helpers import assert_close, make_engine, modes_of

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PM = 0b01000


@pytest.fixture(scope="module")
def sys0():
    return morse_system(seed=0)


# (precision, tolerance against the CUDA-core contraction, tolerance against the oracle)
FORMATS = {"fp16x3": (5, 1e-5, 1e-4), "tf32x3": (2, 1e-5, 1e-4), "bf16x3": (4, 1e-4, 1e-4),
           "bf16": (3, 2e-2, 2e-2)}


@pytest.mark.parametrize("fmt", list(FORMATS))
@pytest.mark.parametrize("mesh", [(3, 3, 3), (4, 4, 4), (6, 6, 6), (5, 3, 4)])
def test_tc_matches_cuda_cores_and_oracle(sys0, mesh, fmt):
    """Meshes with one partial round of 128 partner points (27, 60, 64) and with two (216)."""
    prec, tol_cc, tol_or = FORMATS[fmt]
    prob = oracle.Problem(*sys0, mesh)
    e = make_engine(sys0, mesh, precision=1, prob=prob)
    n = int(np.prod(mesh))
    sub = sample_q(n, 3, seed=n).tolist()
    e.set_precision(prec)
    g1, w1, c1 = (x.cpu().numpy() for x in e.rates(300.0, 0.1, PM, q_subset=sub))
    st1 = e.stats()
    e.check_device()
    e.set_precision(1)
    g0, w0, c0 = (x.cpu().numpy() for x in e.rates(300.0, 0.1, PM, q_subset=sub))
    st0 = e.stats()
    assert c1[3].sum() > 0
    # both contractions walk the same triangular domain (q'' <= q''') of the +- channel
    for k in ("kept", "evaluated"):
        assert st1[k][3] == st0[k][3], k
    assert st1["evaluated"][3] < st1["kept"][3]
    assert np.array_equal(c1, c0)
    assert_close(g1, g0, tol_cc, floor_frac=1e-6, what=f"{fmt}: tensor vs CUDA cores")
    assert_close(w1, w0, 1e-5, floor_frac=1e-6, what="wp")      # WP needs no contraction
    G, WP, CNT = prob.rates(modes_of(sub, 6), channel_mask=PM)
    assert np.array_equal(c1, CNT)
    assert_close(g1, G, tol_or, floor_frac=1e-6, what=f"{fmt}: tensor cores vs oracle")


@pytest.mark.parametrize("fmt", ["tf32x3", "bf16x3"])
def test_tc_formats_adaptive_sigma(sys0, fmt):
    """Adaptive broadening (the 16^3 precision workload's width) through the tensor-core path."""
    prec, _, tol_or = FORMATS[fmt]
    mesh = (6, 6, 6)
    prob = oracle.Problem(*sys0, mesh, sigma=1.0, sigma_adaptive=True)
    e = make_engine(sys0, mesh, precision=prec, prob=prob)
    sub = [5, 77]
    g, _, c = (x.cpu().numpy() for x in e.rates(300.0, 1.0, PM, q_subset=sub, adaptive=True))
    e.check_device()
    G, _, CNT = prob.rates(modes_of(sub, 6), channel_mask=PM)
    assert np.array_equal(c, CNT)
    assert_close(g, G, tol_or, floor_frac=1e-6, what=f"{fmt} adaptive")


def test_tc_all_channels_deterministic(sys0):
    mesh = (4, 4, 4)
    e = make_engine(sys0, mesh, precision=1)
    e.set_tensor_cores(True)
    a = e.rates(300.0, 0.1, 31)[0].cpu().numpy()
    b = e.rates(300.0, 0.1, 31)[0].cpu().numpy()
    assert np.array_equal(a, b)


def test_tc_wait_bound_expires_to_error_status(sys0):
    """A one-clock bound on the tensor-core wait: the kernels give up before their MMAs finish,
    flag the error, wait for the MMAs, free tensor memory and return.  Γ(+-) of that call is NaN,
    fc4_check_device reports FC4_ERR_TIMEOUT once, and the context keeps working."""
    from paper_2510_00518_gb300 import Engine, FC4Error, MIXED
    mesh = (4, 4, 4)
    prob = oracle.Problem(*sys0, mesh)
    e = Engine(*sys0, mesh, precision=MIXED, tensor_cores=True, timeout_cycles=1)
    e.set_modes(prob.modes.omega, prob.modes.vel, prob.modes.evec)
    sub = [1, 2, 3]
    g, _, _ = e.rates(300.0, 0.1, PM, q_subset=sub)
    with pytest.raises(FC4Error) as ei:
        e.check_device()
    assert ei.value.status == 4
    assert np.isnan(g[3].cpu().numpy()).all()
    e.check_device()                                   # the flag was cleared
    e.set_tensor_cores(False)                          # no bounded wait on this path
    g, _, cnt = e.rates(300.0, 0.1, PM, q_subset=sub)
    e.check_device()
    G, _, CNT = prob.rates(modes_of(sub, 6), channel_mask=PM)
    assert np.array_equal(cnt.cpu().numpy(), CNT)
    assert_close(g.cpu().numpy(), G, 1e-4, floor_frac=1e-6, what="after timeout")
