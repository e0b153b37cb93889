"""Mode chunks and partner-point chunks against the oracle (needs a GB300).

A rates call processes its modes in chunks (the paper's all-modes and mode-by-mode strategies,
Results and Algorithm 5; fc4_set_mode_chunk), and the kernels walk the +- triangle q'' <= q''' in
chunks of partner points (1024 in the CUDA-core kernel, 1536 in the tensor-core kernel).  Results
must not depend on the mode chunking (bit for bit: each mode's partials are formed the same way),
and the 12x12x12 mesh (1728 q, two partner chunks in both kernels) must match the oracle's stored
values (tests/golden/mesh12_chunks.npz, written by tests/golden/make_config_goldens.py)."""
import os

import numpy as np
import pytest

import oracle
from synth import morse_system
from tests.helpers import assert_close, make_engine

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def sys0():
    return morse_system(seed=0)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_mode_chunks_bit_identical(sys0, precision):
    mesh = (4, 4, 4)
    e = make_engine(sys0, mesh, precision=precision)
    ref = [x.cpu().numpy() for x in e.rates(300.0, 0.1, 31)]
    st_ref = e.stats()
    assert e.memory()["modes_per_chunk"] == 64 * 6
    per_mode = e.memory()["w_per_mode"]
    for chunk, wlim in ((1, 0), (7, 0), (0, 5 * per_mode)):
        e.set_mode_chunk(chunk, wlim)
        out = [x.cpu().numpy() for x in e.rates(300.0, 0.1, 31)]
        assert e.memory()["modes_per_chunk"] == (chunk or 5)
        for a, b in zip(out, ref):
            assert np.array_equal(a, b)
        st = e.stats()
        for k in st:
            assert np.array_equal(st[k], st_ref[k]), k
    # mode by mode holds partials and W for one mode only
    e.set_mode_chunk(1, 0)
    e2 = make_engine(sys0, mesh, precision=precision)
    e2.set_mode_chunk(1, 0)
    e2.rates(300.0, 0.1, 31)
    m = e2.memory()
    assert m["w_buffer"] == m["w_per_mode"]
    assert m["partials"] == 5 * 64 * 56


def test_mode_chunks_adaptive_subset(sys0):
    mesh = (6, 6, 6)
    prob = oracle.Problem(*sys0, mesh, sigma=1.0, sigma_adaptive=True)
    e = make_engine(sys0, mesh, precision=1, prob=prob)
    sub = [3, 50, 101]
    a = [x.cpu().numpy() for x in e.rates(300.0, 1.0, 31, q_subset=sub, adaptive=True)]
    e.set_mode_chunk(4, 0)
    b = [x.cpu().numpy() for x in e.rates(300.0, 1.0, 31, q_subset=sub, adaptive=True)]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.fixture(scope="module")
def mesh12():
    return np.load(os.path.join(GOLDEN, "mesh12_chunks.npz"))


# (precision, tolerance): FP64; FP32 CUDA cores; tensor cores TF32 x3 and FP16 x3
@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-4), (2, 1e-4), (5, 1e-4)])
@pytest.mark.parametrize("chunk", [0, 1])
def test_mesh12_partner_chunks_match_oracle(sys0, mesh12, precision, tol, chunk):
    from paper_2510_00518_gb300 import Engine
    g = mesh12
    mesh = tuple(int(x) for x in g["mesh"])
    assert int(np.prod(mesh)) > 1536
    e = Engine(*sys0, mesh, precision=precision)
    e.set_modes(g["omega"], g["vel"], g["evec"])
    e.set_mode_chunk(chunk, 0)
    modes = g["modes"]
    nb = 6
    # the stored modes are branches (1, 5) of each q; the call computes all branches of those q
    qs = sorted(set((modes // nb).tolist()))
    out = [x.cpu().numpy() for x in e.rates(float(g["T"][0]), float(g["sigma"]), 31, q_subset=qs)]
    e.check_device()
    pos = np.array([qs.index(m // nb) * nb + m % nb for m in modes])
    G, WP, CNT = g["gamma"][0], g["wp"][0], g["counts"][0]
    assert np.array_equal(out[2][:, pos], CNT)
    floor = 1e-12 if precision == 0 else 1e-6
    assert_close(out[0][:, pos], G, tol, floor_frac=floor, what=f"gamma prec {precision}")
    assert_close(out[1][:, pos], WP, tol, floor_frac=floor, what=f"wp prec {precision}")


@pytest.mark.parametrize("adaptive", [False, True])
def test_ablation_without_compaction_same_results(sys0, adaptive):
    """The uncompacted divergent loop (fc4_set_ablation) evaluates the same processes: identical
    counts, Γ equal to FP32 rounding (each thread sums different processes)."""
    mesh = (4, 4, 4)
    e = make_engine(sys0, mesh, precision=1)
    sigma = 1.0 if adaptive else 0.1
    a = [x.cpu().numpy() for x in e.rates(300.0, sigma, 31, q_subset=[3, 40], adaptive=adaptive)]
    e.set_ablation(True)
    b = [x.cpu().numpy() for x in e.rates(300.0, sigma, 31, q_subset=[3, 40], adaptive=adaptive)]
    e.set_ablation(False)
    assert np.array_equal(a[2], b[2])
    assert_close(b[0], a[0], 1e-5, floor_frac=1e-6, what="gamma")
