"""The two large parity workloads against the oracle's stored values (needs a GB300).

tests/golden/make_config_goldens.py (which calls only oracle/ and synth/) wrote the oracle's Γ, WP
and kept counts together with the harmonic modes it used; the engine takes those modes through
fc4_set_modes, so both sides see the same ω bits and eigenvector gauge.
  config2_8cubed.npz   8x8x8 mesh, seed 0, fixed σ = 0.1 THz, 8 sampled q x 6 branches, 300 and
                       700 K; the GPU computes every mode of the mesh in one call (the bench's
                       launch configuration) and the sampled modes are compared
  config3_16cubed.npz  16x16x16 mesh, seed 1, adaptive σ (scale 1), 300 K, the first of the 145
                       sampled q x 6 branches; computed alone and inside the first 29 of the 145 q
                       (one step of bench.py)
Counts must match bit for bit; Γ and WP within 1e-10 (FP64), within 1e-4 (mixed, FP32 CUDA
cores; TF32 x3 tensor cores) of max(|ref|, 1e-6 x the channel's largest value)."""
import os

import numpy as np
import pytest

from synth import morse_system
from tests.helpers import assert_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    return np.load(os.path.join(GOLDEN, name))


def engine(g, precision):
    from paper_2510_00518_gb300 import Engine
    e = Engine(*morse_system(seed=int(g["seed"])), tuple(int(x) for x in g["mesh"]), precision=precision)
    e.set_modes(g["omega"], g["vel"], g["evec"])
    return e


def compare(out, g, it, tol):
    G, WP, CNT = g["gamma"][it], g["wp"][it], g["counts"][it]
    assert np.array_equal(out[2], CNT)
    floor = 1e-12 if tol < 1e-8 else 1e-6
    assert_close(out[0], G, tol, floor_frac=floor, what="gamma")
    assert_close(out[1], WP, tol, floor_frac=floor, what="wp")


@pytest.fixture(scope="module")
def config2():
    return load("config2_8cubed.npz")


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-4)])
def test_config2_all_modes_sampled_against_oracle(config2, precision, tol):
    g = config2
    e = engine(g, precision)
    modes = g["modes"]
    for it, T in enumerate(g["T"]):
        out = [x.cpu().numpy()[:, modes] for x in e.rates(float(T), float(g["sigma"]), 31)]
        compare(out, g, it, tol)


def test_config2_subset_call_fp64(config2):
    """The sampled q as the call's subset (the oracle's own launch shape)."""
    g = config2
    e = engine(g, 0)
    qs = sorted(set((g["modes"] // 6).tolist()))
    for it, T in enumerate(g["T"]):
        out = [x.cpu().numpy() for x in e.rates(float(T), float(g["sigma"]), 31, q_subset=qs)]
        compare(out, g, it, 1e-10)


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-4), (2, 1e-4)])
def test_config3_sampled_q_against_oracle(precision, tol):
    g = load("config3_16cubed.npz")
    e = engine(g, precision)
    qs = sorted(set((g["modes"] // 6).tolist()))
    out = [x.cpu().numpy() for x in e.rates(float(g["T"][0]), float(g["sigma"]), 31, q_subset=qs, adaptive=True)]
    e.check_device()
    compare(out, g, 0, tol)


def test_config3_bench_step_against_oracle():
    """The stored q inside the bench's own launch: one mixed call on the first 29 of the 145 sampled
    q (default_rng(1).choice(4096, 145), sorted; the stored q is the first).  Its columns must match
    the oracle's values, and equal bit for bit the same q computed alone: every block owns one
    (λ, q') unit and each mode's partials are summed in a fixed order, so the other modes of a call
    do not change a mode's result."""
    from synth.sampling import sample_q
    g = load("config3_16cubed.npz")
    step = sample_q(4096, 145, 1)[:29]
    assert int(step[0]) == int(g["q"][0])
    e = engine(g, 1)
    args = (float(g["T"][0]), float(g["sigma"]), 31)
    full = [x.cpu().numpy()[:, :6] for x in e.rates(*args, q_subset=step, adaptive=True)]
    alone = [x.cpu().numpy() for x in e.rates(*args, q_subset=step[:1], adaptive=True)]
    e.check_device()
    for a, b in zip(full, alone):
        assert np.array_equal(a, b)
    compare(full, g, 0, 1e-4)
