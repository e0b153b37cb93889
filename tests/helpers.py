"""Shared test helpers: seeded systems and engines with the oracle's modes injected."""
import numpy as np

import oracle
from synth import morse_system


def relerr(a, b, floor=0.0):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) / np.maximum(np.maximum(np.abs(a), np.abs(b)), floor)


def assert_close(gpu, ref, rtol, floor_frac=1e-12, what=""):
    """Element-wise |gpu - ref| <= rtol * max(|ref|, floor), floor = floor_frac * max|ref| of the row."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    assert gpu.shape == ref.shape, (gpu.shape, ref.shape)
    scale = np.abs(ref).max(axis=-1, keepdims=True) if ref.ndim > 1 else np.abs(ref).max()
    floor = floor_frac * scale
    err = np.abs(gpu - ref) / np.maximum(np.abs(ref), np.maximum(floor, 1e-300))
    worst = np.unravel_index(np.argmax(err), err.shape)
    assert err.max() <= rtol, f"{what}: max rel err {err.max():.3e} at {worst}: gpu {gpu[worst]} ref {ref[worst]}"


def make_engine(sys, mesh, precision=0, inject=True, prob=None, block_threads=0):
    from paper_2510_00518_gb300 import Engine
    c, p2, p3, p4 = sys
    e = Engine(c, p2, p3, p4, mesh, precision=precision, block_threads=block_threads)
    if inject:
        prob = prob or oracle.Problem(c, p2, p3, p4, mesh)
        e.set_modes(prob.modes.omega, prob.modes.vel, prob.modes.evec)
    return e


def modes_of(q_subset, nb):
    return np.array([q * nb + j for q in q_subset for j in range(nb)], np.int32)


def system(seed=0, perturb=0.01):
    return morse_system(seed=seed, perturb=perturb)
