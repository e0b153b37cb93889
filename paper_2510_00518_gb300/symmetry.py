"""Irreducible q-points: the space-group operations of a crystal and its force constants, the
orbits of the mesh under them, and rates of the whole mesh from one q per orbit.

The mode loops of Algorithms 1 and 3-5 run over N_bands x N_list modes, N_list being the
irreducible q-points.  Argument marshalling only: the operations, orbits and expansion are the
host calls fc4_symmetry_ops, fc4_irreducible_q and fc4_expand_irreducible of libfc4; the rates
of the irreducible points come from fc4_rates on the GPU.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import Engine, FC4Error, _np, _ptr, _structs, load

__all__ = ["symmetry_ops", "irreducible_q", "expand_irreducible", "rates_irreducible"]

TIME_REVERSAL = 1


def _check(lib, st):
    if st != 0:
        raise FC4Error(st, lib.fc4_last_error(None).decode())


def symmetry_ops(crystal, phi2, phi3=None, phi4=None, tol: float = 1e-8, max_ops: int = 48):
    """(W [n, 3, 3] int32, w [n, 3]): operations f -> W f + w of the primitive cell that map the
    atoms and every given cluster set onto themselves (fc4_symmetry_ops)."""
    lib = load()
    keep = []
    c, i2, i3, i4 = _structs(crystal, phi2, phi3, phi4, keep)
    rot = np.zeros((max_ops, 3, 3), np.int32)
    trans = np.zeros((max_ops, 3))
    n = ctypes.c_int(0)
    _check(lib, lib.fc4_symmetry_ops(ctypes.byref(c), ctypes.byref(i2), ctypes.byref(i3),
                                     ctypes.byref(i4), float(tol), int(max_ops), _ptr(rot),
                                     _ptr(trans), ctypes.cast(ctypes.pointer(n), ctypes.c_void_p)))
    return rot[:n.value].copy(), trans[:n.value].copy()


def irreducible_q(mesh, rot, time_reversal: bool = True):
    """(rep [N] int32, irr [n_irr] int32): rep[q] is the smallest q index of the orbit of q
    under the operations ``rot`` (and q -> -q); irr lists the representatives in ascending
    order (fc4_irreducible_q)."""
    lib = load()
    m = _np(mesh, np.int32)
    r = _np(rot, np.int32).reshape(-1, 3, 3)
    N = int(np.prod(m))
    rep = np.zeros(N, np.int32)
    n = ctypes.c_int(0)
    flags = TIME_REVERSAL if time_reversal else 0
    _check(lib, lib.fc4_irreducible_q(_ptr(m), r.shape[0], _ptr(r) if r.size else None, flags,
                                      _ptr(rep), ctypes.cast(ctypes.pointer(n), ctypes.c_void_p)))
    irr = np.flatnonzero(rep == np.arange(N)).astype(np.int32)
    if irr.size != n.value:
        raise FC4Error(1, f"fc4_irreducible_q: {n.value} orbits reported, {irr.size} representatives")
    return rep, irr


def expand_irreducible(mesh, nb: int, rep, omega, sub, deg_tol: float = 1e-5):
    """[n_sets, N*nb] values of every mode from ``sub`` [n_sets, n_irr*nb] on the irreducible
    points, averaged over degenerate branches (fc4_expand_irreducible)."""
    lib = load()
    m = _np(mesh, np.int32)
    N = int(np.prod(m))
    rp = _np(rep, np.int32)
    om = _np(omega, np.float64).reshape(-1)
    s = _np(sub, np.float64)
    s2 = s.reshape(-1, s.shape[-1]) if s.ndim > 1 else s.reshape(1, -1)
    full = np.zeros((s2.shape[0], N * nb))
    _check(lib, lib.fc4_expand_irreducible(_ptr(m), int(nb), _ptr(rp), _ptr(om), float(deg_tol),
                                           s2.shape[0], _ptr(s2), _ptr(full)))
    return full.reshape(s.shape[:-1] + (N * nb,)) if s.ndim > 1 else full[0]


def rates_irreducible(engine: Engine, T: float, sigma_thz: float, channel_mask: int = 31,
                      rot=None, time_reversal: bool = True, deg_tol: float = 1e-5):
    """Γ and WP of every mode of the mesh ([5, N*nb] float64 CUDA tensors) from fc4_rates with
    the fixed width ``sigma_thz`` on the irreducible q-points only, plus the number of those
    points.  ``rot``: the operations of ``symmetry_ops`` (None: time reversal only).  The adaptive
    width is not star-invariant (degenerate modes' velocities depend on the eigenvector basis),
    so it has no irreducible-point form."""
    import torch
    r = np.zeros((0, 3, 3), np.int32) if rot is None else rot
    rep, irr = irreducible_q(engine.mesh, r, time_reversal)
    g, wp, _ = engine.rates(T, sigma_thz, channel_mask, q_subset=irr)
    omega = engine.get_modes()[0]
    sub = np.stack([g.cpu().numpy(), wp.cpu().numpy()])
    full = expand_irreducible(engine.mesh, engine.nb, rep, omega, sub, deg_tol)
    out = torch.from_numpy(full).to(g.device)
    return out[0], out[1], int(irr.size)
