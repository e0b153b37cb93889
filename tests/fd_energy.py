"""Finite differences of the unperturbed Morse energy of a periodic supercell (test helper).

Independent of every cluster, matrix-element and rate code: it evaluates only the pair
potential φ(r) on displaced atoms.  Energy differences are formed bond by bond in a
cancellation-free way, so mixed third and fourth derivatives can be taken accurately."""
from __future__ import annotations

import itertools
import math

import numpy as np

from synth.morse import MorseParams, _shell_cutoffs, bonds


class SupercellEnergy:
    def __init__(self, crystal, size: int, params: MorseParams | None = None, n_shells: int = 2):
        self.c = crystal
        self.L = size
        self.p = params or MorseParams()
        cut = _shell_cutoffs(crystal, n_shells)
        bl = bonds(crystal, cut)
        self.bi = np.array([b[0] for b in bl])
        self.bj = np.array([b[1] for b in bl])
        self.bR = np.array([b[2] for b in bl])
        self.bd = np.array([b[3] for b in bl])
        cells = np.array(list(itertools.product(range(size), repeat=3)))[:, ::-1]  # first axis fastest
        self.cells = cells
        self.ncell = cells.shape[0]
        tgt = (cells[:, None, :] + self.bR[None, :, :]) % size
        self.tgt = tgt[..., 0] + size * (tgt[..., 1] + size * tgt[..., 2])      # (ncell, nbond)
        self.src = np.arange(self.ncell)
        self.Rcart = cells.astype(float) @ crystal.lattice                          # (ncell, 3)

    def delta_energy(self, U: np.ndarray) -> float:
        """E(U) - E(0); U is (ncell, n_atoms, 3) in Å.  Each bond counted from both ends (1/2)."""
        d = self.bd[None, :, :]
        du = U[self.tgt, self.bj[None, :], :] - U[self.src[:, None], self.bi[None, :], :]
        r0 = np.linalg.norm(d, axis=-1)
        dd = d + du
        r1 = np.linalg.norm(dd, axis=-1)
        dr = (2.0 * np.sum(d * du, axis=-1) + np.sum(du * du, axis=-1)) / (r0 + r1)
        x0 = np.exp(-self.p.alpha * (r0 - self.p.r0))
        dx = x0 * np.expm1(-self.p.alpha * dr)
        de = self.p.D * dx * (2.0 * x0 + dx - 2.0)
        return 0.5 * float(np.sum(de))

    def pattern(self, e: np.ndarray, q: np.ndarray, imag: bool = False) -> np.ndarray:
        """Real displacement field Re(ũ_b exp(i q.R_l)) (or Im), ũ_b = e[3b:3b+3] / sqrt(m_b)."""
        ph = np.exp(1j * (self.Rcart @ q))                                          # (ncell,)
        u = e.reshape(self.c.n_atoms, 3) / np.sqrt(self.c.masses)[:, None]
        z = ph[:, None, None] * u[None, :, :]
        return z.imag if imag else z.real

    def mixed_derivative(self, patterns, h: float) -> float:
        """∂^k E / ∂t_1..∂t_k at t = 0 along the given patterns, central differences with one
        Richardson step (error O(h^4))."""
        k = len(patterns)

        def D(hh):
            tot = 0.0
            for s in itertools.product((1.0, -1.0), repeat=k):
                U = sum(si * hh * p for si, p in zip(s, patterns))
                tot += math.prod(s) * self.delta_energy(U)
            return tot / (2.0 ** k * hh ** k)

        return (4.0 * D(h) - D(2.0 * h)) / 3.0
