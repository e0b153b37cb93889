"""Plain FP64 oracle of the three- and four-phonon scattering rates and the RTA conductivity.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA library and never imports it.

Split:
  * this module (NumPy, FP64): q-mesh, dynamical matrix, ``numpy.linalg.eigh`` as the harmonic
    eigensolver (a library primitive), group velocities, occupations, unit constants, κ;
  * ``fc4_oracle.c`` (plain C, FP64, no FMA contraction): enumeration, energy window,
    matrix elements, weights, Γ, WP, process lists and the analytic gradient.

The paper prints only the 3ph absorption loop (Algorithm 1) and the energy window; the readings
used for everything it leaves as black boxes are listed in ``fc4_oracle.c``'s header and below.
Parity of Γ and κ against the paper itself is unpinned (the paper prints no worked example);
they are pinned by invariants, closed forms and brute force in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

from .build import build as _build_lib

# ----------------------------------------------------------------------------- constants
# CODATA 2018 exact / recommended values (SI)
HBAR = 1.054571817e-34        # J s
EV = 1.602176634e-19          # J
AMU = 1.66053906660e-27       # kg
KB = 1.380649e-23             # J/K
ANG = 1e-10                   # m
PS = 1e-12                    # s

# dynamical-matrix eigenvalue eV/(Å² amu) -> ω² in (rad/ps)²
EIG_TO_RADPS2 = EV / (ANG ** 2 * AMU) * PS ** 2


def unit_constants_si() -> tuple[float, float]:
    """(C3, C4): Γ3 = C3/N Σ w|V3|², Γ4 = C4/N² Σ w|V4|² in ps^-1, with V3 in eV/Å³/amu^1.5,
    V4 in eV/Å⁴/amu², ω in rad/ps and δ in ps (so w is in ps⁴ resp. ps⁵).  SI route:
    Γ3 = ħπ/4 V² w, Γ4 = ħ²π/8 V² w, each quantity converted to SI, result converted to ps^-1."""
    fv3 = EV / ANG ** 3 / AMU ** 1.5
    fv4 = EV / ANG ** 4 / AMU ** 2
    c3 = HBAR * math.pi / 4.0 * fv3 ** 2 * PS ** 4 * PS
    c4 = HBAR ** 2 * math.pi / 8.0 * fv4 ** 2 * PS ** 5 * PS
    return c3, c4


def unit_constants_natural() -> tuple[float, float]:
    """Same constants through the natural unit system (amu, Å, ps): energy unit amu Å²/ps²."""
    e_nat = AMU * ANG ** 2 / PS ** 2          # J per natural energy unit
    hbar_nat = HBAR / (e_nat * PS)            # amu Å² / ps
    ev_nat = EV / e_nat                       # natural energy units per eV
    c3 = math.pi / 4.0 * hbar_nat * ev_nat ** 2
    c4 = math.pi / 8.0 * hbar_nat ** 2 * ev_nat ** 2
    return c3, c4


C3, C4 = unit_constants_si()


# ----------------------------------------------------------------------------- mesh

def reciprocal(lattice: np.ndarray) -> np.ndarray:
    """Rows b_i with a_i . b_j = 2π δ_ij, by the cross-product formula
    b_1 = 2π (a_2 x a_3) / (a_1 . (a_2 x a_3)) (cyclic), evaluated left to right in IEEE double."""
    a = [[float(x) for x in row] for row in np.asarray(lattice, dtype=np.float64)]

    def cross(u, v):
        return [u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]]

    c = [cross(a[1], a[2]), cross(a[2], a[0]), cross(a[0], a[1])]
    vol = a[0][0] * c[0][0] + a[0][1] * c[0][1] + a[0][2] * c[0][2]
    f = 2.0 * math.pi / vol
    return np.array([[f * c[i][x] for x in range(3)] for i in range(3)])


def q_coords(mesh) -> np.ndarray:
    """(N, 3) integer coordinates of the Γ-centred mesh, first axis fastest."""
    n1, n2, n3 = mesh
    idx = np.arange(n1 * n2 * n3)
    return np.stack([idx % n1, (idx // n1) % n2, idx // (n1 * n2)], axis=1)


def q_cart(lattice: np.ndarray, mesh) -> np.ndarray:
    """(N, 3) Cartesian q = Σ_k (i_k / n_k) b_k in rad/Å."""
    c = q_coords(mesh).astype(np.float64) / np.asarray(mesh, np.float64)
    return c @ reciprocal(lattice)


# ----------------------------------------------------------------------------- harmonic

class UnstableCrystal(ValueError):
    pass


@dataclass
class Modes:
    omega: np.ndarray      # (N*nb,) rad/ps; 0 for the excluded acoustic modes at Γ
    vel: np.ndarray        # (N*nb, 3) Å/ps
    evec: np.ndarray       # (N, nb, nb) complex; [q, component 3*atom+cart, branch]
    eig: np.ndarray        # (N, nb) raw eigenvalues eV/(Å² amu)


def dynamical_matrix(crystal, phi2, q: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """D(q) = Σ_R Φ2(0a, Rb) exp(i q.R) / sqrt(m_a m_b) (phase on the cell vector R) and its
    q-gradient dD/dq_x = Σ_R i R_x Φ2 exp(i q.R) / sqrt(m_a m_b), both Hermitised."""
    nb = crystal.nb
    D = np.zeros((nb, nb), complex)
    dD = np.zeros((3, nb, nb), complex)
    for at, cell, ph in zip(phi2.atoms, phi2.cells, phi2.phi):
        a, b = int(at[0]), int(at[1])
        R = cell[0].astype(np.float64) @ crystal.lattice
        f = np.exp(1j * float(q @ R)) / math.sqrt(crystal.masses[a] * crystal.masses[b])
        blk = ph.reshape(3, 3) * f
        D[3 * a:3 * a + 3, 3 * b:3 * b + 3] += blk
        for x in range(3):
            dD[x, 3 * a:3 * a + 3, 3 * b:3 * b + 3] += 1j * R[x] * blk
    D = 0.5 * (D + D.conj().T)
    dD = 0.5 * (dD + np.conj(np.transpose(dD, (0, 2, 1))))
    return D, dD


def harmonic(crystal, phi2, mesh, tol: float = 1e-8) -> Modes:
    """ω, v, e on the whole mesh.  ω = sqrt(λ) converted to rad/ps; an eigenvalue below -tol
    (eV/Å²/amu) raises UnstableCrystal; the three lowest branches at Γ are set to ω = 0."""
    qs = q_cart(crystal.lattice, mesh)
    N, nb = qs.shape[0], crystal.nb
    omega = np.zeros((N, nb))
    vel = np.zeros((N, nb, 3))
    evec = np.zeros((N, nb, nb), complex)
    eig = np.zeros((N, nb))
    for iq in range(N):
        D, dD = dynamical_matrix(crystal, phi2, qs[iq])
        lam, v = np.linalg.eigh(D)
        if lam.min() < -tol and not (iq == 0 and np.argmin(lam) < 3):
            raise UnstableCrystal(f"eigenvalue {lam.min():.3e} eV/A^2/amu at q index {iq}")
        eig[iq] = lam
        evec[iq] = v
        w = np.sign(lam) * np.sqrt(np.abs(lam) * EIG_TO_RADPS2)
        for j in range(nb):
            if iq == 0 and j < 3:
                continue
            if w[j] <= 0.0:
                raise UnstableCrystal(f"non-positive ω at q index {iq}, branch {j}")
            omega[iq, j] = w[j]
            g = np.array([np.real(np.conj(v[:, j]) @ dD[x] @ v[:, j]) for x in range(3)])
            vel[iq, j] = g * EIG_TO_RADPS2 / (2.0 * w[j])
    return Modes(omega.reshape(-1), vel.reshape(-1, 3), evec, eig)


def occupations(omega: np.ndarray, T: float) -> np.ndarray:
    """Bose-Einstein n(ω) = 1 / (exp(ħω / k_B T) - 1); 0 where ω = 0 (excluded modes)."""
    out = np.zeros_like(omega)
    m = omega > 0
    out[m] = 1.0 / np.expm1(HBAR * omega[m] * 1e12 / (KB * T))
    return out


def heat_capacity(omega: np.ndarray, T: float) -> np.ndarray:
    """Mode heat capacity C = k_B x² n (n + 1), x = ħω / k_B T (J/K); 0 for ω = 0."""
    n = occupations(omega, T)
    x = HBAR * omega * 1e12 / (KB * T)
    return KB * x * x * n * (n + 1.0)


def kappa(crystal, modes: Modes, T: float, gamma_total: np.ndarray, mesh) -> np.ndarray:
    """RTA κ_αβ = 1/(N V_cell) Σ_λ C_λ v_α v_β / Γ_λ in W/(m K).

    Modes with ω = 0 (excluded) or Γ_λ <= 0 are skipped."""
    N = int(np.prod(mesh))
    C = heat_capacity(modes.omega, T)
    k = np.zeros((3, 3))
    for m in range(modes.omega.shape[0]):
        if modes.omega[m] <= 0.0 or gamma_total[m] <= 0.0:
            continue
        v = modes.vel[m] * 100.0                     # Å/ps -> m/s
        tau = 1e-12 / gamma_total[m]                 # ps^-1 -> s
        k += C[m] * np.outer(v, v) * tau
    return k / (N * crystal.volume * 1e-30)


def kappa_of_F(crystal, modes: Modes, T: float, F: np.ndarray, mesh) -> np.ndarray:
    """κ_αβ = 1/(N V_cell) Σ_λ C_λ v_λα F_λβ in W/(m K) for deviation vectors F [N nb, 3] in
    Å/ps x ps (= Å): the RTA κ is the case F = v / Γ.  Modes with ω = 0 are skipped."""
    N = int(np.prod(mesh))
    C = heat_capacity(modes.omega, T)
    k = np.zeros((3, 3))
    for m in range(modes.omega.shape[0]):
        if modes.omega[m] <= 0.0:
            continue
        k += C[m] * np.outer(modes.vel[m] * 100.0, F[m] * 1e-10)       # m/s x m
    return k / (N * crystal.volume * 1e-30)


def rta_F(modes: Modes, gamma_total: np.ndarray) -> np.ndarray:
    """F⁰_λ = v_λ / Γ_λ (Å), zero for modes with ω = 0 or Γ_λ <= 0."""
    F = np.zeros_like(modes.vel)
    ok = (modes.omega > 0.0) & (gamma_total > 0.0)
    F[ok] = modes.vel[ok] / gamma_total[ok, None]
    return F


# ----------------------------------------------------------------------------- C oracle

class _Problem(ctypes.Structure):
    _fields_ = [
        ("n_atoms", ctypes.c_int), ("nb", ctypes.c_int), ("mesh", ctypes.c_int * 3),
        ("nq", ctypes.c_int), ("lattice", ctypes.c_double * 9), ("recip", ctypes.c_double * 9),
        ("mass", ctypes.c_void_p), ("omega", ctypes.c_void_p), ("vel", ctypes.c_void_p),
        ("evec", ctypes.c_void_p), ("occ", ctypes.c_void_p),
        ("nc3", ctypes.c_int), ("atoms3", ctypes.c_void_p), ("cells3", ctypes.c_void_p),
        ("phi3", ctypes.c_void_p),
        ("nc4", ctypes.c_int), ("atoms4", ctypes.c_void_p), ("cells4", ctypes.c_void_p),
        ("phi4", ctypes.c_void_p),
        ("sigma_adaptive", ctypes.c_int), ("sigma", ctypes.c_double),
        ("c3", ctypes.c_double), ("c4", ctypes.c_double),
        ("sample_all", ctypes.c_int), ("sample_threshold", ctypes.c_ulonglong),
        ("sample_seed", ctypes.c_ulonglong),
    ]


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build_lib()
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER(_Problem)
        vp = ctypes.c_void_p
        lib.fc4o_rates.argtypes = [P, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, vp, vp, vp]
        lib.fc4o_processes.argtypes = [P, ctypes.c_int, ctypes.c_int, vp, ctypes.c_longlong]
        lib.fc4o_processes.restype = ctypes.c_longlong
        lib.fc4o_grad.argtypes = [P, ctypes.c_int, vp, ctypes.c_int, vp, vp, vp]
        lib.fc4o_v3.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]
        lib.fc4o_v4.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, ctypes.c_int, vp]
        lib.fc4o_delta.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4
        lib.fc4o_delta.restype = ctypes.c_double
        lib.fc4o_occupation_factor.argtypes = [ctypes.c_int] + [ctypes.c_double] * 3
        lib.fc4o_occupation_factor.restype = ctypes.c_double
        lib.fc4o_sigma.argtypes = [P, ctypes.c_int, ctypes.c_int]
        lib.fc4o_sigma.restype = ctypes.c_double
        lib.fc4o_bte_offdiag.argtypes = [P, ctypes.c_int, vp, ctypes.c_int, vp, vp]
        lib.fc4o_splitmix64_mix.argtypes = [ctypes.c_ulonglong]
        lib.fc4o_splitmix64_mix.restype = ctypes.c_ulonglong
        _LIB = lib
    return _LIB


def delta(ch: int, w: float, w1: float, w2: float, w3: float = 0.0) -> float:
    """The oracle's energy mismatch Δ of channel ch (canonical parenthesisation)."""
    return _lib().fc4o_delta(ch, w, w1, w2, w3)


def occupation_factor(ch: int, n1: float, n2: float, n3: float = 0.0) -> float:
    """The oracle's occupation factor F of channel ch."""
    return _lib().fc4o_occupation_factor(ch, n1, n2, n3)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


SIGMA_THZ_TO_RADPS = 2.0 * math.pi


def sample_threshold(fraction: float) -> tuple[int, int]:
    """(take every pair, threshold) of the four-phonon sampling estimate: a partner pair is taken
    iff its 64-bit hash is below floor(f 2^64); f >= 1 takes every pair."""
    if not (fraction > 0.0):
        raise ValueError("the sampling fraction must be > 0")
    if fraction >= 1.0:
        return 1, 0xFFFFFFFFFFFFFFFF
    return 0, int(math.ldexp(fraction, 64))


def splitmix64_mix(z: int) -> int:
    """The oracle's SplitMix64 output function (C), for its pins."""
    return int(_lib().fc4o_splitmix64_mix(z & 0xFFFFFFFFFFFFFFFF))


class Problem:
    """A crystal, its clusters, a mesh, the harmonic modes and (T, σ): the oracle's input.

    ``modes`` defaults to the oracle's own harmonic solution; pass a Modes object to evaluate
    the rates for given ω, v, e.  ``sigma`` is a fixed width in THz (σ = 2π value rad/ps) or,
    with ``sigma_adaptive``, the scale factor of the adaptive width."""

    def __init__(self, crystal, phi2, phi3, phi4, mesh, T=300.0, sigma=0.1,
                 sigma_adaptive=False, modes: Modes | None = None, sample_fraction: float = 1.0,
                 sample_seed: int = 0):
        self.crystal, self.phi2, self.phi3, self.phi4 = crystal, phi2, phi3, phi4
        self.mesh = tuple(int(x) for x in mesh)
        self.nq = int(np.prod(self.mesh))
        self.nb = crystal.nb
        self.T = float(T)
        self.sigma = float(sigma)
        self.sigma_adaptive = bool(sigma_adaptive)
        self.modes = modes if modes is not None else harmonic(crystal, phi2, self.mesh)
        self.sample_fraction = float(sample_fraction)
        self.sample_seed = int(sample_seed)
        self._refresh()

    def _refresh(self):
        c = self.crystal
        self._keep = []
        def arr(x, dt):
            a = np.ascontiguousarray(x, dtype=dt)
            self._keep.append(a)
            return a
        s = _Problem()
        s.n_atoms, s.nb = c.n_atoms, c.nb
        s.mesh = (ctypes.c_int * 3)(*self.mesh)
        s.nq = self.nq
        s.lattice = (ctypes.c_double * 9)(*c.lattice.reshape(-1))
        s.recip = (ctypes.c_double * 9)(*reciprocal(c.lattice).reshape(-1))
        s.mass = _ptr(arr(c.masses, np.float64))
        s.omega = _ptr(arr(self.modes.omega, np.float64))
        s.vel = _ptr(arr(self.modes.vel, np.float64))
        ev = np.ascontiguousarray(self.modes.evec, np.complex128)
        s.evec = _ptr(arr(ev.view(np.float64), np.float64))
        s.occ = _ptr(arr(occupations(self.modes.omega, self.T), np.float64))
        s.nc3 = self.phi3.n_clusters
        s.atoms3 = _ptr(arr(self.phi3.atoms, np.int32))
        s.cells3 = _ptr(arr(self.phi3.cells, np.int32))
        s.phi3 = _ptr(arr(self.phi3.phi, np.float64))
        s.nc4 = self.phi4.n_clusters
        s.atoms4 = _ptr(arr(self.phi4.atoms, np.int32))
        s.cells4 = _ptr(arr(self.phi4.cells, np.int32))
        s.phi4 = _ptr(arr(self.phi4.phi, np.float64))
        s.sigma_adaptive = int(self.sigma_adaptive)
        s.sigma = self.sigma * (1.0 if self.sigma_adaptive else SIGMA_THZ_TO_RADPS)
        s.c3, s.c4 = C3, C4
        s.sample_all, s.sample_threshold = sample_threshold(self.sample_fraction)
        s.sample_seed = self.sample_seed & 0xFFFFFFFFFFFFFFFF
        self._s = s

    def with_anharmonic(self, phi3=None, phi4=None) -> "Problem":
        """Same problem and modes with replaced Φ3 / Φ4 clusters."""
        return Problem(self.crystal, self.phi2, phi3 or self.phi3, phi4 or self.phi4, self.mesh,
                       self.T, self.sigma, self.sigma_adaptive, self.modes, self.sample_fraction,
                       self.sample_seed)

    def with_T(self, T: float) -> "Problem":
        return Problem(self.crystal, self.phi2, self.phi3, self.phi4, self.mesh, T, self.sigma,
                       self.sigma_adaptive, self.modes, self.sample_fraction, self.sample_seed)

    def with_sampling(self, fraction: float, seed: int) -> "Problem":
        """Same problem with the four-phonon sampling estimate (fraction f of partner pairs)."""
        return Problem(self.crystal, self.phi2, self.phi3, self.phi4, self.mesh, self.T, self.sigma,
                       self.sigma_adaptive, self.modes, fraction, seed)

    # -- calls into the C oracle -----------------------------------------------------------
    def rates(self, modes=None, channel_mask: int = 31, qp_limit: int = 0):
        """(gamma, wp, counts), each [5][n_modes]: channels 3ph+, 3ph-, 4ph++, 4ph+-, 4ph--."""
        m = np.arange(self.nq * self.nb, dtype=np.int32) if modes is None else \
            np.ascontiguousarray(modes, np.int32)
        g = np.zeros((5, m.size))
        wp = np.zeros((5, m.size))
        cnt = np.zeros((5, m.size), np.int64)
        _lib().fc4o_rates(ctypes.byref(self._s), m.size, _ptr(m), channel_mask, qp_limit,
                          _ptr(g), _ptr(wp), _ptr(cnt))
        return g, wp, cnt

    def processes(self, channel: int, mode: int) -> np.ndarray:
        """Canonical process words of one mode and channel (uint64)."""
        n = _lib().fc4o_processes(ctypes.byref(self._s), channel, mode, None, 0)
        out = np.zeros(max(n, 1), np.uint64)
        _lib().fc4o_processes(ctypes.byref(self._s), channel, mode, _ptr(out), n)
        return out[:n]

    def grad(self, modes, dL_dgamma, channel_mask: int = 31):
        """(dL/dΦ3 [nc3, 27], dL/dΦ4 [nc4, 81]) for L = Σ dL_dgamma[ch, i] Γ_ch(modes[i])."""
        m = np.ascontiguousarray(modes, np.int32)
        dg = np.ascontiguousarray(dL_dgamma, np.float64).reshape(5, m.size)
        g3 = np.zeros((self.phi3.n_clusters, 27))
        g4 = np.zeros((self.phi4.n_clusters, 81))
        _lib().fc4o_grad(ctypes.byref(self._s), m.size, _ptr(m), channel_mask, _ptr(dg),
                         _ptr(g3), _ptr(g4))
        return g3, g4

    def v3(self, s: int, m0: int, m1: int, m2: int) -> complex:
        out = np.zeros(2)
        _lib().fc4o_v3(ctypes.byref(self._s), s, m0, m1, m2, _ptr(out))
        return complex(out[0], out[1])

    def v4(self, s1: int, s2: int, m0: int, m1: int, m2: int, m3: int) -> complex:
        out = np.zeros(2)
        _lib().fc4o_v4(ctypes.byref(self._s), s1, s2, m0, m1, m2, m3, _ptr(out))
        return complex(out[0], out[1])

    def sigma_of(self, ma: int, mb: int) -> float:
        """Broadening (rad/ps) of a process whose free legs are modes ma, mb."""
        return _lib().fc4o_sigma(ctypes.byref(self._s), ma, mb)

    def kappa(self, gamma_total: np.ndarray) -> np.ndarray:
        return kappa(self.crystal, self.modes, self.T, gamma_total, self.mesh)

    # -- iterative Boltzmann equation ------------------------------------------------------
    def bte_offdiag(self, F: np.ndarray, modes=None, channel_mask: int = 31) -> np.ndarray:
        """Δ_λ [n_modes, 3] = Σ_processes γ_p Σ_k s_k (ω_k / ω_λ) F_k (fc4_oracle.c: iterative
        BTE) for deviation vectors F [N nb, 3]."""
        m = np.arange(self.nq * self.nb, dtype=np.int32) if modes is None else \
            np.ascontiguousarray(modes, np.int32)
        Fc = np.ascontiguousarray(F, np.float64).reshape(self.nq * self.nb, 3)
        out = np.zeros((m.size, 3))
        _lib().fc4o_bte_offdiag(ctypes.byref(self._s), m.size, _ptr(m), channel_mask, _ptr(Fc), _ptr(out))
        return out

    def kappa_iterative(self, gamma_total: np.ndarray, channel_mask: int = 31, tol: float = 1e-10,
                        max_iter: int = 200):
        """Iterative solution of the linearised BTE: F⁰ = v / Γ, F^{n+1} = (v + Δ(F^n)) / Γ until
        the relative change of κ is below tol.  Returns (κ, F, iterations, κ of every iterate)."""
        F = rta_F(self.modes, gamma_total)
        ok = (self.modes.omega > 0.0) & (gamma_total > 0.0)
        ks = [kappa_of_F(self.crystal, self.modes, self.T, F, self.mesh)]
        for it in range(1, max_iter + 1):
            D = self.bte_offdiag(F, None, channel_mask)
            Fn = np.zeros_like(F)
            Fn[ok] = (self.modes.vel[ok] + D[ok]) / gamma_total[ok, None]
            F = Fn
            ks.append(kappa_of_F(self.crystal, self.modes, self.T, F, self.mesh))
            if np.abs(ks[-1] - ks[-2]).max() <= tol * np.abs(ks[-1]).max():
                return ks[-1], F, it, ks
        return ks[-1], F, max_iter, ks


# process-word helpers (canonical encodings)
def decode3(word: int, nb: int):
    """3ph word -> (q', j', j'')."""
    j2 = word % nb
    m1 = word // nb
    return m1 // nb, m1 % nb, j2


def decode4(word: int, nb: int, nq: int):
    """4ph word -> (q', j', q'', j'', j''')."""
    j3 = word % nb
    w = word // nb
    j2 = w % nb
    w //= nb
    q2 = w % nq
    m1 = w // nq
    return m1 // nb, m1 % nb, q2, j2, j3


CHANNELS = ("3ph+", "3ph-", "4ph++", "4ph+-", "4ph--")
