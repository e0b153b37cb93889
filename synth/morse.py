"""Synthetic crystals and force-constant clusters from a Morse pair potential.

The paper benchmarks silicon with first-principles force constants (Results section).  Those
are not available here, so every workload is a seeded synthetic crystal whose harmonic (Φ2),
cubic (Φ3) and quartic (Φ4) force constants are analytic derivatives of a Morse pair potential

    φ(r) = D [exp(-2α(r - r0)) - 2 exp(-α(r - r0))].

Construction (the reading used throughout this repository):

* Φ2 comes from the nearest-neighbour shell only, including the tension term φ'/r.  With the
  second-neighbour shell the diamond crystal at a = 5.43 Å has imaginary modes, because
  φ''(r_2NN) < 0.
* Φ3 and Φ4 come from the first two neighbour shells.
* Seeded perturbations of relative size ``perturb`` (default 1 %) multiply the four radial
  derivatives φ', φ'', φ''', φ'''' of each bond.  A bond is an unordered pair of sites, so
  (i, 0; j, R) and (j, 0; i, -R) share one draw.  Every cluster, including the on-site
  (self) terms, is then assembled from the perturbed scalars.  This keeps the index
  permutation symmetry and the translational (acoustic) sum rule of every order exactly.

Cluster format (shared with the C interface):
    atoms [nc][order]        basis-atom index of each leg; leg 0 sits in the home cell
    cells [nc][order-1][3]   integer lattice coordinates of legs 1.. (R = n1 a1 + n2 a2 + n3 a3)
    phi   [nc][3**order]     eV/Å^order, last Cartesian index fastest

Units: Å, amu, eV.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Crystal:
    lattice: np.ndarray       # (3,3) rows a1, a2, a3 in Å
    positions: np.ndarray     # (n,3) Cartesian Å
    masses: np.ndarray        # (n,) amu

    @property
    def n_atoms(self) -> int:
        return int(self.positions.shape[0])

    @property
    def nb(self) -> int:
        return 3 * self.n_atoms

    @property
    def volume(self) -> float:
        return float(abs(np.linalg.det(self.lattice)))


@dataclass
class IFC:
    order: int
    atoms: np.ndarray         # (nc, order) int32
    cells: np.ndarray         # (nc, order-1, 3) int32
    phi: np.ndarray           # (nc, 3**order) float64

    @property
    def n_clusters(self) -> int:
        return int(self.atoms.shape[0])

    def copy(self) -> "IFC":
        return IFC(self.order, self.atoms.copy(), self.cells.copy(), self.phi.copy())


@dataclass
class MorseParams:
    D: float = 2.0            # eV
    alpha: float = 1.5        # 1/Å
    r0: float = 2.35          # Å

    def radial_derivatives(self, r: float) -> np.ndarray:
        """[φ', φ'', φ''', φ''''] at r (closed forms of the Morse function)."""
        x = math.exp(-self.alpha * (r - self.r0))
        D, a = self.D, self.alpha
        return np.array([2 * D * a * (x - x * x),
                         2 * D * a ** 2 * (2 * x * x - x),
                         2 * D * a ** 3 * (x - 4 * x * x),
                         2 * D * a ** 4 * (8 * x * x - x)])

    def energy(self, r: float) -> float:
        x = math.exp(-self.alpha * (r - self.r0))
        return self.D * (x * x - 2 * x)


def diamond_crystal(a: float = 5.43, mass: float = 28.0855) -> Crystal:
    """Two-atom diamond cell: fcc lattice, basis (0,0,0) and (a/4)(1,1,1)."""
    lat = 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
    pos = np.array([[0.0, 0.0, 0.0], [0.25 * a, 0.25 * a, 0.25 * a]])
    return Crystal(lat, pos, np.array([mass, mass]))


def supercell_crystal(base: Crystal, k: int, masses: np.ndarray | None = None) -> Crystal:
    """1 x 1 x k supercell of ``base`` along a3 (n_atoms * k sites)."""
    lat = base.lattice.copy()
    lat[2] = k * base.lattice[2]
    pos = np.concatenate([base.positions + m * base.lattice[2] for m in range(k)])
    if masses is None:
        masses = np.tile(base.masses, k)
    return Crystal(lat, pos, np.asarray(masses, dtype=np.float64))


def batch_crystal(seed: int, a: float = 5.43) -> tuple[Crystal, tuple[int, int, int]]:
    """Crystal ``seed`` of the many-crystal batch: a 1x1xk diamond supercell with k = 1 + seed % 4
    (2, 4, 6 or 8 atoms; 6 to 24 branches), site masses uniform in [10, 120) amu, and a
    Γ-centred mesh of 12³, 10³, 8³ or 6³ q-points for k = 1, 2, 3, 4."""
    k = 1 + seed % 4
    rng = np.random.default_rng(1000 + seed)
    base = diamond_crystal(a)
    masses = rng.uniform(10.0, 120.0, size=2 * k)
    n = {1: 12, 2: 10, 3: 8, 4: 6}[k]
    return supercell_crystal(base, k, masses), (n, n, n)


# ----------------------------------------------------------------------------- neighbours

def _shell_cutoffs(crystal: Crystal, n_shells: int, search: int = 3) -> float:
    """Radius half-way between neighbour shell ``n_shells`` and the next one."""
    d = []
    for i in range(crystal.n_atoms):
        for j in range(crystal.n_atoms):
            for R in itertools.product(range(-search, search + 1), repeat=3):
                v = crystal.positions[j] + np.asarray(R) @ crystal.lattice - crystal.positions[i]
                r = float(np.linalg.norm(v))
                if r > 1e-8:
                    d.append(round(r, 6))
    shells = sorted(set(d))
    return 0.5 * (shells[n_shells - 1] + shells[n_shells])


def bonds(crystal: Crystal, cutoff: float, search: int = 3):
    """All bonds seen from each home atom: list of (i, j, R (3 ints), d = r_jR - r_i0)."""
    out = []
    for i in range(crystal.n_atoms):
        for j in range(crystal.n_atoms):
            for R in itertools.product(range(-search, search + 1), repeat=3):
                v = crystal.positions[j] + np.asarray(R, float) @ crystal.lattice - crystal.positions[i]
                r = float(np.linalg.norm(v))
                if 1e-8 < r < cutoff:
                    out.append((i, j, tuple(int(x) for x in R), v))
    return out


def _bond_class(i: int, j: int, R: tuple) -> tuple:
    """Canonical key of the unordered pair {(i, 0), (j, R)} up to a lattice translation."""
    a = (i, j, R)
    b = (j, i, tuple(-x for x in R))
    return min(a, b)


def bond_factors(crystal: Crystal, cutoff: float, seed: int, perturb: float) -> dict:
    """One draw of four radial-derivative factors (1 + perturb * U(-1, 1)) per unordered bond."""
    keys = sorted({_bond_class(i, j, R) for (i, j, R, _) in bonds(crystal, cutoff)})
    rng = np.random.default_rng(seed)
    out = {}
    for k in keys:
        u = rng.uniform(-1.0, 1.0, size=4)
        out[k] = 1.0 + perturb * u
    return out


# ----------------------------------------------------------------------------- tensors

def _h_derivatives(dphi: np.ndarray, r: float) -> np.ndarray:
    """Derivatives h^(k)(s), k = 1..4, of h(s) = φ(sqrt(2 s)) from φ^(k)(r) (d/ds = (1/r) d/dr)."""
    p1, p2, p3, p4 = dphi
    h1 = p1 / r
    h2 = p2 / r ** 2 - p1 / r ** 3
    h3 = p3 / r ** 3 - 3 * p2 / r ** 4 + 3 * p1 / r ** 5
    h4 = p4 / r ** 4 - 6 * p3 / r ** 5 + 15 * p2 / r ** 6 - 15 * p1 / r ** 7
    return np.array([h1, h2, h3, h4])


def pair_tensor(order: int, d: np.ndarray, dphi: np.ndarray) -> np.ndarray:
    """order-th Cartesian derivative tensor of f(d) = φ(|d|), given the radial derivatives."""
    r = float(np.linalg.norm(d))
    h1, h2, h3, h4 = _h_derivatives(dphi, r)
    I = np.eye(3)
    if order == 2:
        return h2 * np.einsum("a,b->ab", d, d) + h1 * I
    if order == 3:
        return (h3 * np.einsum("a,b,c->abc", d, d, d)
                + h2 * (np.einsum("ab,c->abc", I, d) + np.einsum("ac,b->abc", I, d)
                        + np.einsum("bc,a->abc", I, d)))
    if order == 4:
        dd = np.einsum("a,b->ab", d, d)
        return (h4 * np.einsum("a,b,c,e->abce", d, d, d, d)
                + h3 * (np.einsum("ab,ce->abce", I, dd) + np.einsum("ac,be->abce", I, dd)
                        + np.einsum("ae,bc->abce", I, dd) + np.einsum("bc,ae->abce", I, dd)
                        + np.einsum("be,ac->abce", I, dd) + np.einsum("ce,ab->abce", I, dd))
                + h2 * (np.einsum("ab,ce->abce", I, I) + np.einsum("ac,be->abce", I, I)
                        + np.einsum("ae,bc->abce", I, I)))
    raise ValueError(order)


def _assemble(crystal: Crystal, order: int, cutoff: float, params: MorseParams,
              factors: dict | None) -> IFC:
    """Clusters with leg 0 on home atom x = (i, 0); legs 1.. on x or on the bond partner y.

    A pair term f(r_y - r_x) contributes (-1)^(number of legs on x) * T^(order) to the cluster,
    since d/du_x = -d/dd and d/du_y = +d/dd."""
    acc: dict = {}
    order_keys = []
    for (i, j, R, d) in bonds(crystal, cutoff):
        dphi = params.radial_derivatives(float(np.linalg.norm(d)))
        if factors is not None:
            dphi = dphi * factors[_bond_class(i, j, R)]
        T = pair_tensor(order, d, dphi).reshape(-1)
        for pattern in itertools.product((0, 1), repeat=order - 1):
            n_x = 1 + sum(1 for p in pattern if p == 0)
            atoms = (i,) + tuple(i if p == 0 else j for p in pattern)
            cells = tuple((0, 0, 0) if p == 0 else R for p in pattern)
            key = (atoms, cells)
            if key not in acc:
                acc[key] = np.zeros(3 ** order)
                order_keys.append(key)
            acc[key] += (-1.0) ** n_x * T
    keys = sorted(order_keys)
    atoms = np.array([k[0] for k in keys], dtype=np.int32)
    cells = np.array([k[1] for k in keys], dtype=np.int32).reshape(len(keys), order - 1, 3)
    phi = np.array([acc[k] for k in keys], dtype=np.float64)
    return IFC(order, atoms, cells, phi)


def morse_ifcs(crystal: Crystal, params: MorseParams | None = None, seed: int = 0,
               perturb: float = 0.01, harmonic_shells: int = 1, anharmonic_shells: int = 2):
    """(Φ2, Φ3, Φ4) clusters of ``crystal`` (see module docstring for the construction)."""
    params = params or MorseParams()
    cut2 = _shell_cutoffs(crystal, harmonic_shells)
    cut34 = _shell_cutoffs(crystal, anharmonic_shells)
    f34 = bond_factors(crystal, cut34, seed, perturb) if perturb else None
    # harmonic bonds are a subset of the anharmonic ones: they reuse the same draws
    phi2 = _assemble(crystal, 2, cut2, params, f34)
    phi3 = _assemble(crystal, 3, cut34, params, f34)
    phi4 = _assemble(crystal, 4, cut34, params, f34)
    return phi2, phi3, phi4


def morse_system(seed: int = 0, perturb: float = 0.01, a: float = 5.43, mass: float = 28.0855,
                 params: MorseParams | None = None):
    """The two-atom Morse diamond crystal and its clusters (D=2 eV, α=1.5/Å, r0=2.35 Å)."""
    c = diamond_crystal(a, mass)
    return (c,) + morse_ifcs(c, params, seed=seed, perturb=perturb)


def cell_energy(crystal: Crystal, U: np.ndarray, params: MorseParams | None = None,
                n_shells: int = 2) -> float:
    """Unperturbed Morse energy per cell when every cell's atom b is displaced by U[b] (Å).

    Each unordered bond is listed from both ends, hence the factor 1/2."""
    params = params or MorseParams()
    cut = _shell_cutoffs(crystal, n_shells)
    e = 0.0
    for (i, j, R, d) in bonds(crystal, cut):
        e += 0.5 * params.energy(float(np.linalg.norm(d + U[j] - U[i])))
    return e


def random_cluster_ifcs(crystal: Crystal, order: int, n_clusters: int, seed: int,
                        max_cell: int = 1, scale: float = 1.0) -> IFC:
    """Random clusters whose legs sit on up to ``order`` distinct sites (no pair structure,
    no symmetry): a generic input for kernels that must not assume the Morse structure."""
    rng = np.random.default_rng(seed)
    seen = set()
    atoms, cells, phis = [], [], []
    while len(atoms) < n_clusters:
        a = tuple(int(x) for x in rng.integers(0, crystal.n_atoms, size=order))
        c = tuple(tuple(int(x) for x in rng.integers(-max_cell, max_cell + 1, size=3))
                  for _ in range(order - 1))
        if (a, c) in seen:
            continue
        seen.add((a, c))
        atoms.append(a)
        cells.append(c)
        phis.append(scale * rng.standard_normal(3 ** order))
    return IFC(order, np.array(atoms, np.int32),
               np.array(cells, np.int32).reshape(n_clusters, order - 1, 3),
               np.array(phis, np.float64))
