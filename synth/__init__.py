"""Seeded synthetic inputs shared by the CUDA path's tests, the bench and the oracle's callers.

This package builds crystals and force-constant clusters (the *inputs* of the scattering-rate
method) and draws seeded q-point samples.  It holds none of the method's arithmetic: no
dynamical matrix, no eigenvectors, no matrix elements, no rates.
"""
from .morse import (Crystal, IFC, MorseParams, diamond_crystal, morse_ifcs, morse_system,
                    random_cluster_ifcs, cell_energy, supercell_crystal, batch_crystal)
from .sampling import sample_q

__all__ = ["Crystal", "IFC", "MorseParams", "diamond_crystal", "morse_ifcs", "morse_system",
           "random_cluster_ifcs", "cell_energy", "supercell_crystal", "batch_crystal",
           "sample_q"]
