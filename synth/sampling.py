"""Seeded q-point samples (sorted indices into a Γ-centred mesh, first axis fastest)."""
import numpy as np


def sample_q(n_q: int, k: int, seed: int) -> np.ndarray:
    """``k`` distinct q indices out of ``n_q``, drawn with numpy's default_rng(seed), sorted."""
    if k >= n_q:
        return np.arange(n_q, dtype=np.int32)
    return np.sort(np.random.default_rng(seed).choice(n_q, k, replace=False)).astype(np.int32)
