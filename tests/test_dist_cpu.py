"""Multi-rank logic on CPU (gloo, world size 2): mode sharding and the κ all-reduce.

Each rank evaluates the oracle's rates for its shard of q points, forms its κ contribution with
the Γ of all other modes set to zero (such modes are skipped), and one all-reduce of 9 doubles
must give the κ of the unsharded computation."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2510_00518_gb300.dist import allreduce_kappa, shard_q


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    import oracle
    from synth import morse_system
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        P = oracle.Problem(*morse_system(seed=0), (2, 2, 2))
        qs = shard_q(P.nq, rank, world)
        modes = np.array([q * P.nb + j for q in qs for j in range(P.nb)], np.int32)
        g, _, _ = P.rates(modes, channel_mask=0b11)
        full = np.zeros(P.nq * P.nb)
        full[modes] = g.sum(0)
        part = torch.tensor(P.kappa(full).reshape(-1))
        tot = allreduce_kappa(part).numpy()
        np.save(os.path.join(out_dir, f"k{rank}.npy"), tot)
    finally:
        dist.destroy_process_group()


def test_shard_q_partition():
    for n, w in [(27, 2), (512, 8), (5, 8), (1, 1)]:
        parts = [shard_q(n, r, w) for r in range(w)]
        allq = np.concatenate(parts)
        assert np.array_equal(allq, np.arange(n))
        sizes = [p.size for p in parts]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_q(10, 2, 2)


def test_two_rank_kappa_allreduce(tmp_path):
    import oracle
    from synth import morse_system
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    P = oracle.Problem(*morse_system(seed=0), (2, 2, 2))
    g, _, _ = P.rates(channel_mask=0b11)
    ref = P.kappa(g.sum(0)).reshape(-1)
    for r in range(world):
        k = np.load(tmp_path / f"k{r}.npy")
        assert np.allclose(k, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


class _OracleEngine:
    """The calls sharded_rates_kappa_irreducible makes on an Engine, answered by the oracle."""

    def __init__(self, P):
        self.P, self.mesh, self.nq, self.nb = P, P.mesh, P.nq, P.nb

    def rates(self, T, sigma_thz, channel_mask, q_subset=None):
        qs = np.arange(self.nq) if q_subset is None else np.asarray(q_subset)
        modes = (qs[:, None] * self.nb + np.arange(self.nb)).reshape(-1).astype(np.int32)
        g, wp, cnt = self.P.rates(modes, channel_mask=channel_mask)
        return torch.from_numpy(g), torch.from_numpy(wp), torch.from_numpy(cnt)

    def get_modes(self):
        return self.P.modes.omega, self.P.modes.vel, self.P.modes.evec

    def kappa(self, T, gamma, channel_mask):
        g = gamma.numpy()
        tot = sum(g[ch] for ch in range(5) if channel_mask >> ch & 1)
        return torch.from_numpy(self.P.kappa(tot).reshape(-1))


def _worker_irreducible(rank, world, port, out_dir):
    import oracle
    from synth import morse_system
    from paper_2510_00518_gb300.dist import sharded_rates_kappa_irreducible
    from paper_2510_00518_gb300.symmetry import symmetry_ops
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sysm = morse_system(seed=0, perturb=0.0)
        rot, _ = symmetry_ops(*sysm)
        eng = _OracleEngine(oracle.Problem(*sysm, (4, 4, 4)))
        mine, g, k = sharded_rates_kappa_irreducible(eng, 300.0, 0.1, rot, channel_mask=0b11)
        np.save(os.path.join(out_dir, f"irr{rank}.npy"), mine)
        np.save(os.path.join(out_dir, f"ki{rank}.npy"), k.numpy())
    finally:
        dist.destroy_process_group()


def test_two_rank_irreducible_kappa(tmp_path):
    """The 8 irreducible points of the symmetric 4x4x4 mesh split over two ranks: disjoint blocks
    covering them all, and the all-reduced κ equals the oracle's full-mesh κ."""
    import oracle
    from synth import morse_system
    from paper_2510_00518_gb300 import build as fc4_build
    fc4_build.build()
    world = 2
    mp.start_processes(_worker_irreducible, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    mine = [np.load(tmp_path / f"irr{r}.npy") for r in range(world)]
    allq = np.concatenate(mine)
    assert allq.size == 8 and np.unique(allq).size == 8
    P = oracle.Problem(*morse_system(seed=0, perturb=0.0), (4, 4, 4))
    g, _, _ = P.rates(channel_mask=0b11)
    ref = P.kappa(g.sum(0)).reshape(-1)
    for r in range(world):
        k = np.load(tmp_path / f"ki{r}.npy").reshape(-1)
        assert np.allclose(k, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())


class _OracleGradEngine(_OracleEngine):
    """Adds the calls of the sharded adjoint: fc4_kappa_backward (dκ/dΓ = -C v v / (N V Γ²) of the
    oracle's κ) and fc4_rates_backward (the oracle's analytic gradient for the last rates call)."""

    def __init__(self, P):
        super().__init__(P)
        self.nc3, self.nc4 = P.phi3.n_clusters, P.phi4.n_clusters
        self._modes = None

    def rates(self, T, sigma_thz, channel_mask, q_subset=None):
        qs = np.arange(self.nq) if q_subset is None else np.asarray(q_subset)
        self._modes = (qs[:, None] * self.nb + np.arange(self.nb)).reshape(-1).astype(np.int32)
        self._mask = channel_mask
        return super().rates(T, sigma_thz, channel_mask, q_subset)

    def kappa_backward(self, T, gamma, dk, channel_mask):
        import oracle
        P = self.P
        g = gamma.numpy()
        tot = sum(g[ch] for ch in range(5) if channel_mask >> ch & 1)
        C = oracle.heat_capacity(P.modes.omega, T)
        out = np.zeros_like(g)
        G = dk.numpy()
        for m in range(tot.size):
            if P.modes.omega[m] <= 0 or tot[m] <= 0:
                continue
            v = P.modes.vel[m] * 100.0
            d = -C[m] * (v @ G @ v) * 1e-12 / tot[m] ** 2 / (self.nq * P.crystal.volume * 1e-30)
            for ch in range(5):
                if channel_mask >> ch & 1:
                    out[ch, m] = d
        return torch.from_numpy(out)

    def backward(self, dg):
        g3, g4 = self.P.grad(self._modes, dg.numpy(), self._mask)
        return torch.from_numpy(g3), torch.from_numpy(g4)


def _worker_grad(rank, world, port, out_dir):
    import oracle
    from synth import morse_system
    from paper_2510_00518_gb300.dist import sharded_kappa_gradient
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    if world > 1:
        dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        eng = _OracleGradEngine(oracle.Problem(*morse_system(seed=0), (3, 2, 2)))
        dk = np.array([[1.0, 0.2, 0.0], [0.2, -0.5, 0.1], [0.0, 0.1, 0.3]])
        k, d3, d4 = sharded_kappa_gradient(eng, 300.0, 0.1, dk, channel_mask=0b11)
        np.save(os.path.join(out_dir, f"g{world}_{rank}.npy"), np.concatenate([k.numpy().reshape(-1), d3.numpy().reshape(-1)]))
    finally:
        if world > 1:
            dist.destroy_process_group()


def test_two_rank_gradient_allreduce(tmp_path):
    """dL/dΦ3 of L = Σ G κ with the modes split over two ranks (rates, κ all-reduce, adjoint of each
    rank's own modes, one gradient all-reduce) equals the single-rank result."""
    _worker_grad(0, 1, _free_port(), str(tmp_path))
    mp.start_processes(_worker_grad, args=(2, _free_port(), str(tmp_path)), nprocs=2,
                       start_method="spawn", join=True)
    ref = np.load(tmp_path / "g1_0.npy")
    assert np.abs(ref[9:]).max() > 0
    for r in range(2):
        x = np.load(tmp_path / f"g2_{r}.npy")
        assert np.allclose(x, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
