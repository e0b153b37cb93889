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
