"""Many crystals in one CUDA-graph launch, with a small autotuner.

Each crystal is its own fc4 context (its own cell size, mesh and clusters).  ``BatchRunner``
runs the batch once eagerly (which sizes every buffer), then captures it on one stream into one
CUDA graph; ``run()`` replays it with a single launch.  ``persistent=False`` (the default) captures
every context's ``fc4_rates`` in turn (the tiled kernels for cells of up to two atoms).
``persistent=True`` captures one ``fc4_batch_rates`` call: the four-phonon units of all crystals of
the same cell size (more than two atoms) run as one persistent launch over a shared work list
(largest meshes first); it pays off for many small crystals, whose own launches leave the GPU
partly idle.  ``autotune`` picks the general four-phonon kernel's block size per context by timing
the candidates with CUDA events, and caches the choice in a JSON file keyed by the context's
shape (atoms, mesh, precision, subset size)."""
from __future__ import annotations

import json
import os


def _key(engine, n_q: int) -> str:
    i = engine.info()
    return f"na{i['n_atoms']}_N{i['N']}_p{i['precision']}_nq{n_q}"


def autotune(engine, T: float, sigma_thz: float, channel_mask: int, q_subset, cache: str | None = None,
             candidates=(64, 96, 128), repeats: int = 2) -> int:
    """Block size (threads) of the general four-phonon kernel that runs this call fastest."""
    import torch
    n_q = engine.nq if q_subset is None else len(q_subset)
    key = _key(engine, n_q)
    table = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
    if key in table:
        engine.set_block_threads(table[key])
        return table[key]
    best, best_ms = candidates[-1], float("inf")
    for bt in candidates:
        engine.set_block_threads(bt)
        engine.rates(T, sigma_thz, channel_mask, q_subset=q_subset)       # warm
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(repeats):
            engine.rates(T, sigma_thz, channel_mask, q_subset=q_subset)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / repeats
        if ms < best_ms:
            best, best_ms = bt, ms
    engine.set_block_threads(best)
    table[key] = best
    if cache:
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return best


class BatchRunner:
    """Rates of many contexts as one CUDA graph (one launch per ``run``)."""

    def __init__(self, jobs, T: float, sigma_thz: float, channel_mask: int = 31, persistent: bool = False):
        """jobs: list of (engine, q_subset or None)."""
        import torch
        from . import Batch
        self.jobs = jobs
        self.T, self.sigma, self.mask = T, sigma_thz, channel_mask
        self.stream = torch.cuda.Stream()
        self.batch = Batch([e for e, _ in jobs]) if persistent else None
        qsets = [qs for _, qs in jobs]
        with torch.cuda.stream(self.stream):           # eager pass: sizes all buffers
            if self.batch is not None:
                self.outs = self.batch.rates(T, sigma_thz, channel_mask, q_subsets=qsets, stream=self.stream)
            else:
                self.outs = [eng.rates(T, sigma_thz, channel_mask, q_subset=qs, stream=self.stream)
                             for eng, qs in jobs]
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream, capture_error_mode="thread_local"):
            if self.batch is not None:
                self.batch.rates(T, sigma_thz, channel_mask, q_subsets=qsets, outs=self.outs, stream=self.stream)
            else:
                for (eng, qs), out in zip(jobs, self.outs):
                    eng.rates(T, sigma_thz, channel_mask, q_subset=qs, out=out, stream=self.stream)

    def run(self):
        self.graph.replay()
        return [o[0] for o in self.outs]
