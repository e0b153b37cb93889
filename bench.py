#!/usr/bin/env python3
"""Throughput of the three- and four-phonon scattering-rate path on GB300.

One step = one pass of the hot path over the workload: the 3ph and 4ph rates Γ of every mode
(enumeration, energy window, matrix elements, weights, reduction; fc4_rates with all five
channels) followed by the RTA conductivity κ (fc4_kappa), inputs resident in HBM.  The metric
is kept four-phonon processes per second.  The end-to-end figure ("e2e") times the same work
through the C interface from host buffers: fc4_init (host-to-device copy of the crystal and
clusters, device harmonic solve, phase tables), fc4_rates, fc4_kappa, the device-to-host copy
of Γ, WP, counts and κ, and fc4_destroy.

Workload: two-atom Morse diamond crystal (a = 5.43 Å, m = 28.0855 amu, D = 2 eV, α = 1.5/Å,
r0 = 2.35 Å, seeded 1 % bond perturbations), Γ-centred 8x8x8 mesh (512 q, 3072 modes),
T = 300 K, fixed Gaussian σ = 0.1 THz.  Synthetic: no first-principles force constants.

--impl reference times the FP64 CPU oracle (the test reference) on the same workload, on a
bounded sample of modes and partners per step, on the host's cores.

Multi-GPU (torchrun): each rank computes an independent crystal (seed = rank) of the same size;
no data-path collective ("weak" scaling); the max step time over ranks is reported.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "4ph processes/s on 1 GB300, mixed vs FP64 GPU at κ rel err ≤1e-4; % of roofline"
UNIT = "processes/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="fc4", choices=["fc4", "reference"])
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--mesh", type=int, default=8)
    p.add_argument("--T", type=float, default=300.0)
    p.add_argument("--sigma", type=float, default=0.1)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64-vs-mixed comparison")
    p.add_argument("--no-tc", action="store_true", help="skip the tensor-core +- comparison")
    p.add_argument("--batch", action="store_true",
                   help="time the 24-crystal batch (6-24 branches) as one CUDA graph instead")
    p.add_argument("--cpu-qp", type=int, default=24, help="oracle sample: partners q' < cpu_qp")
    p.add_argument("--cpu-q", type=int, default=2, help="oracle sample: q points (x nb modes)")
    p.add_argument("--block-threads", type=int, default=0)
    p.add_argument("--once", action="store_true",
                   help="one untimed fc4_rates call (for profilers): --mesh, --precision, --mask")
    p.add_argument("--mask", type=int, default=31, help="channel mask of --once")
    p.add_argument("--tc", action="store_true", help="--once with the tensor-core +- contraction")
    p.add_argument("--irreducible", action="store_true",
                   help="irreducible q-points against the full mesh (see run_irreducible)")
    p.add_argument("--symmetric", action="store_true", help="--irreducible on the unperturbed crystal")
    p.add_argument("--cpu-sample", action="store_true",
                   help="only the oracle sample (--cpu-q, --cpu-qp) on the host, one JSON line")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def workload(args, seed):
    from synth import morse_system
    return morse_system(seed=seed), (args.mesh,) * 3


def config_of(args, precision):
    n = args.mesh
    return {"workload": f"morse-diamond-2atom-{n}x{n}x{n}-all-modes", "mesh": [n, n, n], "n_q": n ** 3,
            "nb": 6, "T_K": args.T, "sigma_THz": args.sigma, "channels": "3ph+,3ph-,4ph++,4ph+-,4ph--",
            "precision": precision, "step": "fc4_rates(all modes, 5 channels) + fc4_kappa",
            "l2": "flushed between steps (512 MiB write)"}


# ------------------------------------------------------------------------------ CPU oracle

def cpu_oracle_sample(args, seed=0, qp=None, nq=None):
    """Oracle on a bounded sample of the same workload: cpu_q q points (all branches) and
    partners q' < cpu_qp; returns (kept 4ph processes, seconds, sample description, threads)."""
    import oracle
    from synth.sampling import sample_q
    sysm, mesh = workload(args, seed)
    prob = oracle.Problem(*sysm, mesh, T=args.T, sigma=args.sigma)
    qs = sample_q(int(np.prod(mesh)), nq or args.cpu_q, seed=0)
    modes = np.array([q * 6 + j for q in qs for j in range(6)], np.int32)
    qp = qp or args.cpu_qp
    t0 = time.perf_counter()
    _, _, cnt = prob.rates(modes, channel_mask=0b11100, qp_limit=qp)
    dt = time.perf_counter() - t0
    kept = int(cnt[2:].sum())
    desc = (f"oracle (C, FP64, OpenMP) on {modes.size} modes (q = {qs.tolist()}, all branches), "
            f"4ph channels, partners q' < {qp} of {int(np.prod(mesh))}; {kept} kept processes")
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return kept, dt, desc, threads


def cpu_host_info():
    """(CPU model, logical cores) of the host, best effort."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                if k.strip() in ("model name", "Model") and v.strip():
                    model = v.strip()
                    break
    except OSError:
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return model, os.cpu_count()


def cpu_oracle_one_core(args):
    """The oracle sample on one thread (a child process with OMP_NUM_THREADS=1), 6 modes and a
    quarter of the partners q'; None if the child fails."""
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample", "--cpu-q", "1",
           "--cpu-qp", str(max(2, args.cpu_qp // 4)), "--mesh", str(args.mesh), "--T", str(args.T),
           "--sigma", str(args.sigma)]
    try:
        r = subprocess.run(cmd, env=dict(os.environ, OMP_NUM_THREADS="1"), capture_output=True,
                           text=True, timeout=600)
        return json.loads(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None
    except Exception:
        return None


def clocks_start():
    try:
        out = os.environ.get("FC4_BENCH_OUT")                  # optional folder for the raw samples
        f = open(os.path.join(out, "bench_clocks.csv") if out and os.path.isdir(out) else os.devnull, "w")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                             stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        return p, f
    except Exception:
        return None, None


def clocks_stop(p, f, gpu_index):
    if p is None:
        return None
    p.terminate()
    try:
        out, _ = p.communicate(timeout=5)
    except Exception:
        p.kill()
        out, _ = p.communicate()
    rows = []
    for line in out.splitlines():
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            if int(parts[0]) != gpu_index:
                continue
            rows.append(parts)
        except ValueError:
            continue
    if f:
        f.write(out)
        f.close()
    if not rows:
        return None
    sm = [float(r[1]) for r in rows]
    mx = max(float(r[2]) for r in rows)
    reasons = set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in rows:
        for n, v in zip(names, r[5:9]):
            if v.lower().startswith("active"):
                reasons.add(n)
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(rows)}


# ------------------------------------------------------------------------------ GPU arm

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per (λ, q') unit of the tiled 4ph
# kernel, from one ncu capture of the same kernel on the 6x6x6 seed-0 crystal (279,936 units per
# launch); key (mixed precision, channel, branches).  The bytes are the per-unit W reads, so they
# scale with the unit count.
TRAFFIC_PER_UNIT = {(True, "4ph+-", 6): (4.109239e9 + 19.932e6) / 279936}


def flops_alg(stats, info, nb):
    """Algorithmic FP32 flops of the four-phonon path per channel, counted for the work it
    performs (complex multiply-add = 8 flops, real x complex = 4); where the triangular domain
    applies only the visited candidates and the evaluated processes count:
      window          2 per visited candidate (add, subtract; the comparison is not counted)
      W per (λ, q')   Φ~ = Σ_α Φ e_λ: nc4·27·3·4 / 8 (built once per 8 q'), plus the phase
                      fold Ψ_rb = Σ_c phase Φ~: nc4·27·8, plus W = Σ_bβ e' Ψ: nb·n_keys·9·3na·8
      X per entry     n_keys·9·8 (X[c,d] = Σ_r P_r W_r)
      Y per item      nb²·8 (Y = X times the conjugated third-partner eigenvector)
      per process     V nb·8, weight 30"""
    nc4, nk, N = info["nc4"], info["n_keys"], info["N"]
    out = []
    for ch in range(5):
        if ch < 2:
            out.append(0.0)
            continue
        cand = float(stats["candidates"][ch])
        units = cand / (N * nb ** 3)                   # (λ, q') units
        na = nb // 3
        w = units * (nc4 * 27 * 3 * 4 / 8.0 + nc4 * 27 * 8 + nb * nk * 9 * na * 3 * 8)
        out.append(2.0 * float(stats["visited"][ch]) + w + stats["entries"][ch] * nk * 72.0
                   + stats["items"][ch] * nb * nb * 8.0 + stats["evaluated"][ch] * (8.0 * nb + 30.0))
    return out


def fp64_comparison(args, sysm, mesh, g_mixed, local):
    """FP64 GPU path beside the mixed one: throughput on a sampled q subset of the same workload,
    the largest Γ relative error of the mixed path there, and the κ relative error mixed vs FP64
    on the full 6x6x6 mesh of the same crystal."""
    import torch
    from paper_2510_00518_gb300 import Engine, FP64, MIXED
    from synth.sampling import sample_q
    qs = sample_q(int(np.prod(mesh)), 16, seed=0)
    e64 = Engine(*sysm, mesh, precision=FP64)
    e64.rates(args.T, args.sigma, 31, q_subset=qs)          # warm
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    g64, _, _ = e64.rates(args.T, args.sigma, 31, q_subset=qs)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    kept = int(e64.stats()["kept"][2:].sum())
    modes = torch.tensor([q * 6 + j for q in qs for j in range(6)], device=g64.device)
    gm = g_mixed[:, modes]
    floor = 1e-6 * g64.abs().amax(dim=1, keepdim=True)
    gerr = float(((gm - g64).abs() / torch.maximum(g64.abs(), floor)).max())
    ks = []
    for prec in (MIXED, FP64):
        e = Engine(*sysm, (6, 6, 6), precision=prec)
        g6, _, _ = e.rates(args.T, args.sigma, 31)
        ks.append(e.kappa(args.T, g6, 31).cpu().numpy())
    kerr = float(np.abs(ks[0] - ks[1]).max() / np.abs(ks[1]).max())
    return {"value": kept / (ms * 1e-3), "unit": UNIT, "ms": ms, "kept_4ph": kept,
            "sample": f"16 q points (default_rng(0)) x 6 branches of the {mesh[0]}x{mesh[1]}x{mesh[2]} mesh, 5 channels",
            "gamma_rel_err_max_mixed_vs_fp64": gerr, "kappa_rel_err_mixed_vs_fp64_6x6x6": kerr}


def tensor_core_comparison(args, eng, g_cuda):
    """The 4ph +- channel with its cluster contraction on the tensor cores (tcgen05) beside the
    CUDA-core run of the same step: device time of that channel's kernel (CUDA events, W shared
    with ++ as in the step) and the largest relative Γ difference."""
    import torch
    eng.set_tensor_cores(True)
    try:
        eng.rates(args.T, args.sigma, 0b01100)                  # warm
        gt, _, _ = eng.rates(args.T, args.sigma, 0b01100)
        torch.cuda.synchronize()
        ms = float(eng.timings()["4ph+-"])
        eng.check_device()
    finally:
        eng.set_tensor_cores(False)
    a, b = gt[3], g_cuda[3]
    floor = 1e-6 * b.abs().max()
    err = float(((a - b).abs() / torch.maximum(b.abs(), floor)).max())
    return {"pm_ms": ms, "gamma_pm_rel_err_vs_cuda_cores": err,
            "kernel": "rates4_tc_kernel: tcgen05.mma kind::f16, FP16 hi/lo x 3 products, FP32 accumulation"}


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2510_00518_gb300 import Engine, FP64, MIXED

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prec = MIXED if args.precision == "mixed" else FP64
    sysm, mesh = workload(args, seed=rank)
    eng = Engine(*sysm, mesh, precision=prec, block_threads=args.block_threads, timing=True)
    info = eng.info()
    nb = info["nb"]
    nm = info["N"] * nb
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    g = torch.empty((5, nm), dtype=torch.float64, device=dev)
    wp = torch.empty_like(g)
    cnt = torch.empty((5, nm), dtype=torch.int64, device=dev)
    kap = torch.empty(9, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2

    def step():
        eng.rates(args.T, args.sigma, 31, out=(g, wp, cnt))
        eng.kappa(args.T, g, 31, out=kap)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stats = eng.stats()
    kept4 = int(stats["kept"][2:].sum())

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    k_ms = []
    clk_p, clk_f = clocks_start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    launches0 = eng.timings()["launches"]
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        k_ms.append(eng.timings())
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    clocks = clocks_stop(clk_p, clk_f, local)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = float(np.mean(step_ms))
    launches = (k_ms[-1]["launches"] - launches0) if k_ms else 0
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        kk = torch.tensor([kept4], device=dev, dtype=torch.float64)
        dist.all_reduce(kk)
        kept_total = float(kk.item())
    else:
        kept_total = float(kept4)
    value = kept_total / (ms * 1e-3)

    # dominant kernel (the 4ph channel with the largest device time) and its roofline
    chans = ["4ph++", "4ph+-", "4ph--"]
    avg = {c: float(np.mean([t[c] for t in k_ms])) for c in chans}
    dom = max(avg, key=avg.get)
    ch = 2 + chans.index(dom)
    fl = flops_alg(stats, info, nb)[ch]
    import json as _json
    peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    sm_clock = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    if prec == MIXED:
        peak = 152 * 128 * 2 * 2070e6 / 1e12              # FP32 CUDA-core FLOP/s at max SM clock
        bound_note = "FP32 FMA issue: 152 SMs x 128 lanes x 2 flops x 2.07 GHz (max clock)"
    else:
        peak = 1.25                                         # FP64 (nominal GB300)
        bound_note = "FP64: nominal 1.25 TFLOP/s"
    achieved = fl / (avg[dom] * 1e-3) / 1e12
    units = float(stats["candidates"][ch]) / (info["N"] * nb ** 3)
    per_unit = TRAFFIC_PER_UNIT.get((prec == MIXED, dom, nb))
    traffic = per_unit * units if per_unit else None
    roof = {"bound": "alu", "kernel": f"rates4 {dom}", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
            "traffic_basis": "ncu dram bytes of the same kernel on the 6x6x6 case, per (λ, q') unit, "
                             "times this launch's units" if traffic else None,
            "launch_ms": avg[dom], "alg_flops_per_launch": fl, "peak_basis": bound_note,
            "kernel_ms": avg}

    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": "f32" if prec == MIXED else "f64",
              "data": "synthetic (seeded Morse diamond crystal)", "config": config_of(args, args.precision),
              "kept_4ph_per_step": kept4, "candidates_4ph_per_step": int(stats["candidates"][2:].sum()),
              "evaluated_4ph_per_step": int(stats["evaluated"][2:].sum()),
              "visited_4ph_candidates_per_step": int(stats["visited"][2:].sum()),
              "domain": "triangular where the summand is partner-swap symmetric (one process of each "
                        "swapped pair evaluated with weight 2); kept counts are the rectangular ones",
              "wall_s": wall, "gpu_launches": int(launches), "roofline": roof, "clocks": clocks}

    if not args.no_fp64 and world == 1:
        result["fp64_gpu"] = fp64_comparison(args, sysm, mesh, g, local)
    if prec == MIXED and world == 1 and not args.no_tc and info["n_atoms"] == 2:
        result["tensor_cores_pm"] = tensor_core_comparison(args, eng, g)
        result["tensor_cores_pm"]["cuda_core_pm_ms"] = avg["4ph+-"]

    # end to end through the C interface from host buffers
    if not args.no_e2e:
        import ctypes
        import paper_2510_00518_gb300 as pkg
        c, p2, p3, p4 = sysm
        gh = np.zeros((5, nm))
        wph = np.zeros((5, nm))
        ch_ = np.zeros((5, nm), np.int64)
        kh = np.zeros(9)
        h2d = sum(np.asarray(x).nbytes for x in (c.lattice, c.positions, c.masses, p2.atoms, p2.cells,
                                                 p2.phi, p3.atoms, p3.cells, p3.phi, p4.atoms, p4.cells, p4.phi))
        d2h = gh.nbytes + wph.nbytes + ch_.nbytes + kh.nbytes
        e2e_ms = []
        for i in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            e = Engine(*sysm, mesh, precision=prec, block_threads=args.block_threads)
            g2, wp2, c2 = e.rates(args.T, args.sigma, 31)
            k2 = e.kappa(args.T, g2, 31)
            gh[:] = g2.cpu().numpy()
            wph[:] = wp2.cpu().numpy()
            ch_[:] = c2.cpu().numpy()
            kh[:] = k2.cpu().numpy().reshape(-1)
            e.close()
            torch.cuda.synchronize()
            e2e_ms.append((time.perf_counter() - t1) * 1e3)
        em = float(np.mean(e2e_ms))
        result["e2e"] = {"value": kept_total / (em * 1e-3) if world == 1 else kept4 / (em * 1e-3) * world,
                         "unit": UNIT, "ms_per_step": em, "h2d_bytes_per_step": int(h2d),
                         "d2h_bytes_per_step": int(d2h)}
        result["kappa_W_mK"] = kh.reshape(3, 3).tolist()

    if rank == 0 and world == 1 and not args.no_cpu:
        kept, dt, desc, thr = cpu_oracle_sample(args)
        model, ncpu = cpu_host_info()
        result["cpu_baseline"] = {"value": kept / dt, "unit": UNIT, "cores": thr, "kind": "oracle",
                                  "sample": desc, "seconds": dt, "cpu_model": model, "nproc": ncpu,
                                  "one_core": cpu_oracle_one_core(args)}
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result))


# ------------------------------------------------------------------------------ reference arm

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_oracle_sample(args, qp=2, nq=1)
    kept_tot, secs = 0, 0.0
    desc, thr = "", 1
    for _ in range(args.steps):
        kept, dt, desc, thr = cpu_oracle_sample(args)
        kept_tot += kept
        secs += dt
    v = kept_tot / secs
    ms = secs / args.steps * 1e3
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Morse diamond crystal)",
           "config": config_of(args, "fp64-oracle"),
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": desc,
                            "cpu_model": cpu_host_info()[0], "nproc": cpu_host_info()[1]},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_batch(args):
    """24 synthetic crystals (1x1xk diamond supercells, k = 1..4; 12³/10³/8³/6³ meshes; 4 seeded q
    points each; mixed precision) evaluated as one CUDA graph; metric: kept 4ph processes/s."""
    import torch
    from paper_2510_00518_gb300 import Engine, MIXED
    from paper_2510_00518_gb300.batch import BatchRunner, autotune
    from synth import batch_crystal, morse_ifcs
    from synth.sampling import sample_q
    torch.cuda.set_device(0)
    jobs = []
    for seed in range(24):
        c, mesh = batch_crystal(seed)
        e = Engine(c, *morse_ifcs(c, seed=seed), mesh, precision=MIXED)
        jobs.append((e, sample_q(int(np.prod(mesh)), 4, seed=seed)))
    out_dir = os.environ.get("FC4_BENCH_OUT")
    cache = os.path.join(out_dir, "tune_cache.json") if out_dir and os.path.isdir(out_dir) else None
    for e, qs in jobs:
        if e.n_atoms > 2:
            autotune(e, args.T, args.sigma, 31, qs, cache=cache)
    runner = BatchRunner(jobs, args.T, args.sigma, 31)
    kept = sum(int(e.stats()["kept"][2:].sum()) for e, _ in jobs)
    for _ in range(args.warmup):
        runner.run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        runner.run()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    print(json.dumps({"metric": METRIC + " (batch of 24 crystals, one CUDA graph)", "value": kept / (ms * 1e-3),
                      "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                      "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "batch-24-morse-supercells-6to24-branches", "q_per_crystal": 4,
                                 "meshes": "12^3/10^3/8^3/6^3 for 2/4/6/8 atoms", "graph": "one CUDA graph launch",
                                 "l2": "not flushed (graph replays back to back)"},
                      "kept_4ph_per_step": kept}))


def run_irreducible(args):
    """Rates of the whole mesh from its irreducible q-points (symmetry.rates_irreducible: fc4_rates
    on one q per orbit, host spread over the stars) against the full-mesh step, both followed by
    fc4_kappa, in one process.  ``--symmetric`` takes the unperturbed crystal (48 operations);
    otherwise the bench crystal, whose only symmetry is q -> -q.  Prints one JSON line with both
    step times (wall clock, synchronised, L2 flushed before each step) and the κ difference."""
    import torch
    from synth import morse_system
    from paper_2510_00518_gb300 import Engine, FP64, MIXED
    from paper_2510_00518_gb300.symmetry import rates_irreducible, symmetry_ops
    torch.cuda.set_device(0)
    sysm = morse_system(seed=0, perturb=0.0 if args.symmetric else 0.01)
    mesh = (args.mesh,) * 3
    rot, _ = symmetry_ops(*sysm)
    eng = Engine(*sysm, mesh, precision=MIXED if args.precision == "mixed" else FP64)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def timed(fn):
        out, ts = None, []
        for i in range(args.warmup + args.steps):
            flush.fill_(float(i))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = fn()
            torch.cuda.synchronize()
            if i >= args.warmup:
                ts.append((time.perf_counter() - t0) * 1e3)
        return out, float(np.mean(ts))

    def full():
        g, _, _ = eng.rates(args.T, args.sigma, 31)
        return g, eng.kappa(args.T, g, 31)

    def irreducible():
        g, _, n = rates_irreducible(eng, args.T, args.sigma, 31, rot)
        return g, eng.kappa(args.T, g, 31), n

    (g_f, k_f), ms_f = timed(full)
    (g_i, k_i, n_irr), ms_i = timed(irreducible)
    kf, ki = k_f.cpu().numpy(), k_i.cpu().numpy()
    print(json.dumps({"mode": "irreducible q-points", "crystal": "unperturbed (48 operations)" if args.symmetric
                      else "bench crystal (q -> -q only)", "n_operations": int(len(rot)),
                      "n_q": int(np.prod(mesh)), "n_irreducible": n_irr, "precision": args.precision,
                      "ms_per_step_full": ms_f, "ms_per_step_irreducible": ms_i, "speedup": ms_f / ms_i,
                      "kappa_rel_err": float(np.abs(ki - kf).max() / np.abs(kf).max()),
                      "steps": args.steps, "warmup": args.warmup,
                      "timing": "wall clock around synchronised calls; L2 flushed before each step"}))


def run_once(args):
    """A single rates call on the workload (profiling helper, no timing, no JSON line)."""
    import torch
    from paper_2510_00518_gb300 import Engine, FP64, MIXED
    sysm, mesh = workload(args, seed=0)
    eng = Engine(*sysm, mesh, precision=MIXED if args.precision == "mixed" else FP64,
                 block_threads=args.block_threads, tensor_cores=args.tc)
    g, _, _ = eng.rates(args.T, args.sigma, args.mask)
    torch.cuda.synchronize()
    eng.check_device()
    print("once", args.mesh, args.precision, args.mask, float(g.sum()), eng.stats())


if __name__ == "__main__":
    a = parse()
    if a.cpu_sample:
        kept, dt, desc, thr = cpu_oracle_sample(a)
        print(json.dumps({"value": kept / dt, "unit": UNIT, "cores": thr, "seconds": dt, "sample": desc}))
    elif a.irreducible:
        run_irreducible(a)
    elif a.once:
        run_once(a)
    elif a.batch:
        run_batch(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_gpu(a)
