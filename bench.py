#!/usr/bin/env python3
"""Throughput of the three- and four-phonon scattering-rate path on GB300.

The metric is kept four-phonon processes per second.  Two workloads (synthetic two-atom Morse
diamond crystals: a = 5.43 Å, m = 28.0855 amu, D = 2 eV, α = 1.5/Å, r0 = 2.35 Å, seeded 1 % bond
perturbations; no first-principles force constants):

  precision (default)  16x16x16 mesh (4096 q), seed 1, adaptive σ (scale 1), T = 300 K, the 145
                       q points numpy default_rng(1).choice(4096, 145) (sorted) x 6 branches.
                       One step = fc4_rates (all five channels: enumeration, energy window,
                       matrix elements, weights, reduction) on the next batch of --q-per-step of
                       those q points; the 5 batches of 29 cover the 145 q and are cycled.
  allmodes             8x8x8 mesh, seed 0, fixed σ = 0.1 THz, T = 300 K: one step = fc4_rates of
                       every mode followed by the RTA conductivity κ (fc4_kappa).

Inputs are resident in HBM; L2 is flushed between steps.  Beside the headline (FP32 contraction on
the CUDA cores) the line carries: the FP64 GPU path and every tensor-core operand format on the
first 5 sampled q with their Γ error against FP64 per channel; the all-modes 8x8x8 step in mixed and
FP64 with κ's mixed-vs-FP64 error; the end-to-end rate through the C interface from host buffers
(fc4_init, fc4_rates, device-to-host copy of Γ, WP and counts, fc4_destroy per step); the
roofline of the dominant kernel against the measured FP32 FMA rate (fc4_device_peaks); and the
FP64 CPU oracle on a bounded sample of the same workload on the host cores.

--impl reference times the oracle (the test reference) alone on the same workload.
Multi-GPU (torchrun): each rank runs its own crystal (seed + rank) of the same size; no
data-path collective ("weak" scaling); the max step time over ranks is reported.
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

WORKLOADS = {
    "precision": dict(name="morse-diamond-2atom-{n}x{n}x{n}-145q-adaptive-sigma", seed=1, mesh=16,
                      n_sample=145, sample_seed=1, sigma=1.0, adaptive=True, T=300.0),
    "allmodes": dict(name="morse-diamond-2atom-{n}x{n}x{n}-all-modes", seed=0, mesh=8, n_sample=None,
                     sample_seed=None, sigma=0.1, adaptive=False, T=300.0),
}
PREC_NAMES = ("fp64", "mixed", "tf32x3", "bf16", "bf16x3", "fp16x3")
ARM_Q = 5   # q points of the FP64 and tensor-core arms


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="fc4", choices=["fc4", "reference"])
    p.add_argument("--workload", default="precision", choices=list(WORKLOADS))
    p.add_argument("--precision", default="mixed", choices=list(PREC_NAMES))
    p.add_argument("--q-per-step", type=int, default=29)
    p.add_argument("--mesh", type=int, default=0, help="override the workload's mesh (n x n x n)")
    p.add_argument("--T", type=float, default=0.0, help="override the workload's temperature")
    p.add_argument("--sigma", type=float, default=0.0, help="override σ (THz) or the adaptive scale")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-arms", action="store_true", help="skip the FP64 and tensor-core arms")
    p.add_argument("--no-allmodes", action="store_true", help="skip the 8x8x8 all-modes line")
    p.add_argument("--batch", action="store_true",
                   help="time the 24-crystal batch (6-24 branches) as one CUDA graph instead")
    p.add_argument("--batch-q", type=int, default=4, help="--batch: sampled q points per crystal")
    p.add_argument("--cpu-qp", type=int, default=0, help="oracle sample: partners q' < cpu_qp")
    p.add_argument("--cpu-q", type=int, default=0, help="oracle sample: q points (x nb modes)")
    p.add_argument("--block-threads", type=int, default=0)
    p.add_argument("--once", action="store_true",
                   help="one untimed fc4_rates call on the first batch (for profilers)")
    p.add_argument("--mask", type=int, default=31, help="channel mask of --once")
    p.add_argument("--irreducible", action="store_true",
                   help="irreducible q-points against the full mesh (see run_irreducible)")
    p.add_argument("--symmetric", action="store_true", help="--irreducible on the unperturbed crystal")
    p.add_argument("--fp64-full", action="store_true",
                   help="mixed and FP64 over the whole sample of the workload (one call each), one JSON line")
    p.add_argument("--ablation", action="store_true",
                   help="modes per chunk (all-modes .. mode-by-mode) and compaction ablations, one JSON line")
    p.add_argument("--cpu-sample", action="store_true",
                   help="only the oracle sample (--cpu-q, --cpu-qp) on the host, one JSON line")
    a = p.parse_args()
    w = dict(WORKLOADS[a.workload])
    if a.mesh:
        w["mesh"] = a.mesh
    w["name"] = w["name"].format(n=w["mesh"])
    if a.T:
        w["T"] = a.T
    if a.sigma:
        w["sigma"] = a.sigma
    a.w = w
    if not a.cpu_q:
        a.cpu_q = 3 if w["adaptive"] else 2
    if not a.cpu_qp:
        a.cpu_qp = 3 if w["adaptive"] else 24
    return a


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def system_of(w, rank=0):
    from synth import morse_system
    return morse_system(seed=w["seed"] + rank), (w["mesh"],) * 3


def q_sample(w):
    """The workload's q points (all of the mesh if it has no sample)."""
    from synth.sampling import sample_q
    n = w["mesh"] ** 3
    return np.arange(n, dtype=np.int32) if not w["n_sample"] else sample_q(n, w["n_sample"], w["sample_seed"])


def batches(w, q_per_step):
    """q points of each step: the sample in consecutive batches (all modes: one batch, None)."""
    if not w["n_sample"]:
        return [None]
    qs = q_sample(w)
    return [qs[i:i + q_per_step] for i in range(0, qs.size, q_per_step)]


def config_of(args, precision):
    w = args.w
    n = w["mesh"]
    c = {"workload": w["name"], "mesh": [n, n, n], "n_q_mesh": n ** 3, "nb": 6, "T_K": w["T"],
         "channels": "3ph+,3ph-,4ph++,4ph+-,4ph--", "precision": precision,
         "l2": "flushed between steps (512 MiB write)"}
    if w["adaptive"]:
        c.update({"sigma": f"adaptive, scale {w['sigma']}",
                  "q_sample": f"{w['n_sample']} q = default_rng({w['sample_seed']}).choice({n ** 3}, {w['n_sample']}), sorted",
                  "q_per_step": args.q_per_step,
                  "step": f"fc4_rates (5 channels) on the next {args.q_per_step} of the sampled q "
                          f"({len(batches(w, args.q_per_step))} batches, cycled)"})
    else:
        c.update({"sigma_THz": w["sigma"], "step": "fc4_rates(all modes, 5 channels) + fc4_kappa"})
    return c


# ------------------------------------------------------------------------------ CPU oracle

def cpu_oracle_sample(args, qp=None, nq=None):
    """Oracle on a bounded sample of the workload: the first cpu_q q points of its sample (all
    branches) and partners q' < cpu_qp, four-phonon channels; returns (kept 4ph processes,
    seconds, sample description, threads)."""
    import oracle
    w = args.w
    sysm, mesh = system_of(w)
    prob = oracle.Problem(*sysm, mesh, T=w["T"], sigma=w["sigma"], sigma_adaptive=w["adaptive"])
    from synth.sampling import sample_q
    qs = (q_sample(w) if w["n_sample"] else sample_q(int(np.prod(mesh)), 64, 0))[:nq or args.cpu_q]
    modes = np.array([q * 6 + j for q in qs for j in range(6)], np.int32)
    qp = qp or args.cpu_qp
    t0 = time.perf_counter()
    _, _, cnt = prob.rates(modes, channel_mask=0b11100, qp_limit=qp)
    dt = time.perf_counter() - t0
    kept = int(cnt[2:].sum())
    desc = (f"oracle (C, FP64, OpenMP over modes) on {modes.size} modes (q = {qs.tolist()}, all branches) "
            f"of {w['name']}, 4ph channels, partners q' < {qp} of {int(np.prod(mesh))}; {kept} kept processes")
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
    """The oracle sample on one thread (a child process with OMP_NUM_THREADS=1) on one q point
    and a third of the partners q'; None if the child fails."""
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample", "--workload", args.workload,
           "--cpu-q", "1", "--cpu-qp", str(max(1, args.cpu_qp // 3))]
    if args.mesh:
        cmd += ["--mesh", str(args.mesh)]
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
# kernels, from ncu captures of the same kernels on small cases (fixed σ: 6x6x6 all modes; adaptive
# σ: 8x8x8, 30 modes; see profiles/); key (window kind, channel).  The bytes are the per-unit W
# reads, so they scale with the unit count.
TRAFFIC_PER_UNIT = {("fixed", "4ph+-"): (4.109239e9 + 19.932e6) / 279936,
                    ("adaptive", "4ph+-"): (227.183872e6 + 4.224768e6) / 15360,
                    ("adaptive", "4ph++"): (228.271872e6 + 4.289792e6) / 15360,
                    ("adaptive", "4ph--"): (228.271872e6 + 4.289792e6) / 15360}


def flops_alg(stats, info, nb, adaptive):
    """Algorithmic FP32 flops of the four-phonon path per channel, counted for the work it
    performs (complex multiply-add = 8 flops, real x complex = 4); where the triangular domain
    applies only the visited candidates and the evaluated processes count:
      window          2 per visited candidate (add, subtract; the comparison is not counted);
                      adaptive σ adds 12 per visited (q'', j'', j''') pair (one sixth of the
                      candidates): the velocity difference, its norm and the scale
      W per (λ, q')   Φ~ = Σ_α Φ e_λ: nc4·27·3·4 / 8 (built once per 8 q'), plus the phase
                      fold Ψ_rb = Σ_c phase Φ~: nc4·27·8, plus W = Σ_bβ e' Ψ: nb·n_keys·9·3na·8
      X per entry     n_keys·9·8 (X[c,d] = Σ_r P_r W_r)
      Y per item      nb²·8 (Y = X times the conjugated third-partner eigenvector)
      per process     V nb·8, weight 30 (adaptive: + 12 for the width)"""
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
        vis = float(stats["visited"][ch])
        win = 2.0 * vis + (12.0 * vis / nb if adaptive else 0.0)
        out.append(win + w + stats["entries"][ch] * nk * 72.0 + stats["items"][ch] * nb * nb * 8.0
                   + stats["evaluated"][ch] * (8.0 * nb + 30.0 + (12.0 if adaptive else 0.0)))
    return out


def add_stats(acc, st):
    if acc is None:
        return {k: v.astype(np.float64).copy() for k, v in st.items()}
    for k in acc:
        acc[k] += st[k]
    return acc


def rel_err_per_channel(g, ref):
    """max over modes of |g - ref| / max(|ref|, 1e-6 x the channel's largest |ref|), per channel."""
    import torch
    floor = 1e-6 * ref.abs().amax(dim=1, keepdim=True)
    return ((g - ref).abs() / torch.maximum(ref.abs(), floor.clamp_min(1e-300))).amax(dim=1).tolist()


def time_calls(fn, reps, warm=1):
    """Device time (ms, CUDA events on the current stream) of each of `reps` calls after `warm`."""
    import torch
    for _ in range(warm):
        fn()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        out = fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return out, ts


def precision_arms(args, sysm, mesh, q0, g_mixed_q0):
    """The q points q0 of the workload in FP64 (the reference for every error) and in every
    tensor-core operand format: device time, kept 4ph processes/s, and Γ's relative error per
    channel against FP64."""
    from paper_2510_00518_gb300 import Engine, FP64, PRECISIONS
    w = args.w
    eng = Engine(*sysm, mesh, precision=FP64, timing=True)

    def call():
        return eng.rates(w["T"], w["sigma"], 31, q_subset=q0, adaptive=w["adaptive"])[0]

    g64, ts = time_calls(call, 1)
    kept = int(eng.stats()["kept"][2:].sum())
    out = {"reference": "fp64", "batch_q": [int(x) for x in q0],
           "fp64": {"ms": ts[0], "value": kept / (ts[0] * 1e-3), "kept_4ph": kept,
                    "kernel_ms": {k: v for k, v in eng.timings().items() if k.startswith("4ph")}}}
    out["mixed"] = {"gamma_rel_err_vs_fp64": rel_err_per_channel(g_mixed_q0, g64)}
    for name in ("tf32x3", "bf16", "bf16x3", "fp16x3"):
        eng.set_precision(PRECISIONS[name])
        g, ts = time_calls(call, 1)
        eng.check_device()
        err = rel_err_per_channel(g, g64)
        out[name] = {"ms": ts[0], "value": kept / (ts[0] * 1e-3), "gamma_rel_err_vs_fp64": err,
                     "gamma_rel_err_max": max(err),
                     "kernel_ms": {k: v for k, v in eng.timings().items() if k.startswith("4ph")}}
    eng.close()
    return out


def allmodes_line(args):
    """The all-modes 8x8x8 step (fc4_rates of every mode + fc4_kappa) in mixed precision (3
    timed after 2 warm-up steps, L2 flushed) and once in FP64, with κ's and Γ's mixed-vs-FP64
    relative errors."""
    import torch
    from paper_2510_00518_gb300 import Engine, FP64, MIXED
    w = dict(WORKLOADS["allmodes"])
    w["name"] = w["name"].format(n=w["mesh"])
    sysm, mesh = system_of(w)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    res = {"workload": w["name"]}
    g_k = {}
    for prec, name, reps in ((MIXED, "mixed", 3), (FP64, "fp64", 1)):
        eng = Engine(*sysm, mesh, precision=prec)

        def step():
            flush.fill_(1.0)
            g, _, _ = eng.rates(w["T"], w["sigma"], 31)
            return g, eng.kappa(w["T"], g, 31)

        step()
        ts = []
        for _ in range(reps):
            flush.fill_(0.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            g, _, _ = eng.rates(w["T"], w["sigma"], 31)
            k = eng.kappa(w["T"], g, 31)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        kept = int(eng.stats()["kept"][2:].sum())
        ms = float(np.mean(ts))
        res[name] = {"ms_per_step": ms, "value": kept / (ms * 1e-3), "kept_4ph": kept, "steps": reps}
        g_k[name] = (g.clone(), k.cpu().numpy())
        eng.close()
    k_m, k_d = g_k["mixed"][1], g_k["fp64"][1]
    res["kappa_W_mK_fp64"] = k_d.reshape(3, 3).tolist()
    res["kappa_rel_err_mixed_vs_fp64"] = float(np.abs(k_m - k_d).max() / np.abs(k_d).max())
    res["gamma_rel_err_mixed_vs_fp64"] = rel_err_per_channel(g_k["mixed"][0], g_k["fp64"][0])
    res["speedup_mixed_vs_fp64"] = res["fp64"]["ms_per_step"] / res["mixed"]["ms_per_step"]
    return res


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2510_00518_gb300 import Engine, PRECISIONS, device_peaks

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = args.w
    prec = PRECISIONS[args.precision]
    sysm, mesh = system_of(w, rank)
    eng = Engine(*sysm, mesh, precision=prec, block_threads=args.block_threads, timing=True)
    info = eng.info()
    nb = info["nb"]
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    bl = batches(w, args.q_per_step)
    nm_max = max((len(b) if b is not None else info["N"]) for b in bl) * nb
    g = torch.empty((5, nm_max), dtype=torch.float64, device=dev)
    wp = torch.empty_like(g)
    cnt = torch.empty((5, nm_max), dtype=torch.int64, device=dev)
    kap = torch.empty(9, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2

    def step(i):
        q = bl[i % len(bl)]
        n = (len(q) if q is not None else info["N"]) * nb
        out = (g[:, :n], wp[:, :n], cnt[:, :n])
        eng.rates(w["T"], w["sigma"], 31, q_subset=q, out=out, adaptive=w["adaptive"])
        if q is None:
            eng.kappa(w["T"], g[:, :n], 31, out=kap)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    k_ms, st_acc, kept_steps = [], None, []
    clk_p, clk_f = clocks_start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    launches0 = eng.timings()["launches"]
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step(args.warmup + i)
        ev[i][1].record(stream)
        k_ms.append(eng.timings())               # waits for this step's events
        st = eng.stats()
        kept_steps.append(int(st["kept"][2:].sum()))
        st_acc = add_stats(st_acc, st)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    clocks = clocks_stop(clk_p, clk_f, local)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = float(np.sum(step_ms))
    launches = (k_ms[-1]["launches"] - launches0) if k_ms else 0
    kept_total = float(sum(kept_steps))
    if world > 1:
        t = torch.tensor([tot_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
        kk = torch.tensor([kept_total], device=dev, dtype=torch.float64)
        dist.all_reduce(kk)
        kept_total = float(kk.item())
    value = kept_total / (tot_ms * 1e-3)

    # dominant kernel (the 4ph channel with the largest device time) and its roofline against the
    # measured FP32 (or FP64) FMA rate of this device
    chans = ["4ph++", "4ph+-", "4ph--"]
    tot = {c: float(np.sum([t[c] for t in k_ms])) for c in chans}
    dom = max(tot, key=tot.get)
    ch = 2 + chans.index(dom)
    fl = flops_alg(st_acc, info, nb, w["adaptive"])[ch]
    peaks = device_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    fp64 = prec == PRECISIONS["fp64"]
    peak = peaks["fp64_tflops"] if fp64 else peaks["fp32_tflops"]
    achieved = fl / (tot[dom] * 1e-3) / 1e12
    units = float(st_acc["candidates"][ch]) / (info["N"] * nb ** 3)
    per_unit = TRAFFIC_PER_UNIT.get(("adaptive" if w["adaptive"] else "fixed", dom)) if not fp64 else None
    traffic = per_unit * units / args.steps if per_unit else None
    roof = {"bound": "alu", "kernel": f"rates4 {dom}", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
            "traffic_basis": ("ncu dram bytes of the same kernel on a small case, per (λ, q') unit, times "
                              "the units of one launch") if traffic else None,
            "launch_ms": tot[dom] / args.steps, "alg_flops_per_launch": fl / args.steps,
            "peak_basis": (f"measured {'FP64' if fp64 else 'FP32'} FMA rate of this GPU "
                           f"(fc4_device_peaks: {sms} SMs x 8 blocks of 256 threads, 8 FMA chains each)"),
            "measured_peaks_tflops": peaks, "sms": sms,
            "kernel_ms_per_step": {c: tot[c] / args.steps for c in chans}}

    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "f64" if fp64 else "f32",
              "data": "synthetic (seeded Morse diamond crystal)", "config": config_of(args, args.precision),
              "kept_4ph_timed": int(kept_total), "kept_4ph_per_step": kept_steps,
              "candidates_4ph_timed": int(st_acc["candidates"][2:].sum()),
              "evaluated_4ph_timed": int(st_acc["evaluated"][2:].sum()),
              "visited_4ph_candidates_timed": int(st_acc["visited"][2:].sum()),
              "domain": "triangular where the summand is partner-swap symmetric (one process of each "
                        "swapped pair evaluated with weight 2); kept counts are the rectangular ones",
              "wall_s": wall, "gpu_launches": int(launches), "roofline": roof, "clocks": clocks}

    if world == 1 and not args.no_arms:
        # the arms run on the first ARM_Q sampled q (FP64 takes ~40x the mixed time)
        q0 = q_sample(w)[:ARM_Q] if w["n_sample"] else np.arange(16, dtype=np.int32)
        eng.set_precision(PRECISIONS["mixed"])
        gm, ts = time_calls(lambda: eng.rates(w["T"], w["sigma"], 31, q_subset=q0, adaptive=w["adaptive"])[0], 1)
        gm, m_ms = gm.clone(), ts[0]
        eng.set_precision(prec)
        result["precision_arms"] = precision_arms(args, sysm, mesh, q0, gm)
        fp = result["precision_arms"]["fp64"]
        result["fp64_gpu"] = {"value": fp["value"], "unit": UNIT, "ms": fp["ms"], "mixed_ms_same_batch": m_ms,
                              "speedup_mixed_vs_fp64": fp["ms"] / m_ms,
                              "sample": f"the first {q0.size} q of the workload's sample, all branches",
                              "gamma_rel_err_max_mixed_vs_fp64": max(result["precision_arms"]["mixed"]["gamma_rel_err_vs_fp64"])}
    if world == 1 and not args.no_allmodes and args.workload != "allmodes":
        result["allmodes_8cubed"] = allmodes_line(args)

    # end to end through the C interface from host buffers
    if not args.no_e2e:
        c, p2, p3, p4 = sysm
        h2d = sum(np.asarray(x).nbytes for x in (c.lattice, c.positions, c.masses, p2.atoms, p2.cells,
                                                 p2.phi, p3.atoms, p3.cells, p3.phi, p4.atoms, p4.cells, p4.phi))
        e2e_ms, e2e_kept, d2h = [], 0, 0
        for i in range(max(1, min(args.steps, 3))):
            q = bl[i % len(bl)]
            n = (len(q) if q is not None else info["N"]) * nb
            gh, wph, chh = np.zeros((5, n)), np.zeros((5, n)), np.zeros((5, n), np.int64)
            kh = np.zeros(9)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            e = Engine(*sysm, mesh, precision=prec, block_threads=args.block_threads)
            g2, wp2, c2 = e.rates(w["T"], w["sigma"], 31, q_subset=q, adaptive=w["adaptive"])
            gh[:] = g2.cpu().numpy()
            wph[:] = wp2.cpu().numpy()
            chh[:] = c2.cpu().numpy()
            if q is None:
                kh[:] = e.kappa(w["T"], g2, 31).cpu().numpy().reshape(-1)
            e.close()
            torch.cuda.synchronize()
            e2e_ms.append((time.perf_counter() - t1) * 1e3)
            e2e_kept += int(chh[2:].sum())
            d2h = gh.nbytes + wph.nbytes + chh.nbytes + (kh.nbytes if q is None else 0)
        em = float(np.sum(e2e_ms))
        result["e2e"] = {"value": e2e_kept / (em * 1e-3) * world, "unit": UNIT, "ms_per_step": em / len(e2e_ms),
                         "steps": len(e2e_ms), "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                         "step": "fc4_init (host crystal and clusters) + fc4_rates + copy of Γ, WP, counts to "
                                 "the host + fc4_destroy"}

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
        cpu_oracle_sample(args, qp=1, nq=1)
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
    """24 synthetic crystals (1x1xk diamond supercells, k = 1..4: 2-8 atoms, 6-24 branches; site
    masses U(10, 120) amu; 12^3/10^3/8^3/6^3 meshes; 4 seeded q points each; seeds 0-23; mixed
    precision; fixed σ = 0.1 THz; T = 300 K) as one CUDA graph, in two forms timed in turn: one
    persistent launch per cell size over a shared work list (fc4_batch_rates), and each crystal's
    fc4_rates in turn.  The faster form is the headline.  Metric: kept 4ph processes/s."""
    import torch
    from paper_2510_00518_gb300 import Engine, MIXED
    from paper_2510_00518_gb300.batch import BatchRunner
    from synth import batch_crystal, morse_ifcs
    from synth.sampling import sample_q
    torch.cuda.set_device(0)
    T, sigma = 300.0, 0.1
    jobs = []
    for seed in range(24):
        c, mesh = batch_crystal(seed)
        e = Engine(c, *morse_ifcs(c, seed=seed), mesh, precision=MIXED)
        jobs.append((e, sample_q(int(np.prod(mesh)), args.batch_q, seed=seed)))

    def timed(runner):
        for _ in range(args.warmup):
            runner.run()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            runner.run()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / args.steps

    res = {}
    for name, persistent in (("persistent", True), ("per_crystal", False)):
        runner = BatchRunner(jobs, T, sigma, 31, persistent=persistent)
        ms = timed(runner)
        kept = sum(int(e.stats()["kept"][2:].sum()) for e, _ in jobs)
        res[name] = {"ms_per_step": ms, "value": kept / (ms * 1e-3), "kept_4ph": kept}
    best = min(res, key=lambda k: res[k]["ms_per_step"])
    head = res[best]
    print(json.dumps({"metric": METRIC + " (batch of 24 crystals, one CUDA graph)", "value": head["value"],
                      "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": head["ms_per_step"], "higher_is_better": True, "dtype": "f32",
                      "data": "synthetic", "arms": res,
                      "config": {"workload": "batch-24-morse-supercells-6to24-branches", "q_per_crystal": args.batch_q,
                                 "meshes": "12^3/10^3/8^3/6^3 for 2/4/6/8 atoms", "graph": "one CUDA graph launch",
                                 "four_phonon": {"persistent": "one persistent launch per cell size of more than two atoms (fc4_batch_rates)",
                                                 "per_crystal": "each crystal's fc4_rates in turn"}, "headline_arm": best,
                                 "l2": "not flushed (graph replays back to back)"}}))


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
    args.T, args.sigma = 300.0, 0.1
    sysm = morse_system(seed=0, perturb=0.0 if args.symmetric else 0.01)
    mesh = (args.mesh or 8,) * 3
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


def run_ablation(args):
    """The paper's strategy comparisons on the synthetic crystals, one JSON line:
      modes per chunk (all-modes strategy down to mode-by-mode, Algorithm 5; Results): device time
        of the 8x8x8 all-modes rates step and the device memory the context holds for it;
      compaction vs none (the divergent GPU-only loop, Algorithm 2; Results): the same step, and one
        batch of the 16x16x16 adaptive workload, with the window's entries compacted (default) or
        evaluated by the thread that found them.
    Device times are CUDA events around each call after one warm-up call, L2 flushed before."""
    import torch
    from paper_2510_00518_gb300 import Engine, MIXED
    torch.cuda.set_device(0)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    reps = max(1, min(args.steps, 3))

    def timed(eng, w, q=None):
        eng.rates(w["T"], w["sigma"], 31, q_subset=q, adaptive=w["adaptive"])
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            g, _, _ = eng.rates(w["T"], w["sigma"], 31, q_subset=q, adaptive=w["adaptive"])
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.mean(ts)), g

    w8 = dict(WORKLOADS["allmodes"])
    w8["name"] = w8["name"].format(n=w8["mesh"])
    sysm, mesh = system_of(w8)
    out = {"mode": "ablation", "workload": w8["name"], "precision": "mixed", "steps": reps,
           "timing": "CUDA events per fc4_rates call after one warm-up call; L2 flushed before each"}
    strat = []
    g_ref = None
    for chunk in (0, 768, 96, 12, 1):
        eng = Engine(*sysm, mesh, precision=MIXED, timing=True)
        eng.set_mode_chunk(chunk, 0)
        ms, g = timed(eng, w8)
        mem = eng.memory()
        if g_ref is None:
            g_ref = g.clone()
        strat.append({"modes_per_chunk": mem["modes_per_chunk"], "ms": ms, "context_bytes": mem["total"],
                      "w_buffer_bytes": mem["w_buffer"], "partials_bytes": mem["partials"],
                      "launches": eng.timings()["launches"], "identical_gamma": bool(torch.equal(g, g_ref))})
        eng.close()
    out["modes_per_chunk"] = strat
    comp = {}
    for name, w, q in (("8x8x8 all modes", w8, None),
                       ("16x16x16 adaptive, first 5 sampled q", dict(WORKLOADS["precision"]), None)):
        if w.get("n_sample"):
            w["name"] = w["name"].format(n=w["mesh"])
            q = q_sample(w)[:5]
        s2, m2 = system_of(w)
        eng = Engine(*s2, m2, precision=MIXED, timing=True)
        row = {}
        for flag in (False, True):
            eng.set_ablation(flag)
            ms, g = timed(eng, w, q)
            t = eng.timings()
            row["no_compaction" if flag else "compacted"] = {"ms": ms, "kernel_ms": {k: t[k] for k in ("4ph++", "4ph+-", "4ph--")}}
        eng.close()
        row["slowdown"] = row["no_compaction"]["ms"] / row["compacted"]["ms"]
        comp[name] = row
    out["compaction"] = comp
    print(json.dumps(out))


def run_fp64_full(args):
    """Mixed and FP64 GPU paths over the whole sample of the workload (all 145 q of the precision
    workload in one fc4_rates call each, channels --mask): device times, the speedup, Γ's relative
    error of the mixed path against FP64 per channel (R21's bar), how many modes exceed 1e-4, and
    each channel's absolute error relative to the mode's total Γ over all five channels (the
    quantity κ sees).  One JSON line."""
    import torch
    from paper_2510_00518_gb300 import Engine, FP64, MIXED
    torch.cuda.set_device(0)
    w = args.w
    sysm, mesh = system_of(w)
    qs = q_sample(w)
    mask = args.mask
    res, gam = {}, {}
    for name, prec in (("mixed", MIXED), ("fp64", FP64)):
        e = Engine(*sysm, mesh, precision=prec, timing=True)
        e.rates(w["T"], w["sigma"], mask, q_subset=qs[:1], adaptive=w["adaptive"])        # warm
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        g = e.rates(w["T"], w["sigma"], mask, q_subset=qs, adaptive=w["adaptive"])[0]
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        kept = int(e.stats()["kept"][2:].sum())
        res[name] = {"ms": ms, "value": kept / (ms * 1e-3), "kept_4ph": kept,
                     "kernel_ms": {k: v for k, v in e.timings().items() if k[0] in "34"}}
        if name == "mixed" and mask != 31:
            gtot = e.rates(w["T"], w["sigma"], 31, q_subset=qs, adaptive=w["adaptive"])[0].sum(0)
        elif name == "mixed":
            gtot = g.sum(0)
        gam[name] = g.clone()
        e.close()
    err = rel_err_per_channel(gam["mixed"], gam["fp64"])
    d = (gam["mixed"] - gam["fp64"]).abs()
    floor = 1e-6 * gam["fp64"].abs().amax(dim=1, keepdim=True)
    rel = d / torch.maximum(gam["fp64"].abs(), floor.clamp_min(1e-300))
    n_over = (rel > 1e-4).sum(dim=1).tolist()
    of_total = (d / gtot.abs().clamp_min(1e-300)).amax(dim=1).tolist()
    worst = int(rel[4].argmax()) if mask & 16 else 0
    print(json.dumps({"mode": "mixed vs FP64 over the whole sample", "workload": w["name"], "channel_mask": mask,
                      "n_q": int(qs.size), "arms": res, "speedup_mixed_vs_fp64": res["fp64"]["ms"] / res["mixed"]["ms"],
                      "gamma_rel_err_mixed_vs_fp64": err, "gamma_rel_err_max": max(err),
                      "modes_over_1e-4": n_over, "abs_err_over_total_gamma_max": of_total,
                      "worst_4ph--_mode": {"index": worst, "gamma_fp64": float(gam["fp64"][4, worst]),
                                           "channel_max": float(gam["fp64"][4].abs().max()),
                                           "total_gamma": float(gtot[worst])},
                      "timing": "CUDA events around one fc4_rates call per precision after a 1-q warm-up call"}))


def run_once(args):
    """A single rates call on the first batch of the workload (profiling helper, no timing)."""
    import torch
    from paper_2510_00518_gb300 import Engine, PRECISIONS
    w = args.w
    sysm, mesh = system_of(w)
    eng = Engine(*sysm, mesh, precision=PRECISIONS[args.precision], block_threads=args.block_threads)
    q = batches(w, args.q_per_step)[0]
    g, _, _ = eng.rates(w["T"], w["sigma"], args.mask, q_subset=q, adaptive=w["adaptive"])
    torch.cuda.synchronize()
    eng.check_device()
    print("once", w["name"], args.precision, args.mask, float(g.sum()), eng.stats())


if __name__ == "__main__":
    a = parse()
    if a.cpu_sample:
        kept, dt, desc, thr = cpu_oracle_sample(a)
        print(json.dumps({"value": kept / dt, "unit": UNIT, "cores": thr, "seconds": dt, "sample": desc}))
    elif a.irreducible:
        run_irreducible(a)
    elif a.ablation:
        run_ablation(a)
    elif a.fp64_full:
        run_fp64_full(a)
    elif a.once:
        run_once(a)
    elif a.batch:
        run_batch(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_gpu(a)
