"""Benchmark: FGMRES solves of 2D Stokes (Taylor-Hood P2/P1, 16x16 -> 128x128, 4 levels) on one GB300.

One step = one FGMRES solve to 1e-8 relative residual (zero initial guess, V(1,1) cycles with
Chebyshev-accelerated matrix-full Vanka smoothing) of a seeded N(0,1) right-hand side already resident
in HBM.  The hierarchy (assembly, patch inverses, coarse inverse, eigenvalue estimates) is built once
before timing and kept resident, as a solver service would.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl vk|reference] [--config cfg2]

N > 1 runs under torch.distributed.run as independent replicas (the path does not shard).
--impl reference times the CPU oracle (the plain FP64 NumPy restatement of the method) on the host.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "V-cycle DoF/s; FGMRES solves/s to 1e-8 rel. residual; p50/p99 solve latency"

CONFIGS = {
    # name: (N_coarse, nlevels, k, sweeps, rtol, description)
    "cfg1": (4, 2, 2, 1, 1e-10, "2D Stokes TH P2/P1, 4x4 -> 8x8 (2 levels), FGMRES to 1e-10"),
    "cfg2": (16, 4, 2, 1, 1e-8, "2D Stokes TH P2/P1, 16x16 -> 128x128 (4 levels), FGMRES to 1e-8"),
    "cfg3p3": (16, 3, 3, 1, 1e-8, "2D Stokes TH P3/P2, 16x16 -> 64x64 (3 levels), FGMRES to 1e-8"),
    "cfg3p4": (16, 3, 4, 1, 1e-8, "2D Stokes TH P4/P3, 16x16 -> 64x64 (3 levels), FGMRES to 1e-8"),
    "cfg4": (32, 5, 2, 1, 1e-8, "2D Stokes TH P2/P1, 32x32 -> 512x512 (5 levels), FGMRES to 1e-8"),
    "cfg5": (8, 0, 0, 1, 1e-8, "Serving: Poisson stream of solve requests, N in {16..256} (coarsest 8x8), "
                               "k in {2,3,4}, FGMRES to 1e-8"),
}

HBM_FALLBACK = 6800.0
FP64_NOMINAL_GFLOPS = 1250.0   # GB300 FP64 (vector and tensor) nominal rate


def recorded_traffic(config, prec):
    """DRAM bytes per launch of the dominant kernel from the committed ncu record, or None when the
    record is for another workload or the kernel source changed since the capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)["k_patch_apply"]
        with open(os.path.join(ROOT, "paper_2409_14222_gb300", "csrc", rec["source"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
    except (OSError, KeyError, ValueError):
        return None
    if sha != rec["source_sha256_16"] or config != "cfg2" or prec != "f64":
        return None
    return float(rec["dram_bytes_per_launch"])


def spmv_roofline(kt, key, hbm, peak_kind, kernel):
    """HBM roofline of the finest-level V-cycle residual SpMV from the CUDA events around each launch."""
    n = int(kt["spmv_launches"])
    if n == 0:
        return None
    avg_s = kt["spmv_ms"] / n / 1e3
    gbs = kt[key] / avg_s / 1e9
    return {"kernel": kernel, "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
            "launch_avg_us": avg_s * 1e6, "bytes_per_launch": kt[key], "launches_timed": n,
            "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"}


def schedules(G, L):
    """Launch shape the setup autotuner chose for the patch application of each smoothed level."""
    out = {}
    for l in range(1, L):
        sc = G.apply_schedule(l)
        us = [u for u in sc["cand_us"] if u > 0]
        out[f"level{l}"] = {"split": sc["split"], "threads": sc["threads"], "per_sm": sc["per_sm"],
                            "best_us": min(us) if us else None, "worst_us": max(us) if us else None}
    return out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": HBM_FALLBACK}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index=0):
        self.proc = None
        # scratch file of the samples (only their summary goes into the JSON line); VK_CLOCKS_DIR
        # keeps it somewhere else than the system temporary directory
        import tempfile
        self.path = os.path.join(os.environ.get("VK_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"vk_clocks_bench_{os.getpid()}.csv")
        self.index = index

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for name, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if os.environ.get("VK_BENCH_GLOO") != "1" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_cpu_baseline(cfg, seed=0):
    """The oracle timed as it stands on the host cores: one full FGMRES solve of the workload
    (hierarchy built before timing, like the GPU arm)."""
    from oracle import solver
    import synthetic_inputs as si
    Nc, L, k, sweeps, rtol, _ = cfg
    t0 = time.perf_counter()
    H = solver.Hierarchy(Nc, L, k, sweeps=sweeps)
    t_setup = time.perf_counter() - t0
    b = si.rhs_normal(H.finest.space.ndof, seed)
    t0 = time.perf_counter()
    res = solver.solve(H, b, rtol, 100)
    t = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": 1.0 / t, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"1 full FGMRES solve (seed {seed}, {res.iters} iterations, {t:.1f} s; hierarchy setup "
                      f"{t_setup:.1f} s excluded); NumPy/SciPy FP64, BLAS threads "
                      f"{os.environ.get('OPENBLAS_NUM_THREADS', 'default')}",
            "iterations": res.iters, "seconds": t}


def run_reference(args, cfg):
    """--impl reference: the oracle on the host cores, same metric and config."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    from oracle import solver
    import synthetic_inputs as si
    Nc, L, k, sweeps, rtol, desc = cfg
    H = solver.Hierarchy(Nc, L, k, sweeps=sweeps)
    ndof = H.finest.space.ndof
    # one full solve (untimed warm-up) fixes the iteration count of the workload; each timed step is
    # a bounded sample: the first `sample_iters` FGMRES iterations of a solve, scaled to a full solve
    full = solver.solve(H, si.rhs_normal(ndof, 0), rtol, 100)
    sample_iters = min(3, full.iters)
    for w in range(max(0, args.warmup - 1)):
        solver.solve(H, si.rhs_normal(ndof, 100 + w), rtol, sample_iters)
    times = []
    for s in range(args.steps):
        b = si.rhs_normal(ndof, 1000 + s)
        t0 = time.perf_counter()
        solver.solve(H, b, rtol, sample_iters)
        times.append((time.perf_counter() - t0) * full.iters / sample_iters)
    total = sum(times)
    value = args.steps / total
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    sample = (f"each step: first {sample_iters} FGMRES iterations of a solve, scaled by "
              f"{full.iters}/{sample_iters} (full solve iteration count); hierarchy built before timing")
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": desc, "ndof": ndof, "iterations": full.iters},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "vcycle_dof_per_s": ndof * full.iters * args.steps / total,
        "latency_ms": {"p50": 1e3 * float(np.percentile(times, 50)), "p99": 1e3 * float(np.percentile(times, 99))},
    }
    print(json.dumps(out), flush=True)


def run_vk(args, cfg):
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    from __graft_entry__ import build
    build()
    import paper_2409_14222_gb300 as vk
    import synthetic_inputs as si
    Nc, L, k, sweeps, rtol, desc = cfg
    opts = vk.default_options(sweeps=sweeps)
    if args.prec == "f32":
        opts.factor_prec = vk.VK_PREC_F32
    elif args.prec == "f64e":
        opts.factor_prec = vk.VK_PREC_F64E
    if args.no_graph:
        opts.use_graph = 0
    if args.spmv_warps:
        opts.spmv_warps = args.spmv_warps
    stream = torch.cuda.current_stream()
    G = vk.Hierarchy(Nc, L, k, options=opts)
    ndof = G.ndof()
    # inputs resident in HBM before timing: one RHS per step
    seeds = [rank * 100000 + s for s in range(args.warmup + args.steps)]
    B = [torch.from_numpy(si.rhs_normal(ndof, s)).cuda() for s in seeds]
    x = torch.zeros(ndof, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for w in range(args.warmup):
        G.solve(B[w], x, rtol=rtol, history=False)
    torch.cuda.synchronize()
    G.stats_reset(time_kernels=False)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    iters = []
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        torch.cuda.profiler.start()          # a profiler started with --profile-from-start off sees only this
        for s in range(args.steps):
            flush.fill_(float(s))            # overwrite L2 (256 MiB > 129 MB) between timed solves
            ev[s][0].record(stream)
            out = G.solve(B[args.warmup + s], x, rtol=rtol, history=False)
            ev[s][1].record(stream)
            iters.append(out["iterations"])
            if not out["converged"]:
                raise RuntimeError(f"solve {s} did not converge: {out}")
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    barrier(world)
    st = G.stats()
    times_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = max_over_ranks(sum(times_ms) / 1e3, world)
    value = world * args.steps / total_s
    vcycles = st["vcycles"]
    # dominant kernel: every finest-level patch-apply launch of the same K solves, bracketed by CUDA
    # events on its stream (the solves run through the host-driven FGMRES loop here, because events
    # cannot bracket each iteration of the graph's device-side loop; the kernels and launch
    # configurations are the same)
    G.stats_reset(time_kernels=True)
    for s in range(args.steps):
        flush.fill_(float(s))
        G.solve(B[args.warmup + s], x, rtol=rtol, history=False)
    torch.cuda.synchronize()
    kt = G.stats()
    G.stats_reset(time_kernels=False)       # back to the graph path for the end-to-end pass
    # end to end through the C ABI with host buffers (pinned): H2D copy + solve + D2H copy per step
    bh = [torch.from_numpy(si.rhs_normal(ndof, 7777 + s)).pin_memory() for s in range(args.steps)]
    xh = torch.zeros(ndof, dtype=torch.float64).pin_memory()
    G.solve_host(bh[0].numpy(), xh.numpy(), rtol=rtol)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for s in range(args.steps):
        G.solve_host(bh[s].numpy(), xh.numpy(), rtol=rtol)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    if rank != 0:
        return
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", HBM_FALLBACK))
    apply_avg_s = kt["apply_ms"] / max(kt["apply_launches"], 1) / 1e3
    gbs = kt["apply_bytes"] / apply_avg_s / 1e9
    gflops = kt["apply_flops"] / apply_avg_s / 1e9
    frac_hbm, frac_alu = gbs / hbm, gflops / FP64_NOMINAL_GFLOPS
    if args.prec == "f64" and frac_alu > frac_hbm:
        roof = {"bound": "alu", "achieved": gflops / 1e3, "peak": FP64_NOMINAL_GFLOPS / 1e3, "unit": "TFLOP/s",
                "frac": frac_alu, "traffic": None, "kernel": "k_patch_apply (finest level, FP64 inverses)",
                "peak_source": "GB300 nominal FP64 rate 1.25 TFLOP/s (fp64 FMA pipe)",
                "hbm_view": {"achieved_gbs": gbs, "peak_gbs": hbm, "frac": frac_hbm, "peak_source": peak_kind}}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": frac_hbm, "traffic": None,
                "kernel": f"k_patch_apply (finest level, {args.prec.upper()} inverses)",
                "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"}
    roof["traffic"] = recorded_traffic(args.config, args.prec)
    roof["launch_avg_us"] = apply_avg_s * 1e6
    roof["bytes_per_launch"] = kt["apply_bytes"]
    roof["launches_timed"] = int(kt["apply_launches"])
    roof["spmv"] = spmv_roofline(kt, "spmv_bytes", hbm, peak_kind, "k_sell residual r = b - A x (finest level, FP64)")
    cpu = None
    if not args.no_cpu_baseline:
        cpu = oracle_cpu_baseline(cfg)
    clocks = clk.summary()
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"f64": "f64", "f64e": "f64 vectors; patch inverses as FP32 pairs (48-bit), FP32-pair products",
                  "f32": "f64 vectors, f32 patch inverses"}[args.prec],
        "data": "synthetic",
        "config": {"workload": desc, "ndof": ndof, "levels": L, "k": k, "sweeps": sweeps, "rtol": rtol,
                   "factor_prec": args.prec, "fgmres_loop": "host" if args.no_graph else "CUDA graph (WHILE node)",
                   "rhs": "N(0,1), numpy default_rng(seed)",
                   "l2": "256 MiB buffer overwritten between timed solves (outside the per-solve events)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "apply_schedule": schedules(G, L)},
        "vcycle_dof_per_s": world * ndof * vcycles / total_s,
        "iterations": {"mean": float(np.mean(iters)), "min": int(min(iters)), "max": int(max(iters))},
        "latency_ms": {"p50": float(np.percentile(times_ms, 50)), "p99": float(np.percentile(times_ms, 99))},
        "e2e": {"value": world * args.steps / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": 8 * ndof,
                "d2h_bytes_per_step": 8 * ndof},
        "gpu_launches": int(st["launches"]),
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clocks,
    }
    print(json.dumps(out), flush=True)


def run_batch(args, cfg):
    """cfg4: 16 right-hand sides per step through vk_solve_batch (FP32 V-cycle, BF16/FP16 patch
    inverses on the tensor cores, FP64 FGMRES per column), against plain FP64 single solves."""
    import torch
    from __graft_entry__ import build
    build()
    import paper_2409_14222_gb300 as vk
    import synthetic_inputs as si
    torch.cuda.set_device(0)
    Nc, L, k, sweeps, rtol, desc = cfg
    bp = vk.VK_BATCH_FP16 if args.batch_prec == "fp16" else vk.VK_BATCH_BF16
    t0 = time.perf_counter()
    engines = {"tcgen05": vk.VK_ENGINE_TCGEN05, "mma_sync": vk.VK_ENGINE_MMA_SYNC}
    other = "mma_sync" if args.engine == "tcgen05" else "tcgen05"
    G = vk.Hierarchy(Nc, L, k, options=vk.default_options(sweeps=sweeps, batch_prec=bp,
                                                             batch_engine=engines[args.engine],
                                                             batch_max_iterations=args.batch_maxit))
    setup_s = time.perf_counter() - t0
    n = G.ndof()
    stream = torch.cuda.current_stream()
    nb = args.warmup + args.steps
    Bs = [torch.from_numpy(si.rhs_batch(n, range(16 * i, 16 * i + 16)).T.copy()).cuda() for i in range(min(nb, 4))]
    X = torch.zeros(16, n, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for w in range(args.warmup):
        G.solve_batch(Bs[w % len(Bs)], X, rtol=rtol, maxit=args.batch_maxit)
    torch.cuda.synchronize()
    G.stats_reset(time_kernels=False)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    iters = []
    with ClockSampler(0) as clk:
        torch.cuda.profiler.start()
        for st in range(args.steps):
            flush.fill_(float(st))
            ev[st][0].record(stream)
            out = G.solve_batch(Bs[st % len(Bs)], X, rtol=rtol, maxit=args.batch_maxit)
            ev[st][1].record(stream)
            iters += [o["iterations"] for o in out]
            if not all(o["converged"] for o in out):
                raise RuntimeError("a column did not converge")
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    stt = G.stats()
    times_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(times_ms) / 1e3
    value = 16 * args.steps / total_s
    # tensor-core patch apply, finest level: CUDA events around every launch of the same solves
    G.stats_reset(time_kernels=True)
    for st in range(min(args.steps, 3)):
        G.solve_batch(Bs[st % len(Bs)], X, rtol=rtol, maxit=args.batch_maxit)
    torch.cuda.synchronize()
    kt = G.stats()
    G.stats_reset(time_kernels=False)
    avg_s = kt["apply_ms"] / max(kt["apply_launches"], 1) / 1e3
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", HBM_FALLBACK))
    gbs = kt["batch_apply_bytes"] / avg_s / 1e9
    tflops = kt["batch_apply_flops"] / avg_s / 1e12
    roof = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "traffic": None,
            "kernel": (f"{'k_patch_tc (tcgen05' if args.engine == 'tcgen05' else 'k_patch_mma (mma.sync'}; "
                       f"{args.batch_prec.upper()} inverses x 16 right-hand sides, finest level)"),
            "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})", "launch_avg_us": avg_s * 1e6,
            "bytes_per_launch": kt["batch_apply_bytes"], "tensor_tflops": tflops,
            "tensor_frac_of_bf16_peak": tflops / float(peaks.get("bf16_tflops", 1888.3)),
            "spmv": spmv_roofline(kt, "batch_spmv_bytes", hbm, peak_kind,
                                  "k_mm block residual R = B - A X (finest level, FP32, 16 right-hand sides)")}
    # the same solves with the other tensor-core engine (tcgen05 with TMEM and TMA, or warp-level mma.sync)
    Gm = vk.Hierarchy(Nc, L, k, options=vk.default_options(sweeps=sweeps, batch_prec=bp,
                                                              batch_engine=engines[other],
                                                              batch_max_iterations=args.batch_maxit))
    Xm = torch.zeros_like(X)
    Gm.solve_batch(Bs[0], Xm, rtol=rtol, maxit=args.batch_maxit)
    torch.cuda.synchronize()
    nm = min(args.steps, 3)
    tm = 0.0
    for st in range(nm):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(float(st))
        e0.record(stream)
        Gm.solve_batch(Bs[st % len(Bs)], Xm, rtol=rtol, maxit=args.batch_maxit)
        e1.record(stream)
        torch.cuda.synchronize()
        tm += e0.elapsed_time(e1) / 1e3
    Gm.stats_reset(time_kernels=True)
    Gm.solve_batch(Bs[0], Xm, rtol=rtol, maxit=args.batch_maxit)
    torch.cuda.synchronize()
    km = Gm.stats()
    am = km["apply_ms"] / max(km["apply_launches"], 1) / 1e3
    other_engine = {"engine": other, "solves_per_s": 16 * nm / tm, "patch_apply_us": am * 1e6,
                "patch_apply_gbs": km["batch_apply_bytes"] / am / 1e9,
                "bytes_per_launch": km["batch_apply_bytes"]}
    del Gm, Xm
    # the same solves with the coarsest-level solve in FP32 instead of FP64 (batch_coarse_fp32)
    Gc = vk.Hierarchy(Nc, L, k, options=vk.default_options(sweeps=sweeps, batch_prec=bp,
                                                              batch_engine=engines[args.engine],
                                                              batch_max_iterations=args.batch_maxit,
                                                              batch_coarse_fp32=1))
    Xc = torch.zeros_like(X)
    Gc.solve_batch(Bs[0], Xc, rtol=rtol, maxit=args.batch_maxit)
    torch.cuda.synchronize()
    tc_ = 0.0
    for st in range(nm):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(float(st))
        e0.record(stream)
        oc = Gc.solve_batch(Bs[st % len(Bs)], Xc, rtol=rtol, maxit=args.batch_maxit)
        e1.record(stream)
        torch.cuda.synchronize()
        tc_ += e0.elapsed_time(e1) / 1e3
    fp32_coarse = {"solves_per_s": 16 * nm / tc_, "iterations_mean": float(np.mean([o["iterations"] for o in oc]))}
    del Gc, Xc
    # plain FP64, one right-hand side at a time, same GPU and tolerance
    G64 = vk.Hierarchy(Nc, L, k, options=vk.default_options(sweeps=sweeps))
    x1 = torch.zeros(n, dtype=torch.float64, device="cuda")
    B0 = Bs[0]
    G64.solve(B0[0].contiguous(), x1, rtol=rtol)
    torch.cuda.synchronize()
    nf = min(args.steps, 8)
    errs, t64 = [], 0.0
    G.solve_batch(B0, X, rtol=rtol, maxit=args.batch_maxit)
    for r in range(nf):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(float(r))
        e0.record(stream)
        G64.solve(B0[r].contiguous(), x1, rtol=rtol, history=False)
        e1.record(stream)
        torch.cuda.synchronize()
        t64 += e0.elapsed_time(e1) / 1e3
        errs.append(float(torch.linalg.vector_norm(X[r] - x1) / torch.linalg.vector_norm(x1)))
    fp64 = {"solves_per_s": nf / t64, "ms_per_solve": 1e3 * t64 / nf}
    # FP64 single-right-hand-side kernels at this size: CUDA events around the finest patch apply and
    # the finest residual SpMV (host-driven FGMRES loop, same kernels and launch shapes)
    G64.stats_reset(time_kernels=True)
    G64.solve(B0[0].contiguous(), x1, rtol=rtol, history=False)
    torch.cuda.synchronize()
    k64 = G64.stats()
    G64.stats_reset(time_kernels=False)
    a64 = k64["apply_ms"] / max(k64["apply_launches"], 1) / 1e3
    fp64["patch_apply"] = {"kernel": "k_patch_apply (finest level, FP64 inverses)", "launch_avg_us": a64 * 1e6,
                           "tflops": k64["apply_flops"] / a64 / 1e12,
                           "frac_of_fp64_nominal": k64["apply_flops"] / a64 / 1e9 / FP64_NOMINAL_GFLOPS,
                           "hbm_gbs": k64["apply_bytes"] / a64 / 1e9}
    fp64["spmv"] = spmv_roofline(k64, "spmv_bytes", hbm, peak_kind, "k_sell residual r = b - A x (finest level, FP64)")
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": f"f64 FGMRES per column; f32 V-cycle with f64 coarsest solve; {args.batch_prec} patch inverses "
                 f"(tensor cores, f32 accumulate)",
        "engine": args.engine,
        "data": "synthetic",
        "config": {"workload": desc + ", 16 right-hand sides per step", "ndof": n, "levels": L, "k": k,
                   "rhs_per_step": 16, "rtol": rtol, "setup_s": setup_s,
                   "l2": "256 MiB buffer overwritten between timed steps (outside the events)"},
        "iterations": {"mean": float(np.mean(iters)), "min": int(min(iters)), "max": int(max(iters))},
        "vcycle_dof_per_s": 16 * n * stt["vcycles"] / total_s,
        "latency_ms": {"p50": float(np.percentile(times_ms, 50)), "p99": float(np.percentile(times_ms, 99))},
        "plain_fp64_single_rhs": fp64, "speedup_vs_plain_fp64": value / fp64["solves_per_s"],
        "other_engine": other_engine, "fp32_coarse_solve_variant": fp32_coarse,
        "rel_error_vs_fp64_solution": {"max": max(errs), "mean": float(np.mean(errs)), "columns": nf},
        "gpu_launches": int(stt["launches"]), "roofline": roof, "clocks": clk.summary(),
    }), flush=True)


def serve_pass(vk, srv, reqs, arrivals):
    """Submit reqs at the given arrival offsets (s) from one thread; collect results in order."""
    import threading
    import synthetic_inputs as si
    tickets = [None] * len(reqs)
    rhs = [si.rhs_normal(vk.ndof_of(*key), seed) for key, seed in reqs]
    t0 = time.perf_counter()

    def submitter():
        for i, ((key, seed), ta) in enumerate(zip(reqs, arrivals)):
            delay = t0 + ta - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets[i] = srv.submit(*key, rhs[i], rtol=1e-8)

    th = threading.Thread(target=submitter)
    th.start()
    lat, done_t, iters = [], [], []
    for i in range(len(reqs)):
        while tickets[i] is None:
            time.sleep(1e-4)
        x, res = srv.wait(tickets[i])
        if res["status"] not in (0, 5):
            raise RuntimeError(f"request {i} failed: {res}")
        lat.append(res["latency_ms"])
        iters.append(res["iterations"])
        done_t.append(time.perf_counter() - t0)
    th.join()
    span = max(done_t) - min(arrivals)
    return {"requests": len(reqs), "solves_per_s": len(reqs) / span,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_iterations": float(np.mean(iters))}


def run_serving(args):
    """cfg5: continuous batching of a Poisson request stream (vk_server, C++ runtime)."""
    import torch
    from __graft_entry__ import build
    build()
    import paper_2409_14222_gb300 as vk
    import synthetic_inputs as si
    torch.cuda.set_device(0)
    mix = si.request_mix(args.requests, seed=42)
    keys = lambda N, k: (8, int(np.log2(N // 8)) + 1, k)
    reqs = [(keys(N, k), seed) for N, k, seed in mix]
    uniq = sorted(set(k for k, _ in reqs))
    opts = vk.default_options()
    if args.prec == "f32":
        opts.factor_prec = vk.VK_PREC_F32
    elif args.prec == "f64e":
        opts.factor_prec = vk.VK_PREC_F64E

    def warm(srv, per_key):
        # every hierarchy resident (per_key instances of each key) before any timed request
        for key in uniq:
            ts = [srv.submit(*key, si.rhs_normal(vk.ndof_of(*key), 7), rtol=1e-8) for _ in range(per_key)]
            for t in ts:
                _, res = srv.wait(t)
                if res["status"] not in (0, 5):
                    raise RuntimeError(f"warm-up solve of {key} failed: {res}")

    out_rates = {}
    per_key = min(args.slots, 2)
    srv = vk.Server(slots=args.slots, options=opts, max_per_key=per_key)
    t0 = time.perf_counter()
    warm(srv, per_key)
    warm_s = time.perf_counter() - t0
    ncap = min(len(reqs), 300)
    cap = serve_pass(vk, srv, reqs[:ncap], [0.0] * ncap)
    capacity = cap["solves_per_s"]
    with ClockSampler(0) as clk:
        for mult in (0.5, 1.0, 2.0):
            n = len(reqs) if mult == 1.0 else min(len(reqs), 300)
            arr = si.poisson_arrivals(n, mult * capacity, seed=42 + int(10 * mult))
            out_rates[f"{mult}x"] = serve_pass(vk, srv, reqs[:n], arr)
    st = srv.stats()
    srv.close()
    # plain FP64, one request at a time, same stream at the measured 1x rate
    base = {}
    if not args.no_baseline:
        srv1 = vk.Server(slots=1, options=vk.default_options())
        warm(srv1, 1)
        n1 = min(len(reqs), 300)
        base_cap = serve_pass(vk, srv1, reqs[:n1], [0.0] * n1)
        base_rate = serve_pass(vk, srv1, reqs[:n1], si.poisson_arrivals(n1, capacity, seed=52))
        base = {"capacity_solves_per_s": base_cap["solves_per_s"], "at_1x_rate": base_rate}
        srv1.close()
    one = out_rates["1.0x"]
    print(json.dumps({
        "metric": METRIC, "value": capacity, "unit": "solves/s", "n_gpus": 1, "steps": len(reqs),
        "warmup": len(uniq) * per_key, "ms_per_step": 1e3 / capacity, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"f64": "f64", "f64e": "f64 vectors; FP32-pair patch inverses", "f32": "f64 vectors, f32 patch inverses"}[args.prec],
        "data": "synthetic",
        "config": {"workload": CONFIGS["cfg5"][5], "requests": len(reqs), "slots": args.slots,
                   "distinct_hierarchies": len(uniq), "factor_prec": args.prec, "arrivals": "Poisson, seed 42",
                   "warm_s": warm_s},
        "latency_ms": {"p50": one["p50_ms"], "p99": one["p99_ms"]},
        "rates": out_rates, "capacity": cap, "one_at_a_time_plain_fp64": base,
        "server": st, "clocks": clk.summary(),
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="vk", choices=["vk", "reference"])
    ap.add_argument("--config", default="cfg2", choices=sorted(CONFIGS))
    ap.add_argument("--prec", default="f64", choices=["f64", "f64e", "f32"],
                    help="patch inverses: FP64, FP32-pair emulated FP64, or FP32")
    ap.add_argument("--no-graph", action="store_true",
                    help="host-driven FGMRES loop instead of the whole-solve CUDA graph (for kernel profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--requests", type=int, default=1000, help="cfg5: requests in the 1x stream")
    ap.add_argument("--slots", type=int, default=4, help="cfg5: concurrent solves")
    ap.add_argument("--no-baseline", action="store_true", help="cfg5: skip the one-at-a-time FP64 pass")
    ap.add_argument("--batch-prec", default="bf16", choices=["bf16", "fp16"], help="cfg4: 16-bit inverse format")
    ap.add_argument("--spmv-warps", type=int, default=0, help="SELL threads-per-row rule (warps per SM); 0 = default")
    ap.add_argument("--levels", type=int, default=0, help="override the level count (profiling variants only)")
    ap.add_argument("--rtol", type=float, default=0.0, help="override the tolerance (profiling variants only)")
    ap.add_argument("--batch-maxit", type=int, default=60, help="cfg4: FGMRES basis size per right-hand side")
    ap.add_argument("--engine", default="tcgen05", choices=["tcgen05", "mma_sync"],
                    help="cfg4: tensor-core instruction family of the patch solves")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "vk":
        ap.error("--warmup must be >= 3")
    cfg = CONFIGS[args.config]
    if args.levels or args.rtol:
        # a smaller or looser variant of a workload, for profiler captures (never a bench line)
        Nc, L, k, sweeps, rtol, desc = cfg
        L = args.levels or L
        rtol = args.rtol or rtol
        cfg = (Nc, L, k, sweeps, rtol, f"{desc.split(',')[0]}, {Nc}x{Nc} -> {Nc << (L - 1)}x{Nc << (L - 1)} "
                                         f"({L} levels), rtol {rtol:g} [profiling variant]")
    if args.impl == "reference":
        run_reference(args, cfg)
    elif args.config == "cfg5":
        run_serving(args)
    elif args.config == "cfg4":
        run_batch(args, cfg)
    else:
        run_vk(args, cfg)


if __name__ == "__main__":
    main()
