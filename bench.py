"""Benchmark: FGMRES solves of 2D Stokes (Taylor-Hood P2/P1, 32x32 -> 512x512, 5 levels, 2,364,419
DoFs) on one GB300.

One step = one FGMRES solve to 1e-8 relative residual (zero initial guess, V(1,1) cycles with
Chebyshev-accelerated matrix-full Vanka smoothing, FP64) of a seeded N(0,1) right-hand side already
resident in HBM.  The hierarchy (assembly, patch inverses, coarse inverse, eigenvalue estimates) is
built once before timing and kept resident, as a solver service would.  The default line also nests
sub-records measured in the same run: the 16x16 -> 128x128 P2/P1 workload (148,739 DoFs); the
512x512 workload with FP32-pair patch inverses; its 16-right-hand-side mixed-precision solve (BF16
patch inverses on the tensor cores, FP32 V-cycle, FP64 FGMRES per column) with its error against the
FP64 solutions; a Poisson stream of solve requests through the solve service; (BDM_k, dP_{k-1}) on
5x5 -> 80x80 for k = 2..5; and matrix-full against matrix-free patch setup.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl vk|reference] [--config cfg4]

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
    "cfg4batch": (32, 5, 2, 1, 1e-8, "2D Stokes TH P2/P1, 32x32 -> 512x512 (5 levels), FGMRES to 1e-8"),
    "cfg5": (8, 0, 0, 1, 1e-8, "Serving: Poisson stream of solve requests, N in {16..256} (coarsest 8x8), "
                               "k in {2,3,4}, FGMRES to 1e-8"),
    "stopping": (5, 0, 0, 1, 1e-2, "Stopping-criterion study (Sec. 4.4): manufactured problem, tolerance halving"),
}
DEFAULT_CONFIG = "cfg4"

HBM_FALLBACK = 6800.0
# the oracle's stored whole-solve results (tests/golden/make_golden.py, oracle only): the iteration
# count of a configuration whose oracle solve is too long to repeat here
GOLDEN = {"cfg4": "oracle_p2_32to512.npz", "cfg3p4": "oracle_p4_16to64.npz"}


def golden_iterations(config):
    name = GOLDEN.get(config)
    if not name:
        return None
    p = os.path.join(ROOT, "tests", "golden", name)
    if not os.path.exists(p):
        return None
    with np.load(p) as z:
        return int(z["iterations"])


def recorded_traffic(config, prec, kernel="k_patch_apply"):
    """DRAM bytes per launch of a kernel from the committed ncu record, or None when the record is for
    another workload or the kernel source changed since the capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel]
        with open(os.path.join(ROOT, "paper_2409_14222_gb300", "csrc", rec["source"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
    except (OSError, KeyError, ValueError):
        return None
    if sha != rec["source_sha256_16"] or config != rec.get("config") or prec != rec.get("prec"):
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




# ---- the oracle on the host cores (cpu_baseline and --impl reference) ---------------------------
SAMPLE_ITERS = 3


def oracle_sample_hierarchy(cfg):
    """The oracle hierarchy a bounded sample runs on: the workload's own when its oracle setup and
    iterations take seconds (up to 16x16 -> 128x128 P2), else the 16x16 -> 128x128 P2/P1 hierarchy of
    the same method (same element, patches, smoother, cycle and Krylov method, 148,739 DoFs) whose
    per-DoF cost stands in for the larger mesh."""
    from oracle import solver
    Nc, L, k, sweeps, rtol, _ = cfg
    ndof_target = 2 * (k * (Nc << (L - 1)) + 1) ** 2 + ((k - 1) * (Nc << (L - 1)) + 1) ** 2
    if ndof_target <= 148739:
        key = (Nc, L, k, sweeps)
    else:
        key = (16, 4, k, sweeps)
    t0 = time.perf_counter()
    H = solver.Hierarchy(key[0], key[1], key[2], sweeps=key[3])
    return H, key, ndof_target, time.perf_counter() - t0


def oracle_steps(H, rtol, count, seed0):
    """`count` samples; each is one oracle FGMRES solve stopped after SAMPLE_ITERS iterations (V-cycles,
    products, orthogonalisation, Givens, the final combination and true residual).  Seconds each."""
    from oracle import solver
    import synthetic_inputs as si
    ndof = H.finest.space.ndof
    out = []
    for s in range(count):
        b = si.rhs_normal(ndof, seed0 + s)
        t0 = time.perf_counter()
        solver.solve(H, b, rtol, SAMPLE_ITERS)
        out.append(time.perf_counter() - t0)
    return out


def oracle_target_iterations(config, cfg, H, key):
    """FGMRES iterations of one solve of the target workload by the oracle: the stored oracle result
    when the workload is too large to solve here, else one untimed full oracle solve."""
    from oracle import solver
    import synthetic_inputs as si
    it = golden_iterations(config)
    if it is not None:
        return it, "stored oracle result (tests/golden)"
    if key[:3] == cfg[:3]:
        res = solver.solve(H, si.rhs_normal(H.finest.space.ndof, 0), cfg[4], 100)
        return res.iters, "one untimed full oracle solve (seed 0)"
    return None, "unknown"


def cpu_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def oracle_cpu_baseline(config, cfg, budget_s=15.0):
    """The oracle timed as it stands on the host cores, on a bounded sample (about budget_s of CPU
    work), scaled to solves/s of the workload."""
    H, key, ndof_target, setup_s = oracle_sample_hierarchy(cfg)
    iters, src = oracle_target_iterations(config, cfg, H, key)
    times = oracle_steps(H, cfg[4], 1, 500)
    n = max(1, int(budget_s / max(times[0], 1e-3)))
    times = oracle_steps(H, cfg[4], n, 600)
    mean = float(np.mean(times))
    ndof_s = H.finest.space.ndof
    scale = (ndof_target / ndof_s) * ((iters or SAMPLE_ITERS) / SAMPLE_ITERS)
    return {"value": 1.0 / (mean * scale), "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": (f"{n} oracle FGMRES solves of seeded N(0,1) right-hand sides on the {key[0]}x{key[0]} -> "
                       f"{key[0] << (key[1] - 1)}x{key[0] << (key[1] - 1)} P{key[2]} hierarchy ({ndof_s} DoFs), "
                       f"each stopped after {SAMPLE_ITERS} iterations, {mean:.2f} s each; scaled to one solve of "
                       f"the workload by DoFs ({ndof_target}/{ndof_s}) and iterations ({iters}/{SAMPLE_ITERS}, "
                       f"{src}); oracle setup {setup_s:.1f} s excluded; NumPy/SciPy FP64, BLAS threads "
                       f"{os.environ.get('OPENBLAS_NUM_THREADS', 'default')}"),
            "sample_seconds": mean, "scale_to_one_solve": scale}


def run_reference(args, config, cfg):
    """--impl reference: the oracle on the host cores, same metric, unit and config as the GPU arm.
    Each step is a bounded sample (one oracle solve stopped after SAMPLE_ITERS iterations); ms_per_step
    is that measured sample time, and `value` scales it to solves/s of the workload (the scale factor
    is printed under "extrapolation")."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    H, key, ndof_target, setup_s = oracle_sample_hierarchy(cfg)
    iters, src = oracle_target_iterations(config, cfg, H, key)
    iters = iters or SAMPLE_ITERS
    oracle_steps(H, cfg[4], args.warmup, 100)
    times = oracle_steps(H, cfg[4], args.steps, 1000)
    total = sum(times)
    ndof_s = H.finest.space.ndof
    scale = (ndof_target / ndof_s) * (iters / SAMPLE_ITERS)
    value = args.steps / (total * scale)
    sample = (f"each step: one oracle FGMRES solve of a seeded N(0,1) right-hand side on the {key[0]}x{key[0]} -> "
              f"{key[0] << (key[1] - 1)}x{key[0] << (key[1] - 1)} P{key[2]} hierarchy ({ndof_s} DoFs) stopped "
              f"after {SAMPLE_ITERS} iterations; value = steps / (timed seconds x {scale:.3g}), the scale to one "
              f"solve of the workload by DoFs ({ndof_target}/{ndof_s}) and iterations ({iters}/{SAMPLE_ITERS}, "
              f"{src}); oracle setup {setup_s:.1f} s before timing")
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": cfg[5], "ndof": ndof_target, "iterations": iters},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "extrapolation": {"timed_seconds": total, "sample_ndof": ndof_s, "target_ndof": ndof_target,
                          "sample_iterations": SAMPLE_ITERS, "target_iterations": iters, "scale": scale,
                          "ms_per_step_is": "the measured sample", "value_is": "solves/s of the workload"},
        "vcycle_dof_per_s": ndof_s * SAMPLE_ITERS * args.steps / total,
        "latency_ms": {"p50": 1e3 * float(np.percentile(times, 50)) * scale,
                       "p99": 1e3 * float(np.percentile(times, 99)) * scale},
    }
    print(json.dumps(out), flush=True)


# ---- GPU arm ---------------------------------------------------------------------------------------
def timed_solves(torch, G, B, x, rtol, steps, warmup, flush, world, clk=None):
    """W untimed solves, then K solves each bracketed by CUDA events on the launching stream, with the
    L2 overwritten (256 MiB > 129 MB) before each (outside the events).  Max over ranks."""
    stream = torch.cuda.current_stream()
    for w in range(warmup):
        G.solve(B[w], x, rtol=rtol, history=False)
    torch.cuda.synchronize()
    G.stats_reset(time_kernels=False)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    iters = []
    barrier(world)
    torch.cuda.synchronize()
    if clk is not None:
        clk.__enter__()
    try:
        torch.cuda.profiler.start()          # a profiler started with --profile-from-start off sees only this
        for s in range(steps):
            flush.fill_(float(s))
            ev[s][0].record(stream)
            out = G.solve(B[warmup + s], x, rtol=rtol, history=False)
            ev[s][1].record(stream)
            iters.append(out["iterations"])
            if not out["converged"]:
                raise RuntimeError(f"solve {s} did not converge: {out}")
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    finally:
        if clk is not None:
            clk.__exit__(None, None, None)
    barrier(world)
    st = G.stats()
    times_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = max_over_ranks(sum(times_ms) / 1e3, world)
    return {"total_s": total_s, "times_ms": times_ms, "iters": iters, "vcycles": st["vcycles"],
            "launches": int(st["launches"])}


def kernel_times(torch, G, B, x, rtol, count, warmup, flush):
    """CUDA events around every finest-level patch-apply and V-cycle residual launch of `count` solves
    (host-driven FGMRES loop: events cannot bracket the iterations of the graph's device-side loop; the
    kernels and their launch configurations are the same)."""
    G.stats_reset(time_kernels=True)
    for s in range(count):
        flush.fill_(float(s))
        G.solve(B[warmup + s], x, rtol=rtol, history=False)
    torch.cuda.synchronize()
    kt = G.stats()
    G.stats_reset(time_kernels=False)
    return kt


def apply_roofline(kt, prec, hbm, peak_kind, fp64_tflops, config):
    """Roofline of the dominant kernel, the finest-level patch application: FP64 inverses are bound by
    the FP64 pipe (2 flops per 8-byte entry needs 1.7 TFLOP/s at full HBM bandwidth, above the part's
    FP64 rate), so they are measured against the FMA rate probed in this run; FP32 and FP32-pair
    inverses against the measured HBM bandwidth."""
    n = max(int(kt["apply_launches"]), 1)
    avg_s = kt["apply_ms"] / n / 1e3
    gbs = kt["apply_bytes"] / avg_s / 1e9
    tflops = kt["apply_flops"] / avg_s / 1e12
    hbm_view = {"achieved_gbs": gbs, "peak_gbs": hbm, "frac": gbs / hbm,
                "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"}
    if prec == "f64":
        roof = {"bound": "alu", "achieved": tflops, "peak": fp64_tflops, "unit": "TFLOP/s",
                "frac": tflops / fp64_tflops, "kernel": "k_patch_apply (finest level, FP64 inverses)",
                "peak_source": "FP64 FMA rate measured in this run (vk_measure_fma_rate, of measured)",
                "hbm_view": hbm_view}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                "kernel": f"k_patch_apply (finest level, {prec.upper()} inverses)",
                "peak_source": hbm_view["peak_source"] + ", of measured" if peak_kind == "measured" else
                "fallback 6.8 TB/s, of fallback", "tflops": tflops}
    roof["traffic"] = recorded_traffic(config, prec)
    roof["launch_avg_us"] = avg_s * 1e6
    roof["bytes_per_launch"] = kt["apply_bytes"]
    roof["flops_per_launch"] = kt["apply_flops"]
    roof["launches_timed"] = int(kt["apply_launches"])
    return roof


def make_options(vk, args, sweeps):
    opts = vk.default_options(sweeps=sweeps)
    if args.prec == "f32":
        opts.factor_prec = vk.VK_PREC_F32
    elif args.prec == "f64e":
        opts.factor_prec = vk.VK_PREC_F64E
    if args.no_graph:
        opts.use_graph = 0
    if args.pdl:
        opts.graph_pdl = 1
    if args.spmv_warps:
        opts.spmv_warps = args.spmv_warps
    return opts


def single_rhs_record(vk, torch, si, cfg, args, opts, steps, warmup, flush, world, rank, peaks, clk=None,
                      e2e=True, cell=0):
    """One single-right-hand-side workload: setup, timed solves, kernel times, end-to-end solves."""
    Nc, L, k, sweeps, rtol, desc = cfg
    t0 = time.perf_counter()
    G = vk.Hierarchy(Nc, L, k, options=opts, cell=cell)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    ndof = G.ndof()
    seeds = [rank * 100000 + s for s in range(warmup + steps)]
    B = [torch.from_numpy(si.rhs_normal(ndof, s)).cuda() for s in seeds]
    x = torch.zeros(ndof, dtype=torch.float64, device="cuda")
    t = timed_solves(torch, G, B, x, rtol, steps, warmup, flush, world, clk)
    graph_pdl = int(G.stats()["graph_pdl"])
    kt = kernel_times(torch, G, B, x, rtol, min(steps, 10), warmup, flush)
    rec = {"G": G, "ndof": ndof, "setup_s": setup_s, "timed": t, "kt": kt, "graph_pdl": graph_pdl,
           "value": world * steps / t["total_s"],
           "vcycle_dof_per_s": world * ndof * t["vcycles"] / t["total_s"]}
    if e2e:
        # end to end through the C ABI with host buffers (pinned): H2D copy + solve + D2H copy per step
        bh = [torch.from_numpy(si.rhs_normal(ndof, 7777 + s)).pin_memory() for s in range(steps)]
        xh = torch.zeros(ndof, dtype=torch.float64).pin_memory()
        G.solve_host(bh[0].numpy(), xh.numpy(), rtol=rtol)
        torch.cuda.synchronize()
        barrier(world)
        t1 = time.perf_counter()
        for s in range(steps):
            G.solve_host(bh[s].numpy(), xh.numpy(), rtol=rtol)
        rec["e2e_s"] = max_over_ranks(time.perf_counter() - t1, world)
    return rec


def summary_of(rec, cfg, args, hbm, peak_kind, fp64_tflops, config, prec=None):
    prec = prec or args.prec
    t, kt = rec["timed"], rec["kt"]
    Nc, L, k, sweeps, rtol, desc = cfg
    return {
        "workload": desc, "ndof": rec["ndof"], "value": rec["value"], "unit": "solves/s",
        "ms_per_step": 1e3 * t["total_s"] / len(t["iters"]), "steps": len(t["iters"]),
        "vcycle_dof_per_s": rec["vcycle_dof_per_s"],
        "iterations": {"mean": float(np.mean(t["iters"])), "min": int(min(t["iters"])), "max": int(max(t["iters"]))},
        "latency_ms": {"p50": float(np.percentile(t["times_ms"], 50)), "p99": float(np.percentile(t["times_ms"], 99))},
        "setup_s": rec["setup_s"], "gpu_launches": t["launches"],
        "roofline": apply_roofline(kt, prec, hbm, peak_kind, fp64_tflops, config),
        "spmv": spmv_roofline(kt, "spmv_bytes", hbm, peak_kind, "k_sell residual r = b - A x (finest level, FP64)"),
        "apply_schedule": schedules(rec["G"], L),
    }


def batch_record(vk, torch, si, cfg, args, flush, hbm, peaks, peak_kind, G64=None, fp64_value=None,
                 engine=None, coarse_fp32=0, steps=None, profile=False):
    """16 right-hand sides per step through vk_solve_batch: FP32 V-cycle with BF16 (or FP16) scaled
    patch inverses on the tensor cores, FP64 coarsest solve, FP64 FGMRES per column.  With G64 (the
    FP64 single-right-hand-side hierarchy of the same workload) the first four columns are compared
    with FP64 solves of the same right-hand sides."""
    Nc, L, k, sweeps, rtol, desc = cfg
    bp = vk.VK_BATCH_FP16 if args.batch_prec == "fp16" else vk.VK_BATCH_BF16
    engine = engine or args.engine
    eng = {"tcgen05": vk.VK_ENGINE_TCGEN05, "mma_sync": vk.VK_ENGINE_MMA_SYNC}[engine]
    t0 = time.perf_counter()
    Gb = vk.Hierarchy(Nc, L, k, options=vk.default_options(sweeps=sweeps, batch_prec=bp, batch_engine=eng,
                                                              batch_max_iterations=args.batch_maxit,
                                                              batch_coarse_fp32=coarse_fp32))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    n = Gb.ndof()
    stream = torch.cuda.current_stream()
    Bs = [torch.from_numpy(si.rhs_batch(n, range(16 * i, 16 * i + 16)).T.copy()).cuda() for i in range(2)]
    X = torch.zeros(16, n, dtype=torch.float64, device="cuda")
    nsteps = steps or min(args.steps, 5)
    for w in range(3):
        Gb.solve_batch(Bs[w % 2], X, rtol=rtol, maxit=args.batch_maxit)
    torch.cuda.synchronize()
    Gb.stats_reset(time_kernels=False)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
    iters = []
    if profile:
        torch.cuda.profiler.start()          # a profiler started with --profile-from-start off sees only this
    for st in range(nsteps):
        flush.fill_(float(st))
        ev[st][0].record(stream)
        out = Gb.solve_batch(Bs[st % 2], X, rtol=rtol, maxit=args.batch_maxit)
        ev[st][1].record(stream)
        iters += [o["iterations"] for o in out]
        if not all(o["converged"] for o in out):
            raise RuntimeError("a column did not converge")
    torch.cuda.synchronize()
    if profile:
        torch.cuda.profiler.stop()
    stt = Gb.stats()
    times_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(times_ms) / 1e3
    value = 16 * nsteps / total_s
    # tensor-core patch apply and block residual, finest level: CUDA events around every launch
    Gb.stats_reset(time_kernels=True)
    out = Gb.solve_batch(Bs[0], X, rtol=rtol, maxit=args.batch_maxit)
    torch.cuda.synchronize()
    kt = Gb.stats()
    Gb.stats_reset(time_kernels=False)
    avg_s = kt["apply_ms"] / max(kt["apply_launches"], 1) / 1e3
    gbs = kt["batch_apply_bytes"] / avg_s / 1e9
    tflops = kt["batch_apply_flops"] / avg_s / 1e12
    rec = {
        "workload": desc + ", 16 right-hand sides per step", "engine": engine, "batch_prec": args.batch_prec,
        "coarse_solve": "fp32" if coarse_fp32 else "fp64",
        "value": value, "unit": "solves/s", "steps": nsteps, "ms_per_step": 1e3 * total_s / nsteps,
        "setup_s": setup_s, "vcycle_dof_per_s": 16 * n * stt["vcycles"] / total_s,
        "iterations": {"mean": float(np.mean(iters)), "min": int(min(iters)), "max": int(max(iters))},
        "latency_ms": {"p50": float(np.percentile(times_ms, 50)), "p99": float(np.percentile(times_ms, 99))},
        "gpu_launches": int(stt["launches"]),
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                     "kernel": (f"{'k_patch_tc (tcgen05' if engine == 'tcgen05' else 'k_patch_mma (mma.sync'}; "
                                f"{args.batch_prec.upper()} inverses x 16 right-hand sides, finest level)"),
                     "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})", "launch_avg_us": avg_s * 1e6,
                     "bytes_per_launch": kt["batch_apply_bytes"], "tensor_tflops": tflops,
                     "tensor_frac_of_bf16_peak": tflops / float(peaks.get("bf16_tflops", 1907.0))},
        "spmv": spmv_roofline(kt, "batch_spmv_bytes", hbm, peak_kind,
                              "k_mm block residual R = B - A X (finest level, FP32, 16 right-hand sides)"),
    }
    if G64 is not None:
        errs = []
        x1 = torch.zeros(n, dtype=torch.float64, device="cuda")
        for r in range(4):
            G64.solve(Bs[0][r].contiguous(), x1, rtol=rtol, history=False)
            errs.append(float(torch.linalg.vector_norm(X[r] - x1) / torch.linalg.vector_norm(x1)))
        rec["rel_error_vs_fp64_solution"] = {"max": max(errs), "mean": float(np.mean(errs)), "columns": 4}
    if fp64_value:
        rec["speedup_vs_plain_fp64_one_at_a_time"] = value / fp64_value
    del Gb, X
    torch.cuda.empty_cache()
    return rec


def bdm_records(vk, torch, si, args, flush, world, rank, peaks, hbm, peak_kind, fp64_tflops):
    """(BDM_k, dP_{k-1}) with the interior-penalty form and extended cell patches (Sec. 4.3): the paper's
    5x5 coarsest grid refined four times (80x80, 5 levels), k = 2..5, FGMRES to a 1e-10 reduction, FP64
    (the paper's timing study of this discretization is at four refinements)."""
    out = {}
    for k in (2, 3, 4, 5):
        cfg = (5, 5, k, 1, 1e-10, f"(BDM_{k}, dP_{k - 1}) interior penalty, 5x5 -> 80x80 (5 levels), "
                                   f"extended cell patches, FGMRES to 1e-10")
        rec = single_rhs_record(vk, torch, si, cfg, args, make_options(vk, args, 1), min(args.steps, 5), 3, flush,
                                world, rank, peaks, e2e=False, cell=vk.VK_CELL_BDM)
        out[f"k{k}"] = summary_of(rec, cfg, args, hbm, peak_kind, fp64_tflops, f"bdm{k}")
        del rec
        torch.cuda.empty_cache()
    return out


def patch_assembly_records(vk, torch, si):
    """Matrix-full (patch matrices gathered from the assembled CSR matrix, ASMPatchPC) against matrix-free
    (each patch matrix assembled from the element matrices of the cells it touches, PCPATCH; Sec. 3.1)
    patch setup on the device: the timed gather or assembly plus Gauss-Jordan inversion of every patch on
    every level, the whole setup, the device footprint, and whether the first solve is bit-identical
    (it must be: both build the same patch matrices in the same summation order)."""
    out = {}
    for name, cfg in (("cfg4", CONFIGS["cfg4"]), ("cfg3p4", CONFIGS["cfg3p4"])):
        Nc, L, k, sweeps, rtol, desc = cfg
        rec, xs = {"workload": desc}, []
        for asm in ("matrix_full", "matrix_free"):
            mode = vk.vk.VK_ASSEMBLY_MATRIX_FREE if asm == "matrix_free" else vk.vk.VK_ASSEMBLY_MATRIX_FULL
            t0 = time.perf_counter()
            G = vk.Hierarchy(Nc, L, k, options=vk.default_options(sweeps=sweeps, patch_assembly=mode))
            torch.cuda.synchronize()
            setup_s = time.perf_counter() - t0
            st = G.stats()
            b = torch.from_numpy(si.rhs_normal(G.ndof(), 99)).cuda()
            x = torch.zeros_like(b)
            G.solve(b, x, rtol=rtol, history=False)
            xs.append(x.cpu())
            rec[asm] = {"patch_setup_ms": st["setup_factor_ms"], "setup_s": setup_s,
                        "device_bytes": G.device_bytes()}
            G.close()
            del G, b, x
            torch.cuda.empty_cache()
        rec["first_solve_bit_identical"] = bool(torch.equal(xs[0], xs[1]))
        rec["matrix_free_over_full_patch_setup"] = rec["matrix_free"]["patch_setup_ms"] / rec["matrix_full"]["patch_setup_ms"]
        out[name] = rec
    return out


def run_vk(args, config, cfg):
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    from __graft_entry__ import build
    build()
    import paper_2409_14222_gb300 as vk
    import synthetic_inputs as si
    Nc, L, k, sweeps, rtol, desc = cfg
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", HBM_FALLBACK))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    fp64_tflops = vk.measure_fma_rate(True)
    fp32_tflops = vk.measure_fma_rate(False)
    opts = make_options(vk, args, sweeps)
    clk = ClockSampler(local)
    main = single_rhs_record(vk, torch, si, cfg, args, opts, args.steps, args.warmup, flush, world, rank, peaks, clk)
    s = summary_of(main, cfg, args, hbm, peak_kind, fp64_tflops, config)
    nested = {}
    if config == "cfg4" and world == 1 and not args.no_nested:
        c2 = CONFIGS["cfg2"]
        r2 = single_rhs_record(vk, torch, si, c2, args, make_options(vk, args, c2[3]), args.steps, args.warmup,
                               flush, world, rank, peaks, e2e=False)
        nested["cfg2"] = summary_of(r2, c2, args, hbm, peak_kind, fp64_tflops, "cfg2")
        del r2
        torch.cuda.empty_cache()
        if args.prec == "f64":
            # the same workload with FP32-pair inverses in the symmetric tile layout (about 48-bit
            # entries, FP32-pipe arithmetic, bound by HBM instead of the FP64 pipe), and its solution's
            # difference from the FP64 one on the same right-hand side
            oe = make_options(vk, args, sweeps)
            oe.factor_prec = vk.VK_PREC_F64E
            re_ = single_rhs_record(vk, torch, si, cfg, args, oe, min(args.steps, 10), 3, flush, world, rank, peaks,
                                    e2e=False)
            se = summary_of(re_, cfg, args, hbm, peak_kind, fp64_tflops, config, prec="f64e")
            b0 = torch.from_numpy(si.rhs_normal(main["ndof"], 4242)).cuda()
            xa, xb = torch.zeros_like(b0), torch.zeros_like(b0)
            oa = main["G"].solve(b0, xa, rtol=rtol, history=False)
            ob = re_["G"].solve(b0, xb, rtol=rtol, history=False)
            se["rel_diff_vs_fp64_solution"] = float(torch.linalg.vector_norm(xa - xb) / torch.linalg.vector_norm(xa))
            se["iterations_fp64_vs_f64e"] = [oa["iterations"], ob["iterations"]]
            se["speedup_vs_fp64"] = se["value"] / main["value"]
            se["dtype"] = "f64 vectors; patch inverses as FP32 pairs (48-bit), symmetric tiles, FP32-pair products"
            nested["f64e_symmetric"] = se
            del re_
            torch.cuda.empty_cache()
        nested["batch16"] = batch_record(vk, torch, si, cfg, args, flush, hbm, peaks, peak_kind, G64=main["G"],
                                         fp64_value=main["value"])
        main["G"] = None
        torch.cuda.empty_cache()
        if not args.no_serving:
            srv = serving_record(vk, si, args, args.serve_requests, (1.0,), 8, per_key=1)
            srv["workload"] = CONFIGS["cfg5"][5]
            nested["serving"] = srv
        if not args.no_bdm:
            nested["bdm"] = bdm_records(vk, torch, si, args, flush, world, rank, peaks, hbm, peak_kind, fp64_tflops)
        nested["patch_assembly"] = patch_assembly_records(vk, torch, si)
    if rank != 0:
        return
    cpu = None if args.no_cpu_baseline else oracle_cpu_baseline(config, cfg)
    roof = dict(s["roofline"])
    roof["spmv"] = s["spmv"]
    out = {
        "metric": METRIC, "value": main["value"], "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": s["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"f64": "f64", "f64e": "f64 vectors; patch inverses as FP32 pairs (48-bit), FP32-pair products",
                  "f32": "f64 vectors, f32 patch inverses"}[args.prec],
        "data": "synthetic",
        "config": {"workload": desc, "ndof": main["ndof"], "levels": L, "k": k, "sweeps": sweeps, "rtol": rtol,
                   "factor_prec": args.prec,
                   "fgmres_loop": "host" if args.no_graph else ("CUDA graph (WHILE node), programmatic dependent launch"
                                                                if main["graph_pdl"] else "CUDA graph (WHILE node)"),
                   "rhs": "N(0,1), numpy default_rng(seed)",
                   "l2": "256 MiB buffer overwritten between timed solves (outside the per-solve events)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "apply_schedule": s["apply_schedule"]},
        "vcycle_dof_per_s": main["vcycle_dof_per_s"], "iterations": s["iterations"], "latency_ms": s["latency_ms"],
        "setup_s": main["setup_s"],
        "e2e": {"value": world * args.steps / main["e2e_s"], "unit": "solves/s", "h2d_bytes_per_step": 8 * main["ndof"],
                "d2h_bytes_per_step": 8 * main["ndof"]},
        "gpu_launches": s["gpu_launches"],
        "roofline": roof,
        "fma_rate_measured_here": {"fp64_tflops": fp64_tflops, "fp32_tflops": fp32_tflops,
                                   "how": "vk_measure_fma_rate: independent FMA chains on every SM, best of 5"},
        "nested": nested,
        "cpu_baseline": cpu,
        "clocks": clk.summary(),
    }
    print(json.dumps(out), flush=True)


def run_batch(args, config, cfg):
    """--config cfg4batch: the 16-right-hand-side solve as its own line, with the other tensor-core
    engine, the FP32 coarsest-solve variant and plain FP64 one-at-a-time solves for comparison."""
    import torch
    from __graft_entry__ import build
    build()
    import paper_2409_14222_gb300 as vk
    import synthetic_inputs as si
    torch.cuda.set_device(0)
    Nc, L, k, sweeps, rtol, desc = cfg
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", HBM_FALLBACK))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    G64 = vk.Hierarchy(Nc, L, k, options=vk.default_options(sweeps=sweeps))
    n = G64.ndof()
    x1 = torch.zeros(n, dtype=torch.float64, device="cuda")
    B = [torch.from_numpy(si.rhs_normal(n, 5000 + s)).cuda() for s in range(8)]
    for w in range(3):
        G64.solve(B[w], x1, rtol=rtol, history=False)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    t64 = 0.0
    for r in range(3, 8):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(float(r))
        e0.record(stream)
        G64.solve(B[r], x1, rtol=rtol, history=False)
        e1.record(stream)
        torch.cuda.synchronize()
        t64 += e0.elapsed_time(e1) / 1e3
    fp64_value = 5 / t64
    clk = ClockSampler(0)
    with clk:
        rec = batch_record(vk, torch, si, cfg, args, flush, hbm, peaks, peak_kind, G64=G64, fp64_value=fp64_value,
                           steps=args.steps, profile=True)
    other = "mma_sync" if args.engine == "tcgen05" else "tcgen05"
    rec_other = batch_record(vk, torch, si, cfg, args, flush, hbm, peaks, peak_kind, engine=other, steps=3)
    rec_c32 = batch_record(vk, torch, si, cfg, args, flush, hbm, peaks, peak_kind, coarse_fp32=1, steps=3)
    print(json.dumps({
        "metric": METRIC, "value": rec["value"], "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
        "warmup": 3, "ms_per_step": rec["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": f"f64 FGMRES per column; f32 V-cycle with f64 coarsest solve; {args.batch_prec} patch inverses "
                 f"(tensor cores, f32 accumulate)",
        "data": "synthetic",
        "config": {"workload": rec["workload"], "ndof": n, "levels": L, "k": k, "rhs_per_step": 16, "rtol": rtol,
                   "engine": args.engine,
                   "l2": "256 MiB buffer overwritten between timed steps (outside the events)"},
        "iterations": rec["iterations"], "vcycle_dof_per_s": rec["vcycle_dof_per_s"], "latency_ms": rec["latency_ms"],
        "plain_fp64_single_rhs": {"solves_per_s": fp64_value},
        "speedup_vs_plain_fp64": rec["speedup_vs_plain_fp64_one_at_a_time"],
        "rel_error_vs_fp64_solution": rec["rel_error_vs_fp64_solution"],
        "other_engine": {k_: rec_other[k_] for k_ in ("engine", "value", "roofline")},
        "fp32_coarse_solve_variant": {k_: rec_c32[k_] for k_ in ("value", "iterations")},
        "gpu_launches": rec["gpu_launches"], "roofline": dict(rec["roofline"], spmv=rec["spmv"]),
        "clocks": clk.summary(),
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
        x, res = srv.wait(tickets[i], timeout_ms=600000)
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


def serving_record(vk, si, args, n_req, rate_mults, slots, per_key=2, baseline=True, clk=None):
    """The request stream of the serving workload through vk_server in its two modes on the same arrival
    traces: the group engine (every admitted request shares each FGMRES iteration's launches) and one
    CUDA stream per slot; plus plain FP64 one at a time (one slot).  Arrival rates are multiples of the
    group mode's measured capacity; every hierarchy is resident before the timed passes."""
    mix = si.request_mix(n_req, seed=42)
    keys = lambda N, k: (8, int(np.log2(N // 8)) + 1, k)
    reqs = [(keys(N, k), seed) for N, k, seed in mix]
    uniq = sorted(set(k for k, _ in reqs))
    opts = vk.default_options()
    if args.prec == "f32":
        opts.factor_prec = vk.VK_PREC_F32
    elif args.prec == "f64e":
        opts.factor_prec = vk.VK_PREC_F64E

    def warm(srv, n):
        # every hierarchy resident (n instances of each key) before any timed request
        for key in uniq:
            ts = [srv.submit(*key, si.rhs_normal(vk.ndof_of(*key), 7), rtol=1e-8) for _ in range(n)]
            for t in ts:
                _, res = srv.wait(t)
                if res["status"] not in (0, 5):
                    raise RuntimeError(f"warm-up solve of {key} failed: {res}")

    out = {"requests": len(reqs), "distinct_hierarchies": len(uniq), "slots": slots,
           "rhs": "N(0,1) per request, rtol 1e-8", "arrivals": "Poisson, seed 42 + 10 x rate multiple"}
    capacity = None
    passes = [("group", vk.vk.VK_SERVE_GROUP, slots, per_key), ("streams", vk.vk.VK_SERVE_STREAMS, slots, per_key)]
    if baseline:
        passes.append(("one_at_a_time_plain_fp64", vk.vk.VK_SERVE_STREAMS, 1, 1))
    for name, mode, sl, pk in passes:
        o = vk.default_options() if name.startswith("one_at") else opts
        srv = vk.Server(slots=sl, options=o, max_per_key=pk, mode=mode)
        t0 = time.perf_counter()
        warm(srv, pk)
        warm_s = time.perf_counter() - t0
        st0 = srv.stats()
        cap = serve_pass(vk, srv, reqs, [0.0] * len(reqs))
        if capacity is None:
            capacity = cap["solves_per_s"]
        rates = {}
        if clk is not None and name == "group":
            clk.__enter__()
        for mult in rate_mults:
            arr = si.poisson_arrivals(len(reqs), mult * capacity, seed=42 + int(10 * mult))
            rates[f"{mult}x"] = serve_pass(vk, srv, reqs, arr)
        if clk is not None and name == "group":
            clk.__exit__(None, None, None)
        st = srv.stats()
        srv.close()
        rec = {"capacity_solves_per_s": cap["solves_per_s"], "capacity_pass": cap, "rates": rates,
               "warm_s": warm_s, "builds": st["builds"]}
        if mode == vk.vk.VK_SERVE_GROUP:
            steps = st["group_steps"] - st0["group_steps"]
            rec["requests_per_launch_mean"] = (st["member_steps"] - st0["member_steps"]) / max(steps, 1)
        out[name] = rec
    out["capacity_solves_per_s"] = capacity
    return out


def run_serving(args):
    """cfg5: continuous batching of a Poisson request stream (vk_server, C++ runtime)."""
    import torch
    from __graft_entry__ import build
    build()
    import paper_2409_14222_gb300 as vk
    import synthetic_inputs as si
    torch.cuda.set_device(0)
    clk = ClockSampler(0)
    rec = serving_record(vk, si, args, args.requests, (0.5, 1.0, 2.0), args.slots, baseline=not args.no_baseline,
                         clk=clk)
    g = rec["group"]
    one = g["rates"]["1.0x"]
    print(json.dumps({
        "metric": METRIC, "value": rec["capacity_solves_per_s"], "unit": "solves/s", "n_gpus": 1,
        "steps": rec["requests"], "warmup": rec["distinct_hierarchies"] * 2,
        "ms_per_step": 1e3 / rec["capacity_solves_per_s"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"f64": "f64", "f64e": "f64 vectors; FP32-pair patch inverses", "f32": "f64 vectors, f32 patch inverses"}[args.prec],
        "data": "synthetic",
        "config": {"workload": CONFIGS["cfg5"][5], "requests": rec["requests"], "slots": args.slots,
                   "distinct_hierarchies": rec["distinct_hierarchies"], "factor_prec": args.prec,
                   "server_mode": "group (one launch per stage over all admitted requests)"},
        "latency_ms": {"p50": one["p50_ms"], "p99": one["p99_ms"]},
        "serving": rec, "clocks": clk.summary(),
    }), flush=True)


def run_stopping(args):
    """The stopping-criterion study of Sec. 4.4 on the GPU, for Taylor-Hood P_k/P_{k-1} on triangles,
    Q_k/Q_{k-1} on quadrilaterals (the paper's Taylor-Hood study is on quadrilaterals) and
    (BDM_k, dP_{k-1}) on triangles (broken H^1 velocity error): the
    manufactured problem (Eq. model_problem) on 5x5 -> 5*2^l meshes is solved with relative tolerances
    1e-2, 5e-3, 2.5e-3, ... (halved each time, down to 1e-13), and the relative H^1 velocity error and the
    L^2 pressure error (mean removed) are measured on the device.  For each quantity the reported
    tolerance is the largest of the sequence from which on every tighter tolerance gives an error within
    1 % of the error at the tightest one (the discretisation error)."""
    import torch
    from __graft_entry__ import build
    build()
    import paper_2409_14222_gb300 as vk
    torch.cuda.set_device(0)
    taus = []
    t = 1e-2
    while t >= 1e-13:
        taus.append(t)
        t /= 2
    rows = []
    t_start = time.perf_counter()
    cases = [("triangles", k, lev) for k in (2, 3, 4) for lev in (1, 2, 3, 4)]
    cases += [("quadrilaterals", k, lev) for k in (2, 3) for lev in (1, 2, 3, 4)]
    cases += [("bdm", k, lev) for k in (2, 3, 4, 5) for lev in (1, 2, 3, 4)]
    cell_code = {"triangles": vk.vk.VK_CELL_TRIANGLE, "quadrilaterals": vk.vk.VK_CELL_QUAD, "bdm": vk.vk.VK_CELL_BDM}
    for cell, k, lev in cases:
        if True:
            G = vk.Hierarchy(5, lev + 1, k, options=vk.default_options(sweeps=1), cell=cell_code[cell])
            b = torch.from_numpy(G.manufactured_rhs()).cuda()
            x = torch.zeros_like(b)
            errs, iters, ms = [], [], []
            for tau in taus:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                out = G.solve(b, x, rtol=tau, history=False)
                e1.record()
                errs.append(G.errors(x))
                iters.append(out["iterations"])
                ms.append(e0.elapsed_time(e1))
                if not out["converged"]:
                    break
            def needed(q):
                final = errs[-1][q]
                ok = [abs(e[q] - final) <= 1e-2 * final for e in errs]
                i = len(ok) - 1
                while i > 0 and ok[i - 1]:
                    i -= 1
                return i
            iv, ip = needed(0), needed(2)
            rows.append({"cell": cell, "k": k, "levels_refined": lev, "mesh": f"{5 << lev}x{5 << lev}", "ndof": G.ndof(),
                         "velocity": {"tolerance": taus[iv], "iterations": iters[iv], "h1_rel_error": errs[iv][0],
                                      "solve_ms": ms[iv]},
                         "pressure": {"tolerance": taus[ip], "iterations": iters[ip], "l2_error": errs[ip][2],
                                      "solve_ms": ms[ip]},
                         "tightest": {"tolerance": taus[len(errs) - 1], "h1_rel_error": errs[-1][0],
                                      "l2_rel_error": errs[-1][1], "p_l2_error": errs[-1][2]}})
            G.close()
    print(json.dumps({"metric": "stopping tolerance needed to reach discretisation error (Sec. 4.4)",
                      "config": {"workload": "Taylor-Hood P_k/P_{k-1} on triangles, Q_k/Q_{k-1} on quadrilaterals and "
                                             "(BDM_k, dP_{k-1}) on triangles, manufactured solution, "
                                             "5x5 coarsest grid, V(1,1), FGMRES", "tolerances": "1e-2 halved to 1e-13",
                                 "criterion": "every tighter tolerance within 1 % of the tightest one's error"},
                      "rows": rows, "wall_s": time.perf_counter() - t_start}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="vk", choices=["vk", "reference"])
    ap.add_argument("--config", default=DEFAULT_CONFIG, choices=sorted(CONFIGS))
    ap.add_argument("--prec", default="f64", choices=["f64", "f64e", "f32"],
                    help="patch inverses: FP64, FP32-pair emulated FP64, or FP32")
    ap.add_argument("--no-graph", action="store_true",
                    help="host-driven FGMRES loop instead of the whole-solve CUDA graph (for kernel profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--pdl", action="store_true", help="capture the solve graph with programmatic dependent launch")
    ap.add_argument("--no-nested", action="store_true", help="cfg4: skip the nested records")
    ap.add_argument("--no-serving", action="store_true", help="cfg4: skip the nested serving record")
    ap.add_argument("--no-bdm", action="store_true", help="cfg4: skip the nested BDM records")
    ap.add_argument("--serve-requests", type=int, default=100, help="cfg4: requests of the nested serving record")
    ap.add_argument("--requests", type=int, default=1000, help="cfg5: requests in the 1x stream")
    ap.add_argument("--slots", type=int, default=4, help="cfg5: concurrent solves")
    ap.add_argument("--no-baseline", action="store_true", help="cfg5: skip the one-at-a-time FP64 pass")
    ap.add_argument("--batch-prec", default="bf16", choices=["bf16", "fp16"], help="16-bit inverse format")
    ap.add_argument("--spmv-warps", type=int, default=0, help="SELL threads-per-row rule (warps per SM); 0 = default")
    ap.add_argument("--levels", type=int, default=0, help="override the level count (profiling variants only)")
    ap.add_argument("--rtol", type=float, default=0.0, help="override the tolerance (profiling variants only)")
    ap.add_argument("--batch-maxit", type=int, default=60, help="FGMRES basis size per right-hand side (batch)")
    ap.add_argument("--engine", default="tcgen05", choices=["tcgen05", "mma_sync"],
                    help="tensor-core instruction family of the batched patch solves")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "vk":
        ap.error("--warmup must be >= 3")
    config = args.config
    cfg = CONFIGS[config]
    if args.levels or args.rtol:
        # a smaller or looser variant of a workload, for profiler captures (never a bench line)
        Nc, L, k, sweeps, rtol, desc = cfg
        L = args.levels or L
        rtol = args.rtol or rtol
        cfg = (Nc, L, k, sweeps, rtol, f"{desc.split(',')[0]}, {Nc}x{Nc} -> {Nc << (L - 1)}x{Nc << (L - 1)} "
                                         f"({L} levels), rtol {rtol:g} [profiling variant]")
        config = config + "-variant"
    if args.impl == "reference":
        run_reference(args, config, cfg)
    elif args.config == "cfg5":
        run_serving(args)
    elif args.config == "stopping":
        run_stopping(args)
    elif args.config == "cfg4batch":
        run_batch(args, config, cfg)
    else:
        run_vk(args, config, cfg)


if __name__ == "__main__":
    main()
