"""CPU tests of bench.py's multi-process path (replicas only: the path does not shard, so the only
collectives are the barrier and the max over ranks of the timed region), with the gloo backend and
two ranks on 127.0.0.1."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        out[rank] = bench.max_over_ranks(1.5 + rank, world)
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_barrier_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        assert dict(out) == {0: 2.5, 1: 2.5}


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    port = _free_port()
    env = dict(os.environ, VK_BENCH_GLOO="1", OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--config", "cfg1", "--steps", "1", "--warmup", "1", "--gpus", "2"]
    res = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["unit"] == "solves/s"
    assert rec["value"] > 0 and rec["e2e"]["h2d_bytes_per_step"] == 0
    assert rec["cpu_baseline"]["kind"] == "oracle"


def test_reference_arm_prints_the_time_it_measured():
    # the printed ms_per_step x steps is the measured time of the samples; the extrapolation to one solve
    # of the 512 x 512 workload is a separate, stated factor
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--config", "cfg4", "--steps", "2", "--warmup", "1"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-2000:]
    rec = json.loads([ln for ln in res.stdout.splitlines() if ln.startswith("{")][-1])
    ex = rec["extrapolation"]
    assert abs(rec["ms_per_step"] * rec["steps"] - 1e3 * ex["timed_seconds"]) <= 1e-6 * 1e3 * ex["timed_seconds"]
    assert abs(rec["value"] - rec["steps"] / (ex["timed_seconds"] * ex["scale"])) <= 1e-9 * rec["value"]
    assert ex["target_ndof"] == 2364419 and rec["config"]["ndof"] == 2364419
    assert "512x512" in rec["config"]["workload"]
