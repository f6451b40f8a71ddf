"""Host side of bench.py: the cross-rank aggregation on two gloo ranks, and the reference arm (the
FP64 oracle timed on host cores) run through its real launch paths -- single process and under
torchrun with two ranks, where rank 0 alone prints and the other rank exits 0 without work."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank                     # rank 1 is the slow one
        slowest = bench.max_over_ranks(local_ms, world)
        bench.barrier(world)
        out[rank] = (slowest, bench.weak_scaling_glups(1000, 4, world, slowest))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_on_two_gloo_ranks():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]                              # every rank sees the same job time
    slowest, glups = res[0]
    assert slowest == 15.0
    assert glups == pytest.approx(1000 * 4 * 2 / 0.015 / 1e9)


def test_weak_scaling_formula_single_rank():
    assert bench.weak_scaling_glups(12_800_000, 100, 1, 40.0) == pytest.approx(32.0)


def _json_lines(text):
    return [json.loads(l) for l in text.splitlines() if l.startswith("{")]


def test_reference_arm_single_process():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "cube",
                        "--steps", "3", "--warmup", "1"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["unit"] == "GLUPS" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["steps"] == 3 and d["warmup"] == 1 and d["higher_is_better"] is True


def test_reference_arm_under_torchrun_two_gloo_ranks():
    env = dict(os.environ, LBM_BENCH_BACKEND="gloo")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           "bench.py", "--gpus", "2", "--impl", "reference", "--workload", "cube",
           "--steps", "2", "--warmup", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1                               # rank 0 alone prints
    assert lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2
