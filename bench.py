#!/usr/bin/env python3
"""LBM-LES throughput on one B300: GLUPS and fraction of the HBM roofline.

Workload (default): the synthetic 5 m city, 400 x 400 x 80 = 12.8M cells (2 km x 2 km x 400 m),
Poisson-disk box buildings to a plan-area fraction of 0.35, power-law inflow (alpha 0.25,
u_ref 0.06 at z = 60) from a seeded direction, tau = 0.505, Smagorinsky C = 0.16, FP32 populations.
One benchmark step = one fused D3Q19 stream-collide time step over the whole lattice (the whole
hot path).  The state (1.95 GB in FP32) is 15x the 126 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--store f32|f16s|bf16s]
                    [--workload city400|city256|city1000|cube] [--impl ours|reference]

Prints ONE JSON line on rank 0.  Multi-GPU (torchrun): every rank runs an independent replica of
the workload (the single-domain path has no exchange step here), value = all ranks' cell updates
over the slowest rank's time, "scaling": "weak".
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "city400": dict(nx=400, ny=400, nz=80, seed=1),
    "city256": dict(nx=256, ny=256, nz=64, seed=1),
    "city1000": dict(nx=1000, ny=1000, nz=160, seed=1),
    "cube": None,
}
METRIC = "LBM-LES GLUPS & % HBM roofline, FP32 vs 16-bit storage; adjoint/forward time ratio"
STORE_BYTES = {"f32": 4, "f16s": 2, "bf16s": 2}
DTYPE_NAME = {"f32": "f32", "f16s": "f16-storage/f32-math", "bf16s": "bf16-storage/f32-math"}
SOURCES = ["paper_2607_04516_b300/csrc/lbm_device.cuh", "paper_2607_04516_b300/csrc/lbm_cell.cuh",
           "paper_2607_04516_b300/csrc/lbm_kernels.cu", "paper_2607_04516_b300/csrc/lbm_step.cuh",
           "paper_2607_04516_b300/csrc/lbm_step_kern.cu"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=19000)
    ap.add_argument("--warmup", type=int, default=1000)
    ap.add_argument("--store", default="f32", choices=list(STORE_BYTES))
    ap.add_argument("--workload", default="city400", choices=list(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variants", default="f16s,bf16s,stg,stg_s10,zones,physics,physics_f16s,adjoint,ensemble,ensemble_small,precision",
                    help="extra storage kinds timed after the main measurement ('' = none)")
    ap.add_argument("--e2e-steps", type=int, default=1000)
    ap.add_argument("--adjoint-steps", type=int, default=2000,
                    help="steps of the assimilation run in the adjoint leg (2000 = the full workload)")
    ap.add_argument("--adjoint-recovery", type=int, default=20, help="descent iterations in the adjoint leg")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers
def make_case(workload):
    from paper_2607_04516_b300 import synth
    if workload == "cube":
        return synth.cube_case()
    w = WORKLOADS[workload]
    return synth.city_case(nx=w["nx"], ny=w["ny"], nz=w["nz"], seed=w["seed"])


def source_hash() -> str:
    h = hashlib.sha256()
    for p in SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def recorded_traffic(kernel: str, workload: str, store: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this source."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}_{store}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    s = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    if not m or not s or s.group(1) != source_hash():
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def rows(self) -> int:
        """Samples written so far."""
        self.f.flush()
        try:
            with open(self.f.name) as f:
                return sum(1 for r in f if r.strip())
        except OSError:
            return 0

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, smax, reasons = [], [], set()
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[0]))
                smax.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for k, name in enumerate(names):
                if len(r) > 4 + k and r[4 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("LBM_BENCH_BACKEND") != "gloo" else "gloo")
    return rank, world


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_glups(cells: int, steps: int, world: int, slowest_ms: float) -> float:
    """Whole-job throughput of ``world`` independent replicas: every rank updated ``cells`` cells
    ``steps`` times; the job took as long as its slowest rank."""
    return cells * steps * world / (slowest_ms / 1e3) / 1e9


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------------------- our arm
def layer_kernel_runs(case, store: str) -> bool:
    """A neighbour step of this domain launches the ground/top layer kernel besides the main kernel:
    both z faces no-slip or free-slip (on a lattice of at least 3 x 3 x 2), and the two-cell path
    (16-bit storage, or FP32 from 2^21 cells)."""
    nz, ny, nx = case.solid.shape
    zk = ("noslip", "freeslip")
    return (case.faces[4] in zk and case.faces[5] in zk and nx >= 3 and ny >= 3 and nz >= 2
            and (store != "f32" or nx * ny * nz >= 2 ** 21))


def time_steps(dom, K: int, W: int, world: int, clock_id: str | None):
    """W untimed steps, then K steps with a CUDA event before/after every launch on the domain's
    stream (the library enqueues on the stream the domain was created with)."""
    import torch
    dom.step(W)
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    sampler = ClockSampler(clock_id) if clock_id else None
    # the clock record starts with at least 0.6 s (and 3 samples) of untimed steps under load right
    # before the timed region, so that a short timed region still carries one (every rank runs them)
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < 0.6 or (sampler is not None and sampler.p is not None
                                             and sampler.rows() < 3 and time.perf_counter() - t0 < 10.0):
        dom.step(64)
        torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    parity0 = dom.steps_done % 2
    evs[0].record(dom.stream)
    for k in range(K):
        dom.step(1)
        evs[k + 1].record(dom.stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    clocks = sampler.stop() if sampler else None
    if clocks is not None:
        clocks["window"] = "from 0.6 s of untimed steps right before the timed region to its end"
    barrier(world)
    total_ms = evs[0].elapsed_time(evs[K])
    per = [evs[k].elapsed_time(evs[k + 1]) for k in range(K)]
    # launch k is the neighbour kernel when (parity0 + k) is even
    nb = [t for k, t in enumerate(per) if (parity0 + k) % 2 == 0]
    lc = [t for k, t in enumerate(per) if (parity0 + k) % 2 == 1]
    return total_ms, nb, lc, wall, clocks


def e2e_glups(dom, case, steps: int, world: int):
    """Public-API loop with host buffers: per step the inflow profile goes host -> device
    (lbm_set_inflow_profile, level speeds from pinned host memory), one lbm_step, and 8
    virtual-lidar columns x 10 heights come back device -> pinned host (lbm_sample_columns + an
    asynchronous copy into that step's row of a pinned host array).  The host does not wait per
    step (a serving loop keeps the GPU busy).  The read-back runs on a second stream, from a ring of
    four device sample buffers, so it overlaps the next step; a buffer is sampled into again only
    after its copy has been ordered (stream waits on events, no host wait).  The timed region ends
    when every step's copy has landed."""
    import numpy as np
    import torch
    nz, ny, nx = case.shape
    speed = torch.tensor(case.speed, dtype=torch.float32).pin_memory()
    rng = np.random.default_rng(7)
    fluid_cols = [(int(x), int(y)) for x, y in zip(rng.integers(16, nx - 16, 64), rng.integers(16, ny - 16, 64))
                  if not case.solid[0, y, x]][:8]
    ij = torch.tensor(fluid_cols, dtype=torch.int32, device=dom.device)
    kk = torch.tensor([min(nz - 1, 4 * (i + 1)) for i in range(10)], dtype=torch.int32, device=dom.device)
    ring = [torch.empty((len(fluid_cols), 10, 4), dtype=torch.float32, device=dom.device) for _ in range(4)]
    out_d = ring[0]
    out_h = torch.empty((steps,) + tuple(out_d.shape), dtype=torch.float32).pin_memory()
    from paper_2607_04516_b300 import lbm
    speed_np = speed.numpy()
    copy_stream = torch.cuda.Stream(device=dom.device)
    sampled = [torch.cuda.Event() for _ in ring]
    copied = [torch.cuda.Event() for _ in ring]

    def one_step(k):
        b = k % len(ring)
        dom.set_inflow_profile(speed_np, case.theta)
        dom.step(1)
        if k >= len(ring):
            dom.stream.wait_event(copied[b])           # its previous copy has read the buffer
        lbm.lbm_sample_columns(dom.dom, ij, kk, ring[b])
        sampled[b].record(dom.stream)
        copy_stream.wait_event(sampled[b])
        with torch.cuda.stream(copy_stream):
            out_h[k].copy_(ring[b], non_blocking=True)
        copied[b].record(copy_stream)

    with torch.cuda.stream(dom.stream):
        for k in range(min(10, steps)):
            one_step(k)
        dom.stream.synchronize()
        copy_stream.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for k in range(steps):
            one_step(k)
        dom.stream.synchronize()
        copy_stream.synchronize()
        dt = time.perf_counter() - t0
    out_d = ring[(steps - 1) % len(ring)]
    if not np.isfinite(out_h[-1].numpy()).all():
        raise RuntimeError("e2e: non-finite lidar samples")
    dt = max_over_ranks(dt, world)
    return (case.solid.size * steps * world / dt / 1e9, 4 * len(speed_np), out_d.numel() * 4,
            dt * 1e3 / steps)


def adjoint_leg(world: int, nsteps: int = 2000, iters: int = 20):
    """Boundary assimilation (128 x 128 x 48 city, 24 level speeds + direction, 8 lidar columns x
    10 heights averaged over the last 500 of 2000 steps, checkpoints every 100 steps): time of the
    misfit gradient (forward run + reverse sweep, lbm_lidar_misfit_grad) against 2000 plain FP32
    steps of the same lattice (lbm_step), both with CUDA events on the domain's stream."""
    import numpy as np
    import torch
    from paper_2607_04516_b300 import lbm, synth
    a = synth.assimilation_case()
    if nsteps != a.nsteps:   # shortened run (profiling): same lattice, fewer steps
        a.nsteps, a.n_avg, a.checkpoint_every = nsteps, max(1, nsteps // 4), max(1, min(100, nsteps // 4))
    c = a.case
    dom = lbm.Domain(c.solid, c.faces, c.tau, c.cs, "f32")
    prob = lbm.LidarProblem(dom, a.cols, a.heights, np.zeros((len(a.cols), len(a.heights), 2), np.float32),
                            a.nsteps, a.n_avg, a.checkpoint_every)
    _, mean = prob.misfit(a.speed_true.astype(np.float32), a.theta_true, target=False)
    prob.target = mean[..., :2].float().contiguous()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    guess = a.speed_guess.astype(np.float32)
    prob.misfit_grad(guess, a.theta_guess)                   # warm-up (allocates the workspace)
    dom.set_inflow_profile(guess, a.theta_guess)
    dom.init_fields()
    dom.step(20)
    torch.cuda.synchronize()
    barrier(world)
    ev[0].record(dom.stream)
    dom.step(a.nsteps)
    ev[1].record(dom.stream)
    ev[2].record(dom.stream)
    J0, _ = prob.misfit(guess, a.theta_guess)
    ev[3].record(dom.stream)
    ev[4].record(dom.stream)
    J, g, _ = prob.misfit_grad(guess, a.theta_guess)
    ev[5].record(dom.stream)
    torch.cuda.synchronize()
    fwd, mis, grd = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3]), ev[4].elapsed_time(ev[5])
    fwd, grd = max_over_ranks(fwd, world), max_over_ranks(grd, world)
    # inflow recovery: 20 gradient evaluations, steps along -g / max|g| with a backtracking length
    p0 = np.concatenate([a.speed_guess, [a.theta_guess]])
    p, Jp, step = p0.copy(), float(J), 0.02
    for _ in range(iters):
        Jc, gc, _ = prob.misfit_grad(p[:-1], p[-1])
        Jc, gc = float(Jc), gc.cpu().numpy()
        while step > 1e-6:
            q = p - step * gc / np.abs(gc).max()
            Jq, _ = prob.misfit(q[:-1], q[-1])
            if float(Jq) < Jc:
                p, Jp = q, float(Jq)
                step *= 1.5
                break
            step *= 0.5
    recovery = {"iterations": iters, "J0": float(J), "J": Jp,
                "speed_err0": float(np.abs(p0[:-1] - a.speed_true).max()),
                "speed_err": float(np.abs(p[:-1] - a.speed_true).max()),
                "theta_err0": float(p0[-1] - a.theta_true), "theta_err": float(p[-1] - a.theta_true)}
    nz, ny, nx = c.shape
    out = {"workload": f"assim128: {nx}x{ny}x{nz} synthetic city (seed 4), {a.L} level speeds + direction, "
                       f"{len(a.cols)} lidar columns x {len(a.heights)} heights, mean of the last {a.n_avg} "
                       f"of {a.nsteps} steps, checkpoints every {a.checkpoint_every}",
           "forward_ms": fwd, "misfit_ms": mis, "gradient_ms": grd, "ratio": grd / fwd,
           "J": float(J), "grad_norm": float(torch.linalg.vector_norm(g)), "recovery": recovery}
    del prob, dom
    torch.cuda.empty_cache()
    return out


def ensemble_leg(world: int, steps: int = 40, small: bool = False):
    """Batched ensemble, FP32.  Default workload: a wind rose of 16 inflow directions x 2 speeds on a
    256x256x64 city plus 8 domains of uneven size (96x96x32 .. 320x192x64).  small: 12 directions x
    2 speeds on a 96x96x32 city plus the same 8 uneven domains, where each member's own launch is
    short and launch and tail overhead matter.  Aggregate GLUPS (all cells of all members per
    second) of one single-domain launch per member and step, against the batched launch in the
    autotuned shape, stepped directly and replayed from a CUDA graph; CUDA events on the batch's
    stream."""
    import numpy as np
    import torch
    from paper_2607_04516_b300 import lbm, synth
    if small:
        cases = synth.ensemble_cases(nx=96, ny=96, nz=32, n_dir=12) + synth.uneven_cases()
        label = "12 directions x 2 speeds on a 96x96x32 city (seed 3) + 8 uneven domains 96x96x32 .. 320x192x64"
    else:
        cases = synth.ensemble_cases() + synth.uneven_cases()
        label = "16 directions x 2 speeds on a 256x256x64 city (seed 3) + 8 uneven domains 96x96x32 .. 320x192x64"
    cells = int(sum(c.solid.size for c in cases))
    stream = torch.cuda.Stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        torch.cuda.synchronize()
        ev[0].record(stream)
        fn()
        ev[1].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1])

    with torch.cuda.stream(stream):
        doms = []
        for c in cases:
            d = lbm.Domain(c.solid, c.faces, c.tau, c.cs, "f32", stream=stream)
            d.set_inflow_profile(c.speed.astype(np.float32), c.theta)
            d.init_fields()
            doms.append(d)
        b = lbm.Batch(doms, stream=stream)
        b.shape = 4                        # one single-domain launch per member
        b.step(2)
        seq = timed(lambda: b.step(steps))
        choice, tune_ms = b.autotune(trial_steps=10)
        bat = timed(lambda: b.step(steps))
        b.capture(steps)
        b.launch()
        gra = timed(b.launch)
    barrier(world)
    seq, bat, gra = (max_over_ranks(x, world) for x in (seq, bat, gra))
    g = lambda ms: cells * steps * world / (ms / 1e3) / 1e9
    out = {"workload": f"{label}; {len(cases)} members, {cells} cells, FP32",
           "steps": steps, "sequential_glups": g(seq), "batched_glups": g(bat), "graph_glups": g(gra),
           "graph_vs_sequential": seq / gra, "shape": lbm.BATCH_SHAPES[choice],
           "autotune_ms_per_step": {k: (v if v > 0 else None) for k, v in zip(lbm.BATCH_SHAPES, tune_ms)}}
    del b, doms
    torch.cuda.empty_cache()
    return out


def precision_leg(world: int):
    """Precision sweep: the same synthetic city (seed 1) at 256x256x64, 400x400x80 and
    1000x1000x160 with populations stored as FP32, shifted FP16 and BF16 (FP32 arithmetic).  Per
    size and 16-bit kind: GLUPS over 200 steps; relative L2 of u and of rho - 1 against the FP32
    path after 200 steps (non-solid cells); relative error of the time-mean horizontal wind profile
    (plane mean of |u_h| per height, every 10th state of steps 1..1000).  Plus the relative L2 of u
    against the FP64 oracle on the 64x64x32 cube after 200 steps, per kind."""
    import numpy as np
    import torch
    from paper_2607_04516_b300 import lbm, synth
    out = {}
    for (nx, ny, nz) in ((256, 256, 64), (400, 400, 80), (1000, 1000, 160)):
        case = synth.city_case(nx=nx, ny=ny, nz=nz, seed=1)
        fluid = torch.as_tensor(case.solid == 0, device="cuda")
        res, prof = {}, {}
        for store in ("f32", "f16s", "bf16s"):
            d = lbm.Domain(case.solid, case.faces, case.tau, case.cs, store)
            d.set_inflow_profile(case.speed.astype(np.float32), case.theta)
            d.init_fields(None, case.u0.astype(np.float32))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(d.stream)
            d.step(200)
            e1.record(d.stream)
            rho, u = d.macroscopic()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            res[store] = (rho, u, case.solid.size * 200 / (ms / 1e3) / 1e9)
            acc = torch.zeros(nz, dtype=torch.float64, device="cuda")
            for k in range(80):           # states 210 .. 1000, every 10th
                d.step(10)
                _, uu = d.macroscopic()
                sp = torch.sqrt(uu[..., 0].double() ** 2 + uu[..., 1].double() ** 2)
                acc += (sp * fluid).sum(dim=(1, 2)) / fluid.sum(dim=(1, 2)).clamp(min=1)
            prof[store] = acc / 80
            del d
            torch.cuda.empty_cache()
        r32, u32, g32 = res["f32"]
        row = {"cells": nx * ny * nz, "f32_glups": g32}
        for store in ("f16s", "bf16s"):
            r, u, g = res[store]
            du = torch.linalg.vector_norm((u - u32)[fluid].double()) / torch.linalg.vector_norm(u32[fluid].double())
            dr = torch.linalg.vector_norm((r - r32)[fluid].double()) / torch.linalg.vector_norm((r32 - 1)[fluid].double())
            dp = torch.linalg.vector_norm(prof[store] - prof["f32"]) / torch.linalg.vector_norm(prof["f32"])
            row[store] = {"glups": g, "vs_f32": g / g32, "u_rel_l2_vs_f32_200": float(du),
                          "rho_rel_l2_vs_f32_200": float(dr), "profile_rel_vs_f32_1000": float(dp)}
        out[f"{nx}x{ny}x{nz}"] = row
        del res
        torch.cuda.empty_cache()
    # against the FP64 oracle, 64x64x32 cube, 200 steps
    from oracle import oracle as orc
    cube = synth.cube_case()
    kind = orc.classify(cube.solid, cube.faces)
    ub = orc.expand_profile(cube.speed.astype(np.float32).astype(np.float64), cube.shape[0], 0.0)
    F = orc.init(kind, ub, None, cube.u0.astype(np.float32).astype(np.float64))
    F = orc.run(F, 200, kind, cube.faces, ub, cube.tau, cube.cs)
    _, ur = orc.macros(F, kind, ub)
    fl = kind == orc.FLUID
    vs64 = {}
    for store in ("f32", "f16s", "bf16s"):
        d = lbm.Domain(cube.solid, cube.faces, cube.tau, cube.cs, store)
        d.set_inflow_profile(cube.speed.astype(np.float32), cube.theta)
        d.init_fields(None, cube.u0.astype(np.float32))
        d.step(200)
        _, u = d.macroscopic()
        u = u.cpu().numpy().astype(np.float64)
        vs64[store] = float(np.linalg.norm((u - ur)[fl]) / np.linalg.norm(ur[fl]))
    out["cube64x64x32_u_rel_l2_vs_fp64_200"] = vs64
    # the stated bound on that error: 1e-5 for FP32 storage, 1e-3 for 16-bit storage
    bound = {"f32": 1e-5, "f16s": 1e-3, "bf16s": 1e-3}
    out["meets_u_bound_vs_fp64"] = {s: {"bound": bound[s], "meets": vs64[s] <= bound[s]} for s in vs64}
    return out


def cpu_baseline(case, seconds: float):
    """The FP64 oracle as it stands, on all host cores, over whole-lattice steps of this workload."""
    import numpy as np
    from oracle import oracle as orc
    kind = orc.classify(case.solid, case.faces)
    ub = orc.expand_profile(case.speed.astype(np.float32).astype(np.float64), case.shape[0],
                            float(np.float32(case.theta)))
    F = orc.init(kind, ub, None, None if case.u0 is None else case.u0)
    out = np.empty_like(F)
    steps = 0
    t0 = time.perf_counter()
    while True:
        orc.step(F, kind, case.faces, ub, case.tau, case.cs, out=out)
        F, out = out, F
        steps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    cells = case.solid.size
    return {"value": cells * steps / dt / 1e9, "unit": "GLUPS", "cores": orc.num_threads(),
            "kind": "oracle",
            "sample": f"{steps} full time steps of the {case.shape[2]}x{case.shape[1]}x{case.shape[0]} "
                      f"workload ({cells} cells) in {dt:.1f} s, FP64, OpenMP over z-planes"}


def run_ours(args, rank, world):
    import numpy as np
    import torch
    from paper_2607_04516_b300 import build as lbuild
    from paper_2607_04516_b300 import lbm

    if rank == 0:
        lbuild.build()
    barrier(world)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    case = make_case(args.workload)
    nz, ny, nx = case.shape
    N = nx * ny * nz
    nonsolid = int(N - case.solid.sum())
    props = torch.cuda.get_device_properties(local)
    clock_id = getattr(props, "uuid", None)
    clock_id = f"GPU-{clock_id}" if clock_id is not None and not str(clock_id).startswith("GPU-") else (
        str(clock_id) if clock_id is not None else str(local))

    def build_domain(store, **kw):
        dom = lbm.Domain(case.solid, case.faces, case.tau, case.cs, store, **kw)
        dom.set_inflow_profile(case.speed.astype(np.float32), case.theta)
        dom.init_fields(None, None if case.u0 is None else case.u0.astype(np.float32))
        return dom

    dom = build_domain(args.store)
    total_ms, nb, lc, wall, clocks = time_steps(dom, args.steps, args.warmup, world,
                                                clock_id if rank == 0 else None)
    total_ms = max_over_ranks(total_ms, world)
    diag = dom.diagnostics()
    value = weak_scaling_glups(N, args.steps, world, total_ms)

    sb = STORE_BYTES[args.store]
    alg_bytes = nonsolid * 2 * 19 * sb + N            # read + write every population, + flags
    peak, peak_src = measured_peaks()
    kernels = {"k_step_neighbor": nb, "k_step_local": lc}
    stats = {}
    for name, ts in kernels.items():
        if ts:
            avg = sum(ts) / len(ts)
            stats[name] = {"launches": len(ts), "avg_ms": avg, "total_ms": sum(ts),
                           "achieved_gbs": alg_bytes / (avg / 1e3) / 1e9}
    dominant = max(stats, key=lambda k: stats[k]["total_ms"])
    ach = stats[dominant]["achieved_gbs"]
    traffic = recorded_traffic(dominant, args.workload, args.store)

    e2e_val, h2d, d2h, e2e_ms = e2e_glups(dom, case, args.e2e_steps, world)
    del dom
    torch.cuda.empty_cache()

    variants = {}
    for st in [v for v in args.variants.split(",") if v and v != args.store]:
        if st == "adjoint":
            variants[st] = adjoint_leg(world, args.adjoint_steps, args.adjoint_recovery)
            continue
        if st == "ensemble":
            variants[st] = ensemble_leg(world)
            continue
        if st == "ensemble_small":
            variants[st] = ensemble_leg(world, small=True)
            continue
        if st == "precision":
            variants[st] = precision_leg(world)
            continue
        if st == "zones":
            # FP32 with the boundary relaxation zones (Sec. 3): a top sponge 10 cells deep (rate 0.05
            # at the top) and buffers 16 cells wide next to the open lateral faces (0.02), plus flux
            # balancing; the zones take the general (forced) step kernels
            d2 = build_domain("f32", sponge=(10, 0.05), buffer=(16, 0.02), flux_balance=True)
            K2 = max(200, args.steps // 4)
            t_ms, _, _, _, _ = time_steps(d2, K2, min(args.warmup, 200), world, None)
            t_ms = max_over_ranks(t_ms, world)
            g2 = weak_scaling_glups(N, K2, world, t_ms)
            variants[st] = {"glups": g2, "vs_f32": g2 / value if args.store == "f32" else None,
                            "ms_per_step": t_ms / K2, "sponge": [10, 0.05], "buffer": [16, 0.02],
                            "flux_balance": list(d2.flux_balance_info())}
            del d2
            torch.cuda.empty_cache()
            continue
        if st in ("physics", "physics_f16s"):
            # every per-step physics term of the solver at once: Coriolis at the city's latitude
            # (23.1 deg N, 0.01 s steps, App. E), the relaxation zones and flux balancing as in the
            # zones leg (Sec. 3), and the synthetic von Karman inflow every 10 steps (App. F)
            from paper_2607_04516_b300 import synth
            store = "f16s" if st == "physics_f16s" else "f32"
            omega = lbm.lbm_coriolis_omega(23.1, 0.01)
            d2 = build_domain(store, sponge=(10, 0.05), buffer=(16, 0.02), flux_balance=True,
                              coriolis=tuple(omega))
            d2.configure_stg(synth.stg_uniforms(64, seed=11), n_modes=64, length=20.0, intensity=0.1,
                             stride=10, interpolate=True)
            K2 = max(200, args.steps // 4)
            t_ms, _, _, _, _ = time_steps(d2, K2, min(args.warmup, 200), world, None)
            t_ms = max_over_ranks(t_ms, world)
            g2 = weak_scaling_glups(N, K2, world, t_ms)
            variants[st] = {"glups": g2, "vs_f32": g2 / value if args.store == "f32" else None,
                            "ms_per_step": t_ms / K2, "store": store,
                            "coriolis": [float(v) for v in omega], "sponge": [10, 0.05],
                            "buffer": [16, 0.02], "flux_balance": True, "stg": {"modes": 64, "stride": 10},
                            "nonfinite_after": int(d2.diagnostics()["nonfinite"])}
            del d2
            torch.cuda.empty_cache()
            continue
        if st in ("stg", "stg_s10"):
            # FP32 with the synthetic von Karman inflow (App. F) on the inflow faces: 64 modes,
            # evaluated every step, or every 10 steps with linear interpolation in between
            from paper_2607_04516_b300 import synth
            stride = 10 if st == "stg_s10" else 1
            d2 = build_domain("f32")
            d2.configure_stg(synth.stg_uniforms(64, seed=11), n_modes=64, length=20.0, intensity=0.1,
                             stride=stride, interpolate=True)
            K2 = max(200, args.steps // 4)
            t_ms, _, _, _, _ = time_steps(d2, K2, min(args.warmup, 200), world, None)
            t_ms = max_over_ranks(t_ms, world)
            g2 = weak_scaling_glups(N, K2, world, t_ms)
            variants[st] = {"glups": g2, "vs_f32": g2 / value if args.store == "f32" else None,
                            "ms_per_step": t_ms / K2, "modes": 64, "stride": stride,
                            "launches_per_step": 1 + (0.5 if layer_kernel_runs(case, "f32") else 0.0) + 1 / stride}
            del d2
            torch.cuda.empty_cache()
            continue
        d2 = build_domain(st)
        t_ms, nb2, lc2, _, _ = time_steps(d2, max(200, args.steps // 4), min(args.warmup, 200), world, None)
        t_ms = max_over_ranks(t_ms, world)
        K2 = max(200, args.steps // 4)
        g2 = weak_scaling_glups(N, K2, world, t_ms)
        ab2 = nonsolid * 2 * 19 * STORE_BYTES[st] + N
        avg2 = max(sum(nb2) / len(nb2), sum(lc2) / len(lc2))
        variants[st] = {"glups": g2, "vs_f32": g2 / value if args.store == "f32" else None,
                        "frac_hbm_dominant": ab2 / (avg2 / 1e3) / 1e9 / peak}
        del d2
        torch.cuda.empty_cache()

    if rank != 0:
        return None
    cpu = None if args.no_cpu_baseline else cpu_baseline(case, args.cpu_seconds)
    line = {
        "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME[args.store], "data": "synthetic",
        "config": {"workload": f"{args.workload}: {nx}x{ny}x{nz} synthetic city, 5 m cells" if args.workload != "cube"
                   else "cube 64x64x32", "cells": N, "fluid_cells": nonsolid,
                   "tau": case.tau, "cs_smag": case.cs, "store": args.store, "faces": list(case.faces),
                   "inflow_dir_deg": math.degrees(case.theta),
                   "parallelism": "replicas" if world > 1 else "single-gpu",
                   "l2": "state larger than the 126 MB L2 (no flush between steps)"},
        "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                     "frac": ach / peak, "traffic": traffic, "kernel": dominant,
                     "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "kernels": stats},
        "e2e": {"value": e2e_val, "unit": "GLUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        # one launch per step, and the layer kernel's launch in every neighbour step where it runs
        "gpu_launches": args.steps + (len(nb) if layer_kernel_runs(case, args.store) else 0),
        "clocks": clocks,
        "cpu_baseline": cpu,
        "variants": variants,
        "diagnostics_after": {k: (float(v) if not isinstance(v, int) else v) for k, v in diag.items()},
        "wall_s_timed": wall,
    }
    return line


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The FP64 oracle as it stands on the host cores, same workload and metric; each benchmark
    step is one oracle time step restricted to a slab of z-planes sized so the whole run ends in
    about two minutes."""
    if rank != 0:
        return None
    import numpy as np
    from oracle import oracle as orc
    case = make_case(args.workload)
    nz, ny, nx = case.shape
    kind = orc.classify(case.solid, case.faces)
    ub = orc.expand_profile(case.speed.astype(np.float32).astype(np.float64), nz, float(np.float32(case.theta)))
    F = orc.init(kind, ub, None, case.u0)
    out = np.empty_like(F)
    t0 = time.perf_counter()
    orc.step(F, kind, case.faces, ub, case.tau, case.cs, out=out, z0=0, z1=1)
    plane_s = max(time.perf_counter() - t0, 1e-4)
    budget = 120.0
    planes = int(max(1, min(nz, budget / ((args.steps + args.warmup) * plane_s))))
    z = 0
    for _ in range(args.warmup):
        orc.step(F, kind, case.faces, ub, case.tau, case.cs, out=out, z0=z, z1=z + planes)
        z = (z + planes) % max(1, nz - planes + 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orc.step(F, kind, case.faces, ub, case.tau, case.cs, out=out, z0=z, z1=z + planes)
        z = (z + planes) % max(1, nz - planes + 1)
    dt = time.perf_counter() - t0
    cells = planes * nx * ny * args.steps
    val = cells / dt / 1e9
    sample = (f"each step = one FP64 oracle time step over {planes} z-plane(s) "
              f"({planes * nx * ny} cells) of the {nx}x{ny}x{nz} workload")
    return {"impl": "reference", "metric": METRIC, "value": val, "unit": "GLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {nx}x{ny}x{nz} synthetic city, 5 m cells",
                       "cells": nx * ny * nz, "store": "f64 (oracle)"},
            "cpu_baseline": {"value": val, "unit": "GLUPS", "cores": orc.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world = dist_init()
    line = run_reference(args, rank, world) if args.impl == "reference" else run_ours(args, rank, world)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
