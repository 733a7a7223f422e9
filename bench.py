"""Benchmark of the reduced Kelvin-Voigt hot path on one B300 per rank.

One bench step is one whole pass of the pre-computed-projection pipeline over
the largest single-GPU workload, the 512 x 512 x 384 bone shell (dx = 0.15 mm,
curved bone shell over smooth soft tissue, speckled focused beam, dt = 0.5 x
the stability limit): fold the medium into the step coefficients, zero the
state, project the force (CG to a true relative residual of 1e-8; by default
preconditioned by a multigrid V-cycle, started from the learned network's
potential when one is given with --net; with --projection cg the paper's plain
CG), run 5000 fused time steps with sensor recording and read the traces.
`--workload inclusions256` times the 256^3 inclusions medium (2000 steps) and
`--workload sweep` the 26-case batched sweep instead.

value  = cell-updates of the pass (nx*ny*nz*2000) / pass time, in Gcell/s,
         inputs resident on the device.
e2e    = the same metric through the C ABI with host inputs (pinned host
         medium and force, copied every pass) and the traces read back to the
         host every pass.
Also reported: step-only Gcell/s, projection ms and CG iterations, the roofline
of the step kernel (the dominant kernel) against the measured HBM copy peak,
the clocks seen during the timed region and the FP64 CPU oracle timed on a
bounded sample (cpu_baseline).

`--impl reference` times the FP64 CPU oracle on the same workload instead.
Multi-GPU (torchrun): every rank runs its own replica (the path has no
exchange step); value is the sum over ranks divided by the slowest rank's
time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DEFAULT_STEPS = {"inclusions256": 2000, "bone512": 5000, "sweep": 1000}
GRID = 256
# Algorithmic bytes of one cell-update of the method as printed (3-level
# recurrence of Sec. 3.1): read u^n and u^n-1 (24 B), write u^n+1 (12 B),
# heterogeneous media add the two folded coefficients (8 B); force steps add
# the projected force (12 B). These are the roofline's numerator.
ALG_BYTES_HOMOG = 36
ALG_BYTES_HETEROG = 44
FORCE_BYTES_PER_CELL = 12
# Bytes the storage form of this library moves per cell-update: (u, d) read +
# write 48 B plus the medium (fields A', B' 8 B; one class byte; flux-form
# fields m, e, 1/rho 12 B). Reported beside the algorithmic fraction.
STEP_BYTES_PER_CELL = 56
CLASS_STEP_BYTES_PER_CELL = 49
DIV_STEP_BYTES_PER_CELL = 60


def oracle_cg_iterations(workload_name):
    """Iterations of the oracle's plain CG to 1e-8 on this workload, counted by
    the oracle itself (oracle/plain_cg_iterations.py writes them)."""
    with open(os.path.join(ROOT, "oracle", "plain_cg_iterations.json")) as f:
        return int(json.load(f)[workload_name]["iters"])


def slowest(t, world, device):
    """The job time of independent replicas: the maximum of the per-rank time
    over all ranks (an all-reduce on the process group; identity at world 1)."""
    if world == 1:
        return float(t)
    import torch
    import torch.distributed as dist
    x = torch.tensor([float(t)], dtype=torch.float64, device=device)
    dist.all_reduce(x, op=dist.ReduceOp.MAX)
    return float(x.item())


def job_rate(world, cell_updates_per_rank, t_max):
    """Whole-job Gcell-updates/s: every rank's cell-updates over the slowest rank's time."""
    return world * cell_updates_per_rank / t_max / 1e9


def step_traffic(w, step_cfg, operator, n_force_steps, medium="fields", with_source=False):
    """DRAM bytes per step from the committed ncu capture
    (profiles/kv_step_traffic.json: dram__bytes_read.sum + dram__bytes_write.sum
    of force and plain steps; a two-step launch's bytes over two), averaged over
    this pass's steps (the caller scales it to a launch, like `achieved`); None unless a capture is of this operator, medium encoding
    ("fields" or "classes") and kernel configuration, and either of this grid
    or marked `scale_by_cells` for this workload family (a smaller case of a
    grid too large to capture, scaled by the cell count). with_source: also
    return a one-line description of the capture used."""
    tfile = os.path.join(ROOT, "profiles", "kv_step_traffic.json")
    res = (None, None)
    if os.path.exists(tfile):
        try:
            caps = json.load(open(tfile))["captures"]
            nf = n_force_steps
            for exact in (True, False):
                for c in caps:
                    if not (c["operator"] == operator and c.get("medium", "fields") == medium
                            and c["step_config"] == step_cfg):
                        continue
                    if exact and c["grid"] != [w.nx, w.ny, w.nz]:
                        continue
                    if not exact and not (c.get("scale_by_cells")
                                          and c.get("family") == getattr(w, "family", None)):
                        continue
                    scale = (w.nx * w.ny * w.nz) / float(np.prod(c["grid"]))
                    t = scale * (nf * c["bytes_force_step"] + (w.n_steps - nf) * c["bytes_plain_step"]) \
                        / w.n_steps
                    src = ("stored ncu capture of this grid" if exact else
                           f"stored ncu capture of a {'x'.join(map(str, c['grid']))} case of the same "
                           f"workload and kernel configuration, scaled by the cell count ({scale:.3g}x)")
                    res = (t, src)
                    break
                if res[0] is not None:
                    break
        except (KeyError, ValueError, TypeError):
            res = (None, None)
    return res if with_source else res[0]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="bone512",
                    choices=["inclusions256", "bone512", "sweep"],
                    help="bone512: 512x512x384 bone shell, 5000 steps (the headline, the largest "
                         "single-GPU configuration); inclusions256: 256^3 inclusions, 2000 steps; "
                         "sweep: 26 homogeneous cases on uneven grids, 1000 batched steps")
    ap.add_argument("--operator", default="pointwise", choices=["pointwise", "divergence"],
                    help="spatial operator of the heterogeneous step: pointwise (G/rho) L u "
                         "(Sec. 3.1) or the flux form (1/rho) div(G grad u)")
    ap.add_argument("--medium-encoding", default="auto", choices=["auto", "fields"],
                    help="auto: a medium of at most 256 distinct folded coefficient tuples is "
                         "read as one class byte per node (bit for bit the same step); fields: "
                         "always read the coefficient fields")
    ap.add_argument("--grid", type=int, default=GRID)
    ap.add_argument("--shape", default=None,
                    help="NX,NY,NZ of a smaller bone shell over the same box (profiling captures)")
    ap.add_argument("--time-steps", type=int, default=None,
                    help="time steps of the pass (default: the workload's own)")
    ap.add_argument("--step-config", default=None,
                    help="[variant,]tx,ty,zc,ns of the step kernel instead of autotuning "
                         "(profiling runs; variant 0 one step per sweep, 2 to 4 two steps per sweep)")
    ap.add_argument("--projection", default="auto", choices=["auto", "learned", "mg", "cg"],
                    help="learned: the trained network's potential as the start of the "
                         "multigrid-preconditioned CG (mode 5); mg: that CG from zero (mode 4); cg: "
                         "the paper's plain CG from zero (mode 0); all stop on the same true "
                         "residual. auto: learned for the bone shell (its workload names a "
                         "learned warm start), mg otherwise")
    ap.add_argument("--net", default=None,
                    help="parameters of the warm-start network (.npz written by "
                         "paper_2607_28414_b300.learned --out; default: the committed one)")
    ap.add_argument("--cg-config", type=int, default=None,
                    help="z chunk of the CG passes (default: the CG autotuner's choice)")
    ap.add_argument("--cg-tol", type=float, default=1e-8,
                    help="projection tolerance (1e-8 is the workload's; larger values only for "
                         "short profiling runs)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[5 + q] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def workload(grid, n_steps, kind="bone512", shape=None):
    """The workload of a pass. shape (bone shell only): a smaller grid over the
    same physical box (dx scaled), for captures of the same kernels."""
    from paper_2607_28414_b300 import inputs
    n_steps = DEFAULT_STEPS[kind] if n_steps is None else n_steps
    if kind == "bone512":
        if shape:
            nx, ny, nz = shape
            w = inputs.bone_shell(nx=nx, ny=ny, nz=nz, dx=0.15e-3 * 512 / nx, n_steps=n_steps)
        else:
            w = inputs.bone_shell(n_steps=n_steps)
        w.family = "bone_shell"
        return w
    w = inputs.heterogeneous_inclusions(n=grid, n_steps=n_steps)
    w.family = "inclusions"
    return w


def cpu_oracle_sample(w, dt, cg_iters, n_sample_steps=6, n_sample_iters=6, divform=False):
    """Time the FP64 oracle on a bounded sample of the pass: n_sample_iters CG
    iterations and n_sample_steps time steps of the same workload; the whole
    pass is extrapolated with the GPU's CG iteration count."""
    import oracle as orc
    t0 = time.perf_counter()
    phi, fs, status, st = orc.project(*w.force, w.dx, tol=1e-30, max_iter=n_sample_iters)
    t_cg = (time.perf_counter() - t0) / max(1, st["iters"])
    t0 = time.perf_counter()
    orc.run(w.nx, w.ny, w.nz, w.dx, dt, w.G, w.rho, w.eta, n_sample_steps, w.sensors, fs=fs,
            g=np.ones(n_sample_steps, np.float32), divform=divform)
    t_step = (time.perf_counter() - t0) / n_sample_steps
    total = cg_iters * t_cg + w.n_steps * t_step
    value = w.n_cells * w.n_steps / total / 1e9
    return value, {"cores": orc.get_threads(), "t_cg_iter_s": t_cg, "t_step_s": t_step,
                   "sample": (f"{n_sample_iters} CG iterations + {n_sample_steps} time steps of the "
                              f"{w.nx}x{w.ny}x{w.nz} workload, extrapolated to {cg_iters} CG "
                              f"iterations + {w.n_steps} steps")}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2607_28414_b300 import inputs
    import oracle as orc
    if args.workload == "sweep":
        # the oracle on the sweep's first case (128 x 128 x 192), whose rate per
        # cell-update stands for the sweep's
        n_steps = args.time_steps if args.time_steps is not None else DEFAULT_STEPS["sweep"]
        w = inputs.sweep_cases(n_steps=n_steps)[0]
    else:
        w = workload(args.grid, args.time_steps, args.workload)
    dt = 0.5 * orc.stable_dt(w.G, w.rho, w.eta, w.dx)
    # iterations the paper's plain CG needs to a 1e-8 residual on this workload,
    # counted by the oracle's own CG
    if args.grid != GRID and args.workload == "inclusions256":
        raise SystemExit("--impl reference: the oracle's CG iteration count is stored for the "
                         "256^3 grid only")
    cg_iters = oracle_cg_iterations(args.workload)
    vals = []
    for it in range(args.warmup + args.steps):
        k = 1 if w.n_cells > 50_000_000 else 3  # keeps the whole run within a few minutes
        v, info = cpu_oracle_sample(w, dt, cg_iters, n_sample_steps=k, n_sample_iters=k,
                                    divform=args.operator == "divergence")
        if it >= args.warmup:
            vals.append(v)
    value = float(np.mean(vals))
    ms = w.n_cells * w.n_steps / (value * 1e9) * 1e3
    if args.workload == "sweep":
        metric = f"KV-FDTD Gcell-updates/s (26-case sweep, projections + {w.n_steps} steps)"
        config = {"workload": "sweep_26_cases", "time_steps": w.n_steps,
                  "sampled_case": [w.nx, w.ny, w.nz]}
    else:
        metric = f"KV-FDTD Gcell-updates/s (projection + {w.n_steps} steps)"
        config = {"workload": w.name, "grid": [w.nx, w.ny, w.nz], "time_steps": w.n_steps,
                  "cg_tol": w.tol, "operator": args.operator,
                  "projection": f"plain CG from zero, {cg_iters} iterations (the oracle's count)"}
    line = {"metric": metric, "value": value,
            "unit": "Gcell-updates/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config,
            "cpu_baseline": {"value": value, "unit": "Gcell-updates/s", "cores": info["cores"],
                             "kind": "oracle", "sample": info["sample"] + " (the oracle's own "
                             "plain-CG iteration count to 1e-8 on this workload, "
                             "oracle/plain_cg_iterations.json)"},
            "e2e": {"value": value, "unit": "Gcell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_sweep(args, rank, world):
    """Parameter sweep: 26 homogeneous cases (16 viscosities on 128x128x192, 10
    moduli on cubes of 96..224 nodes), one projection per distinct grid shared
    by the other cases on it, then 1000 steps of all cases in one launch per
    step (CUDA graph). A pass = reset, 11 projections + 15 shares, 1000
    batched steps, traces read."""
    import torch
    from paper_2607_28414_b300 import inputs, kv
    import torch.distributed as dist
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=device)
    stream = torch.cuda.Stream(device)
    torch.cuda.set_stream(stream)
    n_steps = args.time_steps if args.time_steps is not None else DEFAULT_STEPS["sweep"]
    cases = inputs.sweep_cases(n_steps=n_steps)
    hs, forces, owner = [], [], {}
    for w in cases:
        dt = 0.5 * kv.kv_stable_dt(w.nx, w.ny, w.nz, w.dx, w.G, w.rho, w.eta)
        h = kv.kv_create(w.nx, w.ny, w.nz, w.dx, dt, w.G, w.rho, w.eta, stream=stream.cuda_stream)
        kv.kv_set_envelope(h, inputs.push_envelope(n_steps, dt, w.t_push))
        kv.kv_set_sensors(h, w.sensors, n_steps)
        hs.append(h)
        forces.append([torch.from_numpy(a).to(device) for a in w.force])
    b = kv.kv_batch_create(hs)
    N = sum(w.n_cells for w in cases)
    proj_mode = 0 if args.projection == "cg" else 4  # the sweep has no learned start

    def one_pass():
        grids = {}
        for i, (w, h) in enumerate(zip(cases, hs)):
            kv.kv_reset(h)
            key = (w.nx, w.ny, w.nz)
            if key in grids:
                kv.kv_share_force(h, hs[grids[key]])
            else:
                kv.kv_project_force(h, *forces[i], w.tol, 0, proj_mode)
                grids[key] = i
        kv.kv_batch_step(b, n_steps)
        out = torch.empty((n_steps, 256, 3), dtype=torch.float32, device=device)
        for w, h in zip(cases, hs):
            kv.kv_read_traces(h, out[:, :len(w.sensors)])
        return len(grids)

    # projections once so the autotuner runs forced steps too
    one_pass()
    tune_ms = kv.kv_batch_autotune(b, 4)
    cfg = kv.kv_batch_get_config(b)
    for _ in range(args.warmup):
        one_pass()
    torch.cuda.synchronize(device)
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(device)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = kv.kv_batch_launch_count(b) + sum(kv.kv_launch_count(h) for h in hs)
    e0.record(stream)
    for _ in range(args.steps):
        n_proj = one_pass()
    e1.record(stream)
    torch.cuda.synchronize(device)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    t = slowest(e0.elapsed_time(e1) / 1e3, world, device)
    # step-only timing of the batched kernel
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for h in hs:
        kv.kv_reset(h)
    s0.record(stream)
    kv.kv_batch_step(b, n_steps)
    s1.record(stream)
    torch.cuda.synchronize(device)
    t_steps = s0.elapsed_time(s1) / 1e3
    launches = kv.kv_batch_launch_count(b) + sum(kv.kv_launch_count(h) for h in hs) - l0
    kv.kv_batch_destroy(b)
    for h in hs:
        kv.kv_destroy(h)
    value = job_rate(world, N * n_steps * args.steps, t)
    # homogeneous cases: 36 B/cell algorithmic, 48 B/cell moved by the (u, d) form
    n_force = sum(int(inputs.push_envelope(n_steps, 0.5 * kv.kv_stable_dt(
        w.nx, w.ny, w.nz, w.dx, w.G, w.rho, w.eta), w.t_push).sum()) * w.n_cells for w in cases)
    launch_s = t_steps / n_steps
    achieved = (ALG_BYTES_HOMOG * N + FORCE_BYTES_PER_CELL * n_force / n_steps) / launch_s / 1e9
    achieved_storage = (48.0 * N + FORCE_BYTES_PER_CELL * n_force / n_steps) / launch_s / 1e9
    peak, peak_kind = peaks()
    if rank == 0:
        print(json.dumps({
            "metric": f"KV-FDTD Gcell-updates/s (26-case sweep, projections + {n_steps} steps)",
            "value": value, "unit": "Gcell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "sweep_26_cases", "cells": N, "time_steps": n_steps,
                       "projection": ("CG preconditioned by a multigrid V(1,1)-cycle (mode 4)"
                                      if proj_mode == 4 else "plain CG from zero (mode 0)"),
                       "parallelism": f"replicas{world}",
                       "projections_per_pass": n_proj, "batch_config": cfg,
                       "l2": f"state {48 * N / 1e9:.1f} GB > 126 MB L2"},
            "kv_step_gcells": N * n_steps / t_steps / 1e9, "autotune_ms_per_step": tune_ms,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "k_step_batch",
                         "peak_kind": peak_kind,
                         "bytes_model": (f"algorithmic {ALG_BYTES_HOMOG} B/cell (homogeneous, "
                                         f"3-level recurrence) + {FORCE_BYTES_PER_CELL} B/cell "
                                         "on force steps"),
                         "achieved_storage_form": achieved_storage,
                         "frac_storage_form": achieved_storage / peak,
                         "storage_bytes_model": "48 B/cell ((u, d) read + write)"},
            "gpu_launches": int(launches), "clocks": clk, "e2e": None, "cpu_baseline": None}),
            flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "sweep":
        run_sweep(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_2607_28414_b300 import inputs, kv

    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=device)

    def barrier():
        if world > 1:
            dist.barrier()

    w = workload(args.grid, args.time_steps, args.workload,
                 tuple(int(v) for v in args.shape.split(",")) if args.shape else None)
    w.tol = args.cg_tol
    N = w.n_cells
    stream = torch.cuda.Stream(device)  # a non-default stream shared by torch events and libkv
    torch.cuda.set_stream(stream)
    medium_d = [torch.from_numpy(a).to(device) for a in (w.G, w.rho, w.eta)]
    force_d = [torch.from_numpy(a).to(device) for a in w.force]
    div = args.operator == "divergence"
    lim = kv.kv_stable_dt(w.nx, w.ny, w.nz, w.dx, *medium_d)
    if div:
        lim = min(lim, kv.kv_stable_dt_op(w.nx, w.ny, w.nz, w.dx, *medium_d, kv.KV_OP_DIVERGENCE))
    dt = 0.5 * lim
    h = kv.kv_create(w.nx, w.ny, w.nz, w.dx, dt, *medium_d, stream=stream.cuda_stream)
    if div:
        kv.kv_set_operator(h, kv.KV_OP_DIVERGENCE, *medium_d)
    kv.kv_set_medium_encoding(h, kv.KV_MEDIUM_AUTO if args.medium_encoding == "auto"
                              else kv.KV_MEDIUM_FIELDS)
    if args.step_config:
        vals = [int(v) for v in args.step_config.split(",")]
        variant, (tx, ty, zc, ns) = (vals[0], vals[1:]) if len(vals) == 5 else (0, vals)
        kv.kv_set_step_config(h, variant, tx, ty, zc, ns)
        tune_ms = None
    else:
        tune_ms = kv.kv_autotune_step(h, 8)  # picks tile / stages / z chunk; resets the state
    step_cfg = kv.kv_get_step_config(h)
    classes = kv.kv_medium_classes(h) if step_cfg["variant"] == 0 else 0
    medium_enc = "classes" if classes > 0 else "fields"
    two_step = step_cfg["variant"] in (2, 3, 4)  # temporal blocking: one sweep advances two steps
    bytes_per_cell = (CLASS_STEP_BYTES_PER_CELL if classes > 0 else
                      DIV_STEP_BYTES_PER_CELL if div else STEP_BYTES_PER_CELL)
    if two_step:
        bytes_per_cell = STEP_BYTES_PER_CELL / 2  # (u, d) and the fields once per two steps
    if args.cg_config is not None:
        kv.kv_set_cg_config(h, args.cg_config)
        cg_tune_ms = None
    else:
        cg_tune_ms = kv.kv_autotune_cg(h, *force_d, 40)  # trial projections; the pass projects again
    cg_zc = kv.kv_get_cg_config(h)
    g = inputs.push_envelope(w.n_steps, dt, w.t_push)
    n_force_steps = int(g.sum())
    kv.kv_set_envelope(h, g)
    kv.kv_set_sensors(h, w.sensors, w.n_steps)
    traces_d = torch.zeros((w.n_steps, len(w.sensors), 3), dtype=torch.float32, device=device)

    ev = lambda: torch.cuda.Event(enable_timing=True)
    stats_last = {}

    projection = args.projection
    if projection == "auto":
        projection = "learned" if args.workload == "bone512" else "mg"
    proj_mode = {"learned": 5, "mg": 4, "cg": 0}[projection]
    net = None
    if proj_mode == 5:
        from paper_2607_28414_b300 import learned
        net = learned.load_net(args.net or learned.WEIGHTS, (w.nx, w.ny, w.nz),
                               stream=stream.cuda_stream)
        kv.kv_attach_net(h, net)

    def one_pass(step_events=None, medium=medium_d, force=force_d, traces=traces_d):
        kv.kv_set_medium(h, *medium)
        kv.kv_reset(h)
        st = kv.kv_project_force(h, *force, w.tol, 0, proj_mode)
        stats_last.update(st)
        if step_events is not None:
            step_events[0].record(stream)
        kv.kv_step(h, w.n_steps)
        if step_events is not None:
            step_events[1].record(stream)
        kv.kv_read_traces(h, traces)

    for _ in range(args.warmup):
        one_pass()
    torch.cuda.synchronize(device)
    # both projections once, outside the timed region, for the record (the
    # paper's plain CG from zero and the multigrid-preconditioned CG)
    by_mode = {}
    for name, mode in (("cg", 0), ("mg", 4)) + ((("learned_mg", 5),) if net is not None else ()):
        st = kv.kv_project_force(h, *force_d, w.tol, 0, mode)
        by_mode[name] = {"ms": st["ms"], "iters": st["iters"], "rel_res_true": st["rel_res_true"]}

    # ---- timed region: inputs resident on the device ----
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize(device)
    clocks.start()
    launches0 = kv.kv_launch_count(h)
    e0, e1 = ev(), ev()
    step_evs = [(ev(), ev()) for _ in range(args.steps)]
    cg_iters, cg_ms = [], []
    e0.record(stream)
    for k in range(args.steps):
        one_pass(step_evs[k])
        cg_iters.append(stats_last["iters"])
        cg_ms.append(stats_last["ms"])
    e1.record(stream)
    torch.cuda.synchronize(device)
    barrier()
    clk = clocks.stop()
    launches = kv.kv_launch_count(h) - launches0
    t_total = e0.elapsed_time(e1) / 1e3
    t_steps = sum(a.elapsed_time(b) for a, b in step_evs) / 1e3
    t_max = slowest(t_total, world, device)
    value = job_rate(world, N * w.n_steps * args.steps, t_max)
    step_gcells = N * w.n_steps * args.steps / t_steps / 1e9
    # a launch advances steps_per_launch steps (two for the two-step kernels)
    spl = 2 if two_step else 1
    launch_s = spl * t_steps / (w.n_steps * args.steps)
    force_bytes = N * FORCE_BYTES_PER_CELL * n_force_steps / w.n_steps  # per step, averaged
    alg_bytes = spl * (N * ALG_BYTES_HETEROG + force_bytes)             # per launch
    achieved = alg_bytes / launch_s / 1e9
    achieved_storage = spl * (N * bytes_per_cell + force_bytes) / launch_s / 1e9
    peak, peak_kind = peaks()
    traffic, traffic_src = step_traffic(w, step_cfg, args.operator, n_force_steps, medium_enc,
                                        with_source=True)
    if traffic is not None:
        traffic *= spl  # the capture's bytes per step, per launch
    # DRAM rate the stored bytes imply at this run's launch time
    dram_gbs = traffic / launch_s / 1e9 if traffic is not None and launch_s > 0 else None

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        medium_h = [torch.from_numpy(a).pin_memory() for a in (w.G, w.rho, w.eta)]
        force_h = [torch.from_numpy(a).pin_memory() for a in w.force]
        traces_h = torch.zeros((w.n_steps, len(w.sensors), 3), dtype=torch.float32).pin_memory()
        one_pass(None, medium_h, force_h, traces_h)
        torch.cuda.synchronize(device)
        barrier()
        t0 = time.perf_counter()
        f0, f1 = ev(), ev()
        f0.record(stream)
        for _ in range(args.steps):
            one_pass(None, medium_h, force_h, traces_h)
            _ = float(traces_h[-1, 0, 2])  # host reads the result
        f1.record(stream)
        torch.cuda.synchronize(device)
        barrier()
        t_e2e = slowest(max(f0.elapsed_time(f1) / 1e3, 1e-12), world, device)
        e2e = {"value": job_rate(world, N * w.n_steps * args.steps, t_e2e),
               "unit": "Gcell-updates/s", "h2d_bytes_per_step": 6 * N * 4,
               "d2h_bytes_per_step": int(traces_h.numel() * 4),
               "wall_s": time.perf_counter() - t0}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle runs the paper's plain CG: extrapolate with its iteration count
        v, info = cpu_oracle_sample(w, dt, by_mode["cg"]["iters"], divform=div)
        cpu = {"value": v, "unit": "Gcell-updates/s", "cores": info["cores"], "kind": "oracle",
               "sample": info["sample"]}
        # the same oracle on one host core (a smaller sample: 1-2 iterations + 1-2 steps)
        import oracle as orc
        n_all = orc.get_threads()
        orc.set_threads(1)
        try:
            k1 = 1 if N > 50_000_000 else 2
            v1, info1 = cpu_oracle_sample(w, dt, by_mode["cg"]["iters"], k1, k1, divform=div)
        finally:
            orc.set_threads(n_all)
        cpu.update({"value_1_core": v1, "sample_1_core": info1["sample"]})

    kv.kv_destroy(h)
    if net is not None:
        kv.kv_net_destroy(net)
    if rank == 0:
        line = {
            "metric": f"KV-FDTD Gcell-updates/s (projection + {w.n_steps} steps)",
            "value": value, "unit": "Gcell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": w.name, "grid": [w.nx, w.ny, w.nz], "dx_m": w.dx,
                       "time_steps": w.n_steps, "force_steps": n_force_steps, "cg_tol": w.tol,
                       "medium": ("8 seeded spherical inclusions (seed 102), speckled beam"
                                  if args.workload == "inclusions256" else
                                  "bone shell over smooth soft tissue (seed 105), speckled beam"),
                       "operator": args.operator,
                       "medium_encoding": (f"{classes} classes: 1 byte per node + coefficient table"
                                           if classes > 0 else "coefficient fields (FP32)"),
                       "projection": {5: "learned warm start (BF16 U-Net, residual loss) + CG "
                                         "preconditioned by a multigrid V(1,1)-cycle (mode 5)",
                                      4: "CG preconditioned by a multigrid V(1,1)-cycle (mode 4)",
                                      0: "plain CG from zero (mode 0)"}[proj_mode],
                       "reductions": "f64", "parallelism": f"replicas{world}",
                       "l2": f"state {48 * N / 1e9:.1f} GB > 126 MB L2 (inputs larger than L2)"},
            "kv_step_gcells": step_gcells,
            "projection_ms": float(np.mean(cg_ms)), "cg_iters": int(np.median(cg_iters)),
            "projection_by_mode": by_mode,
            "step_config": step_cfg, "autotune_ms_per_step": tune_ms,
            "cg_zc": cg_zc, "cg_autotune_ms_40_iters": cg_tune_ms,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "traffic_source": (f"{traffic_src} (dram__bytes_read.sum + "
                                            "dram__bytes_write.sum per launch, same operator, "
                                            "medium encoding and kernel configuration, "
                                            "profiles/kv_step_traffic.json); not measured in "
                                            "this run" if traffic is not None else
                                            "no stored capture for this configuration"),
                         "kernel": {0: "k_step_tma", 1: "k_step_plain", 2: "k_step2_tma",
                                    3: "k_step2c_tma", 4: "k_step2b_tma"}[step_cfg["variant"]],
                         "steps_per_launch": spl, "cell_steps_per_launch": N * spl,
                         "peak_kind": peak_kind,
                         "bytes_model": (f"algorithmic {ALG_BYTES_HETEROG} B/cell (heterogeneous, "
                                         f"3-level recurrence) + {FORCE_BYTES_PER_CELL} B/cell "
                                         "on force steps"),
                         "launch_us": launch_s * 1e6,
                         "achieved_storage_form": achieved_storage,
                         "frac_storage_form": achieved_storage / peak,
                         "storage_bytes_model": (f"{bytes_per_cell:g} B/cell per step ((u, d) read "
                                                 "+ write 48 B + medium"
                                                 + (", once per two steps" if two_step else "")
                                                 + f") + {FORCE_BYTES_PER_CELL} B/cell on force "
                                                 "steps"),
                         "dram_gbs_from_traffic": dram_gbs,
                         "dram_frac_from_traffic": dram_gbs / peak if dram_gbs is not None else None,
                         "note": ("two steps per launch read and write the state once, so the "
                                  "single step's algorithmic bytes can exceed the copy peak; "
                                  "dram_*_from_traffic is what DRAM moved"
                                  if two_step else None)},
            "gpu_launches": int(launches),
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
