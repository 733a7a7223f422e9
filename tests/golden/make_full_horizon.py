"""Write the FP64 oracle's full-horizon sensor traces of the benchmark
workloads into tests/golden/full_horizon_<name>.npz.

This script calls only the oracle (oracle/) and the seeded input generators
(paper_2607_28414_b300/inputs.py, which hold none of the method's arithmetic);
nothing here comes from the CUDA path. The GPU parity tests read the files and
compare the library's FP32 traces with them over the whole run.

Per workload: the seeded inputs, dt = 0.5 x the oracle's stability limit, the
exact discrete projection of the force (sine-transform Poisson solve, true
relative residual ~1e-15), then the 3-level recurrence of Sec. 3.1 with the
push envelope of Sec. 3.3 for every time step of the workload, recording u at a
subset of the workload's sensors (every `stride`-th). Long runs go in chunks of
`--chunk` steps restarted from the saved (u^n, u^n-1) state, which is the same
recurrence bit for bit; the file is rewritten after every chunk, so a partial
horizon is usable while the rest runs (the file states how many steps it holds).

Usage:
    python tests/golden/make_full_horizon.py inclusions256
    python tests/golden/make_full_horizon.py sweep
    python tests/golden/make_full_horizon.py bone512 [--steps 5000] [--chunk 500]
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as orc  # noqa: E402
from paper_2607_28414_b300 import inputs  # noqa: E402


def digest(*arrays):
    """sha256 over the float32 bytes of the inputs (scalars as float32 too), so
    that a test can check it regenerated the same inputs."""
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(np.asarray(a, np.float32)).tobytes())
    return h.hexdigest()


def out_path(name):
    return os.path.join(HERE, f"full_horizon_{name}.npz")


def run_workload(w, name, stride, chunk, n_steps=None, extra=None):
    n_steps = w.n_steps if n_steps is None else n_steps
    t0 = time.time()
    dt = 0.5 * orc.stable_dt(w.G, w.rho, w.eta, w.dx)
    g = inputs.push_envelope(n_steps, dt, w.t_push)
    sel = np.arange(0, len(w.sensors), stride)
    sensors = np.ascontiguousarray(w.sensors[sel])
    phi, fs, res = orc.project_direct(*w.force, w.dx)
    del phi
    print(f"{name}: projection true rel. residual {res:.2e} ({time.time() - t0:.0f} s)", flush=True)
    meta = dict(workload=w.name, grid=np.array([w.nx, w.ny, w.nz]), dx=w.dx, dt=dt,
                t_push=w.t_push, sensor_index=sel, sensors=sensors,
                input_digest=digest(w.G, w.rho, w.eta, *w.force),
                projection_true_rel_res=res, n_steps_total=n_steps)
    if extra:
        meta.update(extra)
    traces = np.zeros((0, len(sensors), 3))
    u = up = None
    done = 0
    while done < n_steps:
        m = min(chunk, n_steps - done)
        tr, u, up = orc.run(w.nx, w.ny, w.nz, w.dx, dt, w.G, w.rho, w.eta, m, sensors, fs=fs,
                            g=g[done:done + m], u_in=u, uprev_in=up, want_state=True)
        traces = np.concatenate([traces, tr])
        done += m
        np.savez_compressed(out_path(name) + ".tmp.npz", traces=traces.astype(np.float32),
                            n_steps=done, **meta)
        os.replace(out_path(name) + ".tmp.npz", out_path(name))
        print(f"{name}: {done}/{n_steps} steps ({time.time() - t0:.0f} s)", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=["inclusions256", "bone512", "sweep"])
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--chunk", type=int, default=500)
    args = ap.parse_args()
    if args.workload == "inclusions256":
        w = inputs.heterogeneous_inclusions(n=256, n_steps=2000)
        run_workload(w, "inclusions256", 2, args.chunk, args.steps)
    elif args.workload == "bone512":
        w = inputs.bone_shell()
        run_workload(w, "bone512", 8, args.chunk, args.steps)
    else:
        cases = inputs.sweep_cases(n_steps=1000)
        for i in (0, 15, 16):  # eta = 0 and 1.5 on 128x128x192, G = 1 kPa on the 96^3 cube
            run_workload(cases[i], f"sweep_case{i}", 2, args.chunk, args.steps,
                         extra={"case_index": i})


if __name__ == "__main__":
    main()
