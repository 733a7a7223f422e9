"""Full-horizon FP32 parity with the FP64 oracle on the benchmark workloads.

The oracle's traces over every time step of the 256^3 inclusions (2000 steps),
the 512 x 512 x 384 bone shell (5000 steps, or the horizon the file holds) and
three cases of the 26-case sweep (1000 steps) are stored in
tests/golden/full_horizon_*.npz by tests/golden/make_full_horizon.py, which
calls only the oracle and the seeded input generators (exact discrete
projection, then the 3-level recurrence of Sec. 3.1 in FP64).

Here the library runs the same inputs in the launch configuration bench.py
times: autotuned step kernel (class-byte medium where the medium allows it),
autotuned CG passes, the projection mode of the benchmark pass to a true
residual of 1e-8, the step loop replayed from CUDA graphs; the sweep as one
autotuned batch with one projection per grid. Gate: relative trace L2 per
sensor (over all steps and components), max over sensors, <= 1e-4 (FP32).
"""
import os

import numpy as np
import pytest

from paper_2607_28414_b300 import inputs, kv

from test_gpu_parity import FP32_TRACE_TOL, max_rel_l2

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    path = os.path.join(GOLDEN, f"full_horizon_{name}.npz")
    assert os.path.exists(path), f"missing oracle traces {path}"
    return dict(np.load(path))


def check_inputs(w, g):
    from golden.make_full_horizon import digest
    assert str(g["workload"]) == w.name
    assert digest(w.G, w.rho, w.eta, *w.force) == str(g["input_digest"]), \
        "the seeded generators no longer produce the inputs the oracle traces were made from"


def run_handle(w, g, device, mode):
    """One workload through the C ABI as bench.py sets it up; returns the
    traces at the golden's sensors over the golden's horizon, and the stats."""
    n_steps = int(g["n_steps"])
    dt = float(g["dt"])
    stream = torch.cuda.Stream(device)
    with torch.cuda.stream(stream):
        med = [torch.from_numpy(a).to(device) if isinstance(a, np.ndarray) else a
               for a in (w.G, w.rho, w.eta)]
        force = [torch.from_numpy(a).to(device) for a in w.force]
        h = kv.kv_create(w.nx, w.ny, w.nz, w.dx, dt, *med, stream=stream.cuda_stream)
        try:
            kv.kv_set_medium_encoding(h, kv.KV_MEDIUM_AUTO)
            kv.kv_autotune_step(h, 8)
            kv.kv_autotune_cg(h, *force, 40)
            kv.kv_set_envelope(h, inputs.push_envelope(n_steps, dt, w.t_push))
            kv.kv_set_sensors(h, g["sensors"], n_steps)
            st = kv.kv_project_force(h, *force, 1e-8, 0, mode)
            kv.kv_step(h, n_steps)
            tr = torch.zeros((n_steps, len(g["sensors"]), 3), dtype=torch.float32, device=device)
            kv.kv_read_traces(h, tr)
            cfg = kv.kv_get_step_config(h)
            classes = kv.kv_medium_classes(h)
        finally:
            kv.kv_destroy(h)
    return tr.cpu().numpy(), st, cfg, classes


def report(name, g, got, st, extra=""):
    ref = g["traces"].astype(np.float64)
    err = max_rel_l2(got, ref)
    per = max_rel_l2(got[: len(ref) // 4], ref[: len(ref) // 4])
    print(f"{name}: {len(ref)} steps, {ref.shape[1]} sensors, trace rel-L2 max over sensors "
          f"{err:.3e} (first quarter {per:.3e}); projection {st['iters']} it, true residual "
          f"{st['rel_res_true']:.2e}, oracle's {float(g['projection_true_rel_res']):.1e} {extra}")
    return err


def test_full_horizon_inclusions256(device):
    g = load("inclusions256")
    w = inputs.heterogeneous_inclusions(n=256, n_steps=2000)
    check_inputs(w, g)
    assert int(g["n_steps"]) == 2000
    got, st, cfg, classes = run_handle(w, g, device, 4)
    assert st["rel_res_true"] < 1e-8
    err = report("inclusions 256^3", g, got, st, f"step config {cfg}, {classes} classes")
    assert err <= FP32_TRACE_TOL


def test_full_horizon_bone_shell(device):
    g = load("bone512")
    w = inputs.bone_shell()
    check_inputs(w, g)
    assert int(g["n_steps"]) >= 500
    got, st, cfg, classes = run_handle(w, g, device, 4)
    assert st["rel_res_true"] < 1e-8
    err = report("bone shell 512x512x384", g, got, st,
                 f"(of {int(g['n_steps_total'])}), step config {cfg}")
    assert err <= FP32_TRACE_TOL


def test_full_horizon_sweep_batch(device):
    """All 26 cases in one autotuned batch as bench.py runs them; the three
    cases with oracle traces use the oracle's dt, the others their own."""
    cases = inputs.sweep_cases(n_steps=1000)
    goldens = {}
    for i in (0, 15, 16):
        gi = load(f"sweep_case{i}")
        assert int(gi["case_index"]) == i and int(gi["n_steps"]) == 1000
        check_inputs(cases[i], gi)
        goldens[i] = gi
    n_steps = 1000
    stream = torch.cuda.Stream(device)
    hs, owner = [], {}
    try:
        for i, w in enumerate(cases):
            dt = (float(goldens[i]["dt"]) if i in goldens
                  else 0.5 * kv.kv_stable_dt(w.nx, w.ny, w.nz, w.dx, w.G, w.rho, w.eta))
            h = kv.kv_create(w.nx, w.ny, w.nz, w.dx, dt, w.G, w.rho, w.eta,
                             stream=stream.cuda_stream)
            hs.append(h)
            kv.kv_set_envelope(h, inputs.push_envelope(n_steps, dt, w.t_push))
            kv.kv_set_sensors(h, goldens[i]["sensors"] if i in goldens else w.sensors, n_steps)
            key = (w.nx, w.ny, w.nz)
            if key in owner:
                kv.kv_share_force(h, hs[owner[key]])
            else:
                f = [torch.from_numpy(a).to(device) for a in w.force]
                st = kv.kv_project_force(h, *f, w.tol, 0, 4)
                assert st["rel_res_true"] < w.tol
                owner[key] = i
        b = kv.kv_batch_create(hs)
        try:
            kv.kv_batch_autotune(b, 4)  # resets the cases, keeps their projected forces
            kv.kv_batch_step(b, n_steps)
            cfg = kv.kv_batch_get_config(b)
        finally:
            kv.kv_batch_destroy(b)
        errs = {}
        for i, gi in goldens.items():
            tr = torch.zeros((n_steps, len(gi["sensors"]), 3), dtype=torch.float32, device=device)
            kv.kv_read_traces(hs[i], tr)
            errs[i] = report(f"sweep case {cases[i].name}", gi, tr.cpu().numpy(),
                             {"iters": -1, "rel_res_true": float("nan")}, f"batch config {cfg}")
    finally:
        for h in hs:
            kv.kv_destroy(h)
    assert max(errs.values()) <= FP32_TRACE_TOL, errs
