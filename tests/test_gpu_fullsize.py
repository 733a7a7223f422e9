"""Parity at the benchmark's full sizes, in the launch configurations bench.py
times (autotuned kernels, multigrid-preconditioned projection): the 26-case
sweep as one batch (cases checked against the oracle on sampled sensors) and
the 256^3 inclusions with the flux-form operator."""
import numpy as np
import pytest

import oracle as orc
from paper_2607_28414_b300 import inputs, kv

from test_gpu_parity import FP32_TRACE_TOL, max_rel_l2

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_full_size_sweep_batch_against_oracle(device):
    n_steps = 40
    cases = inputs.sweep_cases(n_steps=n_steps)
    stream = torch.cuda.Stream(device)
    hs, dts, forces = [], [], []
    for w in cases:
        dt = 0.5 * kv.kv_stable_dt(w.nx, w.ny, w.nz, w.dx, w.G, w.rho, w.eta)
        h = kv.kv_create(w.nx, w.ny, w.nz, w.dx, dt, w.G, w.rho, w.eta, stream=stream.cuda_stream)
        kv.kv_set_envelope(h, inputs.push_envelope(n_steps, dt, w.t_push))
        kv.kv_set_sensors(h, w.sensors, n_steps)
        hs.append(h)
        dts.append(dt)
        forces.append([torch.from_numpy(a).to(device) for a in w.force])
    owner = {}
    for i, (w, h) in enumerate(zip(cases, hs)):  # one projection per grid, as bench.py
        key = (w.nx, w.ny, w.nz)
        if key in owner:
            kv.kv_share_force(h, hs[owner[key]])
        else:
            st = kv.kv_project_force(h, *forces[i], w.tol, 0, 4)
            assert st["rel_res_true"] < w.tol
            owner[key] = i
    b = kv.kv_batch_create(hs)
    kv.kv_batch_autotune(b, 4)  # resets the cases, keeps their projected forces
    kv.kv_batch_step(b, n_steps)
    # oracle: the eta = 0 and eta = 1.5 cases of the 128 x 128 x 192 grid and the
    # smallest cube, each driven by the oracle's own projection
    for i in (0, 15, 16):
        w = cases[i]
        tr = torch.zeros((n_steps, len(w.sensors), 3), dtype=torch.float32, device=device)
        kv.kv_read_traces(hs[i], tr)
        _, fs, status, _ = orc.project(*w.force, w.dx, tol=1e-12)
        g = inputs.push_envelope(n_steps, dts[i], w.t_push)
        ref = orc.run(w.nx, w.ny, w.nz, w.dx, dts[i], w.G, w.rho, w.eta, n_steps, w.sensors, fs=fs, g=g)
        err = max_rel_l2(tr.cpu().numpy(), ref)
        print(f"sweep case {w.name}: trace rel-L2 {err:.3e}")
        assert err <= FP32_TRACE_TOL
    kv.kv_batch_destroy(b)
    for h in hs:
        kv.kv_destroy(h)


def test_full_size_divergence_form_against_oracle(device):
    w = inputs.heterogeneous_inclusions(n=256, n_steps=2000)
    n_steps = 40
    med = [torch.from_numpy(a).to(device) for a in (w.G, w.rho, w.eta)]
    lim = min(kv.kv_stable_dt(w.nx, w.ny, w.nz, w.dx, *med),
              kv.kv_stable_dt_op(w.nx, w.ny, w.nz, w.dx, *med, kv.KV_OP_DIVERGENCE))
    dt = 0.5 * lim
    h = kv.kv_create(w.nx, w.ny, w.nz, w.dx, dt, *med)
    kv.kv_set_operator(h, kv.KV_OP_DIVERGENCE, *med)
    kv.kv_autotune_step(h, 8)
    g = inputs.push_envelope(n_steps, dt, w.t_push)
    kv.kv_set_envelope(h, g)
    kv.kv_set_sensors(h, w.sensors, n_steps)
    fs = torch.zeros((3, w.nz, w.ny, w.nx), dtype=torch.float32, device=device)
    st = kv.kv_project_force(h, *[torch.from_numpy(a).to(device) for a in w.force], 1e-8, 0, 4, fs)
    assert st["rel_res_true"] < 1e-8
    kv.kv_step(h, n_steps)
    tr = torch.zeros((n_steps, len(w.sensors), 3), dtype=torch.float32, device=device)
    kv.kv_read_traces(h, tr)
    kv.kv_destroy(h)
    fs_np = fs.cpu().numpy()
    ref = orc.run(w.nx, w.ny, w.nz, w.dx, dt, w.G, w.rho, w.eta, n_steps, w.sensors,
                  fs=[fs_np[a] for a in range(3)], g=g, divform=True)
    err = max_rel_l2(tr.cpu().numpy(), ref)
    print(f"256^3 flux form, 40 steps: trace rel-L2 {err:.3e}")
    assert err <= FP32_TRACE_TOL
