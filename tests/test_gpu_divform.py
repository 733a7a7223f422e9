"""The divergence-form heterogeneous operator (1/rho) div(G grad u) +
(1/rho) div(eta grad udot) on the GPU against the FP64 oracle, with the step
kernel variants, CUDA-graph replay, a batch and a pulsed push train.

Tolerances as in the pointwise parity tests: FP64 check mode <= 1e-10 relative
trace L2; FP32 path <= 1e-4; FP32 kernel variants bit for bit (they share
kv_update_div's rounding sequence)."""
import numpy as np
import pytest

import oracle as orc
from paper_2607_28414_b300 import inputs, kv
from paper_2607_28414_b300.runner import Solver, to_device

from test_gpu_parity import TILES, max_rel_l2, ragged_workload, small_heterogeneous

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

DIV = kv.KV_OP_DIVERGENCE


def pulsed(n_steps, dt):
    """Pulsed push train (TIPS-like): 4 pulses of 30 us on, 30 us off."""
    return inputs.pulsed_envelope(n_steps, dt, 30e-6, 30e-6, 4)


def run_div(w, cfg, n_steps, precision=kv.KV_FP32, envelope=None, want_fields=True):
    s = Solver(w, precision=precision, n_steps=n_steps, step_config=cfg, operator=DIV,
               envelope=envelope)
    s.project(tol=1e-12 if precision == kv.KV_FP64 else None)  # oracle: 1e-13
    s.step()
    tr = s.read_traces().cpu().numpy().astype(np.float64)
    fields = None
    if want_fields:
        dt = np.float64 if precision == kv.KV_FP64 else np.float32
        fields = []
        for which in (kv.FIELD_U, kv.FIELD_D):
            for comp in range(3):
                out = np.empty((w.nz, w.ny, w.nx), dt)
                kv.kv_read_field(s.h, which, comp, out)
                fields.append(out)
        fields = np.stack(fields)
    res = (tr, fields, s.dt, s.envelope)
    s.close()
    return res


def oracle_div(w, dt, g, n_steps, want_state=False):
    phi, fs, status, _ = orc.project(*w.force, w.dx, tol=1e-13)
    assert status in ("converged", "zero_rhs")
    return orc.run(w.nx, w.ny, w.nz, w.dx, dt, w.G, w.rho, w.eta, n_steps, w.sensors, fs=fs, g=g,
                   divform=True, want_state=want_state)


def test_divergence_tiles_match_plain_kernel_bitwise(device):
    w = ragged_workload(het=True)
    ref_tr, ref_f, _, _ = run_div(w, {"variant": 1}, 60)
    assert np.abs(ref_f).max() > 0
    ran = 0
    for tx, ty in TILES:
        for ns in (4, 6, 8):
            for zc in (5, 64):
                try:
                    tr, f, _, _ = run_div(w, {"variant": 0, "tx": tx, "ty": ty, "zc": zc, "ns": ns}, 60)
                except kv.KvError as e:
                    assert e.status == kv.KV_ERR_ARG and "shared memory" in str(e)
                    continue
                ran += 1
                assert np.array_equal(tr, ref_tr), (tx, ty, ns, zc)
                assert np.array_equal(f, ref_f), (tx, ty, ns, zc)
    assert ran >= 30


def test_divergence_fp64_matches_oracle(device):
    w = ragged_workload(het=True)
    n = 60
    tr, f, dt, g = run_div(w, {}, n, precision=kv.KV_FP64)
    ref, u_ref, _ = oracle_div(w, dt, g, n, want_state=True)
    assert max_rel_l2(tr, ref) <= 1e-10
    u = f[:3]
    assert np.abs(u - np.stack(u_ref)).max() <= 1e-10 * np.abs(np.stack(u_ref)).max()


def test_divergence_fp32_pulsed_matches_oracle(device):
    w = small_heterogeneous(n=80, n_steps=400)
    tr, _, dt, g = run_div(w, {}, w.n_steps, envelope=pulsed, want_fields=False)
    assert g.sum() > 0 and (np.diff(g) != 0).sum() >= 7  # four separate pulses
    ref = oracle_div(w, dt, g, w.n_steps)
    assert max_rel_l2(tr, ref) <= 1e-4


def test_divergence_differs_from_pointwise_only_when_heterogeneous(device):
    w = ragged_workload(het=True)
    n = 60
    tr_div, _, dt, _ = run_div(w, {}, n, want_fields=False)
    s = Solver(w, n_steps=n, dt=dt)
    s.project()
    s.step()
    tr_pt = s.read_traces().cpu().numpy().astype(np.float64)
    s.close()
    assert max_rel_l2(tr_pt, tr_div) > 1e-3  # sharp inclusions: the operators differ
    # homogeneous medium: the divergence form is the pointwise operator
    wh = ragged_workload(het=False)
    a = Solver(wh, n_steps=n)
    a.project()
    a.step()
    ta = a.read_traces().cpu().numpy()
    b = Solver(wh, n_steps=n, operator=DIV)
    b.project()
    b.step()
    tb = b.read_traces().cpu().numpy()
    a.close()
    b.close()
    assert np.array_equal(ta, tb)


def test_operator_switch_keeps_state_and_checks_dt(device):
    w = ragged_workload(het=True)
    med = [to_device(x, device) for x in (w.G, w.rho, w.eta)]
    lim_p = kv.kv_stable_dt(w.nx, w.ny, w.nz, w.dx, *med)
    lim_d = kv.kv_stable_dt_op(w.nx, w.ny, w.nz, w.dx, *med, DIV)
    lim_host = kv.kv_stable_dt_op(w.nx, w.ny, w.nz, w.dx,
                                  *[np.asarray(x, np.float32) for x in (w.G, w.rho, w.eta)], DIV)
    assert lim_d == pytest.approx(lim_host, rel=1e-12)
    if lim_d < lim_p:  # a dt between the two limits is refused by the divergence form
        h = kv.kv_create(w.nx, w.ny, w.nz, w.dx, 0.5 * (lim_d + lim_p), *med)
        with pytest.raises(kv.KvError) as e:
            kv.kv_set_operator(h, DIV, *med)
        assert e.value.status == kv.KV_ERR_UNSTABLE_DT
        kv.kv_destroy(h)
    h = kv.kv_create(w.nx, w.ny, w.nz, w.dx, 0.5 * min(lim_p, lim_d), *med)
    kv.kv_set_step_config(h, 2, 64, 8, 0, 4)
    with pytest.raises(kv.KvError) as e:
        kv.kv_set_operator(h, DIV, *med)
    assert e.value.status == kv.KV_ERR_UNSUPPORTED
    kv.kv_set_step_config(h, 0, 0, 0, 0, 0)
    kv.kv_set_operator(h, DIV, *med)
    with pytest.raises(kv.KvError) as e:
        kv.kv_set_step_config(h, 2, 64, 8, 0, 4)
    assert e.value.status == kv.KV_ERR_UNSUPPORTED
    assert kv.kv_get_step_config(h)["variant"] == 0
    kv.kv_destroy(h)


def test_divergence_batch_matches_single_handles(device):
    """A batch of divergence-form cases of different sizes advances each case
    exactly as its own handle does."""
    cases = [ragged_workload(70, 37, 45, het=True, seed=3), ragged_workload(45, 40, 33, het=True, seed=8)]
    n = 64
    singles = [run_div(w, {"tx": 64, "ty": 8, "zc": 16, "ns": 4}, n, want_fields=False)[0] for w in cases]
    stream = torch.cuda.Stream(device)
    solvers = [Solver(w, n_steps=n, operator=DIV, stream=stream.cuda_stream) for w in cases]
    for s in solvers:
        s.project()
    b = kv.kv_batch_create([s.h for s in solvers])
    kv.kv_batch_set_config(b, 64, 8, 16, 4)
    kv.kv_batch_step(b, n)
    for s, ref in zip(solvers, singles):
        tr = s.read_traces().cpu().numpy().astype(np.float64)
        assert np.array_equal(tr, ref)
    kv.kv_batch_destroy(b)
    for s in solvers:
        s.close()
