"""Checkpoint/resume, poisoned row padding, and the bounded-wait failure path
(no counterparts in the paper)."""
import numpy as np
import pytest

from paper_2607_28414_b300 import kv
from paper_2607_28414_b300.runner import Solver

from test_gpu_parity import ragged_workload

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def fields(s):
    out = []
    dt = np.float64 if s.precision == kv.KV_FP64 else np.float32
    for which in (kv.FIELD_U, kv.FIELD_D):
        for comp in range(3):
            a = np.empty((s.w.nz, s.w.ny, s.w.nx), dt)
            kv.kv_read_field(s.h, which, comp, a)
            out.append(a)
    return np.stack(out)


@pytest.mark.parametrize("precision", [kv.KV_FP32, kv.KV_FP64])
def test_resume_from_a_checkpoint_is_bit_identical(device, precision):
    w = ragged_workload()  # nx = 70: rows padded to 96
    n1, n2 = 45, 40
    a = Solver(w, precision=precision, n_steps=n1 + n2)
    a.project(tol=1e-10)
    a.step(n1)
    buf = torch.empty(kv.kv_state_bytes(a.h), dtype=torch.uint8, device=device)
    step = kv.kv_save_state(a.h, buf)
    assert step == n1
    a.step(n2)
    ref_tr = a.read_traces().cpu().numpy().copy()
    ref_f = fields(a)

    b = Solver(w, precision=precision, n_steps=n1 + n2, dt=a.dt)
    b.project(tol=1e-10)
    kv.kv_load_state(b.h, buf, step)
    assert kv.kv_steps_taken(b.h) == n1
    b.step(n2)
    tr = b.read_traces().cpu().numpy()
    assert np.array_equal(tr[n1:], ref_tr[n1:])
    assert np.array_equal(fields(b), ref_f)

    # a state whose row padding is NaN continues identically: padding never
    # reaches a result
    host = buf.cpu().numpy().view(np.float64 if precision == kv.KV_FP64 else np.float32).copy()
    px = (w.nx + 31) // 32 * 32
    host.reshape(6, w.nz, w.ny, px)[..., w.nx:] = np.nan
    c = Solver(w, precision=precision, n_steps=n1 + n2, dt=a.dt)
    c.project(tol=1e-10)
    kv.kv_load_state(c.h, host, step)
    c.step(n2)
    assert np.array_equal(c.read_traces().cpu().numpy()[n1:], ref_tr[n1:])
    assert np.array_equal(fields(c), ref_f)
    for s in (a, b, c):
        s.close()


def test_bounded_wait_failure_path(device):
    w = ragged_workload()
    s = Solver(w, n_steps=8)
    s.project()
    assert kv.kv_selftest_wait(s.h) == kv.KV_ERR_TIMEOUT
    assert "timed out" in kv.kv_last_error(s.h)
    with pytest.raises(kv.KvError) as e:
        kv.kv_step(s.h, 1)
    assert e.value.status == kv.KV_ERR_STATE
    s.close()
    # the context is still usable: a fresh handle steps normally
    t = Solver(w, n_steps=8)
    t.project()
    t.step()
    assert np.abs(t.read_traces().cpu().numpy()).max() > 0
    t.close()
