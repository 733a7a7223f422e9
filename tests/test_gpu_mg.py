"""Projection mode 4: CG preconditioned by a multigrid V-cycle. The system and
the stopping rule are the paper's (Sec. 3.2.3), so the oracle checks the same
things as for mode 0: the true residual of the GPU's potential re-evaluated in
FP64, the projected force node by node, and the time steps it drives."""
import numpy as np
import pytest

import oracle as orc
from paper_2607_28414_b300 import inputs, kv
from paper_2607_28414_b300.runner import Solver

from test_gpu_parity import FP32_TRACE_TOL, max_rel_l2, oracle_reference, ragged_workload, small_heterogeneous

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def check_projection(w, s, st, tol, fs):
    assert st["status"] == kv.KV_OK and st["rel_res_true"] < tol
    phi = np.empty((w.nz, w.ny, w.nx), np.float64)
    kv.kv_read_field(s.h, kv.FIELD_PHI, 0, phi)
    b = -orc.div_minus(*w.force, w.dx)
    res = np.linalg.norm(b - orc.apply_A(phi, w.dx)) / np.linalg.norm(b)
    assert res < tol * 1.01
    assert res == pytest.approx(st["rel_res_true"], rel=1e-3)
    g = orc.grad_plus(phi, w.dx)
    fs_np = fs.cpu().numpy()
    for a in range(3):
        expect = w.force[a].astype(np.float64) - g[a]
        assert np.abs(fs_np[a] - expect).max() <= 1e-6 * (np.abs(expect).max() + 1e-30)
    return res


@pytest.mark.parametrize("shape", [(70, 37, 45), (45, 40, 33), (130, 20, 22), (8, 7, 9)])
def test_multigrid_projection_meets_the_same_residual(device, shape):
    w = ragged_workload(*shape, het=min(shape) >= 20, seed=sum(shape))
    s = Solver(w)
    fs = torch.zeros((3, w.nz, w.ny, w.nx), dtype=torch.float32, device=device)
    st4 = kv.kv_project_force(s.h, *s.force, 1e-9, 0, 4, fs)
    check_projection(w, s, st4, 1e-9, fs)
    st0 = kv.kv_project_force(s.h, *s.force, 1e-9, 0, 0)
    print(f"{shape}: mode 4 {st4['iters']} iterations ({st4['ms']:.2f} ms), mode 0 {st0['iters']} "
          f"({st0['ms']:.2f} ms)")
    if min(shape) >= 20:
        assert st4["iters"] * 4 < st0["iters"]
    s.close()


def test_multigrid_projection_drives_the_same_steps(device):
    w = small_heterogeneous()
    dt = 0.5 * orc.stable_dt(w.G, w.rho, w.eta, w.dx)
    ref, _, _ = oracle_reference(w, dt, w.n_steps)
    s = Solver(w, dt=dt)
    st = kv.kv_project_force(s.h, *s.force, 1e-8, 0, 4)
    assert st["rel_res_true"] < 1e-8
    s.step()
    err = max_rel_l2(s.read_traces().cpu().numpy(), ref)
    print(f"80^3 inclusions, mode 4: CG {st['iters']} iterations, trace rel-L2 {err:.3e}")
    assert err <= FP32_TRACE_TOL
    s.close()


def test_multigrid_full_size_and_speed(device):
    """256^3 benchmark configuration: the same 1e-8 true residual as the
    paper's CG, checked by the oracle, in a fraction of its time."""
    w = inputs.heterogeneous_inclusions(n=256, n_steps=2000)
    s = Solver(w, n_steps=4)
    fs = torch.zeros((3, w.nz, w.ny, w.nx), dtype=torch.float32, device=device)
    kv.kv_project_force(s.h, *s.force, 1e-8, 0, 4, fs)  # allocation and warm-up
    st4 = kv.kv_project_force(s.h, *s.force, 1e-8, 0, 4, fs)
    res = check_projection(w, s, st4, 1e-8, fs)
    kv.kv_project_force(s.h, *s.force, 1e-8, 0, 0)
    st0 = kv.kv_project_force(s.h, *s.force, 1e-8, 0, 0)
    print(f"256^3: mode 4 {st4['iters']} iterations {st4['ms']:.1f} ms (oracle residual {res:.3e}); "
          f"mode 0 {st0['iters']} iterations {st0['ms']:.1f} ms; ratio {st0['ms'] / st4['ms']:.1f}")
    assert st4["ms"] * 3 < st0["ms"]
    s.close()


def test_multigrid_needs_fp32(device):
    w = ragged_workload()
    s = Solver(w, precision=kv.KV_FP64)
    with pytest.raises(kv.KvError) as e:
        kv.kv_project_force(s.h, *s.force, 1e-9, 0, 4)
    assert e.value.status == kv.KV_ERR_UNSUPPORTED
    s.close()
