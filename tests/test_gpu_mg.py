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


@pytest.mark.parametrize("shape", [(70, 37, 45), (45, 40, 33), (130, 20, 22), (8, 7, 9), (5, 5, 5), (256, 256, 256)])
def test_preconditioner_matches_the_oracle_cycle(device, shape):
    """kv_apply_preconditioner (the V-cycle every mode-4 iteration applies)
    against the oracle's FP64 cycle (oracle/multigrid.py) on seeded random
    residuals: every node, and r.z. The 5^3 grid is too small to coarsen
    (M = S); the others run two to seven levels."""
    from oracle import multigrid as omg
    nx, ny, nz = shape
    dx = 2e-4
    rng = np.random.default_rng(nx * 7 + ny * 3 + nz)
    r = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    s = torch.cuda.Stream(device)
    with torch.cuda.stream(s):
        dt = 0.5 * kv.kv_stable_dt(nx, ny, nz, dx, 4e3, 1000.0, 0.0)
        h = kv.kv_create(nx, ny, nz, dx, dt, 4e3, 1000.0, 0.0, stream=s.cuda_stream)
        try:
            rd = torch.from_numpy(r).to(device)
            z = torch.full_like(rd, float("nan"))
            rz = kv.kv_apply_preconditioner(h, rd, z)
            z2 = torch.empty_like(rd)
            rz2 = kv.kv_apply_preconditioner(h, rd, z2)  # a second call: the same bits
            z0 = torch.full_like(rd, float("nan"))
            rz0 = kv.kv_apply_preconditioner(h, torch.zeros_like(rd), z0)
            same = bool(torch.equal(z, z2))
            zero_out = bool((z0 == 0).all())
        finally:
            kv.kv_destroy(h)
    got = z.cpu().numpy().astype(np.float64)
    ref = omg.vcycle_grid(r, dx)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    rz_ref = float((r.astype(np.float64)[1:-1, 1:-1, 1:-1] * ref[1:-1, 1:-1, 1:-1]).sum())
    levels = len(omg.levels((nx - 2, ny - 2, nz - 2), dx * dx))
    print(f"{shape}: {levels} levels, max |z - z_oracle| / max |z_oracle| = {err:.2e}, "
          f"r.z rel. error {abs(rz - rz_ref) / rz_ref:.2e}")
    assert np.all(got[0] == 0) and np.all(got[-1] == 0) and np.all(got[:, 0] == 0) and np.all(got[:, :, -1] == 0)
    assert err <= 2e-6  # FP32 through up to seven levels: measured 4e-8 ... 3.1e-7
    assert rz == pytest.approx(rz_ref, rel=1e-6)
    assert same and rz2 == rz
    assert zero_out and rz0 == 0.0


def test_preconditioner_argument_checks(device):
    w = ragged_workload()
    s = Solver(w)
    r = torch.zeros((w.nz, w.ny, w.nx), dtype=torch.float32, device=device)
    with pytest.raises(ValueError):
        kv.kv_apply_preconditioner(s.h, r, torch.zeros((w.nz, w.ny, w.nx + 1), dtype=torch.float32, device=device))
    with pytest.raises(kv.KvError) as e:
        bad = torch.zeros((w.nz, w.ny + 1, w.nx), dtype=torch.float32, device=device)
        kv.kv_apply_preconditioner(s.h, bad, torch.zeros_like(bad))
    assert e.value.status == kv.KV_ERR_ARG
    s.close()
    s64 = Solver(w, precision=kv.KV_FP64)
    with pytest.raises(kv.KvError) as e:
        kv.kv_apply_preconditioner(s64.h, r, torch.zeros_like(r))
    assert e.value.status == kv.KV_ERR_UNSUPPORTED
    s64.close()
