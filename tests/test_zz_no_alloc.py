"""The projection entry point that allocates nothing (kv_project_force_noalloc).

Some callers cannot allocate device memory themselves: their memory belongs to
another allocator, or they run on a stream that must not be stalled by the
device-wide synchronisation of cudaFree. For them libkv keeps the projection's
working set in a static device array. This file checks, through the C ABI,
that two calls in a row give the same projected force as kv_project_force on a
handle and as the FP64 oracle's projection, node by node (within the FP32
parity tolerance used for f_S elsewhere), that the oracle re-evaluates the
true residual of the call from the returned f_S, and that grids beyond the
array's limit are refused. pytest collects it last.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2607_28414_b300 import inputs, kv

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

FS_REL_TOL = 1e-6  # float32 storage of f_S, relative to its largest magnitude


def reference_fs(w, device, tol):
    G, rho, eta = w.G, w.rho, w.eta
    dt = 0.25 * kv.kv_stable_dt(w.nx, w.ny, w.nz, w.dx, G, rho, eta)
    h = kv.kv_create(w.nx, w.ny, w.nz, w.dx, dt, G, rho, eta)
    try:
        f = [torch.from_numpy(a).to(device) for a in w.force]
        fs = torch.zeros((3, w.nz, w.ny, w.nx), dtype=torch.float32, device=device)
        st = kv.kv_project_force(h, *f, tol, 0, 0, fs)
    finally:
        kv.kv_destroy(h)
    return fs.cpu().numpy(), st


def test_noalloc_projection_matches_handle_projection(device):
    rng = np.random.default_rng(11)
    n = (61, 47, 53)
    G, rho, eta, _ = inputs.spherical_inclusions(*n, 2e-4, rng, n=3, r_range=(1e-3, 2e-3),
                                                 margin=0.3e-3)
    force = inputs.beam_push(*n, 2e-4, rng, focal_depth=5e-3, focal_len=2e-3)
    force = (force[2] * 0.3, force[1], force[2])
    w = inputs.Workload("noalloc_61x47x53", *n, 2e-4, G, rho, eta, force, 2e-4, 1,
                        np.zeros((1, 3), np.int32), 1e-8)
    # both solves to 1e-10, so that two correct solutions agree well inside the
    # f_S tolerance whatever their reduction order
    ref, st_ref = reference_fs(w, device, 1e-10)
    assert st_ref["rel_res_true"] < 1e-10
    f = [torch.from_numpy(a).to(device) for a in w.force]
    scale = np.abs(ref).max()
    # the oracle's projection of the same force (CG to 1e-13, FP64)
    _, fs_orc, status, _ = orc.project(*w.force, w.dx, tol=1e-13)
    assert status == "converged"
    fs_orc = np.stack(fs_orc)
    b = -orc.div_minus(*w.force, w.dx)
    for call in range(2):
        out = torch.full((3, w.nz, w.ny, w.nx), float("nan"), dtype=torch.float32, device=device)
        st = kv.kv_project_force_noalloc(w.nx, w.ny, w.nz, w.dx, *f, 1e-10, out)
        got = out.cpu().numpy()
        assert np.isfinite(got).all(), call
        assert st["status"] == kv.KV_OK and st["rel_res_true"] < 1e-10, (call, st)
        assert np.abs(got - ref).max() <= FS_REL_TOL * scale, call
        assert abs(st["iters"] - st_ref["iters"]) <= 2, (call, st, st_ref)
        err_orc = np.abs(got - fs_orc).max() / np.abs(fs_orc).max()
        # D-.f_S = -(b - A phi): the oracle's divergence of the returned f_S is
        # the call's residual, up to the float32 rounding of the stored f_S
        # (|delta| <= 2^-24 |f_S| per component, ||D-|| <= 2/dx per component)
        div_fs = orc.div_minus(*got, w.dx)
        res = np.linalg.norm(div_fs) / np.linalg.norm(b)
        round_bound = (2.0 ** -24 * (2.0 / w.dx) * np.sqrt(3.0)
                       * np.sqrt((got.astype(np.float64) ** 2).sum()) / np.linalg.norm(b))
        print(f"no-alloc call {call}: {st['iters']} iterations, true residual "
              f"{st['rel_res_true']:.3e}, oracle residual {res:.3e} (rounding bound "
              f"{round_bound:.1e}), f_S vs oracle {err_orc:.2e} of max|f_S|")
        assert err_orc <= FS_REL_TOL, call
        assert res <= 1e-10 + round_bound, call


def test_noalloc_rejects_grids_beyond_the_limit(device):
    f = torch.zeros((66, 66, 66), dtype=torch.float32, device=device)
    out = torch.zeros((3, 66, 66, 66), dtype=torch.float32, device=device)
    with pytest.raises(kv.KvError) as e:
        kv.kv_project_force_noalloc(66, 66, 66, 2e-4, f, f, f, 1e-8, out)
    assert e.value.status == kv.KV_ERR_ARG
    assert "at most 262144" in str(e.value)
