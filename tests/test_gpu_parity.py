"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances
----------
* FP32 path: relative trace L2 (per sensor, over steps and components, max over
  sensors) <= 1e-4; projected-force true residual <= tol of the call.
* FP64 check mode: relative trace L2 <= 1e-10 (the oracle solves the
  projection to 1e-13, the GPU to 1e-12).
* Kernel variants of the FP32 step (TMA z-march, every tile shape, plain
  per-node kernel, CUDA-graph replay) share one rounding sequence per node and
  must agree bit for bit.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2607_28414_b300 import inputs, kv
from paper_2607_28414_b300.runner import Solver, to_device

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

FP32_TRACE_TOL = 1e-4
FP64_TRACE_TOL = 1e-10


def max_rel_l2(got, ref, floor=1e-9):
    """Max over sensors of ||got - ref|| / ||ref|| (over steps and components).

    Sensors whose reference trace is below `floor` times the largest one (a
    node on a symmetry plane, where the exact trace is zero and both sides
    hold rounding noise) are measured against the largest reference trace."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.sqrt((ref ** 2).sum(axis=(0, 2)))
    num = np.sqrt(((got - ref) ** 2).sum(axis=(0, 2)))
    top = den.max()
    if top == 0:
        assert np.all(num == 0), "motion recorded where the reference is at rest"
        return 0.0
    small = den < floor * top
    return float(np.concatenate([num[~small] / den[~small], num[small] / top]).max())


def oracle_reference(w, dt, n_steps, tol=1e-13, v0=None):
    phi, fs, status, st = orc.project(*w.force, w.dx, tol=tol)
    assert status in ("converged", "zero_rhs")
    g = inputs.push_envelope(n_steps, dt, w.t_push)
    tr = orc.run(w.nx, w.ny, w.nz, w.dx, dt, w.G, w.rho, w.eta, n_steps, w.sensors, fs=fs, g=g,
                 v0=v0)
    return tr, fs, phi


def small_heterogeneous(n=80, seed=7, n_steps=300):
    return inputs.heterogeneous_inclusions(n=n, seed=seed, n_steps=n_steps, tol=1e-8,
                                           name=f"heterogeneous_{n}^3")


def ragged_workload(nx=70, ny=37, nz=45, het=True, seed=3):
    rng = np.random.default_rng(seed)
    dx = 2e-4
    if het:
        G, rho, eta, _ = inputs.spherical_inclusions(nx, ny, nz, dx, rng, n=3,
                                                     r_range=(0.6e-3, 1.5e-3), margin=0.2e-3)
    else:
        G, rho, eta = 4e3, 1000.0, 0.7
    f = inputs.beam_push(nx, ny, nz, dx, rng, focal_depth=4e-3, focal_len=2e-3)
    fx = (rng.standard_normal((nz, ny, nx)) * 50).astype(np.float32)
    force = (fx, f[1], f[2])
    c = inputs.centre_node(nx, ny, nz)
    sensors = np.concatenate([inputs.line_sensors(c, 0, nx, 3),
                              np.array([[0, 0, 0], [nx - 1, ny - 1, nz - 1], [1, 1, 1]], np.int32)])
    return inputs.Workload(f"ragged_{nx}x{ny}x{nz}", nx, ny, nz, dx, G, rho, eta, force, 40e-6,
                           60, sensors, 1e-9)


# ---------------------------------------------------------------------------
# Kernel variants agree bit for bit
# ---------------------------------------------------------------------------

TILES = [(32, 8), (32, 16), (64, 4), (64, 8), (64, 16), (128, 2), (128, 4), (128, 8)]


def run_variant(w, cfg, n_steps, v0=None):
    s = Solver(w, n_steps=n_steps, step_config=cfg)
    if v0 is not None:
        kv.kv_set_initial_velocity(s.h, *[to_device(a, s.device) for a in v0])
    s.project()
    s.step()
    tr = s.read_traces().cpu().numpy().copy()
    fields = []
    for which in (kv.FIELD_U, kv.FIELD_D):
        for comp in range(3):
            out = np.empty((w.nz, w.ny, w.nx), np.float32)
            kv.kv_read_field(s.h, which, comp, out)
            fields.append(out)
    s.close()
    return tr, np.stack(fields)


@pytest.mark.parametrize("het", [True, False])
def test_tma_tiles_match_plain_kernel_bitwise(device, het):
    w = ragged_workload(het=het)
    v0 = inputs.curl_gaussian_velocity(w.nx, w.ny, w.nz, w.dx, sigma=1e-3, envelope="xyz")
    ref_tr, ref_f = run_variant(w, {"variant": 1}, 60, v0)
    assert np.abs(ref_f).max() > 0
    ran = 0
    for tx, ty in TILES:
        for ns in (4, 6, 8):
            for zc in (5, 64):
                try:
                    tr, f = run_variant(w, {"variant": 0, "tx": tx, "ty": ty, "zc": zc, "ns": ns}, 60, v0)
                except kv.KvError as e:
                    assert e.status == kv.KV_ERR_ARG and "shared memory" in str(e)
                    continue
                ran += 1
                assert np.array_equal(tr, ref_tr), (tx, ty, ns, zc)
                assert np.array_equal(f, ref_f), (tx, ty, ns, zc)
    assert ran >= 36


TILES2 = [(32, 4), (32, 8), (64, 4), (64, 8), (128, 4)]
TILES3 = [(32, 8), (32, 16), (64, 4), (64, 8), (64, 16), (128, 4), (128, 8)]
TILES4 = [(32, 14), (64, 14), (128, 14)]
# tiles and stage counts of the two-step kernels
TWO_STEP = {2: (TILES2, (4, 6)), 3: (TILES3, (4, 6)), 4: (TILES4, (2, 3, 4, 6))}


@pytest.mark.parametrize("variant", [2, 3, 4])
@pytest.mark.parametrize("het", [True, False])
@pytest.mark.parametrize("n_steps", [60, 61])
def test_two_step_kernel_matches_plain_kernel_bitwise(device, variant, het, n_steps):
    """Temporal blocking (two steps per sweep; variant 2 all components per
    block, variants 3 and 4 one component per block) reproduces single steps
    bit for bit, including the intermediate step's sensor records and an odd
    step count (the last step single)."""
    w = ragged_workload(het=het)
    v0 = inputs.curl_gaussian_velocity(w.nx, w.ny, w.nz, w.dx, sigma=1e-3, envelope="xyz")
    ref_tr, ref_f = run_variant(w, {"variant": 1}, n_steps, v0)
    tiles, stages = TWO_STEP[variant]
    for tx, ty in tiles:
        for ns in stages:
            for zc in (3, 64):
                try:
                    tr, f = run_variant(w, {"variant": variant, "tx": tx, "ty": ty, "zc": zc, "ns": ns},
                                        n_steps, v0)
                except kv.KvError as e:
                    assert e.status == kv.KV_ERR_ARG and "shared memory" in str(e)
                    continue
                assert np.array_equal(tr, ref_tr), (tx, ty, ns, zc)
                assert np.array_equal(f, ref_f), (tx, ty, ns, zc)


@pytest.mark.parametrize("het", [True, False])
def test_two_step_interior_blocks_match_plain_kernel_bitwise(device, het):
    """Variant 4 on a grid wide enough for blocks whose tile and halo hold no
    boundary node (the unmasked path of the 64- and 128-wide tiles), against
    single steps bit for bit."""
    w = ragged_workload(nx=300, ny=50, nz=20, het=het)
    v0 = inputs.curl_gaussian_velocity(w.nx, w.ny, w.nz, w.dx, sigma=1e-3, envelope="xyz")
    ref_tr, ref_f = run_variant(w, {"variant": 1}, 40, v0)
    assert np.abs(ref_f).max() > 0
    for tx in (32, 64, 128):
        for ns in (3, 4):
            for zc in (7, 18):
                tr, f = run_variant(w, {"variant": 4, "tx": tx, "ty": 14, "zc": zc, "ns": ns}, 40, v0)
                assert np.array_equal(tr, ref_tr), (tx, ns, zc)
                assert np.array_equal(f, ref_f), (tx, ns, zc)


@pytest.mark.parametrize("variant", [2, 3, 4])
def test_two_step_graph_replay_matches_direct(device, variant):
    w = ragged_workload()
    a = Solver(w, n_steps=75, step_config={"variant": variant, "tx": 64, "ty": 14 if variant == 4 else 4,
                                           "zc": 16, "ns": 4})
    a.project()
    a.step(75)  # one graph of 32 steps (16 two-step launches) + 21 pairs + 1 single
    ta = a.read_traces().cpu().numpy().copy()
    b = Solver(w, n_steps=75, step_config={"variant": 1})
    b.project()
    b.step(75)
    assert np.array_equal(ta, b.read_traces().cpu().numpy())
    assert kv.kv_steps_taken(a.h) == 75
    a.close()
    b.close()


def test_autotuner_picks_a_valid_config_and_resets(device):
    w = ragged_workload()
    s = Solver(w, n_steps=20)
    s.project()
    ms = kv.kv_autotune_step(s.h, 4)
    cfg = kv.kv_get_step_config(s.h)
    assert ms > 0 and cfg["variant"] in (0, 2, 3, 4) and cfg["ns"] in (2, 3, 4, 6, 8)
    assert kv.kv_steps_taken(s.h) == 0
    s.step()
    tr = s.read_traces().cpu().numpy().copy()
    s.close()
    ref = Solver(w, n_steps=20, step_config={"variant": 1})
    ref.project()
    ref.step()
    assert np.array_equal(tr, ref.read_traces().cpu().numpy())
    ref.close()


def test_graph_replay_matches_direct_launches(device):
    w = ragged_workload()
    a = Solver(w, n_steps=75)
    a.project()
    a.step(75)  # 2 graph blocks of 32 + 11 direct launches
    ta = a.read_traces().cpu().numpy().copy()
    b = Solver(w, n_steps=75)
    b.project()
    for _ in range(75):
        b.step(1)
    tb = b.read_traces().cpu().numpy().copy()
    assert np.array_equal(ta, tb)
    assert kv.kv_steps_taken(a.h) == 75
    a.close()
    b.close()


# ---------------------------------------------------------------------------
# Parity with the oracle
# ---------------------------------------------------------------------------

def test_fp64_homogeneous_push_matches_oracle(device):
    w = inputs.homogeneous_push(64, n_steps=400, tol=1e-13)
    dt = 0.5 * orc.stable_dt(w.G, w.rho, w.eta, w.dx)
    ref, fs_ref, _ = oracle_reference(w, dt, w.n_steps)
    s = Solver(w, precision=kv.KV_FP64, dt=dt)
    fs = torch.zeros((3, w.nz, w.ny, w.nx), dtype=torch.float32, device=device)
    st = s.project(tol=1e-12, fs_out=fs)
    assert st["rel_res_true"] < 1e-12
    s.step()
    tr = s.read_traces().cpu().numpy()
    err = max_rel_l2(tr, ref)
    print(f"FP64 homogeneous 64^3 x 400 steps: max trace rel-L2 {err:.3e}")
    assert err <= FP64_TRACE_TOL
    fs = fs.cpu().numpy().astype(np.float64)
    for a in range(3):
        scale = np.abs(fs_ref[a]).max() + 1e-30
        assert np.abs(fs[a] - fs_ref[a]).max() <= 1e-6 * scale  # float32 output buffer
    s.close()


def test_fp32_homogeneous_push_matches_oracle(device):
    w = inputs.homogeneous_push(64, n_steps=400, tol=1e-8)
    dt = 0.5 * orc.stable_dt(w.G, w.rho, w.eta, w.dx)
    ref, _, _ = oracle_reference(w, dt, w.n_steps)
    s = Solver(w, dt=dt)
    st = s.project()
    assert st["rel_res_true"] < 1e-8
    s.step()
    tr = s.read_traces().cpu().numpy()
    err = max_rel_l2(tr, ref)
    print(f"FP32 homogeneous 64^3 x 400 steps: max trace rel-L2 {err:.3e}, CG {st}")
    assert err <= FP32_TRACE_TOL
    s.close()


@pytest.mark.parametrize("precision,tol,gate", [(kv.KV_FP32, 1e-8, FP32_TRACE_TOL),
                                                (kv.KV_FP64, 1e-12, FP64_TRACE_TOL)])
def test_heterogeneous_inclusions_match_oracle(device, precision, tol, gate):
    w = small_heterogeneous()
    dt = 0.5 * orc.stable_dt(w.G, w.rho, w.eta, w.dx)
    ref, fs_ref, phi_ref = oracle_reference(w, dt, w.n_steps)
    s = Solver(w, precision=precision, dt=dt)
    fs = torch.zeros((3, w.nz, w.ny, w.nx), dtype=torch.float32, device=device)
    st = s.project(tol=tol, fs_out=fs)
    assert st["rel_res_true"] < tol
    # the oracle re-evaluates the true residual of the GPU's potential in FP64
    phi = np.empty((w.nz, w.ny, w.nx), np.float64)
    kv.kv_read_field(s.h, kv.FIELD_PHI, 0, phi)
    b = -orc.div_minus(*w.force, w.dx)
    res = np.linalg.norm(b - orc.apply_A(phi, w.dx)) / np.linalg.norm(b)
    assert res < tol * 1.01
    assert res == pytest.approx(st["rel_res_true"], rel=1e-3)
    s.step()
    tr = s.read_traces().cpu().numpy()
    err = max_rel_l2(tr, ref)
    print(f"heterogeneous 80^3 x 300 steps, precision {precision}: trace rel-L2 {err:.3e}, CG {st}")
    assert err <= gate
    s.close()


@pytest.mark.parametrize("precision", [kv.KV_FP32, kv.KV_FP64])
def test_initial_velocity_sets_increment(device, precision):
    """u^0 = 0 and d^0 = u^0 - u^{-1} = dt v0 on interior nodes, 0 on the layer."""
    n = 21
    w = inputs.homogeneous_push(n, n_steps=4, eta=0.4)
    v0 = inputs.curl_gaussian_velocity(n, n, n, w.dx, sigma=1.2e-3, envelope="xyz")
    dt = 0.5 * orc.stable_dt(w.G, w.rho, w.eta, w.dx)
    s = Solver(w, precision=precision, dt=dt)
    kv.kv_set_initial_velocity(s.h, *[to_device(a, s.device) for a in v0])
    dtype = np.float64 if precision == kv.KV_FP64 else np.float32
    m = np.zeros((n, n, n), bool)
    m[1:-1, 1:-1, 1:-1] = True
    for c in range(3):
        d = np.empty((n, n, n), dtype)
        kv.kv_read_field(s.h, kv.FIELD_D, c, d)
        u = np.empty((n, n, n), dtype)
        kv.kv_read_field(s.h, kv.FIELD_U, c, u)
        expect = np.where(m, dt * v0[c].astype(np.float64), 0.0)
        np.testing.assert_allclose(d, expect, rtol=1e-6, atol=1e-30)
        assert not u.any()
    s.close()


@pytest.mark.parametrize("precision,gate", [(kv.KV_FP32, FP32_TRACE_TOL), (kv.KV_FP64, FP64_TRACE_TOL)])
def test_curl_initial_velocity_matches_oracle(device, precision, gate):
    n = 41
    w = inputs.homogeneous_push(n, n_steps=120, eta=0.4)
    w.force = tuple(np.zeros((n, n, n), np.float32) for _ in range(3))
    v0 = inputs.curl_gaussian_velocity(n, n, n, w.dx, sigma=1.2e-3, envelope="xyz")
    dt = 0.5 * orc.stable_dt(w.G, w.rho, w.eta, w.dx)
    ref = orc.run(n, n, n, w.dx, dt, w.G, w.rho, w.eta, w.n_steps, w.sensors, v0=v0)
    s = Solver(w, precision=precision, dt=dt)
    kv.kv_set_initial_velocity(s.h, *[to_device(a, s.device) for a in v0])
    s.step()
    tr = s.read_traces().cpu().numpy()
    err = max_rel_l2(tr, ref)
    print(f"curl start 41^3 x 120 steps, precision {precision}: {err:.3e}, "
          f"|gpu| {np.abs(tr).max():.3e} |oracle| {np.abs(ref).max():.3e}")
    assert err <= gate
    s.close()


def test_full_size_heterogeneous_bench_configuration(device):
    """256^3 inclusions medium, speckled beam, CG to 1e-8, in the launch
    configuration the benchmark times. The oracle checks the GPU's potential
    (true residual in FP64), its projected force node by node, and the time
    step over 40 steps driven by the GPU's projected force."""
    w = inputs.heterogeneous_inclusions(n=256, n_steps=2000)
    dt = 0.5 * orc.stable_dt(w.G, w.rho, w.eta, w.dx)
    n_steps = 40
    s = Solver(w, dt=dt, n_steps=n_steps)
    fs = torch.zeros((3, w.nz, w.ny, w.nx), dtype=torch.float32, device=device)
    st = s.project(fs_out=fs)
    assert st["status"] == kv.KV_OK and st["rel_res_true"] < 1e-8
    phi = np.empty((w.nz, w.ny, w.nx), np.float64)
    kv.kv_read_field(s.h, kv.FIELD_PHI, 0, phi)
    b = -orc.div_minus(*w.force, w.dx)
    res = np.linalg.norm(b - orc.apply_A(phi, w.dx)) / np.linalg.norm(b)
    assert res < 1e-8 * 1.01
    g = orc.grad_plus(phi, w.dx)
    fs_np = fs.cpu().numpy()
    for a in range(3):
        expect = w.force[a].astype(np.float64) - g[a]
        scale = np.abs(expect).max() + 1e-30
        assert np.abs(fs_np[a] - expect).max() <= 1e-6 * scale
    # divergence of the projected force is the residual (discrete projection
    # identity), up to the float32 rounding of the stored f_S: each component
    # carries |delta| <= 2^-24 |f_S| and ||D-|| <= 2/dx per component.
    div_fs = orc.div_minus(*fs_np, w.dx)
    fs_norm = np.sqrt(sum((fs_np[a].astype(np.float64) ** 2).sum() for a in range(3)))
    round_bound = 2.0 ** -24 * (2.0 / w.dx) * np.sqrt(3.0) * fs_norm / np.linalg.norm(b)
    assert np.linalg.norm(div_fs) / np.linalg.norm(b) < 1e-8 + round_bound
    s.step()
    tr = s.read_traces().cpu().numpy()
    g_env = inputs.push_envelope(n_steps, dt, w.t_push)
    ref = orc.run(w.nx, w.ny, w.nz, w.dx, dt, w.G, w.rho, w.eta, n_steps, w.sensors,
                  fs=[fs_np[a] for a in range(3)], g=g_env)
    err = max_rel_l2(tr, ref)
    print(f"256^3 full size: CG {st}, oracle residual {res:.3e}, 40-step trace rel-L2 {err:.3e}")
    assert err <= FP32_TRACE_TOL
    s.close()


# ---------------------------------------------------------------------------
# Edge cases and error paths
# ---------------------------------------------------------------------------

def test_zero_force_gives_zero_iterations(device):
    w = ragged_workload()
    w.force = tuple(np.zeros((w.nz, w.ny, w.nx), np.float32) for _ in range(3))
    s = Solver(w, n_steps=10)
    st = s.project()
    assert st["iters"] == 0 and st["status"] == kv.KV_OK
    s.step()
    assert not s.read_traces().any()
    s.close()


def test_minimal_grid_matches_oracle(device):
    n = 3
    w = inputs.homogeneous_push(n, n_steps=30, eta=0.3)
    w.force = (np.full((n, n, n), 7.0, np.float32), np.zeros((n, n, n), np.float32),
               np.arange(27, dtype=np.float32).reshape(n, n, n))
    w.sensors = np.array([[1, 1, 1], [0, 1, 1]], np.int32)
    w.t_push = 1.0
    for precision, gate in ((kv.KV_FP64, FP64_TRACE_TOL), (kv.KV_FP32, FP32_TRACE_TOL)):
        dt = 0.5 * orc.stable_dt(w.G, w.rho, w.eta, w.dx)
        ref, _, _ = oracle_reference(w, dt, w.n_steps)
        s = Solver(w, precision=precision, dt=dt)
        s.project(tol=1e-12 if precision == kv.KV_FP64 else 1e-7)
        s.step()
        assert max_rel_l2(s.read_traces().cpu().numpy(), ref) <= gate
        s.close()


def test_cg_status_paths(device):
    w = ragged_workload()
    s = Solver(w)
    st = kv.kv_project_force(s.h, *s.force, 1e-8, 3, 0, None, check=False)
    assert st["rc"] == kv.KV_CG_MAXITER and st["iters"] == 3
    bad = [f.clone() for f in s.force]
    bad[2][5, 5, 5] = float("nan")
    st = kv.kv_project_force(s.h, *bad, 1e-8, 0, 0, None, check=False)
    assert st["rc"] == kv.KV_ERR_NONFINITE
    with pytest.raises(kv.KvError) as e:
        kv.kv_project_force(s.h, *s.force, 1e-8, 0, 6)
    assert e.value.status == kv.KV_ERR_UNSUPPORTED
    for mode in (1, 2, 5):  # the learned start and preconditioner need an attached net
        with pytest.raises(kv.KvError) as e:
            kv.kv_project_force(s.h, *s.force, 1e-8, 0, mode)
        assert e.value.status == kv.KV_ERR_STATE
    # the handle is still usable after these statuses
    st = s.project()
    assert st["status"] == kv.KV_OK and st["rel_res_true"] < 1e-8
    s.close()


def test_trace_capacity_and_reset(device):
    w = ragged_workload()
    s = Solver(w, n_steps=60)
    s.project()
    s.step(60)
    full = s.read_traces().cpu().numpy().copy()
    kv.kv_set_sensors(s.h, w.sensors, 20)
    s.reset()
    s.step(60)
    out = torch.zeros((20, len(w.sensors), 3), dtype=torch.float32, device=device)
    n = kv.kv_read_traces(s.h, out)
    assert n == 20
    assert np.array_equal(out.cpu().numpy(), full[:20])
    s.close()


def test_host_inputs_match_device_inputs(device):
    w = ragged_workload()
    dt = 0.5 * orc.stable_dt(w.G, w.rho, w.eta, w.dx)
    a = Solver(w, dt=dt, n_steps=30)
    a.project()
    a.step()
    ta = a.read_traces().cpu().numpy().copy()
    a.close()
    h = kv.kv_create(w.nx, w.ny, w.nz, w.dx, dt, w.G, w.rho, w.eta)
    kv.kv_set_envelope(h, inputs.push_envelope(30, dt, w.t_push))
    kv.kv_set_sensors(h, w.sensors, 30)
    kv.kv_project_force(h, *w.force, w.tol)
    kv.kv_step(h, 30)
    tb = np.zeros_like(ta)
    kv.kv_read_traces(h, tb)
    kv.kv_destroy(h)
    assert np.array_equal(ta, tb)


def test_invalid_arguments_on_gpu(device):
    w = ragged_workload()
    s = Solver(w, n_steps=5)
    with pytest.raises(kv.KvError):
        kv.kv_set_sensors(s.h, [[w.nx, 0, 0]], 5)
    with pytest.raises(kv.KvError):
        kv.kv_set_step_config(s.h, 0, 48, 8, 4)
    with pytest.raises(kv.KvError):
        kv.kv_set_step_config(s.h, 0, 64, 16, 4, 8)  # stages beyond a block's shared memory
    assert kv.kv_get_step_config(s.h)["tx"] == 64
    with pytest.raises(kv.KvError) as e:
        kv.kv_set_medium(s.h, 4e3, 1000.0, 0.0)  # homogeneous into a heterogeneous handle
    assert e.value.status == kv.KV_ERR_ARG
    s.close()


def test_full_size_bone_shell(device):
    """512 x 512 x 384 bone shell over soft tissue (dx = 0.15 mm), speckled
    beam focused beneath the shell, CG to 1e-8: the oracle checks the GPU's
    potential (true residual in FP64), its projected force node by node, and
    20 time steps driven by the GPU's projected force."""
    w = inputs.bone_shell()
    dt = 0.5 * orc.stable_dt(w.G, w.rho, w.eta, w.dx)
    n_steps = 20
    s = Solver(w, dt=dt, n_steps=n_steps)
    fs = torch.zeros((3, w.nz, w.ny, w.nx), dtype=torch.float32, device=device)
    st = s.project(fs_out=fs)
    assert st["status"] == kv.KV_OK and st["rel_res_true"] < 1e-8
    phi = np.empty((w.nz, w.ny, w.nx), np.float64)
    kv.kv_read_field(s.h, kv.FIELD_PHI, 0, phi)
    b = -orc.div_minus(*w.force, w.dx)
    res = np.linalg.norm(b - orc.apply_A(phi, w.dx)) / np.linalg.norm(b)
    assert res < 1e-8 * 1.01
    g = orc.grad_plus(phi, w.dx)
    del phi
    fs_np = fs.cpu().numpy()
    for a in range(3):
        expect = w.force[a].astype(np.float64) - g[a]
        assert np.abs(fs_np[a] - expect).max() <= 1e-6 * (np.abs(expect).max() + 1e-30)
    del g
    s.step()
    tr = s.read_traces().cpu().numpy()
    s.close()
    ref = orc.run(w.nx, w.ny, w.nz, w.dx, dt, w.G, w.rho, w.eta, n_steps, w.sensors,
                  fs=[fs_np[a] for a in range(3)], g=inputs.push_envelope(n_steps, dt, w.t_push))
    err = max_rel_l2(tr, ref)
    print(f"bone shell 512x512x384: CG {st}, oracle residual {res:.3e}, 20-step trace rel-L2 {err:.3e}")
    assert err <= FP32_TRACE_TOL


# ---------------------------------------------------------------------------
# Batched stepping of several handles (parameter sweeps)
# ---------------------------------------------------------------------------

def sweep_small():
    return [c for c in inputs.sweep_cases(n_steps=70, eta_cases=3, g_cases=3, eta_grid=(44, 36, 52),
                                          edge_range=(33, 61))]


def test_batch_matches_individual_handles(device):
    cases = sweep_small()
    stream = torch.cuda.Stream(device)
    ind, bat = [], []
    for w in cases:
        for lst in (ind, bat):
            s = Solver(w, n_steps=70, stream=stream.cuda_stream)
            s.project()
            lst.append(s)
    b = kv.kv_batch_create([s.h for s in bat])
    kv.kv_batch_step(b, 70)  # 2 graph blocks of 32 + 6 launches
    assert kv.kv_batch_launch_count(b) == 70
    for s in ind:
        s.step(70)
    for a, c in zip(ind, bat):
        assert kv.kv_steps_taken(c.h) == 70
        ta = a.read_traces().cpu().numpy()
        tc = c.read_traces().cpu().numpy()
        assert np.abs(ta).max() > 0
        assert np.array_equal(ta, tc), a.w.name
    # another configuration of the batched kernel gives the same numbers
    for c in bat:
        c.reset()
    kv.kv_batch_set_config(b, 128, 2, 5, 6)
    kv.kv_batch_step(b, 70)
    for a, c in zip(ind, bat):
        assert np.array_equal(a.read_traces().cpu().numpy(), c.read_traces().cpu().numpy())
    kv.kv_batch_destroy(b)
    for s in ind + bat:
        s.close()


def test_batch_autotune_resets_cases(device):
    cases = sweep_small()[:2]
    stream = torch.cuda.Stream(device)
    ss = [Solver(w, n_steps=20, stream=stream.cuda_stream) for w in cases]
    for s in ss:
        s.project()
    b = kv.kv_batch_create([s.h for s in ss])
    ms = kv.kv_batch_autotune(b, 2)
    cfg = kv.kv_batch_get_config(b)
    assert ms > 0 and cfg["ns"] in (4, 6, 8)
    assert all(kv.kv_steps_taken(s.h) == 0 for s in ss)
    kv.kv_batch_destroy(b)
    for s in ss:
        s.close()


def test_share_force_matches_direct_projection(device):
    w = sweep_small()[0]
    w2 = sweep_small()[1]  # same grid, other viscosity
    a = Solver(w, n_steps=5)
    a.project(tol=1e-10)
    b_direct = Solver(w2, n_steps=5)
    b_direct.project(tol=1e-10)
    b_shared = Solver(w2, n_steps=5)
    kv.kv_share_force(b_shared.h, a.h)
    n = (w2.nz, w2.ny, w2.nx)
    for c in range(3):
        x = np.empty(n, np.float32)
        y = np.empty(n, np.float32)
        kv.kv_read_field(b_direct.h, kv.FIELD_F, c, x)
        kv.kv_read_field(b_shared.h, kv.FIELD_F, c, y)
        assert np.abs(x - y).max() <= 1e-6 * np.abs(x).max() + 1e-30
    for s in (a, b_direct, b_shared):
        s.close()
