"""Validation of the GPU path against what the paper reports for its own
benchmarks (Sec. 4.4): QIBA-shaped elastic phantoms.

Four homogeneous phantoms (G = 1, 2, 5, 10 kPa, rho = 1000, eta = 0) on
240 x 200 x 200 nodes at dx = 0.25 mm, axial Gaussian push (1/e widths 4.3 /
0.62 / 1.1 mm, focus 30 mm deep, 167 us), solenoidal projection to 1e-8,
dt = 0.5 x the stability limit. The group speed from cross-correlating the
axial velocity traces at lateral offsets 4-14 mm must match sqrt(G/rho); the
paper reports ~1 % for all four (Sec. 4.4), the gate here is 1.2 % (the runs
measure -0.94 ... -1.15 %).
"""
import numpy as np
import pytest

import oracle as orc
from paper_2607_28414_b300 import inputs, kv
from paper_2607_28414_b300.runner import Solver

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("G", [1e3, 2e3, 5e3, 10e3])
def test_qiba_phantom_group_speed(device, G):
    w = inputs.qiba_phantom(G)
    dt = 0.5 * orc.stable_dt(w.G, w.rho, w.eta, w.dx)
    n_steps = int(w.extra["t_window_s"] / dt) + 1
    s = Solver(w, dt=dt, n_steps=n_steps)
    st = s.project()
    assert st["rel_res_true"] < 1e-8
    s.step()
    tr = s.read_traces().cpu().numpy().astype(np.float64)
    s.close()
    vx = np.diff(np.concatenate([np.zeros((1, tr.shape[1])), tr[:, :, 0]]), axis=0) / dt
    c_est = orc.xcorr_group_speed(vx, w.extra["offsets_m"], dt)
    c = np.sqrt(G / 1000.0)
    print(f"QIBA G = {G / 1e3:.0f} kPa: group speed {c_est:.4f} m/s vs {c:.4f} "
          f"({100 * (c_est - c) / c:+.2f} %), {n_steps} steps, CG {st['iters']}")
    assert abs(c_est - c) / c < 0.012


# ---------------------------------------------------------------------------
# General per-step projection (Sec. 3.2) against the pre-computed one (Sec. 3.3)
# ---------------------------------------------------------------------------

def test_per_step_projection_of_a_separable_force_equals_precomputed(device):
    w = inputs.homogeneous_push(40, n_steps=40, eta=0.5, tol=1e-9)
    dt = 0.5 * orc.stable_dt(w.G, w.rho, w.eta, w.dx)
    w.t_push = 12 * dt
    a = Solver(w, dt=dt)
    a.project(tol=1e-9)
    a.step()
    ta = a.read_traces().cpu().numpy().copy()
    a.close()
    b = Solver(w, dt=dt)
    f = [torch.from_numpy(c).to(device) for c in w.force]
    g = inputs.push_envelope(w.n_steps, dt, w.t_push)
    for n in range(w.n_steps):
        kv.kv_step_force(b.h, *[c * float(g[n]) for c in f], 1e-9)
    tb = b.read_traces().cpu().numpy()
    b.close()
    err = np.sqrt(((ta - tb) ** 2).sum()) / np.sqrt((ta ** 2).sum())
    assert err < 1e-5, err


def moving_focus(w, n, dt, speed=0.5):
    """Gaussian push whose focus moves along y at `speed` m/s."""
    c = inputs.centre_node(w.nx, w.ny, w.nz)
    shift = int(round(speed * n * dt / w.dx))
    return inputs.gaussian_push(w.nx, w.ny, w.nz, w.dx, 1e3, 1e-3, 2e-3, (c[0], c[1] - 6 + shift, c[2]))


def test_per_step_projection_moving_focus_matches_oracle(device):
    n = 32
    w = inputs.homogeneous_push(n, n_steps=30, eta=0.3)
    dt = 0.5 * orc.stable_dt(w.G, w.rho, w.eta, w.dx)
    s = Solver(w, dt=dt)
    u = up = None
    ref = []
    for k in range(w.n_steps):
        f = moving_focus(w, k, dt)
        kv.kv_step_force(s.h, *f, 1e-10)
        _, fs, _, _ = orc.project(*f, w.dx, tol=1e-13)
        tr, u_next, u_now = orc.run(n, n, n, w.dx, dt, w.G, w.rho, w.eta, 1, w.sensors, fs=fs, g=[1.0],
                                    u_in=u, uprev_in=up, want_state=True)
        u, up = u_next, u_now
        ref.append(tr[0])
    got = s.read_traces().cpu().numpy()
    s.close()
    ref = np.array(ref)
    den = np.sqrt((ref ** 2).sum(axis=(0, 2)))
    num = np.sqrt(((got - ref) ** 2).sum(axis=(0, 2)))
    m = den > 1e-9 * den.max()
    assert (num[m] / den[m]).max() < 1e-4


def test_precomputed_projection_saves_over_per_step(device):
    """The paper's example (Sec. 3.3): N = 106^3, N_t = 85 steps; the
    pre-computed projection runs one CG, the general solver one per step."""
    w = inputs.homogeneous_push(106, n_steps=85, eta=0.5, tol=1e-8)
    dt = 0.5 * orc.stable_dt(w.G, w.rho, w.eta, w.dx)
    f = [torch.from_numpy(c).to(device) for c in w.force]
    g = inputs.push_envelope(w.n_steps, dt, 1.0)  # force on through the window
    ev = lambda: torch.cuda.Event(enable_timing=True)
    s = Solver(w, dt=dt)
    kv.kv_set_envelope(s.h, g)
    s.project()
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record()
    s.project()
    s.step()
    e1.record()
    torch.cuda.synchronize()
    t_pre = e0.elapsed_time(e1)
    t_gen = {}
    for mode in (0, 3, 4):
        s.reset()
        e2, e3 = ev(), ev()
        e2.record()
        for n in range(w.n_steps):
            kv.kv_step_force(s.h, *f, 1e-8, mode=mode)
        e3.record()
        torch.cuda.synchronize()
        t_gen[mode] = e2.elapsed_time(e3)
    s.close()
    print(f"106^3, 85 steps: pre-computed {t_pre:.1f} ms; per-step projection from zero "
          f"{t_gen[0]:.1f} ms (ratio {t_gen[0] / t_pre:.1f}); from the previous potential "
          f"{t_gen[3]:.1f} ms (ratio {t_gen[3] / t_pre:.1f}); multigrid-preconditioned from zero "
          f"{t_gen[4]:.1f} ms (ratio {t_gen[4] / t_pre:.1f})")
    assert t_gen[0] > 10 * t_pre
    assert t_gen[4] < t_gen[0]
