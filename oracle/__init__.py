"""FP64 CPU oracle for the reduced Kelvin-Voigt shear-wave method.

TEST INFRASTRUCTURE ONLY: the test suite, the package's smoke check and the
CPU-baseline leg of the benchmark may import this package; the product path
(the CUDA library and its Python binding) never does. It shares no code with
the CUDA path: the numerics live in kv_oracle.c (plain loops, FP64) and in the
plain NumPy analysis routines below.

Citations name the paper's sections and equations:
  Sec. 3.1  explicit FDTD update, 7-point Laplacian, eta = 0 stability bound
  Sec. 3.2  solenoidal projection and masked CG (recurrences, stop rule, guards)
  Sec. 3.3  pre-computed projection for separable forces
  Sec. 3.5  Dirichlet outer layer, curl-based initial velocity
  Sec. 4.1  wavespeed from peak arrival times and a distance-time linear fit
  Sec. 4.2  trace-L2 self-convergence
  Sec. 4.3  Kelvin-Voigt dispersion (De_v, Pi_alpha, Eq. alpha_scaling, Table 2)

Parity status: every function here is pinned by a test under tests/ against
closed forms, brute-force dense solves, invariants or numbers the paper prints;
the exact error values of the paper's convergence table and the measured
columns of its Kelvin-Voigt table depend on unstated details and are compared
loosely (see the tests).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None

CG_STATUS = {0: "converged", 1: "maxiter", 2: "breakdown", 3: "nonfinite", 4: "zero_rhs"}


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        i, d = ctypes.c_int, ctypes.c_double
        L.or_set_threads.argtypes = [i]
        L.or_get_threads.restype = i
        L.or_laplacian.argtypes = [i, i, i, d, dp, dp]
        L.or_apply_A.argtypes = [i, i, i, d, dp, dp]
        L.or_div_minus.argtypes = [i, i, i, d, dp, dp, dp, dp]
        L.or_grad_plus.argtypes = [i, i, i, d, dp, dp, dp, dp]
        L.or_cg.argtypes = [i, i, i, d, dp, dp, d, i, dp]
        L.or_cg.restype = i
        L.or_project.argtypes = [i, i, i, d, dp, d, i, dp, dp, dp]
        L.or_project.restype = i
        L.or_run.argtypes = [i, i, i, d, d, dp, dp, dp, dp, dp, i, dp, dp, dp, i, ip, i, dp, dp, dp, i]
        L.or_run.restype = i
        L.or_kv1d_run.argtypes = [i, d, d, d, d, d, d, d, d, i, ip, i, dp]
        L.or_kv1d_run.restype = i
        L.or_conv3d_fwd.argtypes = [i, i, i, i, i, dp, dp, dp, dp]
        L.or_conv3d_bwd.argtypes = [i, i, i, i, i, dp, dp, dp, dp, dp, dp]
        _LIB = L
        set_threads(int(os.environ.get("KV_ORACLE_THREADS", os.cpu_count() or 1)))
    return _LIB


def set_threads(n: int):
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return int(lib().or_get_threads())


def _d(a):
    """Contiguous float64 copy/view and its ctypes pointer."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _null():
    return ctypes.POINTER(ctypes.c_double)()


def _shape(q):
    nz, ny, nx = q.shape
    return nx, ny, nz


def laplacian(q, dx):
    """Sec. 3.1: 7-point Laplacian on interior nodes (0 on the outer layer)."""
    q, qp = _d(q)
    out, op = _d(np.empty_like(q))
    lib().or_laplacian(*_shape(q), dx, qp, op)
    return out


def apply_A(q, dx):
    """Sec. 3.2.3: A q = -L q."""
    q, qp = _d(q)
    out, op = _d(np.empty_like(q))
    lib().or_apply_A(*_shape(q), dx, qp, op)
    return out


def div_minus(fx, fy, fz, dx):
    """Backward-difference divergence on interior nodes (0 on the outer layer)."""
    fx, a = _d(fx)
    fy, b = _d(fy)
    fz, c = _d(fz)
    out, op = _d(np.empty_like(fx))
    lib().or_div_minus(*_shape(fx), dx, a, b, c, op)
    return out


def grad_plus(phi, dx):
    """Forward-difference gradient at every node, phi = 0 beyond the last node."""
    phi, pp = _d(phi)
    g = [np.empty_like(phi) for _ in range(3)]
    ptrs = [_d(x)[1] for x in g]
    lib().or_grad_plus(*_shape(phi), dx, pp, *ptrs)
    return tuple(g)


def cg(b, dx, tol, max_iter, phi0=None):
    """Sec. 3.2.3: masked CG for A phi = b. Returns (phi, status, stats dict)."""
    b, bp = _d(b)
    phi = np.zeros_like(b) if phi0 is None else np.array(phi0, dtype=np.float64, copy=True)
    phi, pp = _d(phi)
    st = np.zeros(3)
    _, sp = _d(st)
    status = lib().or_cg(*_shape(b), dx, bp, pp, float(tol), int(max_iter), sp)
    return phi, CG_STATUS[status], {"iters": int(st[0]), "rel_res": float(st[1]),
                                     "true_rel_res": float(st[2])}


def default_max_iter(nx, ny, nz):
    """Iteration cap of the projection: 20 * max(nx, ny, nz)."""
    return 20 * max(nx, ny, nz)


def project(fx, fy, fz, dx, tol=1e-13, max_iter=None):
    """Sec. 3.2.1 + 3.3: f_S0 = P_S[b0]. Returns (phi, (fsx, fsy, fsz), status, stats)."""
    nz, ny, nx = np.shape(fx)
    if max_iter is None:
        max_iter = 4 * default_max_iter(nx, ny, nz)
    f = np.stack([np.asarray(fx, np.float64), np.asarray(fy, np.float64),
                  np.asarray(fz, np.float64)])
    f, fp = _d(f)
    N = nx * ny * nz
    phi, pp = _d(np.empty(N))
    fs, fsp = _d(np.empty(3 * N))
    st = np.zeros(3)
    _, sp = _d(st)
    status = lib().or_project(nx, ny, nz, dx, fp, float(tol), int(max_iter), pp, fsp, sp)
    fs = fs.reshape(3, nz, ny, nx)
    return (phi.reshape(nz, ny, nx), (fs[0], fs[1], fs[2]), CG_STATUS[status],
            {"iters": int(st[0]), "rel_res": float(st[1]), "true_rel_res": float(st[2])})


def poisson_direct(b, dx, workers=None):
    """Exact discrete solution of A phi = b (A = -L on the interior nodes, phi =
    0 on the outer layer; Sec. 3.2.1 and 3.2.3) through the eigenvectors of the
    Dirichlet 7-point Laplacian: the sine modes s_k(i) = sin(pi k i / (n - 1)),
    k, i = 1 .. n - 2 per axis, with -L s = lam s,
    lam = sum over axes (4/dx^2) sin^2(pi k / (2 (n - 1))).
    So phi = S diag(1/lam) S^-1 b, S the separable sine transform, applied with
    the type-I discrete sine transform of scipy.fft (an FFT library primitive).
    b on the outer layer is ignored. Returns phi (nz, ny, nx) in float64."""
    from scipy.fft import dstn, idstn
    b = np.asarray(b, np.float64)
    nz, ny, nx = b.shape
    if workers is None:
        workers = get_threads()
    bh = dstn(b[1:-1, 1:-1, 1:-1], type=1, workers=workers)
    lam_axis = [4.0 / dx ** 2 * np.sin(np.pi * np.arange(1, n - 1) / (2.0 * (n - 1))) ** 2
                for n in (nz, ny, nx)]
    bh /= lam_axis[0][:, None, None] + lam_axis[1][None, :, None] + lam_axis[2][None, None, :]
    phi = np.zeros((nz, ny, nx))
    phi[1:-1, 1:-1, 1:-1] = idstn(bh, type=1, workers=workers)
    return phi


def project_direct(fx, fy, fz, dx):
    """Sec. 3.2.1 + 3.3 with the exact discrete potential: b = -(D- . f), phi =
    poisson_direct(b), f_S = f - D+ phi. Same result as project() with the CG
    run to convergence, in a few transforms instead of thousands of iterations
    (large grids). Returns (phi, (fsx, fsy, fsz), true relative residual)."""
    b = -div_minus(fx, fy, fz, dx)
    phi = poisson_direct(b, dx)
    res = apply_A(phi, dx)
    res -= b
    res[0], res[-1], res[:, 0], res[:, -1], res[:, :, 0], res[:, :, -1] = 0, 0, 0, 0, 0, 0
    bn = np.linalg.norm(b)
    true_rel = float(np.linalg.norm(res) / bn) if bn > 0 else 0.0
    del res
    g = grad_plus(phi, dx)
    fs = tuple(np.asarray(f, np.float64) - ga for f, ga in zip((fx, fy, fz), g))
    return phi, fs, true_rel


def _field3(v, shape):
    if v is None:
        return None
    return np.stack([np.broadcast_to(np.asarray(c, np.float64), shape) for c in v])


def _medium(x, shape):
    return np.ascontiguousarray(np.broadcast_to(np.asarray(x, np.float64), shape))


def run(nx, ny, nz, dx, dt, G, rho, eta, n_steps, sensors, fs=None, g=None, v0=None,
        u_in=None, uprev_in=None, want_state=False, divform=False):
    """Sec. 3.1 + 3.3: n_steps of the 3-level leapfrog recurrence.

    G, rho, eta: scalars or (nz, ny, nx) maps. fs: (fsx, fsy, fsz) projected force
    pattern or None. g: envelope table g(t_n). v0: initial velocity (3 arrays).
    sensors: (ns, 3) node indices (i, j, k). Returns traces [n_steps, ns, 3]
    (entry n = u^{n+1}) and, with want_state, (u^{n_steps}, u^{n_steps-1}).
    divform: the divergence-form operator (1/rho) div(G grad u) + (1/rho)
    div(eta grad udot) with face-averaged coefficients instead of Sec. 3.1's
    pointwise (G/rho) L u + (eta/rho) L udot.
    """
    shape = (nz, ny, nx)
    mu_a, mup = _d(_medium(G, shape))
    rho_a, rhop = _d(_medium(rho, shape))
    eta_a, etap = _d(_medium(eta, shape))
    keep = [mu_a, rho_a, eta_a]
    fsp = gp = v0p = uinp = uprp = _null()
    n_g = 0
    if fs is not None:
        a, fsp = _d(_field3(fs, shape))
        keep.append(a)
    if g is not None:
        a, gp = _d(np.asarray(g, np.float64))
        n_g = len(a)
        keep.append(a)
    if v0 is not None:
        a, v0p = _d(_field3(v0, shape))
        keep.append(a)
    if u_in is not None:
        a, uinp = _d(_field3(u_in, shape))
        keep.append(a)
    if uprev_in is not None:
        a, uprp = _d(_field3(uprev_in, shape))
        keep.append(a)
    sensors = np.ascontiguousarray(np.asarray(sensors, np.int32).reshape(-1, 3))
    ns = sensors.shape[0]
    sp = sensors.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    traces, tp = _d(np.zeros((n_steps, ns, 3)))
    N = nx * ny * nz
    if want_state:
        uo, uop = _d(np.zeros(3 * N))
        upo, upop = _d(np.zeros(3 * N))
    else:
        uop = upop = _null()
    rc = lib().or_run(nx, ny, nz, dx, dt, mup, rhop, etap, fsp, gp, n_g, v0p, uinp, uprp,
                      int(n_steps), sp, ns, tp, uop, upop, int(bool(divform)))
    if rc != 0:
        raise MemoryError("oracle run failed to allocate")
    if want_state:
        return traces, uo.reshape(3, nz, ny, nx), upo.reshape(3, nz, ny, nx)
    return traces


def kv1d_run(n, dx, dt, mu, rho, eta, omega, amp, n_steps, sensors, t_ramp=0.0):
    """Sec. 4.3: 1D harmonic Kelvin-Voigt chain (same recurrence, 1D Laplacian),
    driven by u_0 = amp r(t) sin(omega t), r a raised-cosine ramp over t_ramp.
    Returns rec[n_steps, ns] (entry s = u^{s+1})."""
    sensors = np.ascontiguousarray(np.asarray(sensors, np.int32))
    rec, rp = _d(np.zeros((n_steps, len(sensors))))
    lib().or_kv1d_run(int(n), dx, dt, mu, rho, eta, omega, amp, float(t_ramp), int(n_steps),
                      sensors.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(sensors), rp)
    return rec


# ---------------------------------------------------------------------------
# Stability (Sec. 3.1, extended to eta > 0 by a von Neumann analysis)
# ---------------------------------------------------------------------------

def stable_dt(G, rho, eta, dx, ndim=3):
    """Largest stable dt of the recurrence for frozen coefficients.

    A mode of -L with eigenvalue lam <= lam_max = 4*ndim/dx^2 follows
    c_{n+1} = (2 - (a+b) lam) c_n - (1 - b lam) c_{n-1}, a = dt^2 G/rho,
    b = dt eta/rho; both roots stay in the unit disc iff lam (a + 2b) <= 4,
    i.e. dt^2 c^2 + 2 dt nu <= h^2 with c^2 = G/rho, nu = eta/rho,
    h^2 = dx^2/ndim. The positive root is taken per node and minimised. At
    eta = 0 it is the paper's bound dt <= (1/c) (sum 1/dx_i^2)^(-1/2).
    """
    G = np.asarray(G, np.float64)
    rho = np.asarray(rho, np.float64)
    eta = np.asarray(eta, np.float64)
    c2 = G / rho
    nu = eta / rho
    h2 = dx * dx / ndim
    with np.errstate(divide="ignore", invalid="ignore"):
        root = np.where(c2 > 0, (-nu + np.sqrt(nu * nu + c2 * h2)) / np.where(c2 > 0, c2, 1.0),
                        h2 / (2.0 * np.where(nu > 0, nu, np.inf)))
    return float(np.min(root))


# ---------------------------------------------------------------------------
# Analysis (Sec. 4)
# ---------------------------------------------------------------------------

def time_to_peak(trace, dt):
    """Sec. 4.1: peak-arrival time of a trace, refined by a 3-point parabola
    through the sample maximum of |trace|. Trace entry n is at t = (n+1) dt."""
    a = np.abs(np.asarray(trace, np.float64))
    m = int(np.argmax(a))
    shift = 0.0
    if 0 < m < len(a) - 1:
        y0, y1, y2 = a[m - 1], a[m], a[m + 1]
        den = y0 - 2.0 * y1 + y2
        if den != 0.0:
            shift = 0.5 * (y0 - y2) / den
    return (m + 1 + shift) * dt


def linear_fit_speed(offsets, times):
    """Sec. 4.1: least-squares slope of offset against arrival time."""
    offsets = np.asarray(offsets, np.float64)
    times = np.asarray(times, np.float64)
    A = np.stack([times, np.ones_like(times)], axis=1)
    coef, *_ = np.linalg.lstsq(A, offsets, rcond=None)
    return float(coef[0])


def trace_rel_l2(trace, ref):
    """Relative L2 norm of a trace difference, per sensor: ||a - r|| / ||r||,
    over time and components. Input shape [n_steps, ns, 3] or [n_steps, ns]."""
    a = np.asarray(trace, np.float64)
    r = np.asarray(ref, np.float64)
    axes = (0, 2) if a.ndim == 3 else (0,)
    num = np.sqrt(np.sum((a - r) ** 2, axis=axes))
    den = np.sqrt(np.sum(r ** 2, axis=axes))
    return num / np.where(den > 0, den, 1.0)


def kv_continuum(omega, mu, rho, eta):
    """Sec. 4.3: exact Kelvin-Voigt plane-wave dispersion.

    rho (i omega)^2 u = (mu + i omega eta) u'' with u ~ exp(i(omega t - k x))
    gives k^2 = rho omega^2 / (mu + i omega eta). Returns (alpha = |Im k|,
    phase speed omega / Re k)."""
    k = omega * np.sqrt(rho / (mu + 1j * omega * eta))
    return float(abs(k.imag)), float(omega / abs(k.real))


def kv_weak_loss_alpha(omega, mu, rho, eta):
    """Sec. 4.3, Eq. alpha_scaling: alpha ~ eta omega^2 / (2 rho c^3) for De_v << 1."""
    c = np.sqrt(mu / rho)
    return eta * omega ** 2 / (2.0 * rho * c ** 3)


def kv_discrete(omega, mu, rho, eta, dx, dt, lam_t=0.0):
    """Exact dispersion of the 1D recurrence (derived from Sec. 3.1).

    With u_i^n = z^n exp(-i k x_i), z = exp(i omega dt), the update gives
    lam = (4/dx^2) sin^2(k dx/2) = -(z-1)^2 / ((a+b) z - b), a = dt^2 mu/rho,
    b = dt eta/rho. Solve for complex k; returns (alpha, phase speed).

    lam_t: eigenvalue of -L over the two transverse directions of a guided
    mode u = U(x) s(y) s(z) on a 3D grid (the 3D recurrence acts on U as the
    1D one with lam replaced by lam + lam_t); 0 for a plane wave."""
    a = dt * dt * mu / rho
    b = dt * eta / rho
    z = np.exp(1j * omega * dt)
    lam = -(z - 1.0) ** 2 / ((a + b) * z - b) - lam_t
    s = np.sqrt(lam * dx * dx / 4.0)
    k = 2.0 / dx * np.arcsin(s)
    return float(abs(k.imag)), float(omega / abs(k.real))


def dirichlet_mode_eigenvalue(n, dx):
    """Eigenvalue of -d^2/dx^2 (3-point) for the first Dirichlet sine mode
    s_j = sin(pi j / (n - 1)), j = 0..n-1, of a line of n nodes with both end
    nodes fixed: (4/dx^2) sin^2(pi / (2 (n - 1)))."""
    return 4.0 / dx ** 2 * np.sin(np.pi / (2.0 * (n - 1))) ** 2


def kv_plane_from_guided(alpha, c, omega, dx, lam_t):
    """Plane-wave (alpha, phase speed) equivalent to a guided mode measured
    with (alpha, c): the guided wavenumber k_x has (4/dx^2) sin^2(k_x dx/2) =
    lam - lam_t, so the plane-wave k has (4/dx^2) sin^2(k dx/2) =
    (4/dx^2) sin^2(k_x dx/2) + lam_t."""
    kx = omega / c - 1j * alpha
    lam = 4.0 / dx ** 2 * np.sin(kx * dx / 2.0) ** 2 + lam_t
    k = 2.0 / dx * np.arcsin(np.sqrt(lam * dx * dx / 4.0))
    return float(abs(k.imag)), float(omega / abs(k.real))


def lockin_fit(rec, xs, dt, omega, n_periods):
    """Sec. 4.3 measurement: complex amplitude of each sensor trace at omega over
    the last n_periods whole periods, then least-squares slopes of ln|U| and of
    the unwrapped phase against position. Returns (alpha, phase speed)."""
    rec = np.asarray(rec, np.float64)
    n_steps = rec.shape[0]
    t = (np.arange(n_steps) + 1) * dt
    period = 2 * np.pi / omega
    n_win = int(round(n_periods * period / dt))
    sl = slice(n_steps - n_win, n_steps)
    ph = np.exp(-1j * omega * t[sl])
    U = (rec[sl] * ph[:, None]).sum(axis=0) * (2.0 / n_win)
    xs = np.asarray(xs, np.float64)
    A = np.stack([xs, np.ones_like(xs)], axis=1)
    la, *_ = np.linalg.lstsq(A, np.log(np.abs(U)), rcond=None)
    phase = np.unwrap(np.angle(U))
    pa, *_ = np.linalg.lstsq(A, phase, rcond=None)
    return float(-la[0]), float(omega / abs(pa[0]))


# ---------------------------------------------------------------------------
# 3D convolution (test reference for the learned warm start's kernels)
# ---------------------------------------------------------------------------

def conv3d_fwd(x, W, bias=None):
    """Direct-loop 3x3x3 convolution, zero padding 1. x: (nz, ny, nx, cin),
    W: (27, cin, cout) with tap t = (dz+1)*9 + (dy+1)*3 + (dx+1), bias: (cout,)."""
    nz, ny, nx, cin = x.shape
    cout = W.shape[2]
    x, xp = _d(x)
    W, wp = _d(W)
    bp = _null()
    if bias is not None:
        bias, bp = _d(bias)
    out, op = _d(np.zeros((nz, ny, nx, cout)))
    lib().or_conv3d_fwd(nx, ny, nz, cin, cout, xp, wp, bp, op)
    return out


def conv3d_bwd(x, W, g):
    """Gradients (d/dx, d/dW, d/dbias) of sum(g * conv3d_fwd(x, W, bias))."""
    nz, ny, nx, cin = x.shape
    cout = W.shape[2]
    x, xp = _d(x)
    W, wp = _d(W)
    g, gp = _d(g)
    gin, gip = _d(np.zeros_like(x))
    gW, gwp = _d(np.zeros_like(W))
    gb, gbp = _d(np.zeros(cout))
    lib().or_conv3d_bwd(nx, ny, nz, cin, cout, xp, wp, gp, gip, gwp, gbp)
    return gin, gW, gb


def xcorr_group_speed(traces, offsets, dt, ref=0):
    """Group speed from cross-correlation of traces at increasing lateral
    offsets (Sec. 4.4): the lag of each trace against the reference trace is
    the argmax of their full cross-correlation, refined by a 3-point parabola;
    the speed is the least-squares slope of offset against lag.
    traces: [n_steps, ns]; offsets: (ns,) metres."""
    tr = np.asarray(traces, np.float64)
    n = tr.shape[0]
    a = tr[:, ref] - tr[:, ref].mean()
    lags = []
    for s in range(tr.shape[1]):
        b = tr[:, s] - tr[:, s].mean()
        cc = np.correlate(b, a, mode="full")  # index n-1 is zero lag
        m = int(np.argmax(cc))
        shift = 0.0
        if 0 < m < len(cc) - 1:
            den = cc[m - 1] - 2 * cc[m] + cc[m + 1]
            if den != 0:
                shift = 0.5 * (cc[m - 1] - cc[m + 1]) / den
        lags.append((m - (n - 1) + shift) * dt)
    off = np.asarray(offsets, np.float64)
    return linear_fit_speed(off - off[ref], np.asarray(lags))
