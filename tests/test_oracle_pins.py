"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed-form
eigenvalues, exactness on quadratics, dense Kronecker solves, a sine-transform
direct solve, manufactured solutions, conserved energies, scalar recurrences of
single modes and the paper's stability bound.
"""
import numpy as np
import pytest

import oracle as orc

DX = 2e-4


def grid_coords(nx, ny, nz, dx=DX):
    x = (np.arange(nx) * dx)[None, None, :]
    y = (np.arange(ny) * dx)[None, :, None]
    z = (np.arange(nz) * dx)[:, None, None]
    return x, y, z


def interior_mask(nx, ny, nz):
    m = np.zeros((nz, ny, nx), bool)
    m[1:-1, 1:-1, 1:-1] = True
    return m


def sine_mode(nx, ny, nz, kx, ky, kz):
    """Discrete Dirichlet eigenvector prod sin(pi k_a i_a / (n_a - 1))."""
    i = np.arange(nx)
    j = np.arange(ny)
    k = np.arange(nz)
    sx = np.sin(np.pi * kx * i / (nx - 1))
    sy = np.sin(np.pi * ky * j / (ny - 1))
    sz = np.sin(np.pi * kz * k / (nz - 1))
    return sz[:, None, None] * sy[None, :, None] * sx[None, None, :]


def sine_eigenvalue(n_axes, k_axes, dx=DX):
    """-L s = lam s with lam = sum_a (4/dx^2) sin^2(pi k_a / (2 (n_a - 1)))."""
    return sum(4.0 / dx ** 2 * np.sin(np.pi * k / (2.0 * (n - 1))) ** 2
               for n, k in zip(n_axes, k_axes))


def dense_negative_laplacian(nx, ny, nz, dx=DX):
    """Textbook matrix of -L on interior unknowns: Kronecker sum of 1D second
    differences tridiag(1, -2, 1)/dx^2 (x fastest)."""
    def T(n):
        m = n - 2
        return (np.diag(-2.0 * np.ones(m)) + np.diag(np.ones(m - 1), 1)
                + np.diag(np.ones(m - 1), -1)) / dx ** 2
    Ix, Iy, Iz = (np.eye(n - 2) for n in (nx, ny, nz))
    L = (np.kron(Iz, np.kron(Iy, T(nx))) + np.kron(Iz, np.kron(T(ny), Ix))
         + np.kron(T(nz), np.kron(Iy, Ix)))
    return -L


def bump(nx, ny, nz, lo, hi, seed=0):
    """Smooth compactly supported bump: prod sin^4 over the node box [lo, hi],
    exactly zero outside it, times a fixed random polynomial-free scale."""
    out = np.zeros((nz, ny, nx))
    rng = np.random.default_rng(seed)
    def w(n, a, b):
        t = np.zeros(n)
        idx = np.arange(a, b + 1)
        t[idx] = np.sin(np.pi * (idx - a) / (b - a)) ** 4
        return t
    out[:] = (w(nz, lo[2], hi[2])[:, None, None] * w(ny, lo[1], hi[1])[None, :, None]
              * w(nx, lo[0], hi[0])[None, None, :])
    return out * (1.0 + rng.uniform())


# ---------------------------------------------------------------------------
# 7-point Laplacian (Sec. 3.1)
# ---------------------------------------------------------------------------

def test_laplacian_exact_on_quadratics():
    nx, ny, nz = 9, 7, 8
    x, y, z = grid_coords(nx, ny, nz)
    q = 3.0 * x ** 2 - 1.5 * y ** 2 + 0.25 * z ** 2 + 2.0 * x * y - 0.7 * y * z + 5 * x - 2 * z + 1
    q = np.broadcast_to(q, (nz, ny, nx))
    L = orc.laplacian(q, DX)
    m = interior_mask(nx, ny, nz)
    expect = 2 * (3.0 - 1.5 + 0.25)
    assert np.allclose(L[m], expect, rtol=1e-8, atol=1e-8 * abs(expect))
    assert np.all(L[~m] == 0.0)


@pytest.mark.parametrize("modes", [(1, 1, 1), (2, 3, 1), (5, 1, 4)])
def test_laplacian_sine_eigenvalues(modes):
    n = (12, 10, 11)
    s = sine_mode(*n, *modes)
    L = orc.laplacian(s, DX)
    lam = sine_eigenvalue(n, modes)
    m = interior_mask(*n)
    np.testing.assert_allclose(L[m], -lam * s[m], rtol=0, atol=1e-9 * lam)


def test_div_and_grad_on_linear_fields():
    nx, ny, nz = 8, 9, 7
    x, y, z = grid_coords(nx, ny, nz)
    sh = (nz, ny, nx)
    fx, fy, fz = (np.broadcast_to(v, sh) for v in (2.0 * x + y, -3.0 * y + z, 0.5 * z + x))
    d = orc.div_minus(fx, fy, fz, DX)
    m = interior_mask(nx, ny, nz)
    np.testing.assert_allclose(d[m], 2.0 - 3.0 + 0.5, rtol=1e-9)
    assert np.all(d[~m] == 0)
    phi = np.broadcast_to(4.0 * x - 2.0 * y + 7.0 * z, sh)
    gx, gy, gz = orc.grad_plus(phi, DX)
    np.testing.assert_allclose(gx[:, :, :-1], 4.0, rtol=1e-9)
    np.testing.assert_allclose(gy[:, :-1, :], -2.0, rtol=1e-9)
    np.testing.assert_allclose(gz[:-1, :, :], 7.0, rtol=1e-9)
    # phi = 0 beyond the last node
    np.testing.assert_allclose(gx[:, :, -1], -phi[:, :, -1] / DX, rtol=1e-12)


def test_div_of_grad_is_laplacian():
    """Mimetic pair: D-(D+ phi) = L phi on the interior when phi vanishes on the
    outer layer (brute-force check on a random field)."""
    n = (9, 8, 10)
    rng = np.random.default_rng(3)
    phi = rng.standard_normal(n[::-1])
    phi[~interior_mask(*n)] = 0
    g = orc.grad_plus(phi, DX)
    d = orc.div_minus(*g, DX)
    L = orc.laplacian(phi, DX)
    np.testing.assert_allclose(d, L, rtol=0, atol=1e-9 * np.abs(L).max())


# ---------------------------------------------------------------------------
# Masked CG (Sec. 3.2.3)
# ---------------------------------------------------------------------------

def test_cg_matches_dense_solve():
    nx, ny, nz = 8, 7, 9
    rng = np.random.default_rng(11)
    b = rng.standard_normal((nz, ny, nx))
    m = interior_mask(nx, ny, nz)
    b[~m] = 0
    A = dense_negative_laplacian(nx, ny, nz)
    x_dense = np.linalg.solve(A, b[1:-1, 1:-1, 1:-1].ravel())
    phi, status, st = orc.cg(b, DX, 1e-14, 1000)
    assert status == "converged"
    np.testing.assert_allclose(phi[1:-1, 1:-1, 1:-1].ravel(), x_dense, rtol=0,
                               atol=1e-12 * np.abs(x_dense).max())
    assert np.all(phi[~m] == 0)
    assert st["true_rel_res"] < 1e-12


def dst_solve(b, dx=DX):
    """Direct solve of -L phi = b by discrete sine transforms written from the
    eigen-decomposition: S_{pq} = sin(pi p q / (n - 1)), S^{-1} = 2/(n-1) S."""
    nz, ny, nx = b.shape
    def S(n):
        p = np.arange(1, n - 1)
        return np.sin(np.pi * np.outer(p, p) / (n - 1))
    Sx, Sy, Sz = S(nx), S(ny), S(nz)
    bi = b[1:-1, 1:-1, 1:-1]
    bh = np.einsum("ai,bj,ck,kji->cba", Sx, Sy, Sz, bi, optimize=True)
    lam = (4 / dx ** 2 * np.sin(np.pi * np.arange(1, nz - 1) / (2 * (nz - 1))) ** 2)[:, None, None] \
        + (4 / dx ** 2 * np.sin(np.pi * np.arange(1, ny - 1) / (2 * (ny - 1))) ** 2)[None, :, None] \
        + (4 / dx ** 2 * np.sin(np.pi * np.arange(1, nx - 1) / (2 * (nx - 1))) ** 2)[None, None, :]
    ph = bh / lam
    scale = (2.0 / (nx - 1)) * (2.0 / (ny - 1)) * (2.0 / (nz - 1))
    phi_i = scale * np.einsum("ai,bj,ck,kji->cba", Sx, Sy, Sz, ph, optimize=True)
    out = np.zeros_like(b)
    out[1:-1, 1:-1, 1:-1] = phi_i
    return out


def test_cg_matches_sine_transform_solve():
    nx, ny, nz = 26, 22, 30
    rng = np.random.default_rng(5)
    b = rng.standard_normal((nz, ny, nx))
    b[~interior_mask(nx, ny, nz)] = 0
    ref = dst_solve(b)
    phi, status, st = orc.cg(b, DX, 1e-13, 5000)
    assert status == "converged"
    np.testing.assert_allclose(phi, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_cg_stopping_rule_and_guards():
    nx = ny = nz = 12
    rng = np.random.default_rng(1)
    b = rng.standard_normal((nz, ny, nx))
    b[~interior_mask(nx, ny, nz)] = 0
    phi, status, st = orc.cg(b, DX, 1e-6, 1000)
    assert status == "converged" and st["rel_res"] < 1e-6
    # one iteration fewer must not have met the tolerance
    _, status2, st2 = orc.cg(b, DX, 1e-6, st["iters"] - 1)
    assert status2 == "maxiter" and st2["rel_res"] >= 1e-6
    # zero right-hand side: phi = 0, no iterations
    phi0, s0, st0 = orc.cg(np.zeros_like(b), DX, 1e-8, 100)
    assert s0 == "zero_rhs" and st0["iters"] == 0 and not phi0.any()
    # non-finite right-hand side
    bn = b.copy()
    bn[5, 5, 5] = np.nan
    _, sn, _ = orc.cg(bn, DX, 1e-8, 100)
    assert sn == "nonfinite"


def test_cg_eigenvector_rhs_converges_in_one_iteration():
    n = (10, 9, 11)
    s = sine_mode(*n, 2, 1, 3)
    lam = sine_eigenvalue(n, (2, 1, 3))
    phi, status, st = orc.cg(s, DX, 1e-12, 50)
    assert st["iters"] == 1 and status == "converged"
    np.testing.assert_allclose(phi, s / lam, atol=1e-12 * np.abs(s / lam).max())


# ---------------------------------------------------------------------------
# Solenoidal projection (Sec. 3.2.1, 3.3)
# ---------------------------------------------------------------------------

def backward_diff(q, axis, dx=DX):
    """D- along an axis (array axis order z, y, x), zero in the first slice."""
    out = np.zeros_like(q)
    sl_hi = [slice(None)] * 3
    sl_lo = [slice(None)] * 3
    sl_hi[axis] = slice(1, None)
    sl_lo[axis] = slice(0, -1)
    out[tuple(sl_hi)] = (q[tuple(sl_hi)] - q[tuple(sl_lo)]) / dx
    return out


def forward_diff(q, axis, dx=DX):
    out = np.zeros_like(q)
    sl_hi = [slice(None)] * 3
    sl_lo = [slice(None)] * 3
    sl_hi[axis] = slice(1, None)
    sl_lo[axis] = slice(0, -1)
    out[tuple(sl_lo)] = (q[tuple(sl_hi)] - q[tuple(sl_lo)]) / dx
    return out


def curl_minus(px, py, pz):
    """Curl built from backward differences; its backward divergence is zero."""
    X, Y, Z = 2, 1, 0
    cx = backward_diff(pz, Y) - backward_diff(py, Z)
    cy = backward_diff(px, Z) - backward_diff(pz, X)
    cz = backward_diff(py, X) - backward_diff(px, Y)
    return cx, cy, cz


def manufactured(n=(20, 18, 22)):
    nx, ny, nz = n
    phi_star = bump(nx, ny, nz, (3, 3, 4), (nx - 5, ny - 4, nz - 4), seed=1)
    psi = [bump(nx, ny, nz, (4 + a, 3, 3 + a), (nx - 6, ny - 5 + a, nz - 4), seed=2 + a)
           for a in range(3)]
    gx, gy, gz = (forward_diff(phi_star, ax) for ax in (2, 1, 0))
    cx, cy, cz = curl_minus(*psi)
    return phi_star, (gx, gy, gz), (cx, cy, cz)


def test_projection_recovers_manufactured_parts():
    phi_star, grad, curl = manufactured()
    f = [g + c for g, c in zip(grad, curl)]
    phi, fs, status, st = orc.project(*f, DX, tol=1e-13)
    assert status == "converged"
    np.testing.assert_allclose(phi, phi_star, atol=1e-9 * np.abs(phi_star).max())
    for a in range(3):
        np.testing.assert_allclose(fs[a], curl[a], atol=1e-9 * np.abs(curl[a]).max())


def test_projection_invariants():
    rng = np.random.default_rng(7)
    n = (18, 16, 20)
    nx, ny, nz = n
    f = [rng.standard_normal((nz, ny, nx)) for _ in range(3)]
    m = interior_mask(nx, ny, nz)
    phi, fs, status, st = orc.project(*f, DX, tol=1e-12)
    assert status == "converged"
    div_f = orc.div_minus(*f, DX)
    div_fs = orc.div_minus(*fs, DX)
    # ||D-.f_S|| / ||D-.f|| equals the true relative residual of the solve
    ratio = np.linalg.norm(div_fs) / np.linalg.norm(div_f)
    assert ratio < 1e-11
    assert ratio == pytest.approx(st["true_rel_res"], rel=1e-2, abs=1e-14)
    # idempotence: P(P f) = P f
    _, fs2, _, _ = orc.project(*fs, DX, tol=1e-12)
    for a in range(3):
        np.testing.assert_allclose(fs2[a], fs[a], atol=1e-9 * np.abs(fs[a]).max())
    # linearity
    g = [rng.standard_normal((nz, ny, nx)) for _ in range(3)]
    _, fsg, _, _ = orc.project(*g, DX, tol=1e-13)
    _, fsc, _, _ = orc.project(*[2.0 * a - 0.5 * b for a, b in zip(f, g)], DX, tol=1e-13)
    for a in range(3):
        np.testing.assert_allclose(fsc[a], 2.0 * fs[a] - 0.5 * fsg[a],
                                   atol=1e-9 * np.abs(fsc[a]).max())


def test_projection_removes_gradients():
    phi_star, grad, _ = manufactured()
    _, fs, status, _ = orc.project(*grad, DX, tol=1e-13)
    for a in range(3):
        assert np.abs(fs[a]).max() < 1e-9 * np.abs(grad[a]).max()


# ---------------------------------------------------------------------------
# Time stepping (Sec. 3.1)
# ---------------------------------------------------------------------------

def mode_coefficients(a_lam, b_lam, n_steps, c0=1.0, cm1=1.0):
    """Closed form of one Laplacian eigenmode under the recurrence:
    c_{n+1} = (2 - (a+b) lam) c_n - (1 - b lam) c_{n-1}, solved through the
    roots of z^2 - (2 - (a+b) lam) z + (1 - b lam) = 0."""
    p = 2.0 - a_lam - b_lam
    q = 1.0 - b_lam
    disc = np.sqrt(complex(p * p - 4 * q))
    z1, z2 = (p + disc) / 2, (p - disc) / 2
    # c_n = P z1^n + Q z2^n with c_0 = c0, c_{-1} = cm1
    M = np.array([[1, 1], [1 / z1, 1 / z2]])
    P, Q = np.linalg.solve(M, np.array([c0, cm1], complex))
    n = np.arange(1, n_steps + 1)
    return (P * z1 ** n + Q * z2 ** n).real


@pytest.mark.parametrize("eta", [0.0, 0.8])
def test_step_sine_mode_closed_form(eta):
    n = (12, 11, 13)
    nx, ny, nz = n
    G, rho = 4e3, 1000.0
    dt = 0.5 * orc.stable_dt(G, rho, eta, DX)
    modes = [(1, 2, 1), (3, 1, 2), (2, 2, 3)]
    u0 = [sine_mode(*n, *mk) for mk in modes]
    um = [0.9 * s for s in u0]  # c_{-1} = 0.9: the mode starts moving
    n_steps = 60
    sensors = np.array([[3, 4, 5], [7, 2, 9]], np.int32)
    tr, u_end, _ = orc.run(nx, ny, nz, DX, dt, G, rho, eta, n_steps, sensors,
                           u_in=u0, uprev_in=um, want_state=True)
    for c, mk in enumerate(modes):
        lam = sine_eigenvalue(n, mk)
        coef = mode_coefficients(dt * dt * G / rho * lam, dt * eta / rho * lam, n_steps,
                                 1.0, 0.9)
        for s, (i, j, k) in enumerate(sensors):
            np.testing.assert_allclose(tr[:, s, c], coef * u0[c][k, j, i], rtol=0,
                                       atol=1e-10 * abs(u0[c][k, j, i]) + 1e-14)
        np.testing.assert_allclose(u_end[c], coef[-1] * u0[c], atol=1e-10)


def energy(u_next, u_cur, A, dx=DX):
    """E^{n+1/2} = sum (u^{n+1}-u^n)^2 / A - <u^{n+1}, L u^n>, A = dt^2 mu/rho,
    with L written here with numpy slicing (interior, Dirichlet layer = 0)."""
    def lap(q):
        out = np.zeros_like(q)
        c = q[1:-1, 1:-1, 1:-1]
        out[1:-1, 1:-1, 1:-1] = (q[2:, 1:-1, 1:-1] + q[:-2, 1:-1, 1:-1] + q[1:-1, 2:, 1:-1]
                                 + q[1:-1, :-2, 1:-1] + q[1:-1, 1:-1, 2:] + q[1:-1, 1:-1, :-2]
                                 - 6 * c) / dx ** 2
        return out
    m = interior_mask(*u_cur.shape[1:][::-1])
    e = 0.0
    for c in range(3):
        v = (u_next[c] - u_cur[c])[m]
        e += np.sum(v * v / A[m]) - np.sum(u_next[c] * lap(u_cur[c]))
    return e


def test_step_conserves_weighted_energy_heterogeneous():
    """eta = 0, no force, pointwise mu(x)/rho(x): the leapfrog conserves
    E^{n+1/2} exactly (to rounding); any index or coefficient slip breaks it."""
    nx, ny, nz = 14, 12, 13
    rng = np.random.default_rng(21)
    mu = rng.uniform(1e3, 10e3, (nz, ny, nx))
    rho = rng.uniform(1000, 1100, (nz, ny, nx))
    dt = 0.5 * orc.stable_dt(mu, rho, 0.0, DX)
    u0 = [rng.standard_normal((nz, ny, nx)) * 1e-6 for _ in range(3)]
    um = [q * 0.97 for q in u0]
    A = dt * dt * mu / rho
    _, ua, uam = orc.run(nx, ny, nz, DX, dt, mu, rho, 0.0, 5, np.zeros((1, 3), np.int32),
                         u_in=u0, uprev_in=um, want_state=True)
    _, ub, ubm = orc.run(nx, ny, nz, DX, dt, mu, rho, 0.0, 137, np.zeros((1, 3), np.int32),
                         u_in=u0, uprev_in=um, want_state=True)
    ea = energy(ua, uam, A)
    eb = energy(ub, ubm, A)
    assert ea > 0
    assert abs(eb - ea) < 1e-10 * abs(ea)
    # with viscosity the same energy decays
    _, uc, ucm = orc.run(nx, ny, nz, DX, 0.5 * orc.stable_dt(mu, rho, 0.5, DX), mu, rho, 0.5, 137,
                         np.zeros((1, 3), np.int32), u_in=u0, uprev_in=um, want_state=True)
    dtv = 0.5 * orc.stable_dt(mu, rho, 0.5, DX)
    _, ud, udm = orc.run(nx, ny, nz, DX, dtv, mu, rho, 0.5, 5, np.zeros((1, 3), np.int32),
                         u_in=u0, uprev_in=um, want_state=True)
    Av = dtv * dtv * mu / rho
    assert energy(uc, ucm, Av) < energy(ud, udm, Av)


def test_stable_dt_reduces_to_paper_bound():
    """Sec. 3.1: at eta = 0, dt_max = (1/c_s) (3/dx^2)^(-1/2)."""
    for G in (1e3, 4e3, 50e3):
        c = np.sqrt(G / 1000.0)
        assert orc.stable_dt(G, 1000.0, 0.0, DX) == pytest.approx(DX / (c * np.sqrt(3)), rel=1e-14)
    # config 1 of the plain method: dt = 0.5 dx / (c sqrt 3) = 28.868 us
    assert 0.5 * orc.stable_dt(4e3, 1000.0, 0.0, DX) == pytest.approx(28.8675e-6, rel=1e-5)


def _grows(dt, eta, n_steps=400):
    nx = ny = nz = 16
    rng = np.random.default_rng(2)
    u0 = [rng.standard_normal((nz, ny, nx)) * 1e-6 for _ in range(3)]
    _, u, _ = orc.run(nx, ny, nz, DX, dt, 4e3, 1000.0, eta, n_steps, np.zeros((1, 3), np.int32),
                      u_in=u0, uprev_in=u0, want_state=True)
    return np.abs(u).max() > 1e-3


def test_stability_bound_separates_growth():
    bound0 = orc.stable_dt(4e3, 1000.0, 0.0, DX)
    assert not _grows(0.95 * bound0, 0.0)
    assert _grows(1.05 * bound0, 0.0)
    # with viscosity the eta = 0 bound is unstable; the viscous bound is not
    boundv = orc.stable_dt(4e3, 1000.0, 1.5, DX)
    assert boundv < 0.2 * bound0
    assert _grows(0.9 * bound0, 1.5, 200)
    assert not _grows(0.95 * boundv, 1.5, 2000)
    assert _grows(1.1 * boundv, 1.5, 2000)


def test_curl_source_symmetry():
    """Sec. 4.1: the curl source drives motion in x-z with u_z odd in x."""
    from paper_2607_28414_b300 import inputs
    n = 25
    v0 = inputs.curl_gaussian_velocity(n, n, n, DX, sigma=1e-3)
    c = n // 2
    sensors = np.array([[c + 4, c, c], [c - 4, c, c]], np.int32)
    dt = 0.5 * orc.stable_dt(4e3, 1000.0, 0.0, DX)
    tr = orc.run(n, n, n, DX, dt, 4e3, 1000.0, 0.0, 40, sensors, v0=v0)
    assert np.abs(tr[:, 0, 2]).max() > 0
    np.testing.assert_allclose(tr[:, 0, 2], -tr[:, 1, 2], atol=1e-12 * np.abs(tr).max())
    np.testing.assert_allclose(tr[:, 0, 1], 0.0, atol=1e-20)


def test_force_linearity_and_separable_envelope():
    """Sec. 3.3: with f = b0 g(t), doubling b0 doubles the response, and the
    envelope enters only through g(t_n)."""
    from paper_2607_28414_b300 import inputs
    n = 20
    f = inputs.gaussian_push(n, n, n, DX, 1e3, 1e-3, 2e-3)
    _, fs, _, _ = orc.project(*f, DX, tol=1e-12)
    dt = 0.5 * orc.stable_dt(4e3, 1000.0, 0.3, DX)
    g = inputs.push_envelope(30, dt, 5 * dt)
    sensors = np.array([[n // 2 + 3, n // 2, n // 2]], np.int32)
    t1 = orc.run(n, n, n, DX, dt, 4e3, 1000.0, 0.3, 30, sensors, fs=fs, g=g)
    t2 = orc.run(n, n, n, DX, dt, 4e3, 1000.0, 0.3, 30, sensors, fs=[2 * a for a in fs], g=g)
    t3 = orc.run(n, n, n, DX, dt, 4e3, 1000.0, 0.3, 30, sensors, fs=fs, g=2 * g)
    np.testing.assert_allclose(t2, 2 * t1, rtol=1e-12, atol=1e-30)
    np.testing.assert_allclose(t3, 2 * t1, rtol=1e-12, atol=1e-30)
    assert g.sum() == 5  # t_n < 5 dt for n = 0..4


# ---------------------------------------------------------------------------
# Divergence-form operator (heterogeneous variant of Sec. 3.1)
# ---------------------------------------------------------------------------

def test_divergence_form_reduces_to_pointwise_when_homogeneous():
    n = (14, 12, 13)
    rng = np.random.default_rng(9)
    u0 = [rng.standard_normal(n[::-1]) * 1e-6 for _ in range(3)]
    dt = 0.5 * orc.stable_dt(4e3, 1000.0, 0.6, DX)
    sens = np.array([[5, 5, 5], [9, 3, 7]], np.int32)
    a = orc.run(*n, DX, dt, 4e3, 1000.0, 0.6, 50, sens, u_in=u0, uprev_in=u0)
    b = orc.run(*n, DX, dt, 4e3, 1000.0, 0.6, 50, sens, u_in=u0, uprev_in=u0, divform=True)
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-12 * np.abs(a).max())


def test_divergence_form_conserves_its_energy():
    """eta = 0: rho (u^{n+1} - 2u^n + u^{n-1}) / dt^2 = K u^n with K symmetric,
    so E = sum rho (u^{n+1} - u^n)^2 / dt^2 - <u^{n+1}, K u^n> is conserved
    (K assembled here from face-averaged moduli with numpy slicing)."""
    nx, ny, nz = 13, 12, 11
    rng = np.random.default_rng(12)
    mu = rng.uniform(1e3, 10e3, (nz, ny, nx))
    rho = rng.uniform(1000, 1100, (nz, ny, nx))
    dt = 0.4 * orc.stable_dt(mu, rho, 0.0, DX)
    u0 = [rng.standard_normal((nz, ny, nx)) * 1e-6 for _ in range(3)]
    um = [q * 0.98 for q in u0]

    def K(q):
        out = np.zeros_like(q)
        c = (slice(1, -1),) * 3
        for ax in range(3):
            for sgn in (-1, 1):
                sl = [slice(1, -1)] * 3
                sl[ax] = slice(1 + sgn, q.shape[ax] - 1 + sgn)
                sl = tuple(sl)
                out[c] += 0.5 * (mu[c] + mu[sl]) * (q[sl] - q[c])
        return out / DX ** 2

    def E(un, uc):
        m = interior_mask(nx, ny, nz)
        return sum(np.sum(rho[m] * (un[c] - uc[c])[m] ** 2) / dt ** 2 - np.sum(un[c] * K(uc[c]))
                   for c in range(3))

    _, ua, uam = orc.run(nx, ny, nz, DX, dt, mu, rho, 0.0, 7, np.zeros((1, 3), np.int32),
                         u_in=u0, uprev_in=um, want_state=True, divform=True)
    _, ub, ubm = orc.run(nx, ny, nz, DX, dt, mu, rho, 0.0, 131, np.zeros((1, 3), np.int32),
                         u_in=u0, uprev_in=um, want_state=True, divform=True)
    ea, eb = E(ua, uam), E(ub, ubm)
    assert ea > 0 and abs(eb - ea) < 1e-10 * abs(ea)


def test_centred_push_mirror_symmetry():
    """A centred Gaussian push along z on a grid whose centre is a node drives
    u_z symmetric in x and y about the centre: the medium, the walls and f_z
    are mirror symmetric, and f_S,z = f_z - D+_z phi keeps the x and y mirror
    symmetry of phi."""
    from paper_2607_28414_b300 import inputs
    n = 21
    f = inputs.gaussian_push(n, n, n, DX, 1e3, 1e-3, 2e-3)
    _, fs, _, _ = orc.project(*f, DX, tol=1e-13)
    dt = 0.5 * orc.stable_dt(4e3, 1000.0, 0.4, DX)
    g = inputs.push_envelope(60, dt, 10 * dt)
    c = n // 2
    sensors = np.array([[c + 3, c, c], [c - 3, c, c], [c, c + 5, c], [c, c - 5, c]], np.int32)
    tr = orc.run(n, n, n, DX, dt, 4e3, 1000.0, 0.4, 60, sensors, fs=fs, g=g)
    scale = np.abs(tr[:, :, 2]).max()
    assert scale > 0
    np.testing.assert_allclose(tr[:, 0, 2], tr[:, 1, 2], rtol=0, atol=1e-10 * scale)
    np.testing.assert_allclose(tr[:, 2, 2], tr[:, 3, 2], rtol=0, atol=1e-10 * scale)
    # (u_x and u_y are driven by the forward-difference gradient of phi,
    # which lives half a node off the centre: they carry no such symmetry
    # once the walls at 0 and n - 1 reflect them.)


def test_divergence_form_energy_decays_with_viscosity():
    """eta > 0 in the flux form: the eta = 0 energy of the same K is not
    conserved but decreases."""
    nx, ny, nz = 12, 11, 10
    rng = np.random.default_rng(5)
    mu = rng.uniform(1e3, 10e3, (nz, ny, nx))
    rho = rng.uniform(1000, 1100, (nz, ny, nx))
    eta = rng.uniform(0.1, 1.0, (nz, ny, nx))
    dt = 0.4 * orc.stable_dt(mu, rho, eta, DX)
    u0 = [rng.standard_normal((nz, ny, nx)) * 1e-6 for _ in range(3)]
    um = [q * 0.98 for q in u0]

    def K(q):
        out = np.zeros_like(q)
        c = (slice(1, -1),) * 3
        for ax in range(3):
            for sgn in (-1, 1):
                sl = [slice(1, -1)] * 3
                sl[ax] = slice(1 + sgn, q.shape[ax] - 1 + sgn)
                sl = tuple(sl)
                out[c] += 0.5 * (mu[c] + mu[sl]) * (q[sl] - q[c])
        return out / DX ** 2

    def E(un, uc):
        m = interior_mask(nx, ny, nz)
        return sum(np.sum(rho[m] * (un[c] - uc[c])[m] ** 2) / dt ** 2 - np.sum(un[c] * K(uc[c]))
                   for c in range(3))

    es = []
    for n in (3, 30, 90):
        _, ua, uam = orc.run(nx, ny, nz, DX, dt, mu, rho, eta, n, np.zeros((1, 3), np.int32),
                             u_in=u0, uprev_in=um, want_state=True, divform=True)
        es.append(E(ua, uam))
    assert es[0] > es[1] > es[2] > 0


# ---------------------------------------------------------------------------
# Body force and initial velocity (Sec. 3.1 a^n with f_S/rho, Sec. 3.3, Sec. 3.5)
# ---------------------------------------------------------------------------

def test_first_forced_step_from_rest_is_dt2_f_over_rho():
    """From rest (u^0 = u^-1 = 0) the Laplacian terms vanish, so one step gives
    u^1 = dt^2 g_0 f_S / rho on every interior node and 0 on the Dirichlet
    layer, node by node, with a heterogeneous rho (a dropped 1/rho, a dt in
    place of dt^2 or a shifted index fails)."""
    nx, ny, nz = 9, 8, 7
    rng = np.random.default_rng(31)
    mu = rng.uniform(1e3, 10e3, (nz, ny, nx))
    rho = rng.uniform(900.0, 2000.0, (nz, ny, nx))
    eta = rng.uniform(0.0, 1.5, (nz, ny, nx))
    fs = [rng.standard_normal((nz, ny, nx)) * 1e3 for _ in range(3)]
    dt = 0.5 * orc.stable_dt(mu, rho, eta, DX)
    g0 = 0.7
    _, u1, u0 = orc.run(nx, ny, nz, DX, dt, mu, rho, eta, 1, np.zeros((1, 3), np.int32), fs=fs,
                        g=[g0], want_state=True)
    m = interior_mask(nx, ny, nz)
    for c in range(3):
        expect = np.where(m, dt * dt * g0 * fs[c] / rho, 0.0)
        np.testing.assert_allclose(u1[c], expect, rtol=1e-14, atol=0)
        assert not u0[c].any()


def test_second_forced_step_by_hand():
    """u^2 = 2u^1 - u^0 + dt^2 [(mu/rho) L u^1 + (eta/rho) L (u^1 - u^0)/dt + g_1 f_S/rho]
    with u^0 = 0 and u^1 = dt^2 g_0 f_S/rho, the Laplacian written here with
    numpy slicing; heterogeneous mu, rho, eta."""
    nx, ny, nz = 10, 9, 8
    rng = np.random.default_rng(32)
    mu = rng.uniform(1e3, 10e3, (nz, ny, nx))
    rho = rng.uniform(900.0, 2000.0, (nz, ny, nx))
    eta = rng.uniform(0.0, 1.5, (nz, ny, nx))
    fs = [rng.standard_normal((nz, ny, nx)) * 1e3 for _ in range(3)]
    dt = 0.5 * orc.stable_dt(mu, rho, eta, DX)
    g = [1.0, 0.4]
    _, u2, _ = orc.run(nx, ny, nz, DX, dt, mu, rho, eta, 2, np.zeros((1, 3), np.int32), fs=fs,
                       g=g, want_state=True)
    m = interior_mask(nx, ny, nz)

    def lap(q):
        out = np.zeros_like(q)
        out[1:-1, 1:-1, 1:-1] = (q[2:, 1:-1, 1:-1] + q[:-2, 1:-1, 1:-1] + q[1:-1, 2:, 1:-1]
                                 + q[1:-1, :-2, 1:-1] + q[1:-1, 1:-1, 2:] + q[1:-1, 1:-1, :-2]
                                 - 6 * q[1:-1, 1:-1, 1:-1]) / DX ** 2
        return out

    for c in range(3):
        u1 = np.where(m, dt * dt * g[0] * fs[c] / rho, 0.0)
        a = (mu / rho) * lap(u1) + (eta / rho) * lap(u1 / dt) + g[1] * fs[c] / rho
        expect = np.where(m, 2.0 * u1 + dt * dt * a, 0.0)
        np.testing.assert_allclose(u2[c], expect, rtol=1e-12, atol=1e-12 * np.abs(expect).max())


def forced_mode_coefficients(a_lam, b_lam, s, n_push, n_steps):
    """One Laplacian eigenmode driven from rest by a constant force of mode
    amplitude F for the first n_push steps, s = dt^2 F / rho:
    c_{n+1} = (2 - (a+b) lam) c_n - (1 - b lam) c_{n-1} + s [n < n_push].
    Closed form: during the push c_n = c_p + P z1^n + Q z2^n with the static
    part c_p = s / (a lam) (the constant solution) and P, Q from c_0 = c_-1 = 0;
    after it, the free recurrence from (c_{n_push}, c_{n_push - 1})."""
    p = 2.0 - a_lam - b_lam
    q = 1.0 - b_lam
    disc = np.sqrt(complex(p * p - 4 * q))
    z1, z2 = (p + disc) / 2, (p - disc) / 2
    cp = s / a_lam
    M = np.array([[1, 1], [1 / z1, 1 / z2]])
    P, Q = np.linalg.solve(M, np.array([-cp, -cp], complex))
    n = np.arange(0, n_push + 1)
    during = (cp + P * z1 ** n + Q * z2 ** n).real  # c_0 .. c_{n_push}
    # free part: c_{n_push + m} = R z1^m + T z2^m from (c_{n_push}, c_{n_push - 1})
    R, T = np.linalg.solve(M, np.array([during[-1], during[-2]], complex))
    m = np.arange(1, n_steps - n_push + 1)
    after = (R * z1 ** m + T * z2 ** m).real
    return np.concatenate([during[1:], after])  # c_1 .. c_{n_steps}


@pytest.mark.parametrize("eta", [0.0, 0.6])
def test_forced_sine_mode_closed_form(eta):
    """Sec. 3.1 + 3.3: a projected force equal to one sine mode (per component,
    different modes) with a step envelope g = 1 for the first 9 steps keeps u
    in that mode; its amplitude follows the forced closed form above, whose
    static part F / (G lam) is the solution of G (-L) u = F. This fixes the
    body-force term's 1/rho and dt^2, G and eta, and the envelope's timing."""
    n = (12, 11, 13)
    G, rho = 4e3, 1300.0
    dt = 0.5 * orc.stable_dt(G, rho, eta, DX)
    modes = [(1, 1, 2), (2, 1, 1), (1, 2, 1)]
    amps = [3e2, -5e2, 7e2]
    fs = [amp * sine_mode(*n, *mk) for amp, mk in zip(amps, modes)]
    n_steps, n_push = 50, 9
    g = np.r_[np.ones(n_push), np.zeros(n_steps - n_push)]
    sensors = np.array([[3, 4, 5], [7, 2, 9], [5, 5, 2]], np.int32)
    tr = orc.run(*n, DX, dt, G, rho, eta, n_steps, sensors, fs=fs, g=g)
    for c, (amp, mk) in enumerate(zip(amps, modes)):
        lam = sine_eigenvalue(n, mk)
        coef = forced_mode_coefficients(dt * dt * G / rho * lam, dt * eta / rho * lam,
                                        dt * dt * amp / rho, n_push, n_steps)
        for s, (i, j, k) in enumerate(sensors):
            shape = sine_mode(*n, *mk)[k, j, i]
            np.testing.assert_allclose(tr[:, s, c], coef * shape, rtol=0,
                                       atol=1e-10 * np.abs(coef).max())
    # the static part: a long push with viscosity settles at u = F / (G lam)
    if eta > 0:
        n_long = 3000
        tr = orc.run(*n, DX, dt, G, rho, eta, n_long, sensors, fs=fs, g=np.ones(n_long))
        for c, (amp, mk) in enumerate(zip(amps, modes)):
            i, j, k = sensors[0]
            static = amp * sine_mode(*n, *mk)[k, j, i] / (G * sine_eigenvalue(n, mk))
            assert tr[-1, 0, c] == pytest.approx(static, rel=1e-6)


@pytest.mark.parametrize("eta", [0.0, 0.5])
def test_initial_velocity_sine_mode_closed_form(eta):
    """Sec. 3.5 start with an initial velocity v0: u^0 = 0, u^-1 = -dt v0, so a
    v0 equal to a sine mode of amplitude V gives mode coefficients with c_0 = 0
    and c_-1 = -dt V (a sign slip or a missing dt fails); on top of a nonzero
    u^0 the start is u^-1 = u^0 - dt v0."""
    n = (11, 12, 10)
    G, rho = 4e3, 1000.0
    dt = 0.5 * orc.stable_dt(G, rho, eta, DX)
    modes = [(2, 1, 1), (1, 1, 1), (1, 3, 2)]
    V = [1e-3, 2e-3, -1.5e-3]
    v0 = [v * sine_mode(*n, *mk) for v, mk in zip(V, modes)]
    n_steps = 40
    sensors = np.array([[3, 4, 5], [6, 8, 2]], np.int32)
    tr = orc.run(*n, DX, dt, G, rho, eta, n_steps, sensors, v0=v0)
    u_start = [0.25e-6 * sine_mode(*n, *mk) for mk in modes]
    tr2 = orc.run(*n, DX, dt, G, rho, eta, n_steps, sensors, v0=v0, u_in=u_start)
    for c, (v, mk) in enumerate(zip(V, modes)):
        lam = sine_eigenvalue(n, mk)
        a, b = dt * dt * G / rho * lam, dt * eta / rho * lam
        coef = mode_coefficients(a, b, n_steps, 0.0, -dt * v)
        coef2 = mode_coefficients(a, b, n_steps, 0.25e-6, 0.25e-6 - dt * v)
        for s, (i, j, k) in enumerate(sensors):
            shape = sine_mode(*n, *mk)[k, j, i]
            np.testing.assert_allclose(tr[:, s, c], coef * shape, rtol=0,
                                       atol=1e-10 * np.abs(coef).max())
            np.testing.assert_allclose(tr2[:, s, c], coef2 * shape, rtol=0,
                                       atol=1e-10 * np.abs(coef2).max())
    # first step: u^1 = dt v0 + dt^2 a^0 with a^0 = (eta/rho) L v0 (u^0 = 0)
    c = 0
    lam = sine_eigenvalue(n, modes[c])
    i, j, k = sensors[0]
    expect = dt * V[c] * sine_mode(*n, *modes[c])[k, j, i] * (1.0 - dt * eta / rho * lam)
    assert tr[0, 0, c] == pytest.approx(expect, rel=1e-12)


# ---------------------------------------------------------------------------
# Exact discrete projection by sine transforms (large-grid reference)
# ---------------------------------------------------------------------------

def test_poisson_direct_matches_dense_solve_and_cg():
    """The transform solve equals the dense Kronecker solve of -L (tiny grid),
    the explicit sine-matrix solve and the oracle's CG at 1e-13."""
    nx, ny, nz = 7, 6, 8
    rng = np.random.default_rng(41)
    b = rng.standard_normal((nz, ny, nx))
    b[~interior_mask(nx, ny, nz)] = 0
    A = dense_negative_laplacian(nx, ny, nz)
    ref = np.zeros_like(b)
    ref[1:-1, 1:-1, 1:-1] = np.linalg.solve(A, b[1:-1, 1:-1, 1:-1].ravel()).reshape(
        nz - 2, ny - 2, nx - 2)
    np.testing.assert_allclose(orc.poisson_direct(b, DX), ref, rtol=0,
                               atol=1e-12 * np.abs(ref).max())
    nx, ny, nz = 26, 22, 30
    b = rng.standard_normal((nz, ny, nx))
    b[~interior_mask(nx, ny, nz)] = 0
    direct = orc.poisson_direct(b, DX)
    np.testing.assert_allclose(direct, dst_solve(b), rtol=0, atol=1e-12 * np.abs(direct).max())
    phi, status, _ = orc.cg(b, DX, 1e-13, 5000)
    assert status == "converged"
    np.testing.assert_allclose(direct, phi, rtol=0, atol=1e-10 * np.abs(direct).max())
    # values on the outer layer of b are ignored, as by the masked CG
    b2 = b.copy()
    b2[0] = 5.0
    np.testing.assert_array_equal(orc.poisson_direct(b2, DX), direct)


def test_project_direct_matches_cg_projection_and_is_solenoidal():
    from paper_2607_28414_b300 import inputs
    rng = np.random.default_rng(42)
    n = (33, 29, 31)
    f = inputs.beam_push(*n, DX, rng, focal_depth=2e-3, focal_len=1e-3)
    f = (f[2] * 0.5 + 10.0, f[1], f[2])
    phi_d, fs_d, res = orc.project_direct(*f, DX)
    assert res < 1e-13
    phi_c, fs_c, status, st = orc.project(*f, DX, tol=1e-13)
    assert status == "converged"
    np.testing.assert_allclose(phi_d, phi_c, rtol=0, atol=1e-11 * np.abs(phi_d).max())
    top = max(np.abs(a).max() for a in fs_d)
    for a, c in zip(fs_d, fs_c):
        np.testing.assert_allclose(a, c, rtol=0, atol=1e-11 * top)
    # D- . f_S = -(b - A phi): the divergence left is the residual
    b = -orc.div_minus(*f, DX)
    assert np.linalg.norm(orc.div_minus(*fs_d, DX)) <= 1e-13 * np.linalg.norm(b)
    # a gradient is removed entirely
    s = sine_mode(*n, 2, 3, 1)
    g = orc.grad_plus(s, DX)
    _, fs_g, _ = orc.project_direct(*g, DX)
    for a, ga in zip(fs_g, g):
        assert np.abs(a).max() <= 1e-12 * np.abs(ga).max()
