"""Seeded synthetic inputs for the reduced Kelvin-Voigt shear-wave solver.

This module builds the *inputs* of the method only: material maps (G, rho, eta),
body-force patterns b0(x), the temporal envelope table g(t_n), sensor lists and
initial velocity fields. It holds none of the method's arithmetic (no stencil,
no projection, no stability bound), so it can feed both the CUDA library and
the CPU oracle without sharing any computation between them.

Conventions
-----------
* Arrays are float32, C-contiguous, shape (nz, ny, nx): x is the fastest axis.
* Node (i, j, k) sits at x = i*dx, y = j*dx, z = k*dx. The outer node layer is
  the Dirichlet layer of the solver.
* Gaussians use the 1/e-width convention exp(-(r/sigma)^2), as in the QIBA
  force model of Sec. 4.4 (Eq. gaussexc).
* Workload recipes name the shapes of the paper's experiments: the Gaussian
  push (Sec. 4.4), soft-tissue moduli, densities and viscosities (Sec. 2.1,
  Sec. 5), a 200 us step push (Sec. 3.3: g(t)=1 during the push).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MM = 1e-3


def _axes(nx: int, ny: int, nz: int, dx: float, centre_ijk):
    ci, cj, ck = centre_ijk
    x = (np.arange(nx, dtype=np.float64) - ci) * dx
    y = (np.arange(ny, dtype=np.float64) - cj) * dx
    z = (np.arange(nz, dtype=np.float64) - ck) * dx
    return x[None, None, :], y[None, :, None], z[:, None, None]


def centre_node(nx: int, ny: int, nz: int):
    """Integer centre node (nx//2, ny//2, nz//2) so that sensors sit on nodes."""
    return (nx // 2, ny // 2, nz // 2)


def gaussian_push(nx, ny, nz, dx, amplitude=1e3, sigma_lat=1 * MM, sigma_ax=2 * MM,
                  centre_ijk=None, axis=2):
    """Separable Gaussian push b0 along one axis (default z).

    b_axis = A exp(-(lateral/sigma_lat)^2 - (axial/sigma_ax)^2), the other two
    components zero. Returns (fx, fy, fz) float32 arrays.
    """
    if centre_ijk is None:
        centre_ijk = centre_node(nx, ny, nz)
    x, y, z = _axes(nx, ny, nz, dx, centre_ijk)
    coords = [x, y, z]
    ax = coords[axis]
    lat = [c for a, c in enumerate(coords) if a != axis]
    val = amplitude * np.exp(-(lat[0] / sigma_lat) ** 2 - (lat[1] / sigma_lat) ** 2
                             - (ax / sigma_ax) ** 2)
    val = np.ascontiguousarray(np.broadcast_to(val, (nz, ny, nx)), dtype=np.float32)
    out = [np.zeros((nz, ny, nx), np.float32) for _ in range(3)]
    out[axis] = val
    return tuple(out)


def lognormal_speckle(rng, shape, sigma=0.3):
    """I.i.d. unit-mean lognormal speckle exp(sigma*xi - sigma^2/2), xi ~ N(0,1)."""
    xi = rng.standard_normal(shape)
    return np.exp(sigma * xi - 0.5 * sigma * sigma)


def beam_push(nx, ny, nz, dx, rng, amplitude=1e3, core=1 * MM, focal_depth=10 * MM,
              focal_len=4 * MM, speckle_sigma=0.3, axis_ij=None, z0=0.0):
    """Non-separable axial beam force f_z: Gaussian core around the beam axis,
    Gaussian focal zone along z, times lognormal speckle.

    f_z = A exp(-(r_perp/core)^2) exp(-((z - z0 - focal_depth)/focal_len)^2) * S(x)
    The beam enters from the z = z0 face; its axis passes through node columns
    axis_ij = (i, j) (default: the x-y centre).
    """
    if axis_ij is None:
        axis_ij = (nx // 2, ny // 2)
    x, y, _ = _axes(nx, ny, nz, dx, (axis_ij[0], axis_ij[1], 0))
    z = (np.arange(nz, dtype=np.float64) * dx)[:, None, None]
    core_prof = np.exp(-(x * x + y * y) / core ** 2)
    ax_prof = np.exp(-((z - z0 - focal_depth) / focal_len) ** 2)
    fz = amplitude * core_prof * ax_prof
    fz = fz * lognormal_speckle(rng, (nz, ny, nx), speckle_sigma)
    fz = np.ascontiguousarray(fz, dtype=np.float32)
    z0s = np.zeros((nz, ny, nx), np.float32)
    return z0s, z0s.copy(), fz


@dataclass
class Inclusion:
    centre: tuple  # metres (x, y, z)
    radius: float
    G: float
    rho: float
    eta: float


def spherical_inclusions(nx, ny, nz, dx, rng, n=8, G_bg=3e3, rho_bg=1000.0, eta_bg=0.5,
                         r_range=(2 * MM, 6 * MM), G_range=(1e3, 10e3),
                         rho_range=(1000.0, 1100.0), eta_range=(0.0, 1.5), margin=1 * MM):
    """Heterogeneous medium: background plus n seeded spheres.

    Each sphere draws r ~ U(r_range), a centre uniform inside the box with a wall
    margin of r + margin, and G, rho, eta uniform in their ranges. A later sphere
    overwrites an earlier one where they overlap. Returns (G, rho, eta, list).
    """
    L = np.array([(nx - 1) * dx, (ny - 1) * dx, (nz - 1) * dx])
    G = np.full((nz, ny, nx), G_bg, np.float64)
    rho = np.full((nz, ny, nx), rho_bg, np.float64)
    eta = np.full((nz, ny, nx), eta_bg, np.float64)
    x = (np.arange(nx) * dx)[None, None, :]
    y = (np.arange(ny) * dx)[None, :, None]
    z = (np.arange(nz) * dx)[:, None, None]
    incl = []
    for _ in range(n):
        r = rng.uniform(*r_range)
        c = [rng.uniform(r + margin, L[a] - r - margin) for a in range(3)]
        g = rng.uniform(*G_range)
        rh = rng.uniform(*rho_range)
        et = rng.uniform(*eta_range)
        inside = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 <= r * r
        G[inside] = g
        rho[inside] = rh
        eta[inside] = et
        incl.append(Inclusion(tuple(c), r, g, rh, et))
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return f32(G), f32(rho), f32(eta), incl


def push_envelope(n_steps, dt, t_push):
    """Step envelope of a push: g_n = 1 while t_n = n*dt < t_push, else 0."""
    n = np.arange(n_steps, dtype=np.float64)
    return (n * dt < t_push).astype(np.float32)


def pulsed_envelope(n_steps, dt, t_on, t_off, n_pulses):
    """Pulsed push train: n_pulses repetitions of t_on on, t_off off."""
    t = np.arange(n_steps, dtype=np.float64) * dt
    period = t_on + t_off
    idx = np.floor(t / period)
    on = (t - idx * period) < t_on
    return (on & (idx < n_pulses)).astype(np.float32)


def harmonic_envelope(n_steps, dt, omega, t_ramp):
    """Harmonic drive g_n = r(t_n) sin(omega t_n), t_n = n dt, with a
    raised-cosine ramp r = (1 - cos(pi t / t_ramp)) / 2 for t < t_ramp."""
    t = np.arange(n_steps, dtype=np.float64) * dt
    r = np.where(t < t_ramp, 0.5 * (1.0 - np.cos(np.pi * t / max(t_ramp, 1e-300))), 1.0)
    return (r * np.sin(omega * t)).astype(np.float32)


def line_sensors(start_ijk, axis, stop, stride=1):
    """Sensors along one axis from start_ijk (inclusive) to stop (exclusive)."""
    pts = []
    for s in range(start_ijk[axis], stop, stride):
        p = list(start_ijk)
        p[axis] = s
        pts.append(p)
    return np.asarray(pts, dtype=np.int32).reshape(-1, 3)


def curl_gaussian_velocity(nx, ny, nz, dx, sigma=3 * MM, peak=1e-3, centre_ijk=None,
                           envelope="xy"):
    """Divergence-free initial velocity v0 = curl(psi * e_y).

    envelope="xy": psi = exp(-(x^2 + y^2)/sigma^2), a Gaussian envelope in the
    x-y plane (Sec. 4.1), so v0 = (0, 0, d(psi)/dx): z motion, odd in x.
    envelope="xyz": psi = exp(-r^2/sigma^2), v0 = (-d(psi)/dz, 0, d(psi)/dx).
    Analytic derivatives at nodes, scaled to a peak speed `peak`.
    """
    if centre_ijk is None:
        centre_ijk = centre_node(nx, ny, nz)
    x, y, z = _axes(nx, ny, nz, dx, centre_ijk)
    if envelope == "xy":
        psi = np.exp(-(x * x + y * y) / sigma ** 2) + 0.0 * z
        vx = np.zeros((nz, ny, nx))
    elif envelope == "xyz":
        psi = np.exp(-(x * x + y * y + z * z) / sigma ** 2)
        vx = np.broadcast_to((2.0 * z / sigma ** 2) * psi, (nz, ny, nx))
    else:
        raise ValueError(envelope)
    vz = np.broadcast_to(-(2.0 * x / sigma ** 2) * psi, (nz, ny, nx))
    s = peak / float(np.sqrt(vx * vx + vz * vz).max())
    f32 = lambda a: np.ascontiguousarray(a * s, dtype=np.float32)
    return f32(vx), np.zeros((nz, ny, nx), np.float32), f32(vz)


# ---------------------------------------------------------------------------
# Workload recipes
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    """One synthetic problem: grid, medium, force pattern, envelope, sensors.

    dt is not part of a workload: the caller takes `cfl_fraction` of the
    stability limit computed by the solver (or by the oracle in tests).
    """
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    G: object  # float (homogeneous) or float32 array (nz, ny, nx)
    rho: object
    eta: object
    force: tuple  # (fx, fy, fz) float32 arrays
    t_push: float
    n_steps: int
    sensors: np.ndarray
    tol: float
    cfl_fraction: float = 0.5
    extra: dict = field(default_factory=dict)

    @property
    def n_cells(self):
        return self.nx * self.ny * self.nz


def homogeneous_push(n=64, dx=0.2 * MM, G=4e3, rho=1000.0, eta=0.0, n_steps=400,
                     t_push=200e-6, tol=1e-10, name=None, ny=None, nz=None):
    """Plain method on a homogeneous grid with the separable Gaussian push along z
    (sigma 1 mm lateral, 2 mm axial, centred, 1e3 N/m^3), sensors on the x line
    through the centre from the centre to the last interior node."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    nx = n
    c = centre_node(nx, ny, nz)
    force = gaussian_push(nx, ny, nz, dx, 1e3, 1 * MM, 2 * MM, c, axis=2)
    sensors = line_sensors(c, 0, nx - 1, 1)
    return Workload(name or f"homogeneous_{nx}x{ny}x{nz}", nx, ny, nz, dx, float(G), float(rho),
                    float(eta), force, t_push, n_steps, sensors, tol)


def heterogeneous_inclusions(n=256, dx=0.2 * MM, seed=102, n_steps=2000, t_push=200e-6,
                             tol=1e-8, n_incl=8, name=None):
    """Heterogeneous medium with 8 seeded spherical inclusions and a speckled
    axial beam focused 10 mm below the z = 0 face; sensors every second node
    on the x line at the focal depth."""
    rng = np.random.default_rng(seed)
    G, rho, eta, incl = spherical_inclusions(n, n, n, dx, rng, n=n_incl)
    force = beam_push(n, n, n, dx, rng)
    kf = int(round(10 * MM / dx))
    sensors = line_sensors((1, n // 2, kf), 0, n - 1, 2)
    return Workload(name or f"heterogeneous_inclusions_{n}^3", n, n, n, dx, G, rho, eta, force,
                    t_push, n_steps, sensors, tol, extra={"inclusions": incl, "seed": seed})


def smooth_field(rng, shape, dx, corr, lo, hi, coarse=8):
    """Smooth random field with correlation length ~corr, affinely mapped to
    [lo, hi]: Gaussian white noise on a lattice of spacing `coarse` nodes,
    Gaussian-filtered (sigma = corr), trilinearly interpolated to `shape`."""
    from scipy.ndimage import gaussian_filter, map_coordinates
    cshape = tuple(max(4, s // coarse + 2) for s in shape)
    w = gaussian_filter(rng.standard_normal(cshape), sigma=corr / (coarse * dx), mode="wrap")
    w = (w - w.min()) / max(w.max() - w.min(), 1e-30)
    axes = [np.arange(s, dtype=np.float64) / coarse for s in shape]
    out = np.empty(shape, np.float32)
    # interpolate plane by plane (z) to bound memory
    zz = axes[0]
    yy, xx = np.meshgrid(axes[1], axes[2], indexing="ij")
    for k in range(shape[0]):
        coords = np.stack([np.full_like(yy, zz[k]), yy, xx])
        out[k] = map_coordinates(w, coords, order=1, mode="nearest")
    return lo + (hi - lo) * out


def bone_shell(nx=512, ny=512, nz=384, dx=0.15 * MM, seed=105, n_steps=5000, t_push=200e-6,
               tol=1e-8, R=40 * MM, centre_above=30 * MM, focus_below=8 * MM, name=None):
    """Large heterogeneous medium: a curved bone shell (spherical cap of inner
    radius R, centre `centre_above` above the z = 0 face on the x-y centre line,
    thickness 3-7 mm from a smooth random field over the angle; G = 50 kPa,
    rho = 1900, eta = 2 Pa s) in soft tissue (G smooth in [1, 5] kPa, rho 1040,
    eta smooth in [0.3, 1.0] Pa s). A speckled axial beam from the top face is
    focused `focus_below` beneath the shell on the axis; sensors every second
    node on the x line at the focal depth."""
    rng = np.random.default_rng(seed)
    shape = (nz, ny, nx)
    G = smooth_field(rng, shape, dx, 5 * MM, 1e3, 5e3)
    eta = smooth_field(rng, shape, dx, 5 * MM, 0.3, 1.0)
    rho = np.full(shape, 1040.0, np.float32)
    cx, cy, cz = (nx // 2) * dx, (ny // 2) * dx, -centre_above
    # thickness over the cap: a smooth 2D field on (x, y), mapped to [3, 7] mm
    thick2d = smooth_field(rng, (1, ny, nx), dx, 5 * MM, 3 * MM, 7 * MM)[0].astype(np.float64)
    y = (np.arange(ny) * dx - cy)[:, None]
    x = (np.arange(nx) * dx - cx)[None, :]
    r_perp2 = x * x + y * y
    for k in range(nz):
        z = k * dx - cz
        r = np.sqrt(r_perp2 + z * z)
        bone = (r >= R) & (r <= R + thick2d)
        G[k][bone] = 50e3
        rho[k][bone] = 1900.0
        eta[k][bone] = 2.0
    z_shell_out = cz + R + float(thick2d[ny // 2, nx // 2])
    focal_depth = z_shell_out + focus_below
    force = beam_push(nx, ny, nz, dx, rng, focal_depth=focal_depth)
    kf = int(round(focal_depth / dx))
    sensors = line_sensors((1, ny // 2, kf), 0, nx - 1, 2)
    return Workload(name or f"bone_shell_{nx}x{ny}x{nz}", nx, ny, nz, dx, G, rho, eta, force,
                    t_push, n_steps, sensors, tol,
                    extra={"seed": seed, "focal_depth_m": focal_depth, "shell_axis_m": z_shell_out})


def sweep_cases(n_steps=1000, dx=0.2 * MM, eta_cases=16, g_cases=10, eta_grid=(128, 128, 192),
                edge_range=(96, 224)):
    """Parameter sweep: eta_cases homogeneous media with eta = linspace(0, 1.5)
    Pa s at G = 4 kPa on one eta_grid (nx, ny, nz), plus g_cases cubes with
    G = linspace(1, 10) kPa (eta = 0) whose edge grows with the wavelength,
    n = round(e0 + (e1 - e0) (sqrt(G/1 kPa) - 1) / (sqrt(10) - 1)); rho = 1000;
    each with the centred Gaussian push along z (sigma 1 mm lateral, 2 mm
    axial, 200 us) and x-line sensors from the centre."""
    cases = []
    nx, ny, nz = eta_grid
    for eta in np.linspace(0.0, 1.5, eta_cases):
        c = centre_node(nx, ny, nz)
        cases.append(Workload(f"sweep_eta{eta:.2f}_{nx}x{ny}x{nz}", nx, ny, nz, dx, 4e3, 1000.0,
                              float(eta), gaussian_push(nx, ny, nz, dx, 1e3, 1 * MM, 2 * MM, c),
                              200e-6, n_steps, line_sensors(c, 0, nx - 1, 1), 1e-8))
    e0, e1 = edge_range
    for G in np.linspace(1e3, 10e3, g_cases):
        n = int(round(e0 + (e1 - e0) * (np.sqrt(G / 1e3) - 1.0) / (np.sqrt(10.0) - 1.0)))
        c = centre_node(n, n, n)
        cases.append(Workload(f"sweep_G{G / 1e3:.0f}kPa_{n}^3", n, n, n, dx, float(G), 1000.0, 0.0,
                              gaussian_push(n, n, n, dx, 1e3, 1 * MM, 2 * MM, c), 200e-6, n_steps,
                              line_sensors(c, 0, n - 1, 1), 1e-8))
    return cases


def random_gaussian_forces_torch(n_fields, shape, dx, seed, device, speckle_sigma=0.3):
    """Generator of force fields for the learned warm start: each field is a sum
    of 1-4 anisotropic Gaussians (centre uniform in the middle half of the box,
    uniformly random rotation from a unit quaternion, 1/e widths U[0.5, 4] mm per
    axis, amplitude 1e3 * lognormal(0, 1) along a random unit direction) times
    unit-mean lognormal speckle. Built with torch on `device` (input
    construction only). Yields (fx, fy, fz) float32 tensors of shape (nz, ny, nx)."""
    import torch
    nx, ny, nz = shape
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    zc = (torch.arange(nz, device=device, dtype=torch.float32) * dx)[:, None, None]
    yc = (torch.arange(ny, device=device, dtype=torch.float32) * dx)[None, :, None]
    xc = (torch.arange(nx, device=device, dtype=torch.float32) * dx)[None, None, :]
    L = torch.tensor([(nx - 1) * dx, (ny - 1) * dx, (nz - 1) * dx], device=device)
    for _ in range(n_fields):
        f = [torch.zeros((nz, ny, nx), device=device) for _ in range(3)]
        k = int(torch.randint(1, 5, (1,), generator=g, device=device).item())
        for _ in range(k):
            c = (0.25 + 0.5 * torch.rand(3, generator=g, device=device)) * L
            q = torch.randn(4, generator=g, device=device)
            q = q / q.norm()
            a, b_, cq, d = q.tolist()
            R = torch.tensor([[a * a + b_ * b_ - cq * cq - d * d, 2 * (b_ * cq - a * d), 2 * (b_ * d + a * cq)],
                              [2 * (b_ * cq + a * d), a * a - b_ * b_ + cq * cq - d * d, 2 * (cq * d - a * b_)],
                              [2 * (b_ * d - a * cq), 2 * (cq * d + a * b_), a * a - b_ * b_ - cq * cq + d * d]],
                             device=device)
            sig = (0.5 + 3.5 * torch.rand(3, generator=g, device=device)) * MM
            amp = 1e3 * float(torch.exp(torch.randn(1, generator=g, device=device)).item())
            dvec = torch.randn(3, generator=g, device=device)
            dvec = dvec / dvec.norm()
            rx, ry, rz = xc - c[0], yc - c[1], zc - c[2]
            e = 0.0
            for ax in range(3):  # coordinate along the rotated axis ax
                proj = R[0, ax] * rx + R[1, ax] * ry + R[2, ax] * rz
                e = e + (proj / sig[ax]) ** 2
            gauss = amp * torch.exp(-e)
            for comp in range(3):
                f[comp] = f[comp] + float(dvec[comp]) * gauss
        speck = torch.exp(speckle_sigma * torch.randn((nz, ny, nx), generator=g, device=device)
                          - 0.5 * speckle_sigma ** 2)
        yield tuple((fc * speck).contiguous() for fc in f)


def qiba_phantom(G, nx=240, ny=200, nz=200, dx=0.25 * MM, x_f=30 * MM, sigma=(4.3 * MM, 0.62 * MM, 1.1 * MM),
                 t_push=167e-6, n_steps=None, offsets=(4 * MM, 14 * MM), name=None):
    """QIBA-shaped elastic phantom (Sec. 4.4): homogeneous G, rho = 1000, eta = 0;
    Gaussian body force along x (axial) b = A exp(-((x - x_f)/sx)^2 - (y/sy)^2 -
    (z/sz)^2) with 1/e widths (4.3, 0.62, 1.1) mm, focus at x_f = 30 mm on the
    y-z centre line, pushed for 167 us; sensors every node along y (lateral) at
    the focal depth from offsets[0] to offsets[1]. n_steps defaults to the time
    the shear wave needs to pass the farthest sensor plus its width."""
    cj, ck = ny // 2, nz // 2
    i_f = int(round(x_f / dx))
    x = ((np.arange(nx) - i_f) * dx)[None, None, :]
    y = ((np.arange(ny) - cj) * dx)[None, :, None]
    z = ((np.arange(nz) - ck) * dx)[:, None, None]
    bx = 1e3 * np.exp(-(x / sigma[0]) ** 2 - (y / sigma[1]) ** 2 - (z / sigma[2]) ** 2)
    bx = np.ascontiguousarray(np.broadcast_to(bx, (nz, ny, nx)), dtype=np.float32)
    zero = np.zeros((nz, ny, nx), np.float32)
    j0, j1 = cj + int(round(offsets[0] / dx)), cj + int(round(offsets[1] / dx))
    sensors = line_sensors((i_f, j0, ck), 1, j1 + 1, 1)
    c = np.sqrt(G / 1000.0)
    if n_steps is None:
        n_steps = 0  # set by the caller from dt: (offsets[1] + 6 mm) / c + t_push
    w = Workload(name or f"qiba_G{G / 1e3:.0f}kPa_{nx}x{ny}x{nz}", nx, ny, nz, dx, float(G), 1000.0, 0.0,
                 (bx, zero, zero.copy()), t_push, n_steps, sensors, 1e-8,
                 extra={"offsets_m": (np.arange(j0, j1 + 1) - cj) * dx, "t_window_s": (offsets[1] + 6 * MM) / c + t_push})
    return w


def guided_mode_case(nx, ny, nz, dx, G, rho, eta, src_i, sensor_i, amp=1e3, src_w=1.5,
                     name=None):
    """Harmonic-benchmark geometry on a 3D grid with Dirichlet walls: a force
    whose z component has the separable shape h(x) s(y) s(z), s the first
    Dirichlet sine mode of the cross-section (s_j = sin(pi j / (n - 1))).

    The force is the forward-difference curl of Psi = y_hat psi,
    psi = H(x) s(y) s(z), H(i) = amp exp(-((i - src_i) / src_w)^2):
    f_x = -(psi_{k+1} - psi_k) / dx, f_y = 0, f_z = (psi_{i+1} - psi_i) / dx
    (psi = 0 beyond the grid). Its backward-difference divergence vanishes on
    every interior node, so the projection leaves it unchanged up to rounding.
    Sensors on the x line through the centre of the cross-section at nodes
    sensor_i (ny, nz odd so that the centre is a node)."""
    assert ny % 2 == 1 and nz % 2 == 1
    i = np.arange(nx, dtype=np.float64)
    H = amp * np.exp(-((i - src_i) / src_w) ** 2)
    sy = np.sin(np.pi * np.arange(ny) / (ny - 1))
    sz = np.sin(np.pi * np.arange(nz) / (nz - 1))
    psi = sz[:, None, None] * sy[None, :, None] * H[None, None, :]
    pad_x = np.concatenate([psi, np.zeros((nz, ny, 1))], axis=2)
    pad_z = np.concatenate([psi, np.zeros((1, ny, nx))], axis=0)
    fz = (pad_x[:, :, 1:] - pad_x[:, :, :-1]) / dx
    fx = -(pad_z[1:] - pad_z[:-1]) / dx
    fy = np.zeros_like(fz)
    sensors = np.stack([np.asarray(sensor_i, np.int32),
                        np.full(len(sensor_i), ny // 2, np.int32),
                        np.full(len(sensor_i), nz // 2, np.int32)], axis=1)
    return Workload(name or f"guided_mode_{nx}x{ny}x{nz}_eta{eta:g}", nx, ny, nz, dx, G, rho, eta,
                    (fx.astype(np.float32), fy.astype(np.float32), fz.astype(np.float32)), 0.0, 0,
                    sensors, 1e-8)
