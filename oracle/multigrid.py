"""FP64 oracle of the multigrid preconditioner of projection modes 4 and 5.

TEST INFRASTRUCTURE ONLY (like the rest of this package): the tests compare
the library's kv_apply_preconditioner with vcycle() below; nothing in the
product path imports it. The paper's projection (Sec. 3.2.3) solves
A phi = b with A = -L (7-point Laplacian, phi = 0 on the outer layer) by plain
CG; the library's mode 4 preconditions that CG with one symmetric V(1,1)-cycle
M, written out here step by step in plain NumPy:

  levels   the interior cells of the grid are level 0; a level of n cells per
           axis coarsens to ceil(n/2) (coarse cell I covers fine cells 2I-1 and
           2I, 1-based), spacing doubled, until a level has at most 64 cells or
           fewer than 4 along an axis
  S        damped Jacobi: S = omega h^2 / 6, omega = 6/7
  A u      (6 u - sum of the six neighbours) / h^2, neighbours off the level 0
  R t      coarse I: (1/8) sum over the fine cells 2I-2 .. 2I+1 per axis of
           w_a w_b w_c t with w = (1/4, 3/4, 3/4, 1/4)
  P e      fine i: per axis 3/4 of the nearer coarse cell (i+1) // 2 and 1/4 of
           the farther one (one lower for odd i, one higher for even i)
  cycle    z1 = S r; r_c = R (r - A z1); e_c = M_c r_c (recursively);
           z2 = z1 + P e_c; z = z2 + S (r - A z2)
  coarsest e = S r, then 32 sweeps e <- e + S (r - A e)
  one level (too small to coarsen): z = S r

Pins: tests/test_oracle_multigrid.py (symmetry and positivity of M, R = P^T/8
from the matrices of the two maps, M against the two-level closed form
(2S - SAS) + (I - SA) P M_c R (I - AS) in dense matrices, contraction of the
two-grid and V-cycle iterations, the one-level case).
"""
from __future__ import annotations

import numpy as np

OMEGA = 6.0 / 7.0
COARSE_SWEEPS = 32
W4 = (0.25, 0.75, 0.75, 0.25)


def levels(n, h2):
    """[(nx, ny, nz, h^2)] from the interior cells n = (nx, ny, nz) down."""
    out = [(int(n[0]), int(n[1]), int(n[2]), float(h2))]
    while len(out) < 12:
        nx, ny, nz, hh = out[-1]
        if nx * ny * nz <= 64 or min(nx, ny, nz) < 4:
            break
        out.append(((nx + 1) // 2, (ny + 1) // 2, (nz + 1) // 2, 4.0 * hh))
    return out


def apply_A(u, h2):
    """(6 u - sum of the six neighbours) / h^2 on an array of interior cells
    (axes z, y, x), neighbours outside the array are 0."""
    p = np.pad(u, 1)
    s = (p[:-2, 1:-1, 1:-1] + p[2:, 1:-1, 1:-1] + p[1:-1, :-2, 1:-1] + p[1:-1, 2:, 1:-1]
         + p[1:-1, 1:-1, :-2] + p[1:-1, 1:-1, 2:])
    return (6.0 * u - s) / h2


def restrict(t, nc):
    """R t onto nc = (ncx, ncy, ncz) coarse cells: the 4 x 4 x 4 weighted sum / 8."""
    ncx, ncy, ncz = nc
    nz, ny, nx = t.shape
    # fine cells 0 .. 2 nc + 1 (1-based fine index 2I-2+a for I = 1..nc, a = 0..3)
    tp = np.zeros((2 * ncz + 2, 2 * ncy + 2, 2 * ncx + 2))
    tp[1:nz + 1, 1:ny + 1, 1:nx + 1] = t
    out = np.zeros((ncz, ncy, ncx))
    for c in range(4):
        for b in range(4):
            for a in range(4):
                out += W4[c] * W4[b] * W4[a] * tp[c:c + 2 * ncz:2, b:b + 2 * ncy:2, a:a + 2 * ncx:2]
    return out / 8.0


def _near_far(n):
    """1-based nearer and farther coarse cell of fine cells 1..n."""
    i = np.arange(1, n + 1)
    near = (i + 1) // 2
    far = np.where(i % 2 == 1, near - 1, near + 1)
    return near, far


def prolong(e, n):
    """P e onto n = (nx, ny, nz) fine cells (trilinear, coarse cells outside 0)."""
    nx, ny, nz = n
    ep = np.pad(e, 1)  # 1-based coarse indices, 0 and nc + 1 are zero
    (xn, xf), (yn, yf), (zn, zf) = _near_far(nx), _near_far(ny), _near_far(nz)
    out = np.zeros((nz, ny, nx))
    for zi, wz in ((zn, 0.75), (zf, 0.25)):
        for yi, wy in ((yn, 0.75), (yf, 0.25)):
            for xi, wx in ((xn, 0.75), (xf, 0.25)):
                out += wz * wy * wx * ep[np.ix_(zi, yi, xi)]
    return out


def _cycle(r, lv, l):
    nx, ny, nz, h2 = lv[l]
    S = OMEGA * h2 / 6.0
    if len(lv) == 1:
        return S * r
    if l == len(lv) - 1:  # coarsest level: damped Jacobi from S r
        e = S * r
        for _ in range(COARSE_SWEEPS):
            e = e + S * (r - apply_A(e, h2))
        return e
    z1 = S * r
    ncx, ncy, ncz, _ = lv[l + 1]
    rc = restrict(r - apply_A(z1, h2), (ncx, ncy, ncz))
    ec = _cycle(rc, lv, l + 1)
    z2 = z1 + prolong(ec, (nx, ny, nz))
    return z2 + S * (r - apply_A(z2, h2))


def vcycle(r, dx):
    """z = M r on the interior cells of r (axes z, y, x) for grid spacing dx."""
    r = np.asarray(r, dtype=np.float64)
    lv = levels((r.shape[2], r.shape[1], r.shape[0]), dx * dx)
    return _cycle(r, lv, 0)


def vcycle_grid(r_grid, dx):
    """M applied to the interior of a full grid array (outer layer ignored);
    returns the full grid with 0 on the outer layer."""
    r_grid = np.asarray(r_grid, dtype=np.float64)
    out = np.zeros_like(r_grid)
    out[1:-1, 1:-1, 1:-1] = vcycle(r_grid[1:-1, 1:-1, 1:-1], dx)
    return out
