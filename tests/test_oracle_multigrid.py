"""Pins of the oracle's multigrid V-cycle (oracle/multigrid.py), the
preconditioner of projection modes 4 and 5 (the paper's system A phi = b of
Sec. 3.2.3; the cycle itself is this library's addition). Each check rests on
something other than the cycle's own code: the matrices of the maps, the
two-level closed form, symmetry, definiteness and contraction."""
import numpy as np
import pytest

from oracle import multigrid as mg


def dense(fn, shape):
    """Matrix of a linear map on arrays of `shape`, column by column."""
    n = int(np.prod(shape))
    cols = []
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        cols.append(np.asarray(fn(e.reshape(shape))).ravel())
    return np.array(cols).T


def test_levels_follow_the_coarsening_rule():
    lv = mg.levels((254, 254, 254), 1.0)
    assert [l[:3] for l in lv] == [(254, 254, 254), (127, 127, 127), (64, 64, 64), (32, 32, 32),
                                   (16, 16, 16), (8, 8, 8), (4, 4, 4)]
    assert [l[3] for l in lv] == [4.0 ** k for k in range(7)]
    assert len(mg.levels((3, 3, 3), 1.0)) == 1           # 27 cells: no coarser level
    assert len(mg.levels((100, 100, 3), 1.0)) == 1        # fewer than 4 along an axis
    assert mg.levels((7, 5, 9), 1.0)[1][:3] == (4, 3, 5)  # ceil(n / 2)


def test_one_level_is_diagonal_scaling():
    rng = np.random.default_rng(0)
    r = rng.standard_normal((3, 3, 3))
    dx = 0.7
    assert np.allclose(mg.vcycle(r, dx), mg.OMEGA * dx * dx / 6.0 * r, rtol=0, atol=1e-15)


def test_operator_is_the_dirichlet_laplacian():
    # A u for u = sin modes of the interior is the textbook eigenvalue
    n, h = 6, 0.5
    z, y, x = np.meshgrid(*(np.arange(1, n + 1),) * 3, indexing="ij")
    u = np.sin(np.pi * x / (n + 1)) * np.sin(2 * np.pi * y / (n + 1)) * np.sin(3 * np.pi * z / (n + 1))
    lam = sum(4.0 / h ** 2 * np.sin(k * np.pi / (2 * (n + 1))) ** 2 for k in (1, 2, 3))
    assert np.allclose(mg.apply_A(u, h * h), lam * u, rtol=0, atol=1e-12 * lam)


def test_restriction_is_prolongation_transposed_over_8():
    nf, nc = (5, 4, 7), (3, 2, 4)
    P = dense(lambda e: mg.prolong(e, nf), (nc[2], nc[1], nc[0]))
    R = dense(lambda t: mg.restrict(t, nc), (nf[2], nf[1], nf[0]))
    assert P.shape == (140, 24) and R.shape == (24, 140)
    assert np.array_equal(R, P.T / 8.0)
    # trilinear interpolation reproduces a constant away from the Dirichlet edge
    e = np.ones((nc[2], nc[1], nc[0]))
    Pe = mg.prolong(e, nf)
    assert Pe[2, 1:3, 1:3].min() == 1.0


def test_two_level_cycle_matches_its_closed_form():
    shape = (5, 6, 8)  # interior (z, y, x): 240 cells -> 4 x 3 x 3 = 36, two levels
    dx = 0.3
    lv = mg.levels((shape[2], shape[1], shape[0]), dx * dx)
    assert len(lv) == 2
    ncx, ncy, ncz, h2c = lv[1]
    h2 = dx * dx
    n, nc = int(np.prod(shape)), ncx * ncy * ncz
    A = dense(lambda u: mg.apply_A(u, h2), shape)
    Ac = dense(lambda u: mg.apply_A(u, h2c), (ncz, ncy, ncx))
    P = dense(lambda e: mg.prolong(e, (shape[2], shape[1], shape[0])), (ncz, ncy, ncx))
    R = P.T / 8.0
    S, Sc = mg.OMEGA * h2 / 6.0, mg.OMEGA * h2c / 6.0
    I, Ic = np.eye(n), np.eye(nc)
    Mc = Sc * Ic
    for _ in range(mg.COARSE_SWEEPS):
        Mc = Mc + Sc * (Ic - Ac @ Mc)
    M_closed = (2 * S * I - S * S * A) + (I - S * A) @ P @ Mc @ R @ (I - S * A)
    M = dense(lambda r: mg.vcycle(r, dx), shape)
    assert np.abs(M - M_closed).max() <= 1e-12 * np.abs(M_closed).max()


@pytest.fixture(scope="module")
def three_level():
    shape = (9, 11, 13)  # 1287 cells -> 7 x 6 x 5 -> 4 x 3 x 3: three levels
    dx = 0.2
    assert len(mg.levels((shape[2], shape[1], shape[0]), dx * dx)) == 3
    M = dense(lambda r: mg.vcycle(r, dx), shape)
    A = dense(lambda u: mg.apply_A(u, dx * dx), shape)
    return M, A


def test_cycle_is_symmetric_positive_definite(three_level):
    M, _ = three_level
    assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0.0


def test_cycle_contracts_as_a_solver(three_level):
    # e <- (I - M A) e: the eigenvalues of M A (those of the symmetric
    # A^1/2 M A^1/2, so real and positive) lie in (0, 2), so the cycle
    # converges as a stationary iteration; measured here 0.52 ... 1.49 (the
    # coarse operator is the rediscretised Laplacian, not P^T A P / 8, so
    # M A can exceed 1), i.e. a contraction of 0.49 per cycle and a condition
    # number of 2.85 for the preconditioned CG (plain CG: cond(A) = 54.5 on
    # this grid, growing with n^2 while the cycle's stays bounded)
    M, A = three_level
    lam = np.sort(np.linalg.eigvals(M @ A).real)
    assert lam.min() > 0.3 and lam.max() < 1.7, (lam.min(), lam.max())
    assert lam.max() / lam.min() < 3.5
    kA = np.linalg.eigvalsh(A)
    assert kA.max() / kA.min() > 15 * lam.max() / lam.min()
