"""Host logic of the divergence-form stability limit (no GPU needed: scalar and
host-array media are evaluated on the CPU inside libkv).

The limit must bound the true spectrum: for eta = 0 the leapfrog recursion of
the flux operator is stable iff dt^2 lambda_max(M^{-1} K) <= 4 (M = diag(rho)).
lambda_max is computed here by power iteration on a numpy assembly of K, an
independent route to the same quantity."""
import numpy as np
import pytest

from paper_2607_28414_b300 import kv

DX = 2e-4


def flux_apply(mu, q, dx):
    """K q on interior nodes (face moduli = means of the two nodes), 0 elsewhere."""
    out = np.zeros_like(q)
    c = (slice(1, -1),) * 3
    for ax in range(3):
        for sgn in (-1, 1):
            sl = [slice(1, -1)] * 3
            sl[ax] = slice(1 + sgn, q.shape[ax] - 1 + sgn)
            sl = tuple(sl)
            out[c] += 0.5 * (mu[c] + mu[sl]) * (q[sl] - q[c])
    return -out / dx ** 2  # positive semi-definite sign


def lambda_max(mu, rho, dx, iters=400, seed=0):
    rng = np.random.default_rng(seed)
    q = np.zeros_like(mu)
    q[1:-1, 1:-1, 1:-1] = rng.standard_normal(tuple(s - 2 for s in mu.shape))
    lam = 0.0
    for _ in range(iters):
        # symmetric form M^{-1/2} K M^{-1/2}
        y = flux_apply(mu, q / np.sqrt(rho), dx) / np.sqrt(rho)
        lam = float(np.sum(q * y) / np.sum(q * q))
        q = y / np.linalg.norm(y)
    return lam


@pytest.fixture(scope="module")
def lib_loaded():
    try:
        kv.lib()
    except OSError as e:  # library not built
        pytest.skip(str(e))


def test_divergence_limit_bounds_the_spectrum(lib_loaded):
    rng = np.random.default_rng(4)
    n = (12, 11, 10)
    mu = rng.uniform(1e3, 20e3, n[::-1])
    rho = rng.uniform(900, 1200, n[::-1])
    mu32, rho32 = mu.astype(np.float32), rho.astype(np.float32)
    dt = kv.kv_stable_dt_op(*n, DX, mu32, rho32, 0.0, kv.KV_OP_DIVERGENCE)
    lam = lambda_max(mu32.astype(np.float64), rho32.astype(np.float64), DX)
    assert dt ** 2 * lam <= 4.0
    # and it is not vacuous: within a factor 2 of the true limit
    assert dt ** 2 * lam > 1.0


def test_divergence_limit_equals_pointwise_when_homogeneous(lib_loaded):
    n = (9, 8, 7)
    a = kv.kv_stable_dt(*n, DX, 5e3, 1000.0, 0.8)
    b = kv.kv_stable_dt_op(*n, DX, 5e3, 1000.0, 0.8, kv.KV_OP_DIVERGENCE)
    G = np.full(n[::-1], 5e3, np.float32)
    c = kv.kv_stable_dt_op(*n, DX, G, 1000.0, 0.8, kv.KV_OP_DIVERGENCE)
    assert a == pytest.approx(b, rel=1e-15) and a == pytest.approx(c, rel=1e-12)


def test_divergence_limit_uses_neighbour_moduli(lib_loaded):
    """A stiff boundary node enters the divergence limit only through the face
    mean of its interior neighbour, (6 G_i + sum of neighbours) / 12; the
    pointwise limit takes every node's own wave speed, boundary included."""
    n = (6, 6, 6)
    G = np.full(n[::-1], 2e3, np.float32)
    G[0, 3, 3] = 50e3  # boundary node (k = 0) next to interior node (3, 3, 1)
    p = kv.kv_stable_dt_op(*n, DX, G, 1000.0, 0.0, kv.KV_OP_POINTWISE)
    d = kv.kv_stable_dt_op(*n, DX, G, 1000.0, 0.0, kv.KV_OP_DIVERGENCE)
    h2 = DX ** 2 / 3
    gbar = (6 * 2e3 + 5 * 2e3 + 50e3) / 12
    assert d == pytest.approx(np.sqrt(h2 * 1000.0 / gbar), rel=1e-6)
    assert p == pytest.approx(np.sqrt(h2 * 1000.0 / 50e3), rel=1e-6)


def test_operator_argument_is_checked(lib_loaded):
    with pytest.raises(kv.KvError) as e:
        kv.kv_stable_dt_op(8, 8, 8, DX, 3e3, 1000.0, 0.0, 7)
    assert e.value.status == kv.KV_ERR_ARG
