"""Pins of the oracle's direct-loop 3D convolution (the reference of the
learned warm start's tensor-core kernels): a single-tap kernel is a shift,
a centre-only identity kernel returns its input, and both gradients agree
with central finite differences in FP64."""
import numpy as np

import oracle as orc


def test_conv_identity_and_shift():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((5, 6, 7, 3))
    W = np.zeros((27, 3, 3))
    W[13] = np.eye(3)  # centre tap
    np.testing.assert_allclose(orc.conv3d_fwd(x, W), x, atol=1e-15)
    W = np.zeros((27, 3, 3))
    W[14] = np.eye(3)  # dx = +1: out[x] = in[x + 1], zero beyond the last voxel
    out = orc.conv3d_fwd(x, W, bias=np.array([1.0, 2.0, 3.0]))
    np.testing.assert_allclose(out[:, :, :-1], x[:, :, 1:] + [1.0, 2.0, 3.0], atol=1e-15)
    np.testing.assert_allclose(out[:, :, -1], np.zeros((5, 6, 3)) + [1.0, 2.0, 3.0], atol=1e-15)


def test_conv_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((4, 5, 6, 2))
    W = rng.standard_normal((27, 2, 3))
    b = rng.standard_normal(3)
    g = rng.standard_normal((4, 5, 6, 3))
    loss = lambda x_, W_, b_: float(np.sum(g * orc.conv3d_fwd(x_, W_, b_)))
    gin, gW, gb = orc.conv3d_bwd(x, W, g)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (2, 3, 4, 1), (3, 4, 5, 0), (1, 0, 5, 1)]:
        e = np.zeros_like(x)
        e[idx] = h
        fd = (loss(x + e, W, b) - loss(x - e, W, b)) / (2 * h)
        assert abs(fd - gin[idx]) < 1e-6 * max(1.0, abs(fd))
    for idx in [(0, 0, 0), (13, 1, 2), (26, 1, 1), (7, 0, 2)]:
        e = np.zeros_like(W)
        e[idx] = h
        fd = (loss(x, W + e, b) - loss(x, W - e, b)) / (2 * h)
        assert abs(fd - gW[idx]) < 1e-6 * max(1.0, abs(fd))
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        fd = (loss(x, W, b + e) - loss(x, W, b - e)) / (2 * h)
        assert abs(fd - gb[c]) < 1e-6 * max(1.0, abs(fd))
