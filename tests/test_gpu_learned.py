"""The learned warm start: tensor-core convolution kernels against the FP64
oracle, training on the GPU, and the warm start inside the projection.

Tolerances (BF16 operands, FP32 accumulation): with operands rounded to BF16
on both sides, an FP32-accumulated convolution matches the FP64 reference to
~1e-6 relative (FP32 output) and to BF16 rounding, 2^-8 relative, when its
output is stored in BF16; gradients likewise. The gates are 1e-4 (FP32 output)
and 5e-3 (BF16 output), relative to the largest reference magnitude.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2607_28414_b300 import inputs, kv, learned

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SHAPE = (21, 10, 7)  # a multiple of no convolution tile in any axis


def bf16_tensor(rng, shape, device, scale=1.0):
    a = torch.from_numpy((rng.standard_normal(shape) * scale).astype(np.float32)).to(device)
    return a.to(torch.bfloat16)


def to64(t):
    return t.float().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("cin,cout", [(16, 16), (16, 32), (32, 64), (64, 16), (64, 64)])
def test_conv_forward_matches_oracle(device, cin, cout):
    rng = np.random.default_rng(cin * 100 + cout)
    nx, ny, nz = SHAPE
    x = bf16_tensor(rng, (nz, ny, nx, cin), device)
    W = bf16_tensor(rng, (27, cin, cout), device, 0.1)
    b = torch.from_numpy(rng.standard_normal(cout).astype(np.float32)).to(device)
    ref = orc.conv3d_fwd(to64(x), to64(W), b.cpu().numpy().astype(np.float64))
    out32 = torch.empty((nz, ny, nx, cout), dtype=torch.float32, device=device)
    kv.kv_nn_conv3d_fwd(SHAPE, cin, cout, x, W, b, out32)
    scale = np.abs(ref).max()
    assert np.abs(out32.cpu().numpy() - ref).max() <= 1e-4 * scale
    out16 = torch.empty((nz, ny, nx, cout), dtype=torch.bfloat16, device=device)
    kv.kv_nn_conv3d_fwd(SHAPE, cin, cout, x, W, b, out16, relu=True)
    assert np.abs(to64(out16) - np.maximum(ref, 0)).max() <= 5e-3 * scale


@pytest.mark.parametrize("cin,cout,shape", [
    (16, 16, SHAPE), (16, 32, SHAPE), (16, 64, SHAPE), (32, 16, SHAPE), (32, 32, SHAPE), (32, 64, SHAPE),
    (64, 16, SHAPE), (64, 32, SHAPE), (64, 64, SHAPE),
    # several chunks of 8 x 8 (x 4) x 16 voxels per block, ragged in x, y and z
    (16, 16, (61, 37, 35)), (32, 32, (29, 23, 41)), (64, 64, (26, 21, 37)),
])
def test_conv_gradients_match_oracle(device, cin, cout, shape):
    rng = np.random.default_rng(7 + cin + cout + shape[2])
    nx, ny, nz = shape
    x = bf16_tensor(rng, (nz, ny, nx, cin), device)
    W = bf16_tensor(rng, (27, cin, cout), device, 0.1)
    g = bf16_tensor(rng, (nz, ny, nx, cout), device)
    gin_ref, gW_ref, gb_ref = orc.conv3d_bwd(to64(x), to64(W), to64(g))
    Wt = torch.empty((27, cout, cin), dtype=torch.bfloat16, device=device)
    kv.kv_nn_conv3d_flip(cin, cout, W, Wt)
    gin = torch.empty((nz, ny, nx, cin), dtype=torch.float32, device=device)
    kv.kv_nn_conv3d_fwd(shape, cout, cin, g, Wt, None, gin)
    assert np.abs(gin.cpu().numpy() - gin_ref).max() <= 1e-4 * np.abs(gin_ref).max()
    gW = torch.zeros((27, cin, cout), dtype=torch.float32, device=device)
    gb = torch.zeros(cout, dtype=torch.float32, device=device)
    kv.kv_nn_conv3d_bwd_weight(shape, cin, cout, x, g, gW, gb)
    assert np.abs(gW.cpu().numpy() - gW_ref).max() <= 1e-4 * np.abs(gW_ref).max()
    assert np.abs(gb.cpu().numpy() - gb_ref).max() <= 1e-4 * np.abs(gb_ref).max()


def small_pairs(n, shape, seed, device):
    return learned.make_pairs(shape, inputs.random_gaussian_forces_torch(n, shape, learned.DX, seed, device),
                              tol=1e-10)


def test_training_lowers_the_loss(device):
    shape = (24, 24, 24)
    B, P, _ = small_pairs(6, shape, 3, device)
    net = kv.kv_net_create([16, 16], shape)
    kv.kv_net_init(net, 1)
    losses = learned.train(net, B, P, shape, epochs=12, lr=2e-3)
    kv.kv_net_destroy(net)
    assert np.isfinite(losses).all()
    assert np.mean(losses[-6:]) < 0.5 * np.mean(losses[:6])


def test_residual_loss_training_lowers_the_residual(device):
    """Training on the squared residual |b - A phi_hat|^2 lowers it; the loss
    the net reports equals the oracle's residual of the net's own prediction
    (in the net's unit-RMS scaling of b)."""
    shape = (24, 24, 24)
    B, P, _ = small_pairs(6, shape, 4, device)
    net = kv.kv_net_create([16, 16], shape)
    kv.kv_net_init(net, 3)
    kv.kv_net_set_loss(net, kv.KV_LOSS_RESIDUAL)
    losses = learned.train(net, B, P, shape, epochs=12, lr=2e-3)
    assert np.isfinite(losses).all()
    assert np.mean(losses[-6:]) < 0.5 * np.mean(losses[:6])
    phi = torch.empty_like(B[0])
    kv.kv_net_predict(net, shape, learned.DX, B[0], phi)
    b = B[0].double().cpu().numpy()
    r = b - orc.apply_A(phi.double().cpu().numpy(), learned.DX)
    r[0], r[-1], r[:, 0], r[:, -1], r[:, :, 0], r[:, :, -1] = 0, 0, 0, 0, 0, 0
    s2 = b.size / (b ** 2).sum()  # the net's scale s = 1/rms(b), squared
    expect = (r ** 2).sum() * s2 / b.size
    # a train step reports the loss of the forward pass before its update: compare
    # with a step at learning rate 0, whose weights stay those of the prediction
    got = kv.kv_net_train_step(net, shape, learned.DX, B[0], P[0], 0.0)
    kv.kv_net_destroy(net)
    assert got == pytest.approx(expect, rel=2e-2)


def test_warm_start_reaches_the_same_residual_and_saves_iterations(device):
    """Zero start and learned start stop on the same true residual (checked by
    the oracle on the learned-start potential); after a short training the
    learned start needs fewer CG iterations on held-out fields."""
    shape = (40, 40, 40)
    B, P, _ = small_pairs(48, shape, 5, device)
    net = kv.kv_net_create([16, 32, 64], shape)
    kv.kv_net_init(net, 2)
    learned.train(net, B, P, shape, epochs=6, lr=2e-3)
    held = list(inputs.random_gaussian_forces_torch(6, shape, learned.DX, 10_005, device))
    res = learned.evaluate(net, shape, held, tol=1e-8)
    print("warm start on 40^3:", res)
    assert res["max_rel_res_learned"] < 1e-8 and res["max_rel_res_plain"] < 1e-8
    assert res["max_rel_res_mg"] < 1e-8 and res["max_rel_res_learned_mg"] < 1e-8
    assert res["learned_iters"] < res["plain_iters"]
    # independent check of the learned-start potential by the oracle
    h = learned.projection_handle(shape)
    kv.kv_attach_net(h, net)
    st = kv.kv_project_force(h, *held[0], 1e-8, 0, 1)
    phi = np.empty(shape[::-1], np.float64)
    kv.kv_read_field(h, kv.FIELD_PHI, 0, phi)
    b = -orc.div_minus(*[f.cpu().numpy() for f in held[0]], learned.DX)
    r = np.linalg.norm(b - orc.apply_A(phi, learned.DX)) / np.linalg.norm(b)
    assert r < 1e-8 and r == pytest.approx(st["rel_res_true"], rel=1e-3)
    kv.kv_destroy(h)
    kv.kv_net_destroy(net)


def test_flexible_cg_with_the_net_meets_the_same_residual(device):
    """Mode 2 (flexible CG, the net as preconditioner) stops on the same true
    residual as the zero-start CG, checked by the oracle on its potential, and
    its projected force matches mode 0's node by node."""
    shape = (40, 40, 40)
    net = learned.load_net(learned.WEIGHTS, shape)
    held = list(inputs.random_gaussian_forces_torch(3, shape, learned.DX, 10_009, device))
    h = learned.projection_handle(shape)
    kv.kv_attach_net(h, net)
    try:
        for f in held:
            fs0 = torch.zeros((3,) + shape[::-1], dtype=torch.float32, device=device)
            fs2 = torch.zeros_like(fs0)
            st0 = kv.kv_project_force(h, *f, 1e-8, 0, 0, fs0)
            st2 = kv.kv_project_force(h, *f, 1e-8, 0, 2, fs2)
            phi = np.empty(shape[::-1], np.float64)
            kv.kv_read_field(h, kv.FIELD_PHI, 0, phi)
            b = -orc.div_minus(*[c.cpu().numpy() for c in f], learned.DX)
            r = np.linalg.norm(b - orc.apply_A(phi, learned.DX)) / np.linalg.norm(b)
            print(f"flexible CG 40^3: {st2['iters']} iterations (plain CG {st0['iters']}), "
                  f"true residual {st2['rel_res_true']:.2e}, oracle {r:.2e}")
            assert st2["status"] == kv.KV_OK and st2["rel_res_true"] < 1e-8
            assert r < 1e-8 and r == pytest.approx(st2["rel_res_true"], rel=1e-3)
            a, c = fs0.cpu().numpy(), fs2.cpu().numpy()
            assert np.abs(a - c).max() <= 1e-6 * np.abs(a).max()
    finally:
        kv.kv_destroy(h)
        kv.kv_net_destroy(net)


def test_trained_net_gains_at_128(device):
    """What the trained network (the committed residual-loss net) gains on
    held-out fields at its training size, 128^3, at a true residual of 1e-8:
    as a flexible-CG preconditioner it cuts the plain CG's iterations at least
    tenfold (about 30x measured); as a warm start it saves plain-CG iterations
    (about 10 % here); with the multigrid-preconditioned CG the projection is
    at least twice as fast in wall time as the paper's plain CG (2.7x here,
    5.4x at 256^3, where the multigrid cycle carries the gain). Every mode
    stops on the same residual."""
    shape = (128, 128, 128)
    net = learned.load_net(learned.WEIGHTS, shape)
    warm = list(inputs.random_gaussian_forces_torch(1, shape, learned.DX, 20_127, device))
    held = list(inputs.random_gaussian_forces_torch(4, shape, learned.DX, 20_128, device))
    try:
        learned.evaluate(net, shape, warm, tol=1e-8, modes=(0, 1, 2, 4, 5))  # first-call costs
        res = learned.evaluate(net, shape, held, tol=1e-8, modes=(0, 1, 2, 4, 5))
    finally:
        kv.kv_net_destroy(net)
    print("trained net at 128^3:", res)
    for name in ("plain", "learned", "fcg", "mg", "learned_mg"):
        assert res[f"max_rel_res_{name}"] < 1e-8, name
    assert res["fcg_iters"] * 10 <= res["plain_iters"]
    assert res["learned_iters"] < res["plain_iters"]
    assert res["speedup_ms_learned_mg"] >= 2.0
