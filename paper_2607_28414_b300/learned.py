"""Learned warm start of the projection: data, training and evaluation.

Training pairs (b, phi) come from the library's own projection (CG to a true
residual of 1e-10) on random Gaussian force fields; the net (kv_net_*) is
trained by the library's tensor-core forward/backward kernels; evaluation
compares kv_project_force with mode 0 (zero start), mode 1 (learned start),
mode 4 (multigrid-preconditioned CG) and mode 5 (learned start with the
preconditioned CG) at the same tolerance. This module only orchestrates calls through the binding.

    python -m paper_2607_28414_b300.learned --train 2000 --train-n 128 --eval 200 --eval-n 256
    python -m paper_2607_28414_b300.learned --conv-bench 64,64,96 --reps 3   # one layer's kernels
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import inputs, kv

DX = 0.2 * inputs.MM


WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "unet_residual.npz")


def load_net(path=WEIGHTS, max_shape=(128, 128, 128), stream=None):
    """A net with the parameters stored by `--out` (default: the committed
    residual-loss net), activations allocated for grids up to max_shape."""
    d = np.load(path)
    net = kv.kv_net_create([int(c) for c in d["channels"]], tuple(max_shape), stream=stream)
    kv.kv_net_set_params(net, np.ascontiguousarray(d["params"], np.float32))
    return net


def projection_handle(shape, dx=DX, stream=None):
    """A handle whose only use is the projection (the medium does not enter it)."""
    nx, ny, nz = shape
    dt = 0.5 * kv.kv_stable_dt(nx, ny, nz, dx, 4e3, 1000.0, 0.0)
    return kv.kv_create(nx, ny, nz, dx, dt, 4e3, 1000.0, 0.0, stream=stream)


def make_pairs(shape, forces, tol=1e-10, dx=DX, device="cuda:0"):
    """Stack (b, phi) float32 pairs [n, nz, ny, nx] on the device."""
    import torch
    nx, ny, nz = shape
    h = projection_handle(shape, dx)
    B, P, iters = [], [], []
    try:
        for f in forces:
            st = kv.kv_project_force(h, *f, tol)
            iters.append(st["iters"])
            b = torch.empty((nz, ny, nx), dtype=torch.float64, device=device)
            phi = torch.empty_like(b)
            kv.kv_read_field(h, 4, 0, b)
            kv.kv_read_field(h, kv.FIELD_PHI, 0, phi)
            B.append(b.float())
            P.append(phi.float())
    finally:
        kv.kv_destroy(h)
    return torch.stack(B), torch.stack(P), iters


def train(net, B, P, shape, epochs=3, lr=1e-3, dx=DX, seed=0, log=None):
    """Adam over the pairs in a seeded random order; cosine learning-rate decay."""
    import torch
    n = B.shape[0]
    rng = np.random.default_rng(seed)
    steps = epochs * n
    losses = []
    k = 0
    for ep in range(epochs):
        order = rng.permutation(n)
        for i in order:
            lr_k = lr * 0.5 * (1.0 + np.cos(np.pi * k / max(1, steps)))
            losses.append(kv.kv_net_train_step(net, shape, dx, B[i], P[i], lr_k))
            k += 1
        if log:
            log(f"epoch {ep}: mean loss {np.mean(losses[-n:]):.4e}")
    return losses


MODES = {0: "plain", 1: "learned", 2: "fcg", 4: "mg", 5: "learned_mg"}


def evaluate(net, shape, forces, tol=1e-8, dx=DX, device="cuda:0", modes=(0, 1, 4, 5)):
    """Projection of each field at the same tolerance with each mode: 0 the
    paper's CG from zero, 1 the learned start, 2 flexible CG with the net as
    preconditioner, 4 multigrid-preconditioned CG from zero, 5 the learned
    start with the multigrid-preconditioned CG.
    Returns mean iterations and milliseconds per mode (keys <name>_iters,
    <name>_ms, max_rel_res_<name>) and the wall-time ratios to mode 0."""
    h = projection_handle(shape, dx)
    kv.kv_attach_net(h, net)
    rows = {m: [] for m in modes}
    n = 0
    try:
        for f in forces:
            n += 1
            for mode in modes:
                st = kv.kv_project_force(h, *f, tol, 0, mode)
                rows[mode].append((st["iters"], st["ms"], st["rel_res_true"]))
    finally:
        kv.kv_destroy(h)
    out = {"fields": n}
    for mode in modes:
        a = np.array(rows[mode])
        name = MODES[mode]
        out[f"{name}_iters"] = float(a[:, 0].mean())
        out[f"{name}_ms"] = float(a[:, 1].mean())
        out[f"max_rel_res_{name}"] = float(a[:, 2].max())
    if 0 in modes:
        for mode in modes:
            if mode != 0:
                out[f"speedup_ms_{MODES[mode]}"] = out["plain_ms"] / out[f"{MODES[mode]}_ms"]
        if 1 in modes:
            out["speedup_ms"] = out["speedup_ms_learned"]
    return out


def conv_bench(cin, cout, n, reps=20, warmup=3, seed=0):
    """Event-timed forward and weight-gradient convolutions of one layer
    (cin -> cout channels on n^3 voxels, random BF16 tensors) on the current
    stream: mean ms per call and TFLOP/s (2 n^3 27 cin cout per call)."""
    import torch
    dev = torch.device("cuda:0")
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    shape = (n, n, n)
    x = torch.randn((n, n, n, cin), device=dev, generator=gen).to(torch.bfloat16)
    g = torch.randn((n, n, n, cout), device=dev, generator=gen).to(torch.bfloat16)
    W = (0.1 * torch.randn((27, cin, cout), device=dev, generator=gen)).to(torch.bfloat16)
    y = torch.empty((n, n, n, cout), device=dev, dtype=torch.bfloat16)
    gW = torch.zeros((27, cin, cout), device=dev)
    st = torch.cuda.current_stream(dev).cuda_stream
    flop = 2.0 * n ** 3 * 27 * cin * cout
    out = {"cin": cin, "cout": cout, "n": n, "reps": reps}
    for name, fn in (("fwd", lambda: kv.kv_nn_conv3d_fwd(shape, cin, cout, x, W, None, y, stream=st)),
                     ("wgrad", lambda: kv.kv_nn_conv3d_bwd_weight(shape, cin, cout, x, g, gW, stream=st))):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(reps):
            fn()
        t1.record()
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / reps
        out[f"{name}_ms"] = ms
        out[f"{name}_tflops"] = flop / ms / 1e9
    return out


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--conv-bench", default=None, metavar="CIN,COUT,N",
                    help="time one layer's forward and weight-gradient kernels and exit")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--train-n", type=int, default=128)
    ap.add_argument("--eval", type=int, default=200)
    ap.add_argument("--eval-n", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--channels", default="16,32,64,64")
    ap.add_argument("--seed", type=int, default=104)
    ap.add_argument("--out", default=None, help="write the trained parameters and their recipe (.npz)")
    ap.add_argument("--modes", default="0,1,4,5",
                    help="projection modes compared on the held-out fields (2: flexible CG)")
    ap.add_argument("--load", default=None,
                    help="evaluate the parameters of this .npz (from --out) instead of training")
    ap.add_argument("--loss", default="mse", choices=["mse", "residual"],
                    help="mse: squared error of the potential; residual: squared residual "
                         "|b - A phi_hat|^2 of the prediction")
    args = ap.parse_args()
    if args.conv_bench:
        cin, cout, n = (int(v) for v in args.conv_bench.split(","))
        print(json.dumps(conv_bench(cin, cout, n, reps=args.reps)))
        return
    device = torch.device("cuda:0")
    tshape = (args.train_n,) * 3
    eshape = (args.eval_n,) * 3
    modes = tuple(int(m) for m in args.modes.split(","))
    held = lambda: inputs.random_gaussian_forces_torch(args.eval, eshape, DX, args.seed + 1_000_000, device)
    if args.load:  # evaluation of stored parameters only
        net = load_net(args.load, eshape)
        res = evaluate(net, eshape, held(), modes=modes)
        d = np.load(args.load)
        res.update({"params_file": os.path.basename(args.load), "loss": str(d["loss"]),
                    "protocol": str(d["protocol"]), "eval_shape": eshape})
        kv.kv_net_destroy(net)
        print(json.dumps(res))
        return
    ch = [int(c) for c in args.channels.split(",")]
    t0 = time.perf_counter()
    B, P, it = make_pairs(tshape, inputs.random_gaussian_forces_torch(args.train, tshape, DX, args.seed, device))
    t_data = time.perf_counter() - t0
    net = kv.kv_net_create(ch, tuple(max(a, b) for a, b in zip(tshape, eshape)))
    kv.kv_net_init(net, args.seed)
    kv.kv_net_set_loss(net, kv.KV_LOSS_RESIDUAL if args.loss == "residual" else kv.KV_LOSS_MSE)
    t0 = time.perf_counter()
    losses = train(net, B, P, tshape, args.epochs, args.lr, log=print)
    t_train = time.perf_counter() - t0
    del B, P
    res = evaluate(net, eshape, held(), modes=modes)
    res.update({"loss": args.loss, "train_fields": args.train, "train_shape": tshape, "eval_shape": eshape,
                "channels": ch, "epochs": args.epochs, "data_s": t_data, "train_s": t_train,
                "train_cg_iters_mean": float(np.mean(it)), "final_loss": float(np.mean(losses[-50:])),
                "first_loss": float(np.mean(losses[:50])), "params": kv.kv_net_num_params(net)})
    if args.out:  # parameters and how they were made (.npz)
        np.savez_compressed(args.out, params=kv.kv_net_get_params(net), channels=np.array(ch),
                            loss=args.loss, seed=args.seed,
                            protocol=(f"{args.train} fields at {args.train_n}^3 (seed {args.seed}), "
                                      f"plain-CG potentials at 1e-10, {args.epochs} epochs of Adam "
                                      f"(lr {args.lr:g}, cosine), {args.loss} loss"))
    kv.kv_net_destroy(net)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
