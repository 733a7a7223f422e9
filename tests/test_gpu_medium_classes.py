"""Class-encoded media: an FP32 medium with at most 256 distinct folded
coefficient tuples ((A', B') for the pointwise operator of Sec. 3.1, (m, e,
1/rho) for the flux form) is read by the TMA step kernel as one class byte per
node plus a table of the FP32 tuples.

The table holds the folded values bit for bit, so the class path must agree
bit for bit with the field path (KV_MEDIUM_FIELDS) and with the plain per-node
kernel, and, like them, match the FP64 oracle to a trace rel-L2 of 1e-4.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2607_28414_b300 import inputs, kv
from paper_2607_28414_b300.runner import Solver, to_device

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def run(w, n_steps, encoding=kv.KV_MEDIUM_AUTO, step_config=None, operator=kv.KV_OP_POINTWISE):
    s = Solver(w, n_steps=n_steps, step_config=step_config, operator=operator)
    kv.kv_set_medium_encoding(s.h, encoding)
    classes = kv.kv_medium_classes(s.h)
    s.project()
    s.step()
    tr = s.read_traces().cpu().numpy().copy()
    fields = []
    for which in (kv.FIELD_U, kv.FIELD_D):
        for comp in range(3):
            out = np.empty((w.nz, w.ny, w.nx), np.float32)
            kv.kv_read_field(s.h, which, comp, out)
            fields.append(out)
    s.close()
    return classes, tr, np.stack(fields)


def inclusion_workload(nx=70, ny=37, nz=45, seed=3):
    rng = np.random.default_rng(seed)
    dx = 2e-4
    G, rho, eta, _ = inputs.spherical_inclusions(nx, ny, nz, dx, rng, n=3, r_range=(0.6e-3, 1.5e-3),
                                                 margin=0.2e-3)
    f = inputs.beam_push(nx, ny, nz, dx, rng, focal_depth=4e-3, focal_len=2e-3)
    c = inputs.centre_node(nx, ny, nz)
    sensors = np.concatenate([inputs.line_sensors(c, 0, nx, 3),
                              np.array([[1, 1, 1], [nx - 2, ny - 2, nz - 2]], np.int32)])
    return inputs.Workload(f"inclusions_{nx}x{ny}x{nz}", nx, ny, nz, dx, G, rho, eta, tuple(f), 40e-6, 60,
                           sensors, 1e-9)


def banded_workload(k, nx=64, ny=24, nz=30, seed=5):
    """A medium of exactly k distinct (G, rho, eta) triples (shear modulus
    cycling through k values along the node index); nx is a multiple of 32, so
    no row padding adds a class."""
    w = inclusion_workload(nx, ny, nz, seed)
    idx = np.arange(nx * ny * nz).reshape(nz, ny, nx) % k
    G = (2e3 + 10.0 * idx).astype(np.float32)
    rho = np.full((nz, ny, nx), 1000.0, np.float32)
    eta = np.full((nz, ny, nx), 0.5, np.float32)
    return inputs.Workload(f"bands{k}", nx, ny, nz, w.dx, G, rho, eta, w.force, w.t_push, 40, w.sensors,
                           w.tol)


@pytest.mark.parametrize("cfg", [None, {"variant": 0, "tx": 32, "ty": 8, "zc": 7, "ns": 6},
                                 {"variant": 0, "tx": 128, "ty": 4, "zc": 64, "ns": 4}])
def test_classes_match_fields_and_plain_kernel_bitwise(device, cfg):
    w = inclusion_workload()
    c_auto, tr, f = run(w, 60, kv.KV_MEDIUM_AUTO, cfg)
    c_fld, tr_f, f_f = run(w, 60, kv.KV_MEDIUM_FIELDS, cfg)
    _, tr_p, f_p = run(w, 60, kv.KV_MEDIUM_AUTO, {"variant": 1})
    assert 2 <= c_auto <= 8 and c_fld == 0  # background, up to 3 spheres, row padding
    assert np.abs(f).max() > 0
    assert np.array_equal(tr, tr_f) and np.array_equal(f, f_f)
    assert np.array_equal(tr, tr_p) and np.array_equal(f, f_p)


@pytest.mark.parametrize("op", [kv.KV_OP_POINTWISE, kv.KV_OP_DIVERGENCE])
def test_batch_of_class_encoded_handles_reads_the_fields(device, op):
    """Batched stepping of handles whose step reads class bytes: the batch
    kernel reads the coefficient fields and matches each handle's own step."""
    cases = [inclusion_workload(70, 37, 45, seed=3), inclusion_workload(45, 40, 33, seed=8)]
    n = 64
    cfg = {"variant": 0, "tx": 64, "ty": 8, "zc": 16, "ns": 4}
    singles = [run(w, n, kv.KV_MEDIUM_AUTO, cfg, op)[1] for w in cases]
    stream = torch.cuda.Stream(device)
    solvers = [Solver(w, n_steps=n, operator=op, stream=stream.cuda_stream) for w in cases]
    for s in solvers:
        kv.kv_set_medium_encoding(s.h, kv.KV_MEDIUM_AUTO)
        assert kv.kv_medium_classes(s.h) > 0
        s.project()
    b = kv.kv_batch_create([s.h for s in solvers])
    kv.kv_batch_set_config(b, 64, 8, 16, 4)
    kv.kv_batch_step(b, n)
    for s, ref in zip(solvers, singles):
        assert np.array_equal(s.read_traces().cpu().numpy(), ref)
    kv.kv_batch_destroy(b)
    for s in solvers:
        s.close()


def test_class_count_limit(device):
    c256, tr, f = run(banded_workload(256), 40)
    c257, _, _ = run(banded_workload(257), 40)
    assert c256 == 256 and c257 == 0
    _, tr_f, f_f = run(banded_workload(256), 40, kv.KV_MEDIUM_FIELDS)
    assert np.array_equal(tr, tr_f) and np.array_equal(f, f_f)


@pytest.mark.parametrize("cfg", [None, {"variant": 0, "tx": 32, "ty": 8, "zc": 7, "ns": 6},
                                 {"variant": 0, "tx": 64, "ty": 8, "zc": 64, "ns": 4},
                                 {"variant": 0, "tx": 128, "ty": 4, "zc": 16, "ns": 4}])
def test_flux_form_classes_match_fields_and_plain_kernel_bitwise(device, cfg):
    w = inclusion_workload(seed=4)
    div = kv.KV_OP_DIVERGENCE
    c_auto, tr, f = run(w, 60, kv.KV_MEDIUM_AUTO, cfg, div)
    c_fld, tr_f, f_f = run(w, 60, kv.KV_MEDIUM_FIELDS, cfg, div)
    _, tr_p, f_p = run(w, 60, kv.KV_MEDIUM_AUTO, {"variant": 1}, div)
    assert 2 <= c_auto <= 8 and c_fld == 0
    assert np.abs(f).max() > 0
    assert np.array_equal(tr, tr_f) and np.array_equal(f, f_f)
    assert np.array_equal(tr, tr_p) and np.array_equal(f, f_p)


def test_flux_form_keeps_fields_when_density_is_not_fixed_by_the_moduli(device):
    """Two regions with the same G and eta but different rho share (m, e) and
    differ in 1/rho: the flux form reads the fields, the pointwise operator
    (A' = m/rho) still has two classes."""
    w = inclusion_workload(48, 24, 30)
    rho = np.full((w.nz, w.ny, w.nx), 1000.0, np.float32)
    rho[:, :, w.nx // 2:] = 1100.0
    w2 = inputs.Workload("rho_step", w.nx, w.ny, w.nz, w.dx, np.full_like(rho, 3e3), rho,
                         np.full_like(rho, 0.5), w.force, w.t_push, 20, w.sensors, w.tol)
    c_div, tr, f = run(w2, 20, kv.KV_MEDIUM_AUTO, None, kv.KV_OP_DIVERGENCE)
    c_pt, _, _ = run(w2, 20, kv.KV_MEDIUM_AUTO)
    assert c_div == 0 and c_pt >= 2
    _, tr_f, f_f = run(w2, 20, kv.KV_MEDIUM_FIELDS, None, kv.KV_OP_DIVERGENCE)
    assert np.array_equal(tr, tr_f) and np.array_equal(f, f_f)


def test_field_path_for_continuous_and_fp64_media(device):
    w = inclusion_workload(40, 33, 35)
    rng = np.random.default_rng(11)
    G = (3e3 * (1 + 0.1 * rng.random((w.nz, w.ny, w.nx)))).astype(np.float32)
    s = Solver(w, n_steps=5)
    kv.kv_set_medium_encoding(s.h, kv.KV_MEDIUM_AUTO)
    assert kv.kv_medium_classes(s.h) > 0
    med = [to_device(a, s.device) for a in (G, w.rho, w.eta)]
    kv.kv_set_medium(s.h, *med)  # continuous: the fields are read
    assert kv.kv_medium_classes(s.h) == 0
    kv.kv_set_medium(s.h, *s.medium)  # back to the inclusions
    assert kv.kv_medium_classes(s.h) > 0
    kv.kv_set_operator(s.h, kv.KV_OP_DIVERGENCE, *s.medium)
    assert kv.kv_medium_classes(s.h) > 0  # (m, e, 1/rho) of the flux form
    kv.kv_set_operator(s.h, kv.KV_OP_POINTWISE, *s.medium)
    assert kv.kv_medium_classes(s.h) > 0
    kv.kv_set_medium_encoding(s.h, kv.KV_MEDIUM_FIELDS)
    assert kv.kv_medium_classes(s.h) == 0
    with pytest.raises(kv.KvError):
        kv.kv_set_medium_encoding(s.h, 7)
    s.close()
    s64 = Solver(w, n_steps=5, precision=kv.KV_FP64)
    kv.kv_set_medium_encoding(s64.h, kv.KV_MEDIUM_AUTO)
    assert kv.kv_medium_classes(s64.h) == 0
    s64.close()


def test_classes_match_oracle(device):
    w = inclusion_workload(48, 40, 44, seed=9)
    s = Solver(w, n_steps=120)
    kv.kv_set_medium_encoding(s.h, kv.KV_MEDIUM_AUTO)
    assert kv.kv_medium_classes(s.h) > 0
    s.project(tol=1e-9)
    s.step()
    tr = s.read_traces().cpu().numpy().astype(np.float64)
    dt = s.dt
    s.close()
    phi, fs, status, _ = orc.project(*w.force, w.dx, tol=1e-13)
    g = inputs.push_envelope(120, dt, w.t_push)
    ref = orc.run(w.nx, w.ny, w.nz, w.dx, dt, w.G, w.rho, w.eta, 120, w.sensors, fs=fs, g=g)
    den = np.sqrt((ref ** 2).sum(axis=(0, 2)))
    num = np.sqrt(((tr - ref) ** 2).sum(axis=(0, 2)))
    keep = den > 1e-9 * den.max()
    assert keep.sum() >= 3
    assert (num[keep] / den[keep]).max() <= 1e-4
