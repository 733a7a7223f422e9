"""Python binding of libkv (include/kv.h): argument marshalling only.

Every function keeps the C name and forwards to the CUDA library; nothing here
computes any part of the method. Arrays may be NumPy arrays or torch tensors
(CPU tensors and NumPy arrays are host fields, CUDA tensors device fields);
scalars become KV_SCALAR fields. A non-OK status raises KvError, which carries
the status code and libkv's one-line message. The library must be built
(`python -m paper_2607_28414_b300.build`); importing this module without it
raises ImportError, and there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkv.so")

KV_OK = 0
KV_ERR_ARG = 1
KV_ERR_CUDA = 2
KV_ERR_OOM = 3
KV_ERR_UNSTABLE_DT = 4
KV_ERR_NONFINITE = 5
KV_CG_BREAKDOWN = 6
KV_CG_MAXITER = 7
KV_ERR_TIMEOUT = 8
KV_ERR_STATE = 9
KV_ERR_UNSUPPORTED = 10

KV_FP32 = 0
KV_FP64 = 1
KV_SCALAR = 0
KV_HOST = 1
KV_DEVICE = 2
KV_OP_POINTWISE = 0
KV_OP_DIVERGENCE = 1
KV_MEDIUM_AUTO = 0
KV_MEDIUM_FIELDS = 1

FIELD_U, FIELD_D, FIELD_PHI, FIELD_F = 0, 1, 2, 3


class KvField(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("value", ctypes.c_double), ("where", ctypes.c_int)]


class KvCgStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("refinements", ctypes.c_int), ("status", ctypes.c_int),
                ("rel_res_true", ctypes.c_double), ("rel_res_recursive", ctypes.c_double),
                ("ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KvError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_status_name(status)}: {message}")
        self.status = status


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libkv is not built ({LIB_PATH} missing); run "
                              "python -m paper_2607_28414_b300.build")
        L = ctypes.CDLL(LIB_PATH)
        H = ctypes.c_void_p
        i, d, vp = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        F = KvField
        L.kv_status_string.restype = ctypes.c_char_p
        L.kv_status_string.argtypes = [i]
        L.kv_last_error.restype = ctypes.c_char_p
        L.kv_last_error.argtypes = [H]
        L.kv_stable_dt.argtypes = [i, i, i, d, F, F, F, ctypes.POINTER(d)]
        L.kv_create.argtypes = [ctypes.POINTER(H), i, i, i, d, d, F, F, F, i, vp]
        L.kv_set_medium.argtypes = [H, F, F, F]
        L.kv_selftest_wait.argtypes = [H]
        L.kv_state_bytes.argtypes = [H]
        L.kv_state_bytes.restype = ctypes.c_longlong
        L.kv_save_state.argtypes = [H, vp, i, ctypes.POINTER(ctypes.c_longlong)]
        L.kv_load_state.argtypes = [H, vp, i, ctypes.c_longlong]
        L.kv_stable_dt_op.argtypes = [i, i, i, d, F, F, F, i, ctypes.POINTER(d)]
        L.kv_set_operator.argtypes = [H, i, F, F, F]
        L.kv_set_medium_encoding.argtypes = [H, i]
        L.kv_medium_classes.argtypes = [H]
        L.kv_medium_classes.restype = i
        L.kv_set_envelope.argtypes = [H, vp, i, i]
        L.kv_set_sensors.argtypes = [H, vp, i, i]
        L.kv_reset.argtypes = [H]
        L.kv_set_initial_velocity.argtypes = [H, F, F, F]
        L.kv_project_force.argtypes = [H, F, F, F, d, i, i, vp, ctypes.POINTER(KvCgStats)]
        L.kv_clear_force.argtypes = [H]
        L.kv_step_force.argtypes = [H, F, F, F, d, i, i, ctypes.POINTER(KvCgStats)]
        L.kv_step.argtypes = [H, i]
        L.kv_steps_taken.argtypes = [H]
        L.kv_steps_taken.restype = ctypes.c_longlong
        L.kv_read_traces.argtypes = [H, vp, i, ctypes.POINTER(i)]
        L.kv_read_field.argtypes = [H, i, i, vp, i]
        L.kv_sync.argtypes = [H]
        L.kv_set_step_config.argtypes = [H, i, i, i, i, i]
        L.kv_set_cg_config.argtypes = [H, i]
        L.kv_get_cg_config.argtypes = [H, ctypes.POINTER(ctypes.c_int)]
        L.kv_autotune_cg.argtypes = [H, F, F, F, i, ctypes.POINTER(d)]
        L.kv_get_step_config.argtypes = [H, ctypes.POINTER(ctypes.c_int)]
        L.kv_autotune_step.argtypes = [H, i, ctypes.POINTER(d)]
        L.kv_launch_count.argtypes = [H]
        L.kv_launch_count.restype = ctypes.c_longlong
        L.kv_destroy.argtypes = [H]
        L.kv_apply_preconditioner.argtypes = [H, i, i, i, vp, vp, ctypes.POINTER(d)]
        L.kv_project_force_noalloc.argtypes = [i, i, i, d, vp, vp, vp, d, i, vp,
                                               ctypes.POINTER(KvCgStats), vp]
        L.kv_batch_create.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(vp)]
        L.kv_batch_set_config.argtypes = [vp, i, i, i, i]
        L.kv_batch_get_config.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        L.kv_batch_autotune.argtypes = [vp, i, ctypes.POINTER(d)]
        L.kv_batch_step.argtypes = [vp, i]
        L.kv_batch_launch_count.argtypes = [vp]
        L.kv_batch_launch_count.restype = ctypes.c_longlong
        L.kv_batch_destroy.argtypes = [vp]
        L.kv_share_force.argtypes = [H, H]
        L.kv_net_create.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(ctypes.c_int), i, i, i, vp]
        L.kv_net_destroy.argtypes = [vp]
        L.kv_net_num_params.argtypes = [vp]
        L.kv_net_num_params.restype = ctypes.c_longlong
        L.kv_net_init.argtypes = [vp, ctypes.c_ulonglong]
        L.kv_net_set_loss.argtypes = [vp, i]
        L.kv_net_get_params.argtypes = [vp, vp]
        L.kv_net_set_params.argtypes = [vp, vp]
        L.kv_net_train_step.argtypes = [vp, i, i, i, d, vp, vp, d, ctypes.POINTER(d)]
        L.kv_net_predict.argtypes = [vp, i, i, i, d, vp, vp]
        L.kv_attach_net.argtypes = [H, vp]
        L.kv_nn_conv3d_fwd.argtypes = [i, i, i, i, i, vp, vp, vp, vp, i, i, vp]
        L.kv_nn_conv3d_flip.argtypes = [i, i, vp, vp, vp]
        L.kv_nn_conv3d_bwd_weight.argtypes = [i, i, i, i, i, vp, vp, vp, vp, vp]
        for name in ("kv_stable_dt", "kv_create", "kv_set_medium", "kv_set_envelope",
                     "kv_set_sensors", "kv_reset", "kv_set_initial_velocity", "kv_project_force",
                     "kv_clear_force", "kv_step_force", "kv_step", "kv_read_traces", "kv_read_field", "kv_sync",
                     "kv_set_step_config", "kv_get_step_config", "kv_autotune_step",
                     "kv_destroy", "kv_project_force_noalloc", "kv_batch_create",
                     "kv_batch_set_config", "kv_batch_get_config", "kv_batch_autotune",
                     "kv_batch_step", "kv_batch_destroy", "kv_share_force", "kv_net_create",
                     "kv_net_destroy", "kv_net_init", "kv_net_set_loss", "kv_net_get_params", "kv_net_set_params",
                     "kv_net_train_step", "kv_net_predict", "kv_attach_net", "kv_nn_conv3d_fwd",
                     "kv_nn_conv3d_flip", "kv_nn_conv3d_bwd_weight"):
            getattr(L, name).restype = ctypes.c_int
        _LIB = L
    return _LIB


def _status_name(s):
    try:
        return lib().kv_status_string(int(s)).decode()
    except Exception:
        return str(s)


def _check(st, h=None):
    if st != KV_OK:
        msg = lib().kv_last_error(h).decode(errors="replace")
        raise KvError(st, msg)


def _producers_done(t):
    """libkv works on its handle's own stream, which is not ordered with
    torch's: wait until the work torch has queued on the tensor's device
    (which may still be writing `t`, or may later overwrite it) is done."""
    import torch
    torch.cuda.current_stream(t.device).synchronize()


def field(x, keep):
    """KvField for a scalar, NumPy array or torch tensor (float32, dense,
    C-contiguous). `keep` collects objects that must outlive the call. A CUDA
    tensor is complete on torch's current stream before libkv reads it."""
    if x is None:
        return KvField(None, 0.0, KV_SCALAR)
    if isinstance(x, (int, float, np.floating, np.integer)):
        return KvField(None, float(x), KV_SCALAR)
    if isinstance(x, np.ndarray):
        a = np.ascontiguousarray(x, dtype=np.float32)
        keep.append(a)
        return KvField(a.ctypes.data, 0.0, KV_HOST)
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(x, torch.Tensor):
        if x.dtype != torch.float32 or not x.is_contiguous():
            x = x.contiguous().to(torch.float32)
        keep.append(x)
        if x.is_cuda:
            _producers_done(x)
        return KvField(x.data_ptr(), 0.0, KV_DEVICE if x.is_cuda else KV_HOST)
    raise TypeError(f"unsupported field type {type(x)}")


def _ptr(x, keep):
    """Raw pointer and kv_where of a NumPy array or torch tensor."""
    if isinstance(x, np.ndarray):
        keep.append(x)
        return x.ctypes.data, KV_HOST
    import torch
    if isinstance(x, torch.Tensor):
        keep.append(x)
        if x.is_cuda:
            _producers_done(x)
        return x.data_ptr(), (KV_DEVICE if x.is_cuda else KV_HOST)
    raise TypeError(f"unsupported buffer type {type(x)}")


def _check_f32_buffer(fn, name, t, numel):
    """Raise ValueError unless t is a contiguous float32 torch tensor of numel elements."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{fn}: {name} must be a torch tensor, got {type(t).__name__}")
    if t.dtype != torch.float32:
        raise ValueError(f"{fn}: {name} must be float32, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{fn}: {name} must be contiguous")
    if t.numel() != numel:
        raise ValueError(f"{fn}: {name} holds {t.numel()} elements, expected {numel}")


def kv_stable_dt(nx, ny, nz, dx, G, rho, eta):
    keep = []
    out = ctypes.c_double()
    _check(lib().kv_stable_dt(nx, ny, nz, dx, field(G, keep), field(rho, keep), field(eta, keep),
                              ctypes.byref(out)))
    return out.value


def kv_stable_dt_op(nx, ny, nz, dx, G, rho, eta, op):
    keep = []
    out = ctypes.c_double()
    _check(lib().kv_stable_dt_op(nx, ny, nz, dx, field(G, keep), field(rho, keep), field(eta, keep),
                                 int(op), ctypes.byref(out)))
    return out.value


def kv_create(nx, ny, nz, dx, dt, G, rho, eta, precision=KV_FP32, stream=None):
    keep = []
    h = ctypes.c_void_p()
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(lib().kv_create(ctypes.byref(h), nx, ny, nz, dx, dt, field(G, keep), field(rho, keep),
                           field(eta, keep), precision, s))
    return h


def kv_set_medium(h, G, rho, eta):
    keep = []
    _check(lib().kv_set_medium(h, field(G, keep), field(rho, keep), field(eta, keep)), h)


def kv_set_operator(h, op, G, rho, eta):
    keep = []
    _check(lib().kv_set_operator(h, int(op), field(G, keep), field(rho, keep), field(eta, keep)), h)


def kv_set_medium_encoding(h, encoding):
    """KV_MEDIUM_AUTO (class bytes for a medium of at most 256 (A', B') pairs) or KV_MEDIUM_FIELDS."""
    _check(lib().kv_set_medium_encoding(h, int(encoding)), h)


def kv_medium_classes(h):
    """Number of medium classes the step reads (0: the coefficient fields)."""
    return int(lib().kv_medium_classes(h))


def kv_selftest_wait(h):
    """Runs the bounded-wait failure path; returns the kv_status (KV_ERR_TIMEOUT)."""
    return int(lib().kv_selftest_wait(h))


def kv_state_bytes(h):
    return int(lib().kv_state_bytes(h))


def kv_save_state(h, buf):
    """Copy the state (u^n, d^n in the handle's padded layout) into buf, a
    NumPy array or CUDA tensor of kv_state_bytes(h) bytes; returns the step."""
    keep = []
    p, where = _ptr(buf, keep)
    step = ctypes.c_longlong()
    _check(lib().kv_save_state(h, p, where, ctypes.byref(step)), h)
    return step.value


def kv_load_state(h, buf, step):
    keep = []
    p, where = _ptr(buf, keep)
    _check(lib().kv_load_state(h, p, where, int(step)), h)


def kv_set_envelope(h, g):
    keep = []
    if isinstance(g, np.ndarray):
        g = np.ascontiguousarray(g, np.float32)
    p, where = _ptr(g, keep)
    _check(lib().kv_set_envelope(h, p, int(len(g)), where), h)


def kv_set_sensors(h, ijk, capacity):
    ijk = np.ascontiguousarray(np.asarray(ijk, np.int32).reshape(-1, 3))
    _check(lib().kv_set_sensors(h, ijk.ctypes.data, ijk.shape[0], int(capacity)), h)


def kv_reset(h):
    _check(lib().kv_reset(h), h)


def kv_set_initial_velocity(h, vx, vy, vz):
    keep = []
    _check(lib().kv_set_initial_velocity(h, field(vx, keep), field(vy, keep), field(vz, keep)), h)


def kv_project_force(h, fx, fy, fz, tol, max_iter=0, mode=0, fs_out=None, check=True):
    """Returns the stats dict. With check=False a CG status (maxiter,
    breakdown, non-finite) is returned in stats['status'] instead of raised."""
    keep = []
    st = KvCgStats()
    fs_ptr = None
    if fs_out is not None:
        fs_ptr, where = _ptr(fs_out, keep)
        if where != KV_DEVICE:
            raise ValueError("fs_out must be a CUDA tensor")
    rc = lib().kv_project_force(h, field(fx, keep), field(fy, keep), field(fz, keep), float(tol),
                                int(max_iter), int(mode), fs_ptr, ctypes.byref(st))
    d = st.as_dict()
    d["rc"] = rc
    if check or rc not in (KV_CG_MAXITER, KV_CG_BREAKDOWN, KV_ERR_NONFINITE):
        _check(rc, h)
    return d


def kv_apply_preconditioner(h, r, z):
    """z = M r with the mode-4 multigrid V-cycle (see include/kv.h). r, z:
    contiguous float32 CUDA tensors of shape (nz, ny, nx), the handle's grid.
    Returns r.z over the interior."""
    import torch
    for name, t in (("r", r), ("z", z)):
        if not isinstance(t, torch.Tensor) or t.dim() != 3:
            raise ValueError(f"kv_apply_preconditioner: {name} must be a 3D torch tensor (nz, ny, nx)")
        _check_f32_buffer("kv_apply_preconditioner", name, t, r.numel())
        if not t.is_cuda:
            raise ValueError("kv_apply_preconditioner takes device tensors")
    if tuple(z.shape) != tuple(r.shape):
        raise ValueError("kv_apply_preconditioner: r and z differ in shape")
    nz, ny, nx = (int(v) for v in r.shape)
    rz = ctypes.c_double()
    _check(lib().kv_apply_preconditioner(h, nx, ny, nz, ctypes.c_void_p(r.data_ptr()),
                                         ctypes.c_void_p(z.data_ptr()), ctypes.byref(rz)), h)
    return rz.value


def kv_project_force_noalloc(nx, ny, nz, dx, fx, fy, fz, tol, fs_out, max_iter=0, stream=None):
    """Projection without device allocation (working set in libkv's static
    device array; see include/kv.h). fx, fy, fz, fs_out: CUDA tensors.
    Returns the stats dict.

    The library reads nx*ny*nz contiguous float32 values per force component
    and writes 3*nx*ny*nz to fs_out, so every buffer is checked for type, dtype,
    contiguity, element count and device here, before any pointer is passed."""
    n = int(nx) * int(ny) * int(nz)
    for name, t, want in (("fx", fx, n), ("fy", fy, n), ("fz", fz, n), ("fs_out", fs_out, 3 * n)):
        _check_f32_buffer("kv_project_force_noalloc", name, t, want)
    keep = []
    ptrs = []
    for t in (fx, fy, fz, fs_out):
        ptr, where = _ptr(t, keep)
        if where != KV_DEVICE:
            raise ValueError("kv_project_force_noalloc takes device tensors")
        ptrs.append(ptr)
    st = KvCgStats()
    s = None if stream is None else ctypes.c_void_p(int(stream))
    rc = lib().kv_project_force_noalloc(int(nx), int(ny), int(nz), float(dx), ptrs[0], ptrs[1],
                                        ptrs[2], float(tol), int(max_iter), ptrs[3],
                                        ctypes.byref(st), s)
    _check(rc, None)
    return st.as_dict()


def kv_step_force(h, fx, fy, fz, tol, max_iter=0, mode=3):
    """One step with this step's force projected on its own (mode 0: CG from
    zero, mode 3: from the previous potential); returns the projection's stats."""
    keep = []
    st = KvCgStats()
    _check(lib().kv_step_force(h, field(fx, keep), field(fy, keep), field(fz, keep), float(tol),
                               int(max_iter), int(mode), ctypes.byref(st)), h)
    return st.as_dict()


def kv_clear_force(h):
    _check(lib().kv_clear_force(h), h)


def kv_step(h, n):
    _check(lib().kv_step(h, int(n)), h)


def kv_steps_taken(h):
    return int(lib().kv_steps_taken(h))


def kv_read_traces(h, out):
    """Fill `out` (NumPy array or torch tensor, float32 for KV_FP32 / float64 for
    KV_FP64, at least [n_steps, n_sensors, 3]); returns the steps written."""
    keep = []
    p, where = _ptr(out, keep)
    n = ctypes.c_int()
    _check(lib().kv_read_traces(h, p, where, ctypes.byref(n)), h)
    return n.value


def kv_read_field(h, which, comp, out):
    keep = []
    p, where = _ptr(out, keep)
    _check(lib().kv_read_field(h, int(which), int(comp), p, where), h)
    return out


def kv_sync(h):
    _check(lib().kv_sync(h), h)


def kv_set_step_config(h, variant=-1, tx=0, ty=0, zc=0, ns=0):
    _check(lib().kv_set_step_config(h, int(variant), int(tx), int(ty), int(zc), int(ns)), h)


def kv_get_step_config(h):
    cfg = (ctypes.c_int * 5)()
    _check(lib().kv_get_step_config(h, cfg), h)
    return dict(zip(("variant", "tx", "ty", "zc", "ns"), list(cfg)))


def kv_set_cg_config(h, zc):
    _check(lib().kv_set_cg_config(h, int(zc)), h)


def kv_get_cg_config(h):
    zc = ctypes.c_int()
    _check(lib().kv_get_cg_config(h, ctypes.byref(zc)), h)
    return zc.value


def kv_autotune_cg(h, fx, fy, fz, iters=40):
    keep = []
    out = ctypes.c_double()
    _check(lib().kv_autotune_cg(h, field(fx, keep), field(fy, keep), field(fz, keep), int(iters),
                                ctypes.byref(out)), h)
    return out.value


def kv_autotune_step(h, trial_steps=8):
    best = ctypes.c_double()
    _check(lib().kv_autotune_step(h, int(trial_steps), ctypes.byref(best)), h)
    return best.value


def kv_launch_count(h):
    return int(lib().kv_launch_count(h))


def kv_destroy(h):
    if h:
        lib().kv_destroy(h)


def kv_batch_create(handles):
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h
                                             for h in handles])
    b = ctypes.c_void_p()
    _check(lib().kv_batch_create(ctypes.byref(b), len(handles), arr))
    return b


def kv_batch_set_config(b, tx, ty, zc, ns):
    _check(lib().kv_batch_set_config(b, int(tx), int(ty), int(zc), int(ns)))


def kv_batch_get_config(b):
    cfg = (ctypes.c_int * 4)()
    _check(lib().kv_batch_get_config(b, cfg))
    return dict(zip(("tx", "ty", "zc", "ns"), list(cfg)))


def kv_batch_autotune(b, trial_steps=4):
    best = ctypes.c_double()
    _check(lib().kv_batch_autotune(b, int(trial_steps), ctypes.byref(best)))
    return best.value


def kv_batch_step(b, n):
    _check(lib().kv_batch_step(b, int(n)))


def kv_batch_launch_count(b):
    return int(lib().kv_batch_launch_count(b))


def kv_batch_destroy(b):
    if b:
        lib().kv_batch_destroy(b)


def kv_share_force(dst, src):
    _check(lib().kv_share_force(dst, src), dst)


def _dptr(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    _producers_done(t)
    return t.data_ptr()


def _stream(stream):
    return None if stream is None else ctypes.c_void_p(int(stream))


def kv_net_create(channels, max_shape, stream=None):
    """channels: per level (16/32/64); max_shape: (nx, ny, nz)."""
    ch = (ctypes.c_int * len(channels))(*channels)
    n = ctypes.c_void_p()
    _check(lib().kv_net_create(ctypes.byref(n), len(channels), ch, int(max_shape[0]),
                               int(max_shape[1]), int(max_shape[2]), _stream(stream)))
    return n


def kv_net_destroy(n):
    if n:
        lib().kv_net_destroy(n)


def kv_net_num_params(n):
    return int(lib().kv_net_num_params(n))


def kv_net_init(n, seed=0):
    _check(lib().kv_net_init(n, ctypes.c_ulonglong(seed)))


KV_LOSS_MSE, KV_LOSS_RESIDUAL = 0, 1


def kv_net_set_loss(n, kind):
    """Training loss of the net: KV_LOSS_MSE (potential) or KV_LOSS_RESIDUAL
    (squared residual of the prediction)."""
    _check(lib().kv_net_set_loss(n, int(kind)))


def kv_net_get_params(n):
    out = np.empty(kv_net_num_params(n), np.float32)
    _check(lib().kv_net_get_params(n, out.ctypes.data))
    return out


def kv_net_set_params(n, params):
    p = np.ascontiguousarray(params, np.float32)
    assert p.size == kv_net_num_params(n)
    _check(lib().kv_net_set_params(n, p.ctypes.data))


def kv_net_train_step(n, shape, dx, b, phi, lr):
    loss = ctypes.c_double()
    _check(lib().kv_net_train_step(n, int(shape[0]), int(shape[1]), int(shape[2]), float(dx),
                                   _dptr(b), _dptr(phi), float(lr), ctypes.byref(loss)))
    return loss.value


def kv_net_predict(n, shape, dx, b, phi_out):
    _check(lib().kv_net_predict(n, int(shape[0]), int(shape[1]), int(shape[2]), float(dx), _dptr(b),
                                _dptr(phi_out)))
    return phi_out


def kv_attach_net(h, n):
    _check(lib().kv_attach_net(h, n), h)


def kv_nn_conv3d_fwd(shape, cin, cout, x, W, bias, out, relu=False, stream=None):
    _check(lib().kv_nn_conv3d_fwd(int(shape[0]), int(shape[1]), int(shape[2]), int(cin), int(cout),
                                  _dptr(x), _dptr(W), None if bias is None else _dptr(bias),
                                  _dptr(out), int(out.dtype.is_floating_point and out.element_size() == 4),
                                  int(relu), _stream(stream)))


def kv_nn_conv3d_flip(cin, cout, W, Wt, stream=None):
    _check(lib().kv_nn_conv3d_flip(int(cin), int(cout), _dptr(W), _dptr(Wt), _stream(stream)))


def kv_nn_conv3d_bwd_weight(shape, cin, cout, x, g, gW, gb=None, stream=None):
    _check(lib().kv_nn_conv3d_bwd_weight(int(shape[0]), int(shape[1]), int(shape[2]), int(cin),
                                         int(cout), _dptr(x), _dptr(g), _dptr(gW),
                                         None if gb is None else _dptr(gb), _stream(stream)))


def kv_last_error(h=None):
    return lib().kv_last_error(h).decode(errors="replace")


def exported_symbols():
    """Names declared in include/kv.h (used by the load test)."""
    import re
    hdr = os.path.join(_HERE, "..", "include", "kv.h")
    src = open(hdr).read()
    return sorted(set(re.findall(r"\b(kv_[a-z_0-9]+)\s*\(", src)))
