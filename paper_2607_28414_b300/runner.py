"""Drive one workload through libkv: create, project the force once, step, read
traces (the pre-computed projection pipeline of Sec. 3.3). Only calls the
binding; all arithmetic happens in the CUDA library."""
from __future__ import annotations

import numpy as np

from . import inputs
from . import kv


def to_device(x, device):
    """Arrays become CUDA tensors on `device`; scalars pass through."""
    import torch
    if isinstance(x, np.ndarray):
        return torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(device)
    return x


class Solver:
    """Owns one libkv handle for a workload."""

    def __init__(self, w: inputs.Workload, precision=kv.KV_FP32, dt=None, n_steps=None,
                 device="cuda:0", stream=None, step_config=None, operator=kv.KV_OP_POINTWISE,
                 envelope=None):
        import torch
        self.w = w
        self.device = torch.device(device)
        self.precision = precision
        self.n_steps = w.n_steps if n_steps is None else n_steps
        self.medium = [to_device(x, self.device) for x in (w.G, w.rho, w.eta)]
        self.force = [to_device(f, self.device) for f in w.force]
        if dt is None:
            lim = kv.kv_stable_dt(w.nx, w.ny, w.nz, w.dx, *self.medium)
            if operator != kv.KV_OP_POINTWISE:
                lim = min(lim, kv.kv_stable_dt_op(w.nx, w.ny, w.nz, w.dx, *self.medium, operator))
            dt = w.cfl_fraction * lim
        self.dt = dt
        self.h = kv.kv_create(w.nx, w.ny, w.nz, w.dx, dt, *self.medium, precision=precision,
                              stream=stream)
        if operator != kv.KV_OP_POINTWISE:
            kv.kv_set_operator(self.h, operator, *self.medium)
        if step_config:
            kv.kv_set_step_config(self.h, **step_config)
        self.envelope = (inputs.push_envelope(self.n_steps, dt, w.t_push) if envelope is None
                         else envelope(self.n_steps, dt))
        kv.kv_set_envelope(self.h, self.envelope)
        kv.kv_set_sensors(self.h, w.sensors, self.n_steps)
        self.trace_dtype = torch.float64 if precision == kv.KV_FP64 else torch.float32
        self.traces = torch.zeros((self.n_steps, len(w.sensors), 3), dtype=self.trace_dtype,
                                  device=self.device)
        self.stats = None

    def project(self, tol=None, max_iter=0, fs_out=None):
        self.stats = kv.kv_project_force(self.h, *self.force, self.w.tol if tol is None else tol,
                                         max_iter, 0, fs_out)
        return self.stats

    def step(self, n=None):
        kv.kv_step(self.h, self.n_steps if n is None else n)

    def read_traces(self, out=None):
        out = self.traces if out is None else out
        n = kv.kv_read_traces(self.h, out)
        return out[:n]

    def reset(self):
        kv.kv_reset(self.h)

    def close(self):
        if self.h:
            kv.kv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
