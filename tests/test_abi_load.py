"""CPU checks of the C-ABI library: it loads, exports every symbol the header
declares, and its host-side logic (stability limit, argument checks) works
without a GPU."""
import ctypes
import subprocess

import numpy as np
import pytest

import oracle as orc
from paper_2607_28414_b300 import build as kvbuild
from paper_2607_28414_b300 import kv


@pytest.fixture(scope="module")
def lib():
    kvbuild.build()
    return kv.lib()


def test_header_symbols_exported(lib):
    names = kv.exported_symbols()
    assert "kv_step" in names and "kv_project_force" in names and "kv_create" in names
    nm = subprocess.run(["nm", "-D", "--defined-only", kv.LIB_PATH], capture_output=True,
                        text=True, check=True).stdout
    exported = {line.split()[-1] for line in nm.splitlines() if line.strip()}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)


def test_stable_dt_scalar_matches_oracle(lib):
    for G, rho, eta in [(4e3, 1000.0, 0.0), (3e3, 1000.0, 0.5), (50e3, 1900.0, 2.0), (1e3, 1040.0, 1.5)]:
        got = kv.kv_stable_dt(16, 16, 16, 2e-4, G, rho, eta)
        assert got == pytest.approx(orc.stable_dt(G, rho, eta, 2e-4), rel=1e-12)


def test_stable_dt_host_arrays_match_oracle(lib):
    rng = np.random.default_rng(4)
    n = (9, 8, 7)
    G = rng.uniform(1e3, 10e3, n[::-1]).astype(np.float32)
    rho = rng.uniform(1000, 1100, n[::-1]).astype(np.float32)
    eta = rng.uniform(0, 1.5, n[::-1]).astype(np.float32)
    got = kv.kv_stable_dt(*n, 1.5e-4, G, rho, eta)
    assert got == pytest.approx(orc.stable_dt(G, rho, eta, 1.5e-4), rel=1e-12)
    # mixing a host array with a scalar is fine
    got2 = kv.kv_stable_dt(*n, 1.5e-4, G, 1000.0, 0.0)
    assert got2 == pytest.approx(orc.stable_dt(G, 1000.0, 0.0, 1.5e-4), rel=1e-12)


def test_argument_errors_without_gpu(lib):
    with pytest.raises(kv.KvError) as e:
        kv.kv_stable_dt(2, 16, 16, 2e-4, 4e3, 1000.0, 0.0)
    assert e.value.status == kv.KV_ERR_ARG
    with pytest.raises(kv.KvError) as e:
        kv.kv_stable_dt(16, 16, 16, 2e-4, 4e3, -1.0, 0.0)
    assert e.value.status == kv.KV_ERR_ARG
    with pytest.raises(kv.KvError) as e:
        kv.kv_create(16, 16, 16, 2e-4, 1.0, 4e3, 1000.0, 0.0)
    assert e.value.status == kv.KV_ERR_UNSTABLE_DT
    assert "stability limit" in str(e.value)
    with pytest.raises(kv.KvError) as e:
        kv.kv_create(16, 16, 16, 2e-4, 1e-6, 4e3, 1000.0, 0.0, precision=7)
    assert e.value.status == kv.KV_ERR_ARG


def test_status_strings(lib):
    assert kv._status_name(kv.KV_CG_MAXITER) == "KV_CG_MAXITER"
    assert kv._status_name(99) == "KV_UNKNOWN"


def test_noalloc_wrapper_rejects_bad_buffers_before_the_call(lib, monkeypatch):
    """The allocation-free projection reads nx*ny*nz float32 values per force
    component and writes 3*nx*ny*nz: the binding refuses anything else before
    a pointer reaches the library (which is replaced here by a trap)."""
    torch = pytest.importorskip("torch")

    class Trap:
        def __getattr__(self, name):
            raise AssertionError(f"library called: {name}")

    monkeypatch.setattr(kv, "lib", lambda: Trap())
    n = (5, 4, 3)
    good = torch.zeros(n[::-1], dtype=torch.float32)
    out = torch.zeros((3,) + n[::-1], dtype=torch.float32)
    bad = [
        (good.double(), good, good, out, "float32"),
        (good, torch.zeros((3, 4, 2), dtype=torch.float32), good, out, "elements"),
        (good, good, good.transpose(0, 2).contiguous().transpose(0, 2), out, "contiguous"),
        (good, good, good, out[:2], "elements"),
        (good, good, good.numpy(), out, "torch tensor"),
    ]
    for fx, fy, fz, fo, what in bad:
        with pytest.raises(ValueError) as e:
            kv.kv_project_force_noalloc(*n, 2e-4, fx, fy, fz, 1e-8, fo)
        assert what in str(e.value)
    # well-formed host tensors pass these checks and are refused as host memory
    with pytest.raises(ValueError) as e:
        kv.kv_project_force_noalloc(*n, 2e-4, good, good, good, 1e-8, out)
    assert "device" in str(e.value)
