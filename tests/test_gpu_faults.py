"""Failure handling made on the host: an injected device-allocation failure
(ZMC_FAULT=alloc in the environment, read at each call) must come back as
ZMC_ERR_OOM with the caller's output untouched, and the handle must work
again once the fault is gone.  Nothing here faults, traps or stalls a GPU:
the library refuses before it calls cudaMalloc."""
import ctypes
import math

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zmc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_07916_gb300 import build
    build.build()
    from paper_1902_07916_gb300 import zmc as mod
    return mod


def sentinel_result(zmc):
    out = zmc.zmc_result()
    out.value = out.std = 12345.0
    out.status = -7
    return out


def test_injected_allocation_failure_single(zmc, monkeypatch):
    h = zmc.zmc_create(3, [0.0] * 3, [10.0] * 3, 4, 1000, 5, 2, 2.0, 0)
    try:
        zmc.zmc_set_integrand(h, "sin_sum")
        monkeypatch.setenv("ZMC_FAULT", "alloc")
        out = sentinel_result(zmc)
        rc = zmc.lib.zmc_integrate(h, None, ctypes.byref(out))
        assert rc == zmc.ZMC_ERR_OOM
        assert (out.value, out.std, out.status) == (12345.0, 12345.0, -7)
        assert "injected" in zmc.zmc_last_error(h)
        monkeypatch.delenv("ZMC_FAULT")
        r = zmc.zmc_integrate(h)
        assert r.status == zmc.ZMC_OK and math.isfinite(r.value) and r.samples > 0
    finally:
        zmc.zmc_destroy(h)


def test_injected_allocation_failure_batch(zmc, monkeypatch):
    hs = []
    try:
        for seed in (1, 2):
            h = zmc.zmc_create(2, [0.0] * 2, [1.0] * 2, 3, 64, 4, 2, 1.0, seed)
            hs.append(h)
            zmc.zmc_set_integrand(h, "genz_corner", [1.0, 2.0])
        monkeypatch.setenv("ZMC_FAULT", "alloc")
        arr = (ctypes.c_void_p * 2)(*[h.value for h in hs])
        outs = (zmc.zmc_result * 2)(sentinel_result(zmc), sentinel_result(zmc))
        rc = zmc.lib.zmc_integrate_batch(2, arr, None, outs)
        assert rc == zmc.ZMC_ERR_OOM
        assert all((o.value, o.status) == (12345.0, -7) for o in outs)
        monkeypatch.delenv("ZMC_FAULT")
        res = zmc.zmc_integrate_batch(hs)
        assert all(r.status == zmc.ZMC_OK and r.samples > 0 for r in res)
    finally:
        for h in hs:
            zmc.zmc_destroy(h)
