"""Python binding of the C ABI in include/zmc.h (ctypes; marshalling only).

Every function has the name of the C entry point it calls.  Status codes
other than ZMC_OK raise ZmcError, except the result statuses ZMC_ERR_BUDGET
and ZMC_ERR_NONFINITE of an integration, which are returned with the result
(the result is still valid: see zmc_integrate in the header).

The library must have been built (``paper_1902_07916_gb300.build.build()``);
importing this module without it raises ImportError -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# ZMC_LIBRARY selects another build of the library (the bounds-guarded test
# build, _build_checked/libzmc.so); the default is the in-tree build.
LIB_PATH = os.environ.get("ZMC_LIBRARY") or os.path.join(_HERE, "_build", "libzmc.so")

ZMC_OK = 0
ZMC_ERR_ARG = 1
ZMC_ERR_COMPILE = 2
ZMC_ERR_BUDGET = 3
ZMC_ERR_NONFINITE = 4
ZMC_ERR_OOM = 5
ZMC_ERR_CUDA = 6
ZMC_ERR_TIMEOUT = 7
ZMC_ERR_NOINTEGRAND = 8
ZMC_ERR_CHECK = 9

ZMC_FP64 = 0
ZMC_FP32_FP64ACC = 1
ZMC_FP32_KAHAN = 2
PRECISIONS = {"fp64": ZMC_FP64, "fp32_fp64acc": ZMC_FP32_FP64ACC,
              "fp32_kahan": ZMC_FP32_KAHAN}

ZMC_MAX_DIM = 16
ZMC_MAX_DEPTH = 16
ZMC_PLAN_FIELDS = 5
ZMC_TUNE_SHAPE = 1
ZMC_TUNE_PLAN = 2

_D = ZMC_MAX_DEPTH


class zmc_result(ctypes.Structure):
    _fields_ = [
        ("value", ctypes.c_double),
        ("std", ctypes.c_double),
        ("cells_evaluated", ctypes.c_int64),
        ("samples", ctypes.c_int64),
        ("levels_run", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("cells_per_level", ctypes.c_int64 * _D),
        ("flagged_per_level", ctypes.c_int64 * _D),
        ("theta_per_level", ctypes.c_double * _D),
        ("mu_per_level", ctypes.c_double * _D),
        ("sigma_per_level", ctypes.c_double * _D),
        ("min_margin_per_level", ctypes.c_double * _D),
        ("work_plan", ctypes.c_int64 * ZMC_PLAN_FIELDS),
    ]


class ZmcError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__("zmc error %d: %s" % (code, message))
        self.code = code


@dataclass
class Result:
    value: float
    std: float
    cells_evaluated: int
    samples: int
    levels_run: int
    status: int
    cells_per_level: list
    flagged_per_level: list
    theta_per_level: list
    mu_per_level: list
    sigma_per_level: list
    min_margin_per_level: list
    work_plan: list


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libzmc.so is not built (%s); run "
                          "paper_1902_07916_gb300.build.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    H = ctypes.c_void_p
    P = ctypes.POINTER
    sig = {
        "zmc_create": [P(H), ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double),
                       ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                       ctypes.c_double, ctypes.c_uint64],
        "zmc_set_integrand": [H, ctypes.c_char_p, P(ctypes.c_double), ctypes.c_int],
        "zmc_set_precision": [H, ctypes.c_int],
        "zmc_set_limits": [H, ctypes.c_int64, ctypes.c_int64],
        "zmc_integrate": [H, ctypes.c_void_p, P(zmc_result)],
        "zmc_enqueue": [H, ctypes.c_void_p],
        "zmc_read_result": [H, ctypes.c_void_p, P(zmc_result)],
        "zmc_integrate_batch": [ctypes.c_int, P(H), ctypes.c_void_p, P(zmc_result)],
        "zmc_set_trace": [H, ctypes.c_int],
        "zmc_trace_level": [H, ctypes.c_int, P(ctypes.c_int64), P(ctypes.c_int64),
                            P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
                            P(ctypes.c_uint32)],
        "zmc_philox_words": [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                             ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64,
                             ctypes.c_void_p, ctypes.c_void_p],
        "zmc_uniforms": [ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32,
                         ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                         ctypes.c_void_p, ctypes.c_void_p],
        "zmc_set_launch": [H, ctypes.c_int, ctypes.c_int],
        "zmc_launch_shape": [H, P(ctypes.c_int), P(ctypes.c_int)],
        "zmc_set_work_plan": [H, P(ctypes.c_int64)],
        "zmc_set_tuning": [H, ctypes.c_int],
        "zmc_set_profiling": [H, ctypes.c_int],
        "zmc_profile": [H, P(ctypes.c_double), P(ctypes.c_int)],
        "zmc_run_info": [H, P(ctypes.c_int64), P(ctypes.c_int64), P(ctypes.c_int64)],
        "zmc_pipe_probe": [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
        "zmc_level_stats_noalloc": [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int64,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p],
        "zmc_check_expression": [ctypes.c_char_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_char_p, ctypes.c_size_t],
        "zmc_last_error": [H],
        "zmc_destroy": [H],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name == "zmc_last_error" else ctypes.c_int
    return lib


_lib = _load()
lib = _lib


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


def _check(rc: int, h=None):
    if rc != ZMC_OK:
        msg = _lib.zmc_last_error(h)
        raise ZmcError(rc, msg.decode() if msg else "")


def _result(r: zmc_result) -> Result:
    L = r.levels_run
    return Result(r.value, r.std, r.cells_evaluated, r.samples, r.levels_run, r.status,
                  list(r.cells_per_level[:L]), list(r.flagged_per_level[:L]),
                  list(r.theta_per_level[:L]), list(r.mu_per_level[:L]),
                  list(r.sigma_per_level[:L]), list(r.min_margin_per_level[:L]),
                  list(r.work_plan))


def _doubles(values):
    arr = (ctypes.c_double * max(1, len(values)))(*[float(v) for v in values])
    return arr


# ----------------------------------------------------------------- calls

def zmc_create(dim, lo, hi, k, n, num_trials, depth, sigma_multiplier, seed):
    h = ctypes.c_void_p()
    _check(_lib.zmc_create(ctypes.byref(h), int(dim), _doubles(lo), _doubles(hi), int(k),
                           int(n), int(num_trials), int(depth), float(sigma_multiplier),
                           int(seed) & 0xFFFFFFFFFFFFFFFF))
    return h


def zmc_set_integrand(h, name_or_expr: str, params=()):
    params = list(params)
    _check(_lib.zmc_set_integrand(h, name_or_expr.encode(), _doubles(params) if params else None,
                                  len(params)), h)


def zmc_set_precision(h, mode):
    if isinstance(mode, str):
        mode = PRECISIONS[mode]
    _check(_lib.zmc_set_precision(h, int(mode)), h)


def zmc_set_limits(h, max_cells_per_level, max_samples):
    _check(_lib.zmc_set_limits(h, int(max_cells_per_level), int(max_samples)), h)


_RESULT_STATUSES = (ZMC_OK, ZMC_ERR_BUDGET, ZMC_ERR_NONFINITE)


def zmc_integrate(h, stream=None) -> Result:
    out = zmc_result()
    rc = _lib.zmc_integrate(h, _stream_ptr(stream), ctypes.byref(out))
    if rc not in _RESULT_STATUSES:
        _check(rc, h)
    return _result(out)


def zmc_enqueue(h, stream=None):
    _check(_lib.zmc_enqueue(h, _stream_ptr(stream)), h)


def zmc_read_result(h, stream=None) -> Result:
    out = zmc_result()
    rc = _lib.zmc_read_result(h, _stream_ptr(stream), ctypes.byref(out))
    if rc not in _RESULT_STATUSES:
        _check(rc, h)
    return _result(out)


def zmc_integrate_batch(handles, stream=None) -> list:
    n = len(handles)
    arr = (ctypes.c_void_p * max(1, n))(*[h.value for h in handles])
    outs = (zmc_result * max(1, n))()
    rc = _lib.zmc_integrate_batch(n, arr, _stream_ptr(stream), outs)
    if rc not in _RESULT_STATUSES:
        _check(rc)
    return [_result(outs[i]) for i in range(n)]


def zmc_set_trace(h, on: bool):
    _check(_lib.zmc_set_trace(h, 1 if on else 0), h)


def zmc_trace_level(h, level: int, dim: int, trials: int) -> dict:
    cells = ctypes.c_int64()
    flagged = ctypes.c_int64()
    _check(_lib.zmc_trace_level(h, level, ctypes.byref(cells), ctypes.byref(flagged),
                                None, None, None, None), h)
    C, F = cells.value, flagged.value
    stats4 = np.zeros(4)
    sums = np.zeros((max(C, 0), trials, 2))
    cstats = np.zeros((max(C, 0), 2))
    parents = np.zeros((max(F, 0), dim), dtype=np.uint32)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(_lib.zmc_trace_level(h, level, None, None, dp(stats4), dp(sums), dp(cstats),
                                parents.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))), h)
    return {"cells": C, "flagged": F, "mu": stats4[0], "sigma": stats4[1],
            "theta": stats4[2], "min_margin": stats4[3], "sums": sums,
            "cell_stats": cstats, "parents_out": parents}


def zmc_philox_words(seed, c0, c1, c2, c3, count, out_ptr, stream=None):
    _check(_lib.zmc_philox_words(int(seed) & 0xFFFFFFFFFFFFFFFF, c0 & 0xFFFFFFFF,
                                 c1 & 0xFFFFFFFF, c2 & 0xFFFFFFFF, c3 & 0xFFFFFFFF,
                                 int(count), ctypes.c_void_p(int(out_ptr)),
                                 _stream_ptr(stream)))


def zmc_uniforms(seed, level, slot, trial, dim, mode, first, count, out_ptr, stream=None):
    if isinstance(mode, str):
        mode = PRECISIONS[mode]
    _check(_lib.zmc_uniforms(int(seed) & 0xFFFFFFFFFFFFFFFF, int(level), int(slot) & 0xFFFFFFFF,
                             int(trial) & 0xFFFFFFFF, int(dim), int(mode), int(first),
                             int(count), ctypes.c_void_p(int(out_ptr)), _stream_ptr(stream)))


def zmc_set_launch(h, threads=0, ctas_per_sm=0):
    _check(_lib.zmc_set_launch(h, int(threads), int(ctas_per_sm)), h)


def zmc_set_work_plan(h, plan=None):
    """plan: five ints (target_units, min_unit_groups, lane_tile_groups,
    lane_tile_max_groups, lane_tile_min_tiles), or None for the default."""
    arr = None
    if plan is not None:
        arr = (ctypes.c_int64 * ZMC_PLAN_FIELDS)(*[int(v) for v in plan])
    _check(_lib.zmc_set_work_plan(h, arr), h)


def zmc_set_tuning(h, flags=ZMC_TUNE_SHAPE):
    _check(_lib.zmc_set_tuning(h, int(flags)), h)


def zmc_launch_shape(h):
    t, g = ctypes.c_int(), ctypes.c_int()
    _check(_lib.zmc_launch_shape(h, ctypes.byref(t), ctypes.byref(g)), h)
    return t.value, g.value


def zmc_set_profiling(h, on: bool):
    _check(_lib.zmc_set_profiling(h, 1 if on else 0), h)


def zmc_profile(h, depth: int):
    """(per-level sampling-kernel milliseconds, levels that had cells)."""
    ms = (ctypes.c_double * max(1, depth))()
    levels = ctypes.c_int()
    _check(_lib.zmc_profile(h, ms, ctypes.byref(levels)), h)
    return list(ms[:depth]), levels.value


def zmc_run_info(h):
    """(kernels per run, host->device bytes and device->host bytes per call)."""
    k, i, o = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.zmc_run_info(h, ctypes.byref(k), ctypes.byref(i), ctypes.byref(o)), h)
    return k.value, i.value, o.value


def zmc_pipe_probe(kind, iters, blocks, threads, sink_ptr, clocks_ptr, stream=None):
    """Device pointers: sink (blocks * threads uint32), clocks (blocks * 6 int64)."""
    _check(_lib.zmc_pipe_probe(int(kind), int(iters), int(blocks), int(threads),
                               ctypes.c_void_p(int(sink_ptr)), ctypes.c_void_p(int(clocks_ptr)),
                               _stream_ptr(stream)))


def zmc_level_stats_noalloc(sums_ptr, cells, trials, n, volume, sigma_multiplier,
                            cell_stats_ptr, level_stats_ptr, stream=None):
    """Device pointers in, device pointers out; allocates nothing."""
    _check(_lib.zmc_level_stats_noalloc(
        ctypes.c_void_p(int(sums_ptr)), int(cells), int(trials), int(n), float(volume),
        float(sigma_multiplier), ctypes.c_void_p(int(cell_stats_ptr)),
        ctypes.c_void_p(int(level_stats_ptr)), _stream_ptr(stream)))


def zmc_check_expression(expr: str, dim: int, precision="fp64", cc=(10, 3)):
    """Compile an expression integrand with NVRTC for compute capability cc
    without a device.  Returns the compiler's log; raises ZmcError (with the
    log) when it does not compile."""
    mode = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    if expr.startswith("expr:"):
        expr = expr[5:]
    buf = ctypes.create_string_buffer(1 << 16)
    rc = _lib.zmc_check_expression(expr.encode(), int(dim), mode, int(cc[0]), int(cc[1]), buf,
                                   ctypes.sizeof(buf))
    log = buf.value.decode(errors="replace")
    if rc != ZMC_OK:
        raise ZmcError(rc, log)
    return log


def zmc_last_error(h=None) -> str:
    m = _lib.zmc_last_error(h)
    return m.decode() if m else ""


def zmc_destroy(h):
    _check(_lib.zmc_destroy(h))


class Integrator:
    """Owning wrapper of one handle (argument marshalling only)."""

    def __init__(self, dim, lo, hi, k, n, num_trials, depth, sigma_multiplier, seed,
                 integrand=None, params=(), precision=ZMC_FP64, limits=None):
        self.dim, self.trials = int(dim), int(num_trials)
        self.h = zmc_create(dim, lo, hi, k, n, num_trials, depth, sigma_multiplier, seed)
        try:
            if integrand is not None:
                zmc_set_integrand(self.h, integrand, params)
            zmc_set_precision(self.h, precision)
            if limits is not None:
                zmc_set_limits(self.h, *limits)
        except Exception:
            self.close()
            raise

    def integrate(self, stream=None) -> Result:
        return zmc_integrate(self.h, stream)

    def enqueue(self, stream=None):
        zmc_enqueue(self.h, stream)

    def read_result(self, stream=None) -> Result:
        return zmc_read_result(self.h, stream)

    def trace(self, on=True):
        zmc_set_trace(self.h, on)

    def trace_level(self, level):
        return zmc_trace_level(self.h, level, self.dim, self.trials)

    def close(self):
        if getattr(self, "h", None) is not None:
            zmc_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
