"""The C ABI library loads without a GPU, exports every entry point that
include/zmc.h declares, and validates arguments on the host."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "zmc.h")


@pytest.fixture(scope="module")
def zmc():
    from paper_1902_07916_gb300 import build
    build.build()
    from paper_1902_07916_gb300 import zmc as mod
    return mod


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"ZMC_API\s+[\w\s\*]+?\b(zmc_\w+)\s*\(", text)))


def test_header_declares_the_abi():
    names = declared_symbols()
    for must in ["zmc_create", "zmc_set_integrand", "zmc_set_precision", "zmc_set_limits",
                 "zmc_integrate", "zmc_enqueue", "zmc_read_result", "zmc_integrate_batch",
                 "zmc_last_error", "zmc_destroy", "zmc_philox_words", "zmc_set_trace",
                 "zmc_trace_level"]:
        assert must in names


def test_library_exports_every_declared_symbol(zmc):
    lib = ctypes.CDLL(zmc.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_result_struct_matches_header(zmc):
    # 2 doubles, 2 int64, 2 int32, then 6 arrays of 16 eight-byte values and
    # the five int64 of the work plan
    assert ctypes.sizeof(zmc.zmc_result) == 16 + 16 + 8 + 6 * 16 * 8 + 5 * 8


@pytest.mark.parametrize("kw,bad", [
    ({"dim": 0}, "dim"), ({"dim": 17}, "dim"), ({"k": 1}, "k"), ({"n": 1}, "n"),
    ({"num_trials": 1}, "num_trials"), ({"depth": 0}, "depth"), ({"depth": 17}, "depth"),
    ({"sigma_multiplier": -1.0}, "sigma"), ({"sigma_multiplier": float("nan")}, "sigma"),
    ({"hi": [0.0, 1.0]}, "lo"), ({"k": 70000}, "k^dim"),
])
def test_create_rejects_bad_arguments(zmc, kw, bad):
    args = dict(dim=2, lo=[0.0, 0.0], hi=[1.0, 1.0], k=3, n=100, num_trials=4, depth=2,
                sigma_multiplier=1.0, seed=1)
    args.update(kw)
    if "dim" in kw and kw["dim"] > 0:
        args["lo"] = [0.0] * kw["dim"]
        args["hi"] = [1.0] * kw["dim"]
    with pytest.raises(zmc.ZmcError) as e:
        zmc.zmc_create(**args)
    assert e.value.code == zmc.ZMC_ERR_ARG
    assert bad.split("^")[0] in zmc.zmc_last_error(None)


def test_integrand_validation_on_host(zmc):
    h = zmc.zmc_create(3, [0.0] * 3, [1.0] * 3, 2, 16, 2, 1, 0.0, 0)
    try:
        with pytest.raises(zmc.ZmcError) as e:
            zmc.zmc_set_integrand(h, "no_such_integrand")
        assert e.value.code == zmc.ZMC_ERR_ARG
        with pytest.raises(zmc.ZmcError) as e:
            zmc.zmc_set_integrand(h, "genz_gauss", [1.0, 2.0])   # needs 2*dim
        assert "takes 6 parameters" in zmc.zmc_last_error(h)
        with pytest.raises(zmc.ZmcError):
            zmc.zmc_set_integrand(h, "gauss_norm", [-0.1])
        with pytest.raises(zmc.ZmcError):
            zmc.zmc_set_integrand(h, "constant", [float("inf")])
        with pytest.raises(zmc.ZmcError):
            zmc.zmc_set_integrand(h, "expr:x[0]; }")            # not one expression
        zmc.zmc_set_integrand(h, "genz_corner", [1.0, 2.0, 3.0])
        with pytest.raises(zmc.ZmcError):
            zmc.zmc_set_precision(h, 7)
        with pytest.raises(zmc.ZmcError):
            zmc.zmc_set_limits(h, 7, 1 << 40)                   # below level 1 (8 cells)
        zmc.zmc_set_limits(h, 8, 8 * 16 * 2)
    finally:
        zmc.zmc_destroy(h)


def test_integrate_without_integrand_reports_it(zmc):
    h = zmc.zmc_create(1, [0.0], [1.0], 2, 16, 2, 1, 0.0, 0)
    try:
        with pytest.raises(zmc.ZmcError) as e:
            zmc.zmc_integrate(h)
        assert e.value.code == zmc.ZMC_ERR_NOINTEGRAND
    finally:
        zmc.zmc_destroy(h)


# ------------------------------------------------------- expressions, no device

@pytest.mark.parametrize("precision", ["fp64", "fp32_fp64acc", "fp32_kahan"])
@pytest.mark.parametrize("expr,dim", [
    ("sin(x[0] + x[1] + x[2])", 3),
    ("(x[0] < p[0] ? p[1] : 0.0) * (1.0 + x[1])", 2),
    ("exp(-(x[0]*x[0] + x[1]*x[1]) / 2e-4) * erf(x[2])", 3),
    ("x[15] * x[0]", 16),
])
def test_expressions_compile_without_a_device(zmc, precision, expr, dim):
    # the embedded device headers must compile under NVRTC in every mode
    zmc.zmc_check_expression(expr, dim, precision, cc=(10, 3))


def test_expression_compile_errors_without_a_device(zmc):
    with pytest.raises(zmc.ZmcError) as e:
        zmc.zmc_check_expression("x[0] + no_such_function(x[1])", 2, "fp32_fp64acc")
    assert e.value.code == zmc.ZMC_ERR_COMPILE
    assert "no_such_function" in str(e.value)
    with pytest.raises(zmc.ZmcError) as e:
        zmc.zmc_check_expression("x[0]; x[1]", 2)
    assert e.value.code == zmc.ZMC_ERR_COMPILE
    with pytest.raises(zmc.ZmcError) as e:
        zmc.zmc_check_expression("x[0]", 17)
    assert e.value.code == zmc.ZMC_ERR_ARG
    with pytest.raises(zmc.ZmcError) as e:
        zmc.zmc_check_expression("", 2)
    assert e.value.code == zmc.ZMC_ERR_ARG


def test_work_plan_and_tuning_validation_on_host(zmc):
    h = zmc.zmc_create(3, [0.0] * 3, [1.0] * 3, 2, 16, 2, 1, 0.0, 0)
    try:
        for bad in ([0, 1024, 64, 1024, 1 << 18], [(1 << 18) + 1, 1024, 64, 1024, 1 << 18],
                    [1 << 18, 0, 64, 1024, 1 << 18], [1 << 18, 1024, -1, 1024, 1 << 18],
                    [1 << 18, 1024, 64, 1024, 0]):
            with pytest.raises(zmc.ZmcError) as e:
                zmc.zmc_set_work_plan(h, bad)
            assert e.value.code == zmc.ZMC_ERR_ARG and "work plan" in zmc.zmc_last_error(h)
        zmc.zmc_set_work_plan(h, [1 << 17, 512, 32, 512, 1 << 16])
        zmc.zmc_set_work_plan(h, None)
        with pytest.raises(zmc.ZmcError) as e:
            zmc.zmc_set_tuning(h, 4)
        assert e.value.code == zmc.ZMC_ERR_ARG
        zmc.zmc_set_tuning(h, zmc.ZMC_TUNE_SHAPE | zmc.ZMC_TUNE_PLAN)
        zmc.zmc_set_tuning(h, 0)
    finally:
        zmc.zmc_destroy(h)


def test_build_id_follows_the_sources(tmp_path, monkeypatch):
    # The tuner's file cache (ZMC_TUNE_CACHE) keys its entries by this id:
    # the same sources give the same id, the checked build and any changed
    # source another.
    import shutil
    from paper_1902_07916_gb300 import build as b
    srcs = [os.path.join(b.CSRC, f) for f in b.SOURCES]
    a = b._build_id(srcs, False)
    assert re.fullmatch(r"0x[0-9a-f]{16}ULL", a)
    assert a == b._build_id(srcs, False)
    assert a != b._build_id(srcs, True)
    csrc = tmp_path / "csrc"
    shutil.copytree(b.CSRC, csrc)
    (csrc / "select.cu").write_text((csrc / "select.cu").read_text() + "\n")
    monkeypatch.setattr(b, "CSRC", str(csrc))
    assert b._build_id([str(csrc / f) for f in b.SOURCES], False) != a
