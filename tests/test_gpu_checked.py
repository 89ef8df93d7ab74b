"""The bounds-guarded build of the library (ZMC_CHECKED).

compute-sanitizer is closed here, so the library can be built with a check
before every access to a partial-sum, cell-statistics or parent-list buffer:
an index outside the buffer raises the run's status to ZMC_ERR_CHECK (with
the failing site) and skips the access.  This test builds that library (two
registry integrands: sin_sum and genz_corner), runs workloads that exercise
every guarded site -- tiles cut into several units, lane tiles, deeper
levels, the budget rule, a batch and an expression integrand -- in a child
process that loads it, and requires status OK and results equal bit for bit
to the normal build's.  With ZMC_FAULT=capacity the kernels are told half of
level 1's size as their capacity (the buffers keep their real size, so no
access leaves its allocation) and the guard of the cell statistics fires.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [
    # (name, integrand, params, dim, lo, hi, k, n, trials, depth, m, seed, precision, limits)
    ("sin3d_fp64", "sin_sum", [], 3, 0.0, 10.0, 4, 1000, 5, 2, 2.0, 0, "fp64", None),
    ("sin6_fp64_two_levels", "sin_sum", [], 6, 0.0, 10.0, 4, 256, 10, 2, 1.5, 2, "fp64", None),
    ("sin6_fp32_lane_tiles", "sin_sum", [], 6, 0.0, 1.0, 6, 1280, 8, 1, 1.0, 12,
     "fp32_fp64acc", None),
    ("corner3_kahan_chunks", "genz_corner", [1.0, 2.0, 3.0], 3, 0.0, 1.0, 2, 1 << 16, 4, 3, 0.5,
     3, "fp32_kahan", None),
    ("corner5_fp64_deep", "genz_corner", [1.0, 2.0, 3.0, 4.0, 5.0], 5, 0.0, 1.0, 2, 33, 4, 3,
     0.5, 3, "fp64", None),
    ("corner2_budget", "genz_corner", [6.0, 6.0], 2, 0.0, 1.0, 3, 50, 4, 3, 0.0, 11, "fp64",
     [20, 1 << 40]),
    ("expr_sin2", "expr:sin(x[0] + x[1])", [], 2, 0.0, 3.0, 4, 301, 5, 3, 1.0, 7, "fp64", None),
]

CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
from paper_1902_07916_gb300 import zmc
cases = json.loads(sys.argv[2])
out = {}
for c in cases:
    name, fn, p, d, a, b, k, n, T, depth, m, seed, prec, limits = c
    h = zmc.zmc_create(d, [a] * d, [b] * d, k, n, T, depth, m, seed)
    try:
        zmc.zmc_set_integrand(h, fn, p)
        zmc.zmc_set_precision(h, prec)
        if limits:
            zmc.zmc_set_limits(h, *limits)
        r = zmc.zmc_integrate(h)
        out[name] = [r.value, r.std, r.flagged_per_level, r.cells_per_level, r.status]
    except zmc.ZmcError as e:
        out[name] = ["error", e.code, str(e)]
    finally:
        zmc.zmc_destroy(h)
# the registry cases as one batch in the FP32-mixed mode
hs = []
for c in cases:
    name, fn, p, d, a, b, k, n, T, depth, m, seed, prec, limits = c
    if fn.startswith("expr:"):
        continue
    h = zmc.zmc_create(d, [a] * d, [b] * d, k, n, T, depth, m, seed)
    zmc.zmc_set_integrand(h, fn, p)
    zmc.zmc_set_precision(h, "fp32_fp64acc")
    hs.append(h)
try:
    res = zmc.zmc_integrate_batch(hs)
    out["batch"] = [[r.value, r.std, r.flagged_per_level, r.status] for r in res]
except zmc.ZmcError as e:
    out["batch"] = ["error", e.code, str(e)]
finally:
    for h in hs:
        zmc.zmc_destroy(h)
print(json.dumps(out))
"""


def run_child(lib, cases, env_extra=None):
    env = dict(os.environ)
    env["ZMC_LIBRARY"] = lib
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, json.dumps(cases)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


@pytest.fixture(scope="module")
def libs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_07916_gb300 import build
    return build.build(), build.build(checked=True)


def test_checked_build_matches_the_normal_build(libs):
    normal, checked = libs
    a = run_child(normal, CASES)
    b = run_child(checked, CASES)
    for name in a:
        assert b[name] == a[name], (name, a[name], b[name])
    for name, row in b.items():
        if name == "batch":
            assert row[0] != "error" and all(r[3] in (0, 3) for r in row), row
        else:
            assert row[0] != "error" and row[4] in (0, 3), (name, row)   # OK or BUDGET


def test_checked_build_reports_an_index_outside_its_buffer(libs):
    _, checked = libs
    out = run_child(checked, CASES[:1], {"ZMC_FAULT": "capacity"})
    row = out[CASES[0][0]]
    assert row[0] == "error" and row[1] == 9, row                       # ZMC_ERR_CHECK
    assert "bounds check failed (site 5)" in row[2], row                # cell statistics
