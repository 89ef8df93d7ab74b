"""zmc_level_stats_noalloc against the library's own selection step.

Some callers cannot allocate device memory: their device memory is all owned
by their own pool or arena, or their loop cannot afford the synchronisation
an allocation may imply.  zmc_level_stats_noalloc serves them: it computes a
level's per-cell statistics and threshold from per-(cell, trial) sums the
caller holds, with its scratch in a fixed static device array.

This test runs a traced integration through the existing entry point
(zmc_integrate), hands the traced sums of a level to the no-allocation entry
point through the C ABI twice in a row, and checks the per-cell (mean,
spread) and (mu, sigma, theta) it writes against the traced values of the
library's selection step, to 1e-12 relative.  It needs nothing from other
test files, so it passes alone in a fresh process and after the rest.
"""
import math

import numpy as np
import pytest

from paper_1902_07916_gb300.workloads import Workload

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module")
def zmc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_07916_gb300 import build
    build.build()
    from paper_1902_07916_gb300 import zmc as mod
    return mod


CASES = [
    # 64 cells: one CTA
    (Workload("sin3", "sin_sum", 3, [0.0] * 3, [10.0] * 3, 4, 1000, 5, 2, 2.0, 0), 1),
    # 7776 cells: several CTAs and their arrival ticket
    (Workload("corner5", "genz_corner", 5, [0.0] * 5, [1.0] * 5, 6, 37, 4, 2, 0.5, 3,
              [1.0, 2.0, 3.0, 4.0, 5.0]), 1),
    # a refined level
    (Workload("gauss3", "gauss_norm", 3, [-1.0] * 3, [1.0] * 3, 4, 64, 6, 2, 0.5, 8, [0.2]), 2),
]


@pytest.mark.parametrize("w,level", CASES, ids=[c[0].name for c in CASES])
def test_noalloc_matches_library_selection(zmc, w, level):
    import torch
    with zmc.Integrator(w.dim, w.lo, w.hi, w.k, w.n, w.trials, w.depth, w.sigma_multiplier,
                        w.seed, w.integrand, w.params) as it:
        it.trace(True)
        it.integrate()
        lv = it.trace_level(level)
    C = lv["cells"]
    assert C > 0
    volume = math.prod((b - a) / w.k ** level for a, b in zip(w.lo, w.hi))
    stream = torch.cuda.current_stream()
    sums = torch.tensor(lv["sums"], dtype=torch.float64, device="cuda").contiguous()
    cell_stats = torch.empty((C, 2), dtype=torch.float64, device="cuda")
    level_stats = torch.empty(3, dtype=torch.float64, device="cuda")
    for _ in range(2):   # two calls in a row share the static scratch
        cell_stats.fill_(float("nan"))
        level_stats.fill_(float("nan"))
        zmc.zmc_level_stats_noalloc(sums.data_ptr(), C, w.trials, w.n, volume,
                                    w.sigma_multiplier, cell_stats.data_ptr(),
                                    level_stats.data_ptr(), stream)
        torch.cuda.synchronize()
        got = cell_stats.cpu().numpy()
        ref = lv["cell_stats"]
        scale = np.abs(ref[:, 0]).max() + 1e-300
        assert np.all(np.abs(got[:, 0] - ref[:, 0]) <= RTOL * scale)
        np.testing.assert_allclose(got[:, 1], ref[:, 1], rtol=RTOL, atol=1e-300)
        mu, sigma, theta = level_stats.cpu().tolist()
        assert math.isclose(mu, lv["mu"], rel_tol=RTOL)
        assert math.isclose(sigma, lv["sigma"], rel_tol=RTOL, abs_tol=1e-300)
        assert math.isclose(theta, lv["theta"], rel_tol=RTOL)


def test_noalloc_rejects_sizes_beyond_its_scratch(zmc):
    import torch
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(zmc.ZmcError) as e:
        zmc.zmc_level_stats_noalloc(buf.data_ptr(), 1048577, 2, 10, 1.0, 1.0, buf.data_ptr(),
                                    buf.data_ptr())
    assert e.value.code == zmc.ZMC_ERR_ARG
    assert "1048576" in zmc.zmc_last_error(None)
