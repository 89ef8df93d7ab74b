"""zmc_level_stats_noalloc against the oracle and the library's own
selection step.

Some callers cannot allocate device memory: their device memory is all owned
by their own pool or arena, or their loop cannot afford the synchronisation
an allocation may imply.  zmc_level_stats_noalloc serves them: it computes a
level's per-cell statistics and threshold from per-(cell, trial) sums the
caller holds, with its scratch in a fixed static device array.

The tests hand per-(cell, trial) sums to the no-allocation entry point
through the C ABI twice in a row and check the per-cell (mean, spread) and
(mu, sigma, theta) it writes, to 1e-12 relative, against the oracle's
statistics and threshold (Sec. 2.1) on the same sums, and for traced levels
also against the library's own selection step (zmc_integrate).  The largest
case fills every slot of the static scratch (1,048,576 cells).  Nothing is
needed from other test files, so the file passes alone in a fresh process
and after the rest.
"""
import math

import numpy as np
import pytest

from oracle import zmc_oracle as O
from paper_1902_07916_gb300.workloads import Workload

pytestmark = pytest.mark.gpu

RTOL = 1e-12
MAX_CELLS = 1048576


@pytest.fixture(scope="module")
def zmc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_07916_gb300 import build
    build.build()
    from paper_1902_07916_gb300 import zmc as mod
    return mod


def noalloc_twice(zmc, sums_np, trials, n, volume, m):
    """Two calls in a row on the same inputs; returns both (cell_stats, level_stats)."""
    import torch
    C = sums_np.shape[0]
    stream = torch.cuda.current_stream()
    sums = torch.tensor(sums_np.reshape(C, trials, 2), dtype=torch.float64,
                        device="cuda").contiguous()
    cell_stats = torch.empty((C, 2), dtype=torch.float64, device="cuda")
    level_stats = torch.empty(3, dtype=torch.float64, device="cuda")
    out = []
    for _ in range(2):   # the calls share the static scratch
        cell_stats.fill_(float("nan"))
        level_stats.fill_(float("nan"))
        zmc.zmc_level_stats_noalloc(sums.data_ptr(), C, trials, n, volume, m,
                                    cell_stats.data_ptr(), level_stats.data_ptr(), stream)
        torch.cuda.synchronize()
        out.append((cell_stats.cpu().numpy().copy(), level_stats.cpu().tolist()))
    return out


def check_against(got_cells, got_level, mean, spread, level3):
    scale = np.abs(mean).max() + 1e-300
    assert np.all(np.abs(got_cells[:, 0] - mean) <= RTOL * scale)
    np.testing.assert_allclose(got_cells[:, 1], spread, rtol=RTOL, atol=1e-300)
    for g, r in zip(got_level, level3):
        assert math.isclose(g, r, rel_tol=RTOL, abs_tol=1e-300), (got_level, level3)


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
def test_noalloc_matches_oracle_and_library_selection(zmc, w, level):
    with zmc.Integrator(w.dim, w.lo, w.hi, w.k, w.n, w.trials, w.depth, w.sigma_multiplier,
                        w.seed, w.integrand, w.params) as it:
        it.trace(True)
        it.integrate()
        lv = it.trace_level(level)
    C = lv["cells"]
    assert C > 0
    volume = math.prod((b - a) / w.k ** level for a, b in zip(w.lo, w.hi))
    _, mean, spread = O.cell_statistics(lv["sums"], volume, w.n)
    oracle3 = O.threshold(spread, w.sigma_multiplier)
    for got_cells, got_level in noalloc_twice(zmc, lv["sums"], w.trials, w.n, volume,
                                              w.sigma_multiplier):
        check_against(got_cells, got_level, mean, spread, oracle3)
        check_against(got_cells, got_level, lv["cell_stats"][:, 0], lv["cell_stats"][:, 1],
                      (lv["mu"], lv["sigma"], lv["theta"]))


def test_noalloc_full_scratch_against_oracle(zmc):
    # exactly the bound: 1024 CTAs of 1024 cells, every scratch slot and the
    # arrival ticket after the last one in use; synthetic sums (2 trials)
    C, T, n, volume, m = MAX_CELLS, 2, 1000, 1.0 / 1024, 1.5
    rng = np.random.default_rng(20260)
    sums = np.empty((C, T, 2))
    sums[..., 0] = rng.normal(300.0, 40.0, size=(C, T))
    sums[..., 1] = np.abs(rng.normal(9e4, 1e3, size=(C, T)))
    _, mean, spread = O.cell_statistics(sums, volume, n)
    oracle3 = O.threshold(spread, m)
    for got_cells, got_level in noalloc_twice(zmc, sums, T, n, volume, m):
        check_against(got_cells, got_level, mean, spread, oracle3)


def test_noalloc_nonfinite_sums_propagate(zmc):
    # not reported as an error (the header says so): the cell's statistics
    # and the level's threshold become non-finite, the other cells are exact
    C, T, n, volume, m = 3000, 3, 50, 0.25, 1.0
    rng = np.random.default_rng(7)
    sums = np.abs(rng.normal(10.0, 2.0, size=(C, T, 2)))
    sums[17, 1, 0] = np.inf
    _, mean, spread = O.cell_statistics(np.delete(sums, 17, axis=0), volume, n)
    (got_cells, got_level), _ = noalloc_twice(zmc, sums, T, n, volume, m)
    assert not math.isfinite(got_level[2])
    keep = np.ones(C, dtype=bool)
    keep[17] = False
    np.testing.assert_allclose(got_cells[keep, 0], mean, rtol=RTOL)
    np.testing.assert_allclose(got_cells[keep, 1], spread, rtol=RTOL, atol=1e-300)


def test_noalloc_rejects_sizes_beyond_its_scratch(zmc):
    import torch
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(zmc.ZmcError) as e:
        zmc.zmc_level_stats_noalloc(buf.data_ptr(), MAX_CELLS + 1, 2, 10, 1.0, 1.0,
                                    buf.data_ptr(), buf.data_ptr())
    assert e.value.code == zmc.ZMC_ERR_ARG
    assert str(MAX_CELLS) in zmc.zmc_last_error(None)
