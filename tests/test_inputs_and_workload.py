"""Generator recipe and the work counts (host logic, no GPU)."""
import math

import numpy as np
import pytest

from paper_1607_06303_gb300 import workload
from paper_1607_06303_gb300.inputs import batch_sizes, make_T, n_negative


@pytest.mark.parametrize("n,p,order", [(0, 0.5, "random"), (1, 0.5, "random"), (256, 0.5, "random"),
                                       (1000, 0.1, "sorted"), (333, 0.25, "random")])
def test_recipe(n, p, order):
    T = make_T(n, p, seed=0, order=order)
    assert T.shape == (n, n) and T.flags["F_CONTIGUOUS"] and T.dtype == np.float64
    d = np.diag(T)
    assert int((d < 0).sum()) == n_negative(n, p)
    assert np.all((np.abs(d) >= 0.5) & (np.abs(d) <= 2.0))
    assert np.all(np.tril(T, -1) == 0)
    if order == "sorted" and n:
        s = np.sign(d)
        assert np.all(np.diff(s) <= 0)      # positives first
    if n >= 256:
        off = T[np.triu_indices(n, 1)]
        assert abs(off.std() * math.sqrt(n) - 1.0) < 0.05
        assert abs(off.mean()) < 0.01


def test_reproducible():
    np.testing.assert_array_equal(make_T(100, 0.5, seed=3), make_T(100, 0.5, seed=3))
    assert not np.array_equal(make_T(100, 0.5, seed=3), make_T(100, 0.5, seed=4))


def test_batch_sizes():
    ns, ps = batch_sizes(2000, seed=0)
    assert min(ns) >= 32 and max(ns) <= 2048 and len(ns) == 2000
    assert 0 <= min(ps) and max(ps) <= 1
    # log-uniform: median near sqrt(32*2048) = 256
    assert 180 < np.median(ns) < 360


@pytest.mark.parametrize("n,p,seed", [(1, 0.5, 0), (2, 0.5, 1), (5, 0.5, 0), (64, 0.5, 1), (200, 0.1, 2),
                                      (150, 0.9, 3), (90, 0.0, 4)])
def test_useful_flops_matches_oracle_count(oracle_mod, n, p, seed):
    T = make_T(n, p, seed=seed)
    assert workload.useful_flops(np.sign(np.diag(T))) == oracle_mod.useful_flops(T)


def test_mm_and_swaps():
    assert workload.mm_flops(16384) == 6 * math.comb(16384, 3)
    assert workload.swaps(np.array([-1, 1, -1, 1, 1])) == 1 + 2 + 2
    assert workload.swaps(np.array([1, 1, -1])) == 0
    # 16384 at p = 0.5: useful flops ~ n^3/2
    s = np.sign(np.diag(make_T(4096, 0.5, seed=0)))
    assert abs(workload.useful_flops(s) / (4096 ** 3 / 2) - 1) < 0.01
