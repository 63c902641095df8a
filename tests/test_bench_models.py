"""The flop models bench.py divides by (float64 roofline), checked against a
brute-force count of the block-sum terms (Section 5.3): every (row, k,
column) triple with k in the K-blocks strictly between the row's and the
column's block, 6 flops in the matrix-multiply form, 2 (equal signs, Y only)
or 4 (opposite signs, X only) in the arithmetic-efficient form."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def brute(n, b, signs):
    nb = (n + b - 1) // b
    mm = eff = 0
    for i in range(n):
        for j in range(n):
            I, J = i // b, j // b
            if J < I + 2:
                continue
            k_between = (J - I - 1) * b          # interior K-blocks are full
            mm += 6 * k_between
            eff += (2 if signs[i] == signs[j] else 4) * k_between
    return mm, eff


@pytest.mark.parametrize("n,b", [(1, 16), (40, 16), (64, 16), (97, 16), (130, 32), (200, 64)])
def test_block_sum_flop_models(n, b):
    rng = np.random.default_rng(n * 131 + b)
    signs = np.where(rng.random(n) < 0.4, -1.0, 1.0)
    mm, eff = brute(n, b, signs)
    assert bench.block_sum_flops(n, b) == mm
    assert bench.block_sum_flops_efficient(n, b, signs) == eff


def test_efficient_is_between_third_and_two_thirds_of_mm():
    # all one sign: 2 of the MM form's 6 flops per term; alternating signs: 4 of 6 at most
    n, b = 256, 16
    same = np.ones(n)
    assert 3 * bench.block_sum_flops_efficient(n, b, same) == bench.block_sum_flops(n, b)
    alt = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    e = bench.block_sum_flops_efficient(n, b, alt)
    assert bench.block_sum_flops(n, b) / 3 < e < 2 * bench.block_sum_flops(n, b) / 3 + 1
