"""Work counts of the method (Section 3), from the diagonal signs alone.

useful_flops: the operations of Algorithm 3's inner sums, the metric's
"useful" work: 2 per term of an equal-sign entry (U^2 = I) and 4 per term of
an opposite-sign entry (TU = UT), an entry (i, j) having j - i - 1 terms.
mm_flops: the matrix-multiply form of Algorithms 4-6, which forms both block
sums everywhere: 6 flops per (i < k < j) triple, n^3 to leading order.
ps_flops: the Parlett-Sylvester estimate of Section 3 for k swaps.
"""
import math

import numpy as np


def _pair_gap_sum(pos: np.ndarray) -> int:
    """sum over pairs a < b of (pos[b] - pos[a] - 1) for increasing positions."""
    m = len(pos)
    if m < 2:
        return 0
    pos = pos.astype(np.int64)
    ranks = np.arange(m, dtype=np.int64)
    prefix = np.concatenate(([0], np.cumsum(pos)[:-1]))
    return int(np.sum(ranks * (pos - 1) - prefix))


def term_counts(signs):
    """(equal-sign terms, opposite-sign terms) of Algorithm 3's inner sums."""
    s = np.asarray(signs)
    n = len(s)
    all_terms = math.comb(n, 3) if n >= 3 else 0
    idx = np.arange(n)
    same = _pair_gap_sum(idx[s > 0]) + _pair_gap_sum(idx[s < 0])
    return same, all_terms - same


def useful_flops(signs) -> int:
    same, opp = term_counts(signs)
    return 2 * same + 4 * opp


def mm_flops(n: int) -> int:
    return 6 * math.comb(n, 3) if n >= 3 else 0


def swaps(signs) -> int:
    """#{i < j : s_i < 0 < s_j}: adjacent swaps that put positives first."""
    s = np.asarray(signs)
    neg_before = np.cumsum(s < 0) - (s < 0)
    return int(np.sum(neg_before[s > 0]))


def ps_flops(signs) -> float:
    s = np.asarray(signs)
    n = len(s)
    npos, nneg = int(np.sum(s > 0)), int(np.sum(s < 0))
    k = swaps(s)
    w = 12.0 * n * k + npos * nneg * n
    if k > 0:
        w += 2.0 * n * min(npos, nneg) * (n + max(npos, nneg))
    return w
