"""Seeded synthetic inputs: dense real upper-triangular T with a prescribed
inertia (number of negative diagonal entries).

This module serves both the CUDA path and the oracle.  It holds none of the
method's arithmetic: it only draws random numbers.

Recipe (the paper's forced-inertia workload, Section 6, with a Gaussian
strictly-upper part in place of a Schur form):
  1. the sign pattern: exactly n_neg = floor(p*n + 0.5) negative diagonal
     entries, at positions drawn uniformly without replacement
     (order="random"), or all positives first (order="sorted");
  2. |t_ii| ~ U[0.5, 2], i = 1..n;
  3. strictly-upper t_ij ~ N(0, 1/n), drawn column by column (j outer,
     i = 1..j-1 inner);
  the strictly lower triangle is zero.
Matrices are numpy float64 arrays in column-major (Fortran) order.
"""
import math

import numpy as np


def n_negative(n: int, p: float) -> int:
    return int(math.floor(p * n + 0.5))


def sign_pattern(rng, n: int, n_neg: int, order: str) -> np.ndarray:
    s = np.ones(n)
    if n_neg <= 0:
        return s
    if order == "random":
        s[rng.permutation(n)[:n_neg]] = -1.0
    elif order == "sorted":
        s[n - n_neg:] = -1.0
    else:
        raise ValueError("order must be 'random' or 'sorted'")
    return s


def make_T(n: int, p: float = 0.5, seed: int = 0, order: str = "random",
           n_neg: int = None) -> np.ndarray:
    """Upper-triangular T (column-major float64) from the recipe above."""
    if n < 0:
        raise ValueError("n must be >= 0")
    rng = np.random.Generator(np.random.PCG64(seed))
    k = n_negative(n, p) if n_neg is None else int(n_neg)
    s = sign_pattern(rng, n, k, order)
    mags = rng.uniform(0.5, 2.0, size=n)
    T = np.zeros((n, n), dtype=np.float64, order="F")
    if n == 0:
        return T
    m = n * (n - 1) // 2
    off = rng.standard_normal(m) * (1.0 / math.sqrt(n))
    o = 0
    for j in range(1, n):
        T[:j, j] = off[o:o + j]
        o += j
    T[np.arange(n), np.arange(n)] = s * mags
    return T


def make_orthogonal(n: int, seed: int = 0) -> np.ndarray:
    """Seeded n x n orthogonal matrix (column-major float64): the Q factor of
    a standard normal matrix, columns signed so that R's diagonal is
    positive (Haar-distributed)."""
    if n < 0:
        raise ValueError("n must be >= 0")
    rng = np.random.Generator(np.random.PCG64(seed))
    G = rng.standard_normal((n, n))
    if n == 0:
        return np.zeros((0, 0), order="F")
    Q, R = np.linalg.qr(G)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return np.asfortranarray(Q * d)


def make_schur_pair(n: int, p: float = 0.5, seed: int = 0, order: str = "random"):
    """A real Schur pair (Q, T): T from make_T, Q from make_orthogonal, so
    that A = Q T Q^T has T's (real) eigenvalues."""
    return make_orthogonal(n, seed + 7919), make_T(n, p, seed=seed, order=order)


def make_T_complex(n: int, p: float = 0.5, seed: int = 0, order: str = "random") -> np.ndarray:
    """Complex upper-triangular T (column-major complex128): the real recipe's
    sign pattern and |Re t_ii| ~ U[0.5, 2], Im t_ii ~ N(0, 1); strictly upper
    re and im parts each N(0, 1/(2n)) (so |t_ij|^2 has mean 1/n)."""
    if n < 0:
        raise ValueError("n must be >= 0")
    rng = np.random.Generator(np.random.PCG64(seed))
    k = n_negative(n, p)
    s = sign_pattern(rng, n, k, order)
    mags = rng.uniform(0.5, 2.0, size=n)
    ims = rng.standard_normal(n)
    T = np.zeros((n, n), dtype=np.complex128, order="F")
    if n == 0:
        return T
    m = n * (n - 1) // 2
    sd = 1.0 / math.sqrt(2.0 * n)
    re = rng.standard_normal(m) * sd
    im = rng.standard_normal(m) * sd
    o = 0
    for j in range(1, n):
        T[:j, j] = re[o:o + j] + 1j * im[o:o + j]
        o += j
    T[np.arange(n), np.arange(n)] = s * mags + 1j * ims
    return T


def make_A(n: int, seed: int = 0) -> np.ndarray:
    """A general real n x n matrix with entries uniform in [-50, 50] (the
    matrices whose Schur forms make the paper's Section 6 workload);
    column-major float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.asfortranarray(rng.uniform(-50.0, 50.0, size=(n, n)))


def make_T_schur(n: int, seed: int = 0, n_neg: int = None) -> np.ndarray:
    """The paper's workload (Section 6): the real part of the complex Schur
    form of a random n x n matrix with entries uniform in [-50, 50]; inertia
    roughly balanced.  With n_neg given, the diagonal keeps its magnitudes but
    all signs are made positive except at n_neg random positions (the paper's
    forced inertia).  Column-major float64; needs scipy (host only)."""
    import scipy.linalg
    rng = np.random.Generator(np.random.PCG64(seed))
    A = rng.uniform(-50.0, 50.0, size=(n, n))
    Tc, _ = scipy.linalg.schur(A, output="complex")
    T = np.asfortranarray(np.triu(Tc.real))
    if n_neg is not None:
        d = np.abs(np.diag(T))
        s = np.ones(n)
        s[rng.permutation(n)[:int(n_neg)]] = -1.0
        T[np.arange(n), np.arange(n)] = s * d
    return T


def batch_sizes(count: int, seed: int = 0, n_min: int = 32, n_max: int = 2048):
    """Sizes n_i = round(exp(U[ln n_min, ln n_max])) and inertias p_i ~ U[0,1]
    of a batch of independent problems."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ln = rng.uniform(math.log(n_min), math.log(n_max), size=count)
    ns = np.clip(np.floor(np.exp(ln) + 0.5).astype(np.int64), n_min, n_max)
    ps = rng.uniform(0.0, 1.0, size=count)
    return [int(x) for x in ns], [float(x) for x in ps]


def make_batch(count: int, seed: int = 0, n_min: int = 32, n_max: int = 2048):
    """A batch of independent problems: list of (T_i, seed_i), T_i from make_T
    with n_i, p_i from batch_sizes and random diagonal order."""
    ns, ps = batch_sizes(count, seed, n_min, n_max)
    return [make_T(n, p, seed=seed * 1000003 + i + 1, order="random")
            for i, (n, p) in enumerate(zip(ns, ps))]
