"""The statistics behind the mixed variants' acceptance test, on the CPU.

The refinement accepts U when both residual norms, ||TU - UT||_F and
||U^2 - I||_F (the two defining equations of sign(T), Section 2), are below
the tolerance.  By default the norms are estimated from Z, n x 128 with
independent +-1 entries: ||R||_F ~ ||R Z||_F / sqrt(128).  Per probe z the
summand X = ||R z||^2 = z^T A z (A = R^T R, positive semidefinite) has
E X = tr A = ||R||_F^2 and E X^2 = (tr A)^2 + 2 (||A||_F^2 - sum a_ii^2)
<= 3 (tr A)^2.  Maurer's inequality for sums of independent nonnegative
variables, P(E S - S >= t) <= exp(-t^2 / (2 sum E X_i^2)), then bounds the
chance that a residual r times above the tolerance passes:
exp(-(1 - 1/r^2)^2 m / 6) for m probes -- below 1e-9 for r = 10, m = 128."""
import itertools
import math

import numpy as np


def _moments_by_enumeration(A):
    m = A.shape[0]
    xs = []
    for signs in itertools.product((-1.0, 1.0), repeat=m):
        z = np.array(signs)
        xs.append(z @ A @ z)
    xs = np.array(xs)
    return xs.mean(), (xs ** 2).mean()


def test_quadratic_form_moments_exact():
    rng = np.random.default_rng(3)
    for trial in range(6):
        m = 4 + trial % 4
        R = rng.standard_normal((m + 2, m)) * rng.uniform(0.1, 3.0, size=m)   # uneven columns
        A = R.T @ R
        mean, second = _moments_by_enumeration(A)
        tr = np.trace(A)
        assert math.isclose(mean, tr, rel_tol=1e-12)
        closed = tr ** 2 + 2.0 * (np.sum(A * A) - np.sum(np.diag(A) ** 2))
        assert math.isclose(second, closed, rel_tol=1e-12)
        assert second <= 3.0 * tr ** 2 * (1 + 1e-12)
    # the constant 3 is approached: A = all-ones (rank one, equal diagonal)
    m = 10
    A = np.ones((m, m))
    _, second = _moments_by_enumeration(A)
    assert second / np.trace(A) ** 2 > 2.7


def _pass_bound(ratio, probes):
    return math.exp(-(1.0 - 1.0 / ratio ** 2) ** 2 * probes / 6.0)


def test_acceptance_bound_at_the_library_setting():
    assert _pass_bound(10.0, 128) < 1e-9
    # fewer probes would not give it
    assert _pass_bound(10.0, 64) > 1e-9


def test_false_acceptance_rate_seeded():
    """A residual 1.5x the tolerance passes the 128-probe estimate no more
    often than the bound allows (seeded Monte Carlo; the bound is loose)."""
    rng = np.random.default_rng(11)
    n, probes, trials, ratio = 48, 128, 3000, 1.5
    R = np.triu(rng.standard_normal((n, n)))
    tol = np.linalg.norm(R) / ratio
    passes = 0
    for _ in range(trials):
        Z = rng.choice((-1.0, 1.0), size=(n, probes))
        est = np.linalg.norm(R @ Z) / math.sqrt(probes)
        passes += est <= tol
    assert passes / trials <= _pass_bound(ratio, probes)
    # and the estimate is unbiased in the square
    Z = rng.choice((-1.0, 1.0), size=(n, 20000))
    assert math.isclose(np.linalg.norm(R @ Z) ** 2 / 20000, np.linalg.norm(R) ** 2, rel_tol=0.02)
