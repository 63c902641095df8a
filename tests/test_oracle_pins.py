"""Pins of the CPU oracle against facts fixed by the paper and by mathematics,
independent of the oracle's own code:

* hand-worked small cases (tests/golden/sign_small.txt, Algorithm 3 and the
  2x2 closed form u_12 = t_12 (u_11 - u_22)/(t_11 - t_22));
* the spectral definition sign(A) = Z sign(D) Z^{-1} (Section 1), by the
  oracle's long-double brute force AND by numpy's eigendecomposition;
* scipy.linalg.signm (a library routine for the same function);
* the Newton iteration X <- (X + X^{-1})/2, a textbook route to sign(A);
* the Parlett-Sylvester identity for a sign-sorted diagonal (Section 2):
  U = [I X; 0 -I] with T11 X - X T22 = 2 T12, by scipy's Sylvester solver;
* invariants UT = TU, U^2 = I, trace U = n_+ - n_- (Sections 1-2);
* special cases: all t_ii > 0 gives I, all < 0 gives -I, diagonal T gives
  sign(D), all exactly (Section 3);
* the principal-window property: u_ij depends only on T[i..j, i..j]
  (Algorithm 3's index ranges), so the oracle on a window equals the full
  oracle there bit for bit;
* the flop count of Algorithm 3's inner sums in closed form (Section 3).
A dropped term, a wrong sign, a shifted sum index or a transposed operand in
the oracle fails at least the brute-force, Newton, signm and invariant pins.
"""
import fractions
import math
import os

import numpy as np
import pytest

from paper_1607_06303_gb300.inputs import make_T

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sign_small.txt")


def _parse_golden():
    cases, lines = [], []
    with open(GOLDEN) as f:
        for raw in f:
            s = raw.split("#")[0].strip()
            if s:
                lines.append(s)
    i = 0
    while i < len(lines):
        n = int(lines[i]); i += 1
        T = [[float(fractions.Fraction(x)) for x in lines[i + r].split()] for r in range(n)]; i += n
        U = [[float(fractions.Fraction(x)) for x in lines[i + r].split()] for r in range(n)]; i += n
        cases.append((np.array(T), np.array(U)))
    return cases


def relerr(A, B):
    return np.linalg.norm(A - B) / max(np.linalg.norm(B), 1e-300)


def test_golden_hand_cases(oracle_mod):
    cases = _parse_golden()
    assert len(cases) == 5
    for T, U in cases:
        got = oracle_mod.sign_tri(T)
        np.testing.assert_allclose(got, U, rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", range(6))
def test_2x2_closed_form(oracle_mod, seed):
    rng = np.random.default_rng(100 + seed)
    a, c = rng.uniform(0.5, 2, 2) * rng.choice([-1, 1], 2)
    b = rng.standard_normal()
    U = oracle_mod.sign_tri(np.array([[a, b], [0, c]]))
    sa, sc = np.sign(a), np.sign(c)
    expect = b * (sa - sc) / (a - c)
    assert U[0, 0] == sa and U[1, 1] == sc and U[1, 0] == 0.0
    assert abs(U[0, 1] - expect) <= 1e-15 * max(1, abs(expect))


@pytest.mark.parametrize("n", [3, 4, 5, 7, 9, 12])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_brute_force_spectral(oracle_mod, n, seed):
    for p in (0.5, 0.25):
        T = make_T(n, p, seed=seed)
        U = oracle_mod.sign_tri(T)
        Ub = oracle_mod.sign_spectral(T)
        assert relerr(U, Ub) < 1e-10
        # numpy eigendecomposition: an implementation that shares nothing
        w, V = np.linalg.eig(T)
        Ue = (V * np.sign(w.real)) @ np.linalg.inv(V)
        assert relerr(U, Ue.real) < 1e-9


@pytest.mark.parametrize("n,p,order", [(40, 0.5, "random"), (80, 0.3, "random"), (100, 0.5, "sorted")])
def test_scipy_signm(oracle_mod, n, p, order):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    T = make_T(n, p, seed=7, order=order)
    U = oracle_mod.sign_tri(T)
    Us = scipy_linalg.signm(T)
    assert relerr(U, Us) < 1e-9


def test_newton_iteration(oracle_mod):
    # X_{k+1} = (X_k + X_k^{-1})/2 converges quadratically to sign(A)
    n = 200
    T = make_T(n, 0.5, seed=3)
    X = T.copy()
    for _ in range(60):
        Xn = 0.5 * (X + np.linalg.inv(X))
        if np.linalg.norm(Xn - X) <= 1e-15 * np.linalg.norm(Xn):
            X = Xn
            break
        X = Xn
    U = oracle_mod.sign_tri(T)
    assert relerr(U, X) < 1e-11


@pytest.mark.parametrize("p", [0.1, 0.5])
def test_sylvester_sorted(oracle_mod, p):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    n = 150
    T = make_T(n, p, seed=4, order="sorted")
    npos = int((np.diag(T) > 0).sum())
    T11, T12, T22 = T[:npos, :npos], T[:npos, npos:], T[npos:, npos:]
    # T11 X - X T22 = 2 T12  <=>  T11 X + X (-T22) = 2 T12
    X = scipy_linalg.solve_sylvester(T11, -T22, 2 * T12)
    U = oracle_mod.sign_tri(T)
    np.testing.assert_array_equal(U[:npos, :npos], np.eye(npos))
    np.testing.assert_array_equal(U[npos:, npos:], -np.eye(n - npos))
    assert relerr(U[:npos, npos:], X) < 1e-11


@pytest.mark.parametrize("n,p,seed", [(300, 0.5, 0), (257, 0.1, 1), (333, 0.9, 2)])
def test_invariants(oracle_mod, n, p, seed):
    T = make_T(n, p, seed=seed)
    U = oracle_mod.sign_tri(T)
    I = np.eye(n)
    nU, nT = np.linalg.norm(U), np.linalg.norm(T)
    assert np.linalg.norm(U @ U - I) <= 1e-12 * nU ** 2
    assert np.linalg.norm(U @ T - T @ U) <= 1e-12 * nT * nU
    npos = int((np.diag(T) > 0).sum())
    assert np.trace(U) == npos - (n - npos)
    assert np.all(np.tril(U, -1) == 0)
    assert np.all(np.diag(U) == np.sign(np.diag(T)))


def test_trivial_inertia_and_diagonal(oracle_mod):
    n = 50
    T = make_T(n, 0.0, seed=5)
    np.testing.assert_array_equal(oracle_mod.sign_tri(T), np.eye(n))
    Tn = make_T(n, 1.0, seed=5)
    np.testing.assert_array_equal(oracle_mod.sign_tri(Tn), -np.eye(n))
    D = np.diag(np.diag(make_T(n, 0.5, seed=6)))
    np.testing.assert_array_equal(oracle_mod.sign_tri(D), np.diag(np.sign(np.diag(D))))


def test_window_property_bitexact(oracle_mod):
    n = 120
    T = make_T(n, 0.5, seed=8)
    U = oracle_mod.sign_tri(T)
    for a, b in [(0, 50), (17, 90), (70, 120), (33, 34)]:
        Uw = oracle_mod.sign_tri(T[a:b, a:b])
        np.testing.assert_array_equal(Uw, U[a:b, a:b])


def test_antidiag_schedule_bitexact(oracle_mod):
    for n, p in [(257, 0.5), (130, 0.2)]:
        T = make_T(n, p, seed=9)
        U1 = oracle_mod.sign_tri(T, schedule="paper")
        U2 = oracle_mod.sign_tri(T, schedule="antidiag", threads=4)
        np.testing.assert_array_equal(U1, U2)


def test_status_codes(oracle_mod):
    T = make_T(6, 0.5, seed=1)
    T[3, 3] = 0.0
    assert oracle_mod.sign_tri_status(T) == oracle_mod.ZERO_EIGENVALUE
    T[3, 3] = np.nan
    assert oracle_mod.sign_tri_status(T) == oracle_mod.NONFINITE
    T[3, 3] = np.inf
    assert oracle_mod.sign_tri_status(T) == oracle_mod.NONFINITE
    assert oracle_mod.sign_tri_status(np.zeros((0, 0))) == oracle_mod.OK


@pytest.mark.parametrize("n", [1, 2, 3, 10, 37])
def test_flop_count_closed_forms(oracle_mod, n):
    # all signs equal: every term uses U^2 = I (2 flops): 2 * C(n,3)
    T = make_T(n, 0.0, seed=2)
    assert oracle_mod.useful_flops(T) == 2 * math.comb(n, 3)
    # alternating signs: pairs at odd distance differ (4 flops per term),
    # pairs at even distance agree (2 flops per term)
    d = np.array([(1.0 if i % 2 == 0 else -1.0) for i in range(n)])
    Ta = np.diag(d) + np.triu(np.ones((n, n)), 1)
    expect = sum((n - g) * (g - 1) * (4 if g % 2 else 2) for g in range(1, n))
    assert oracle_mod.useful_flops(Ta) == expect


# ---- the Schur route (Section 1; Algorithm 3's first step) ----------------

@pytest.mark.parametrize("n,p", [(5, 0.4), (20, 0.5), (60, 0.3)])
def test_sign_schur_vs_signm(oracle_mod, n, p):
    # A = Q T Q^T with orthogonal Q: sign(A) from scipy's own routine on A,
    # which knows nothing of the Schur pair (a transposed Q, or U applied on
    # the wrong side, fails this)
    sl = pytest.importorskip("scipy.linalg")
    from paper_1607_06303_gb300.inputs import make_schur_pair
    Q, T = make_schur_pair(n, p, seed=n)
    A = Q @ T @ Q.T
    S = oracle_mod.sign_schur(Q, T)
    ref = sl.signm(A)
    assert np.linalg.norm(S - ref) <= 1e-12 * np.linalg.norm(ref)


def test_sign_schur_real_schur_of_A(oracle_mod):
    # the use the route is for: A with real eigenvalues, its real Schur form
    # from LAPACK, against the spectral definition V sign(L) V^{-1}
    sl = pytest.importorskip("scipy.linalg")
    rng = np.random.Generator(np.random.PCG64(5))
    n = 40
    V = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / math.sqrt(n)
    lam = rng.uniform(0.5, 2.0, n) * np.where(rng.random(n) < 0.4, -1.0, 1.0)
    A = V @ np.diag(lam) @ np.linalg.inv(V)
    T, Z = sl.schur(A, output="real")
    assert np.allclose(np.tril(T, -1), 0.0, atol=1e-12)   # real spectrum: T triangular
    S = oracle_mod.sign_schur(Z, np.triu(T))
    ref = V @ np.diag(np.sign(lam)) @ np.linalg.inv(V)
    assert np.linalg.norm(S - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("n,p", [(1, 0.0), (2, 0.5), (33, 0.5), (64, 0.1)])
def test_sign_schur_invariants(oracle_mod, n, p):
    from paper_1607_06303_gb300.inputs import make_schur_pair
    Q, T = make_schur_pair(n, p, seed=3 * n + 1)
    A = Q @ T @ Q.T
    S = oracle_mod.sign_schur(Q, T)
    I = np.eye(n)
    assert np.linalg.norm(S @ S - I) <= 1e-12 * max(1.0, np.linalg.norm(S) ** 2)
    assert np.linalg.norm(A @ S - S @ A) <= 1e-12 * np.linalg.norm(A) * np.linalg.norm(S)
    npos = int(np.sum(np.diag(T) > 0))
    assert abs(np.trace(S) - (npos - (n - npos))) <= 1e-10 * n
    # Q = I reduces to the triangular oracle exactly
    assert np.array_equal(oracle_mod.sign_schur(np.eye(n), T), oracle_mod.sign_tri(T))


# ---- complex T (the Schur form of a general matrix is complex) ------------

def _paper_matrix(n, seed):
    # Section 6's workload: entries uniform in [-50, 50]
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-50.0, 50.0, size=(n, n))


@pytest.mark.parametrize("n,seed", [(8, 1), (30, 2), (60, 3)])
def test_complex_schur_route_vs_signm(oracle_mod, n, seed):
    # a general real A through its complex Schur form (LAPACK), against
    # scipy's signm of A itself; sign(A) of a real A is real
    sl = pytest.importorskip("scipy.linalg")
    A = _paper_matrix(n, seed)
    T, Z = sl.schur(A, output="complex")
    S = oracle_mod.sign_schur_complex(Z, T)
    ref = sl.signm(A)
    assert np.linalg.norm(S - ref) <= 1e-11 * np.linalg.norm(ref)
    assert np.abs(S.imag).max() <= 1e-11 * np.abs(S).max()


def test_complex_spectral_definition(oracle_mod):
    # complex triangular T with distinct eigenvalues: V sign(Re L) V^{-1}
    rng = np.random.Generator(np.random.PCG64(11))
    n = 12
    T = np.triu(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / 3.0
    d = (rng.uniform(0.5, 2.0, n) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
         + 1j * rng.uniform(-2.0, 2.0, n))
    T[np.arange(n), np.arange(n)] = d
    lam, V = np.linalg.eig(T)
    ref = V @ np.diag(np.sign(lam.real)) @ np.linalg.inv(V)
    U = oracle_mod.sign_tri_complex(T)
    assert np.linalg.norm(U - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.array_equal(np.diag(U), np.sign(d.real).astype(complex))
    assert np.all(np.tril(U, -1) == 0)


def test_complex_2x2_and_invariants(oracle_mod):
    t11, t12, t22 = 1.5 - 0.5j, 0.3 + 2.0j, -0.7 + 1.1j
    U = oracle_mod.sign_tri_complex(np.array([[t11, t12], [0, t22]]))
    assert U[0, 0] == 1 and U[1, 1] == -1
    assert abs(U[0, 1] - t12 * 2 / (t11 - t22)) <= 1e-15 * abs(U[0, 1])
    rng = np.random.Generator(np.random.PCG64(12))
    n = 40
    T = np.triu(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(n)
    T[np.arange(n), np.arange(n)] = (rng.uniform(0.5, 2.0, n) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
                                     + 1j * rng.standard_normal(n))
    U = oracle_mod.sign_tri_complex(T)
    assert np.linalg.norm(U @ U - np.eye(n)) <= 1e-12 * np.linalg.norm(U) ** 2
    assert np.linalg.norm(U @ T - T @ U) <= 1e-12 * np.linalg.norm(U) * np.linalg.norm(T)


def test_complex_reduces_to_real(oracle_mod):
    # a real T in complex form gives the real oracle's U bit for bit
    T = make_T(50, 0.4, seed=7)
    U = oracle_mod.sign_tri_complex(T.astype(complex))
    assert np.array_equal(U.real, oracle_mod.sign_tri(T))
    assert np.all(U.imag == 0)


def test_complex_imaginary_axis_is_an_error(oracle_mod):
    # sign is undefined on the imaginary axis (Section 1)
    T = np.array([[1.0 + 1j, 0.5], [0, 2.0j]])
    with pytest.raises(oracle_mod.OracleError) as e:
        oracle_mod.sign_tri_complex(T)
    assert e.value.status == oracle_mod.ZERO_EIGENVALUE


# ---- general phi: Parlett's substitution (Section 2, Algorithm 1) ----------

def _spread_T(n, seed, lo=1.0, hi=3.0):
    # distinct, well separated diagonal entries in random order
    rng = np.random.Generator(np.random.PCG64(seed))
    T = np.triu(rng.standard_normal((n, n))) / math.sqrt(n)
    T[np.arange(n), np.arange(n)] = rng.permutation(np.linspace(lo, hi, n))
    return np.asfortranarray(T)


@pytest.mark.parametrize("n", [5, 20, 40])
def test_funm_vs_scipy(oracle_mod, n):
    sl = pytest.importorskip("scipy.linalg")
    T = _spread_T(n, n)
    for phi, ref in (("exp", sl.expm(T)), ("log", sl.logm(T)), ("sqrt", sl.sqrtm(T))):
        F = oracle_mod.funm(T, phi)
        assert np.linalg.norm(F - ref) <= 1e-12 * np.linalg.norm(ref), phi
        assert np.all(np.tril(F, -1) == 0)


def test_funm_identities(oracle_mod):
    sl = pytest.importorskip("scipy.linalg")
    T = _spread_T(30, 3)
    S = oracle_mod.funm(T, "sqrt")
    assert np.linalg.norm(S @ S - T) <= 1e-13 * np.linalg.norm(T)
    L = oracle_mod.funm(T, "log")
    assert np.linalg.norm(sl.expm(L) - T) <= 1e-12 * np.linalg.norm(T)
    E, Em = oracle_mod.funm(T, "exp"), oracle_mod.funm(-T, "exp")
    assert np.linalg.norm(E @ Em - np.eye(30)) <= 1e-12 * np.linalg.norm(E) * np.linalg.norm(Em)
    for F in (S, L, E):
        assert np.linalg.norm(F @ T - T @ F) <= 1e-13 * np.linalg.norm(F) * np.linalg.norm(T)


def test_funm_2x2_and_sign(oracle_mod):
    T = np.array([[1.5, 0.7], [0.0, 0.4]])
    F = oracle_mod.funm(T, "exp")
    assert F[0, 0] == math.exp(1.5) and F[1, 1] == math.exp(0.4)
    assert abs(F[0, 1] - 0.7 * (math.exp(1.5) - math.exp(0.4)) / 1.1) <= 1e-15 * abs(F[0, 1])
    # the sign function through Eq. 1 alone agrees with Algorithm 3's mix of
    # Eqs. 1 and 2 when the diagonal entries are well separated (with close
    # equal-sign entries Eq. 1 divides by their small difference, which is
    # why Algorithm 3 takes Eq. 2 there)
    T = _spread_T(60, 8)
    T[np.arange(60), np.arange(60)] *= np.where(np.arange(60) % 3 == 0, -1.0, 1.0)
    U = oracle_mod.sign_tri(T)
    assert np.linalg.norm(oracle_mod.funm(T, "sign") - U) <= 1e-12 * np.linalg.norm(U)


def test_funm_errors(oracle_mod):
    T = np.array([[1.0, 0.5], [0.0, 1.0]])       # repeated eigenvalue
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.funm(T, "exp")
    T = np.array([[-1.0, 0.5], [0.0, 2.0]])      # log of a negative eigenvalue
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.funm(T, "log")


@pytest.mark.parametrize("n,seed", [(1, 4), (8, 5), (30, 6), (60, 7)])
def test_sign_general_vs_signm(oracle_mod, n, seed):
    # the oracle's general route (LAPACK's complex Schur form, then the
    # complex sign and Q U Q^H) against scipy's signm of A itself
    sl = pytest.importorskip("scipy.linalg")
    A = _paper_matrix(n, seed)
    S = oracle_mod.sign_general(A)
    ref = sl.signm(A)
    assert S.dtype == np.float64
    assert np.linalg.norm(S - ref) <= 1e-11 * np.linalg.norm(ref)


def test_sign_general_closed_form(oracle_mod):
    # A = P B P^{-1} with B block diagonal: 2 x 2 blocks [a b; -b a]
    # (eigenvalues a +- ib, sign = sign(a) I) and 1 x 1 blocks d; so
    # sign(A) = P sign(B) P^{-1} with sign(B) diagonal +-1, no Schur form
    # involved.  Also S^2 = I, AS = SA, trace S = n_+ - n_-.
    pytest.importorskip("scipy.linalg")
    rng = np.random.Generator(np.random.PCG64(21))
    n = 40
    B = np.zeros((n, n))
    sB = np.zeros(n)
    i = 0
    while i < n:
        a = rng.uniform(0.5, 3.0) * (1.0 if rng.random() < 0.5 else -1.0)
        if i + 1 < n and rng.random() < 0.6:
            b = rng.uniform(0.5, 3.0)
            B[i:i + 2, i:i + 2] = [[a, b], [-b, a]]
            sB[i:i + 2] = np.sign(a)
            i += 2
        else:
            B[i, i] = a
            sB[i] = np.sign(a)
            i += 1
    P = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / math.sqrt(n)
    Pi = np.linalg.inv(P)
    A = P @ B @ Pi
    ref = P @ np.diag(sB) @ Pi
    S = oracle_mod.sign_general(A)
    assert np.linalg.norm(S - ref) <= 1e-11 * np.linalg.norm(ref)
    assert np.linalg.norm(S @ S - np.eye(n)) <= 1e-11 * np.linalg.norm(S) ** 2
    assert np.linalg.norm(A @ S - S @ A) <= 1e-11 * np.linalg.norm(A) * np.linalg.norm(S)
    assert abs(np.trace(S) - sB.sum()) <= 1e-9


def test_sign_general_of_triangular(oracle_mod):
    # an upper triangular A is its own Schur form: the real oracle's U
    pytest.importorskip("scipy.linalg")
    T = make_T(50, 0.5, seed=8)
    assert np.linalg.norm(oracle_mod.sign_general(T) - oracle_mod.sign_tri(T)) <= \
        1e-12 * np.linalg.norm(oracle_mod.sign_tri(T))
