"""CPU oracle for U = sign(T) of a real upper-triangular T.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use it; the library never does.  It shares no code with the
CUDA path.  The arithmetic lives in oracle.c (plain C, float64, no FMA
contraction); this module only marshals numpy arrays.

Matrices are numpy float64 arrays in column-major (Fortran) order, element
(i, j) of an n x n matrix at offset i + j*n.
"""
import ctypes
import os

import numpy as np

from . import build as _build

OK, BAD_ARG, ZERO_EIGENVALUE, NONFINITE = 0, 1, 2, 3

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        for name in ("oracle_sign_tri", "oracle_sign_spectral"):
            f = getattr(L, name)
            f.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int]
            f.restype = ctypes.c_int
        L.oracle_sign_tri_count.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_longlong)]
        L.oracle_sign_tri_count.restype = ctypes.c_int
        L.oracle_sign_tri_antidiag.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int,
                                               ctypes.c_int]
        L.oracle_sign_tri_antidiag.restype = ctypes.c_int
        L.oracle_sign_schur.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int,
                                        ctypes.c_int]
        L.oracle_sign_schur.restype = ctypes.c_int
        L.oracle_sign_tri_complex.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int]
        L.oracle_sign_tri_complex.restype = ctypes.c_int
        L.oracle_sign_schur_complex.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int]
        L.oracle_sign_schur_complex.restype = ctypes.c_int
        L.oracle_funm.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int]
        L.oracle_funm.restype = ctypes.c_int
        L.oracle_max_threads.argtypes = []
        L.oracle_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


class OracleError(RuntimeError):
    def __init__(self, status):
        super().__init__("oracle status %d" % status)
        self.status = status


def _colmajor(T):
    T = np.asarray(T, dtype=np.float64)
    if T.ndim != 2 or T.shape[0] != T.shape[1]:
        raise ValueError("T must be square")
    return np.asfortranarray(T)


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def sign_tri(T, *, threads=None, schedule="paper"):
    """sign(T) by the Parlett-Higham substitution (Eqs. 1 and 2 entry by
    entry).  schedule='paper' visits columns left to right, each bottom to
    top; 'antidiag' visits by anti-diagonal (OpenMP, bit-identical)."""
    T = _colmajor(T)
    n = T.shape[0]
    U = np.zeros((n, n), dtype=np.float64, order="F")
    ld = max(n, 1)
    if schedule == "paper":
        st = lib().oracle_sign_tri(n, _ptr(T), ld, _ptr(U), ld)
    elif schedule == "antidiag":
        st = lib().oracle_sign_tri_antidiag(n, _ptr(T), ld, _ptr(U), ld, int(threads or 0))
    else:
        raise ValueError(schedule)
    if st != OK:
        raise OracleError(st)
    return U


def sign_tri_status(T):
    """Status code of Algorithm 3 on T (0 when it succeeds)."""
    T = _colmajor(T)
    n = T.shape[0]
    U = np.zeros((n, n), dtype=np.float64, order="F")
    return lib().oracle_sign_tri(n, _ptr(T), max(n, 1), _ptr(U), max(n, 1))


def useful_flops(T):
    """Floating-point operations executed by the inner sums of Algorithm 3."""
    T = _colmajor(T)
    n = T.shape[0]
    U = np.zeros((n, n), dtype=np.float64, order="F")
    c = ctypes.c_longlong(0)
    st = lib().oracle_sign_tri_count(n, _ptr(T), max(n, 1), _ptr(U), max(n, 1), ctypes.byref(c))
    if st != OK:
        raise OracleError(st)
    return int(c.value)


def sign_spectral(T):
    """Brute force sign(T) = Z sign(D) Z^{-1} in long double (n <= 64)."""
    T = _colmajor(T)
    n = T.shape[0]
    U = np.zeros((n, n), dtype=np.float64, order="F")
    st = lib().oracle_sign_spectral(n, _ptr(T), max(n, 1), _ptr(U), max(n, 1))
    if st != OK:
        raise OracleError(st)
    return U


def sign_schur(Q, T, *, threads=None):
    """sign(A) = Q sign(T) Q^T for the real Schur pair A = Q T Q^T (Section 1:
    the route through a Schur decomposition; Algorithm 3's first step)."""
    Q = _colmajor(Q)
    T = _colmajor(T)
    if Q.shape != T.shape:
        raise ValueError("Q and T must have the same shape")
    n = T.shape[0]
    S = np.zeros((n, n), dtype=np.float64, order="F")
    st = lib().oracle_sign_schur(n, _ptr(Q), max(n, 1), _ptr(T), max(n, 1), _ptr(S), max(n, 1), int(threads or 0))
    if st != OK:
        raise OracleError(st)
    return S


def _ccolmajor(M):
    M = np.asarray(M, dtype=np.complex128)
    if M.ndim != 2 or M.shape[0] != M.shape[1]:
        raise ValueError("matrix must be square")
    return np.asfortranarray(M)


def sign_tri_complex(T):
    """sign(T) of a complex upper triangular T (complex128): u_ii =
    sign(Re t_ii), then Eqs. 1 and 2 entry by entry (Algorithm 3)."""
    T = _ccolmajor(T)
    n = T.shape[0]
    U = np.zeros((n, n), dtype=np.complex128, order="F")
    st = lib().oracle_sign_tri_complex(n, _ptr(T), max(n, 1), _ptr(U), max(n, 1))
    if st != OK:
        raise OracleError(st)
    return U


def sign_schur_complex(Q, T):
    """sign(A) = Q sign(T) Q^H for a complex Schur pair A = Q T Q^H (Section
    1's route; Algorithm 3's first step)."""
    Q = _ccolmajor(Q)
    T = _ccolmajor(T)
    if Q.shape != T.shape:
        raise ValueError("Q and T must have the same shape")
    n = T.shape[0]
    S = np.zeros((n, n), dtype=np.complex128, order="F")
    st = lib().oracle_sign_schur_complex(n, _ptr(Q), max(n, 1), _ptr(T), max(n, 1), _ptr(S), max(n, 1))
    if st != OK:
        raise OracleError(st)
    return S


def sign_general(A):
    """sign(A) of a general real A by the paper's route (Section 1): the
    complex Schur form A = Q T Q^H from LAPACK (scipy.linalg.schur, a library
    step), then sign_schur_complex; returns the real part (A real makes
    sign(A) real; the imaginary part left is rounding)."""
    import scipy.linalg
    A = np.asarray(A, dtype=np.float64)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be square")
    if A.shape[0] == 0:
        return np.zeros((0, 0), order="F")
    T, Z = scipy.linalg.schur(A, output="complex")
    return np.asfortranarray(sign_schur_complex(Z, np.triu(T)).real)


PHI = {"exp": 1, "log": 2, "sqrt": 3, "sign": 4}


def funm(T, phi):
    """phi(T) of an upper triangular T with distinct diagonal entries by
    Parlett's substitution (Section 2, Algorithm 1): f_ii = phi(t_ii), then
    each f_ij from entry (i, j) of TF = FT.  phi: "exp", "log", "sqrt"
    (principal branches, t_ii > 0 for the last two) or "sign"."""
    T = _colmajor(T)
    n = T.shape[0]
    F = np.zeros((n, n), dtype=np.float64, order="F")
    st = lib().oracle_funm(n, _ptr(T), max(n, 1), _ptr(F), max(n, 1), PHI[phi])
    if st != OK:
        raise OracleError(st)
    return F


def max_threads():
    return int(lib().oracle_max_threads())
