"""The oracle pins must catch plausible mistakes.  Each case below plants one
mistake in a copy of oracle.c (on the CPU, in a temporary directory), builds
it, and checks that the independent pins used in test_oracle_pins.py
(numpy-eigendecomposition brute force, UT = TU, U^2 = I) reject it."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_1607_06303_gb300.inputs import make_T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

# (name, text in the Algorithm 3 routine, replacement)
MUTANTS = [
    ("dropped t_ij term", "AT(T, ldt, i, j) * (uii - ujj) / den + s / den", "s / den"),
    ("sign of commutator sum", "s = s + (a - b);", "s = s + (b - a);"),
    ("sum starts at k=i", "for (int k = i + 1; k <= j - 1; k++) {", "for (int k = i; k <= j - 1; k++) {"),
    ("transposed operand", "s = s + AT(U, ldu, i, k) * AT(U, ldu, k, j);",
     "s = s + AT(U, ldu, i, k) * AT(U, ldu, j, k);"),
    ("sign of U^2 branch", "AT(U, ldu, i, j) = -s / (uii + ujj);", "AT(U, ldu, i, j) = s / (uii + ujj);"),
    ("denominator reversed", "double den = AT(T, ldt, i, i) - AT(T, ldt, j, j);",
     "double den = AT(T, ldt, j, j) - AT(T, ldt, i, i);"),
    ("row/column swapped in T", "double b = AT(T, ldt, i, k) * AT(U, ldu, k, j);",
     "double b = AT(T, ldt, k, j) * AT(U, ldu, i, k);"),
    ("branch test inverted", "if (uii + ujj == 0.0) {\n                double s = 0.0;\n                for (int k = i + 1; k <= j - 1; k++) {",
     "if (uii + ujj != 0.0 && 0) {\n                double s = 0.0;\n                for (int k = i + 1; k <= j - 1; k++) {"),
]


def _build_mutant(tmp_path, old, new):
    src = open(SRC).read()
    body_start = src.index("int oracle_sign_tri_count(")
    body_end = src.index("int oracle_sign_tri(int n")
    body = src[body_start:body_end]
    assert old in body, old
    src = src[:body_start] + body.replace(old, new, 1) + src[body_end:]
    c = tmp_path / "mut.c"
    c.write_text(src)
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", str(c), "-o", str(so), "-lm"],
                   check=True, capture_output=True)
    L = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    L.oracle_sign_tri.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int]
    L.oracle_sign_tri.restype = ctypes.c_int
    return L


def _run(L, T):
    T = np.asfortranarray(T)
    n = T.shape[0]
    U = np.zeros((n, n), order="F")
    dp = ctypes.POINTER(ctypes.c_double)
    L.oracle_sign_tri(n, T.ctypes.data_as(dp), n, U.ctypes.data_as(dp), n)
    return U


def _pins_pass(L):
    for n, p, seed in [(8, 0.5, 0), (11, 0.3, 1), (60, 0.5, 2)]:
        T = make_T(n, p, seed=seed)
        U = _run(L, T)
        if not np.all(np.isfinite(U)):
            return False
        if n <= 12:
            w, V = np.linalg.eig(T)
            Ue = ((V * np.sign(w.real)) @ np.linalg.inv(V)).real
            if np.linalg.norm(U - Ue) > 1e-9 * np.linalg.norm(Ue):
                return False
        I = np.eye(n)
        if np.linalg.norm(U @ U - I) > 1e-12 * np.linalg.norm(U) ** 2:
            return False
        if np.linalg.norm(U @ T - T @ U) > 1e-12 * np.linalg.norm(T) * np.linalg.norm(U):
            return False
    return True


def test_unmutated_passes(tmp_path):
    L = _build_mutant(tmp_path, "s = s + (a - b);", "s = s + (a - b);")
    assert _pins_pass(L)


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_rejected(tmp_path, name, old, new):
    L = _build_mutant(tmp_path, old, new)
    assert not _pins_pass(L), name
