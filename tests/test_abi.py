"""The C-ABI library loads and exports every function that include/signtri.h
declares; argument checks that return before any CUDA call (no GPU needed)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "signtri.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\**\s*([a-z_0-9]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1607_06303_gb300 import build
    build.build()
    import paper_1607_06303_gb300 as p
    return p


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("sign_tri", "sign_tri_host", "signtri_workspace_bytes", "signtri_set_workspace",
                     "signtri_status_string", "signtri_inertia", "signtri_get_info", "signtri_set_cutoff"):
        assert required in names


def test_exports_every_declared_symbol(lib):
    from paper_1607_06303_gb300 import signtri
    out = subprocess.run(["nm", "-D", "--defined-only", signtri.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    for name in declared_functions():
        assert name in exported, name
        assert name in signtri.exported_symbols(), name
    L = lib.load()
    for name in declared_functions():
        assert hasattr(L, name)


def test_status_strings(lib):
    assert lib.signtri_status_string(0) == "SIGNTRI_OK"
    assert lib.signtri_status_string(2) == "SIGNTRI_ERR_ZERO_EIGENVALUE"
    assert lib.signtri_status_string(99) == "SIGNTRI_ERR_UNKNOWN"


def test_host_side_argument_checks(lib):
    # these return before touching CUDA
    assert lib.sign_tri(-1, 0, 1, 0, 1, 1, 0) == lib.Status.ERR_BAD_ARG
    assert lib.sign_tri(0, 0, 1, 0, 1, 1, 0) == lib.Status.OK
    assert lib.sign_tri(4, 0, 4, 0, 4, 1, 0) == lib.Status.ERR_BAD_ARG          # NULL T
    assert lib.sign_tri(4, 16, 3, 16, 4, 1, 0) == lib.Status.ERR_BAD_ARG        # ldt < n
    assert lib.sign_tri(4, 16, 4, 16, 4, 17, 0) == lib.Status.ERR_BAD_ARG       # bad variant
    assert lib.sign_tri_host(-3, 0, 1, 0, 1, 0, 0) == lib.Status.ERR_BAD_ARG
    assert lib.signtri_set_cutoff(48) == lib.Status.ERR_BAD_ARG
    assert lib.signtri_set_cutoff(0) == lib.Status.OK
    assert lib.signtri_workspace_bytes(-1, 1) == 0
    assert lib.signtri_workspace_bytes(16384, 1) > 0
    assert lib.signtri_workspace_bytes(100, 1) >= 0
    info = lib.signtri_get_info()
    assert info.n == -3 and info.bad_index == -1


def test_profile_counters_host_side(lib):
    # counters are host state: readable and resettable without a GPU; bad
    # classes are rejected
    import ctypes
    L = lib.load()
    v = ctypes.c_double(-1.0)
    assert L.signtri_profile_read_flops(99, ctypes.byref(v)) == lib.Status.ERR_BAD_ARG
    assert L.signtri_profile_read_bytes(-1, ctypes.byref(v)) == lib.Status.ERR_BAD_ARG
    assert L.signtri_profile_read_bytes(lib.signtri.KC_BLOCK_SUMS_TC, None) == lib.Status.ERR_BAD_ARG
    assert lib.signtri_profile_reset() == lib.Status.OK
    assert lib.signtri_profile_read_bytes(lib.signtri.KC_BLOCK_SUMS_TC) == 0.0
    assert lib.signtri_profile_read_flops(lib.signtri.KC_RESIDUAL) == 0.0
    assert lib.signtri_kernel_class_name(lib.signtri.KC_BLOCK_SUMS_TC) == "block_sums_tc"


def _header_text():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return re.sub(r"//.*", "", txt)


def _c_kind(decl):
    """'ptr', or the base type of a C declaration without its name."""
    decl = " ".join(decl.replace("const", " ").split())
    if "*" in decl:
        return "ptr"
    words = decl.split()
    base = " ".join(words[:-1]) if len(words) > 1 else words[0]
    return {"signtri_variant": "int", "signtri_status": "int", "signtri_phi": "int"}.get(base, base)


def _ctypes_kind(t):
    import ctypes
    if t in (ctypes.c_void_p, ctypes.c_char_p) or (isinstance(t, type) and issubclass(t, ctypes._Pointer)):
        return "ptr"
    return {ctypes.c_int: "int", ctypes.c_size_t: "size_t", ctypes.c_double: "double",
            ctypes.c_longlong: "long long"}[t]


def test_binding_signatures_match_header():
    """Every prototype of include/signtri.h against the ctypes signature the
    binding installs: same arity, same kind (pointer, int, size_t, double,
    long long) in every position and in the return type."""
    from paper_1607_06303_gb300 import signtri
    protos = re.findall(r"^\s*((?:const\s+)?[a-z_]+\s*\**)\s*([a-z_0-9]+)\s*\(([^)]*)\)\s*;", _header_text(),
                        flags=re.M)
    assert len(protos) == len(declared_functions())
    for ret, name, params in protos:
        res, args = signtri._SIGNATURES[name]
        params = " ".join(params.split())
        c_args = [] if params in ("", "void") else [_c_kind(p) for p in params.split(",")]
        assert c_args == [_ctypes_kind(a) for a in args], name
        assert _c_kind(ret + " r") == _ctypes_kind(res), name
    assert set(signtri._SIGNATURES) == {p[1] for p in protos}


def test_binding_constants_match_header():
    """Variant and status codes, kernel classes and the signtri_info layout."""
    import ctypes

    from paper_1607_06303_gb300 import signtri
    txt = _header_text()
    enums = {k: int(v) for k, v in re.findall(r"\b(SIGNTRI_[A-Z0-9_]+)\s*=\s*(\d+)", txt)}
    for v in signtri.Variant:
        assert enums["SIGNTRI_" + v.name] == v.value
    for s in signtri.Status:
        assert enums["SIGNTRI_" + s.name] == s.value
    alias = {"OFFDIAG_LEAF_F32": "OFFDIAG_LEAF_MIXED"}
    kcs = {k[len("SIGNTRI_KC_"):]: v for k, v in enums.items() if k.startswith("SIGNTRI_KC_")}
    for k, v in kcs.items():
        assert getattr(signtri, "KC_" + alias.get(k, k)) == v, k
    body = re.search(r"typedef struct \{(.*?)\}\s*signtri_info;", txt, flags=re.S).group(1)
    fields = []
    for decl in body.split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        words = decl.split(" ", 1) if not decl.startswith("long long") else ["long long", decl[10:]]
        fields += [(n.strip(), words[0]) for n in words[1].split(",")]
    kinds = {"int": ctypes.c_int, "double": ctypes.c_double, "long long": ctypes.c_longlong}
    assert [(f, kinds[t]) for f, t in fields] == [(f, t) for f, t in signtri.Info._fields_]


class _FakeCudaTensor:
    """Attributes sign()'s checks read, without a GPU."""

    def __init__(self, n, ptr, dtype=None, cuda=True, contiguous=True, device="cuda:0", shape=None):
        import torch
        self.shape = shape or (n, n)
        self.dtype = dtype or torch.float64
        self.is_cuda = cuda
        self._contig = contiguous
        self.device = torch.device(device)
        self._ptr = ptr

    def dim(self):
        return len(self.shape)

    def is_contiguous(self):
        return self._contig

    def numel(self):
        out = 1
        for s in self.shape:
            out *= s
        return out

    def data_ptr(self):
        return self._ptr


def test_sign_operand_checks():
    """sign() rejects, before any library call, operands that would make the
    kernels read or write outside a tensor: wrong dtype, shape, layout,
    device, or an output overlapping T."""
    import torch

    from paper_1607_06303_gb300.signtri import check_operands
    F = _FakeCudaTensor
    T = F(8, 1 << 20)
    check_operands(T)
    check_operands(T, F(8, (1 << 20) + 512))                  # adjacent, not overlapping
    check_operands(F(0, 4096), F(0, 4096))                    # empty: nothing to overlap
    bad = [(F(8, 4096, dtype=torch.float32), None), (F(8, 4096, cuda=False), None),
           (F(8, 4096, shape=(8, 9)), None), (F(8, 4096, contiguous=False), None),
           (T, F(9, 4096)), (T, F(8, 4096, device="cuda:1")), (T, F(8, (1 << 20) + 504)),
           (T, F(8, (1 << 20) - 8)), (T, F(8, 1 << 20)), (T, F(8, 4096, dtype=torch.float32))]
    for t, u in bad:
        with pytest.raises(ValueError):
            check_operands(t, u)
    with pytest.raises(ValueError):
        from paper_1607_06303_gb300 import sign
        sign(torch.zeros(4, 4, dtype=torch.float64))           # a CPU tensor never reaches the library


def _elements(base, ld, rows, cols):
    """Byte offsets of the doubles of a column-major block."""
    return {base + 8 * (i + j * ld) for j in range(cols) for i in range(rows)}


def _bytes(base, ld, rows, cols):
    return {b + q for b in _elements(base, ld, rows, cols) for q in range(8)}


def _cuda_visible():
    import torch
    return torch.cuda.is_available()


@pytest.mark.skipif(_cuda_visible(), reason="accepted calls would launch kernels on made-up pointers")
def test_overlapping_operands_rejected(lib):
    """Output blocks that share an element with an input block are rejected
    with SIGNTRI_ERR_BAD_ARG before any CUDA call; disjoint blocks (also when
    interleaved in one array through their leading dimensions) pass the check
    and, with no GPU here, stop at the first CUDA call.  Checked against a
    brute-force intersection of the blocks' elements."""
    import random
    BAD, CUDA = lib.Status.ERR_BAD_ARG, lib.Status.ERR_CUDA
    rng = random.Random(7)
    base = 1 << 32
    cases = 0
    for _ in range(400):
        n = rng.randint(1, 9)
        ldt, ldu = n + rng.choice([0, 0, 1, 3, n]), n + rng.choice([0, 0, 2, n])
        off = 8 * rng.randint(-3 * n * ldu, 3 * n * ldt) + (rng.choice([1, 4]) if rng.random() < 0.1 else 0)
        pT, pU = base, base + off
        expect = BAD if _bytes(pT, ldt, n, n) & _bytes(pU, ldu, n, n) else CUDA
        assert lib.sign_tri(n, pT, ldt, pU, ldu, 1, 0) == expect, (n, ldt, ldu, off)
        assert lib.sign_tri_noalloc(n, pT, ldt, pU, ldu, 0) == expect, (n, ldt, ldu, off)
        cases += expect == BAD
    assert 50 < cases < 350          # both outcomes exercised
    # rectangular blocks: X (m x p) of the Sylvester solve against C (m x p)
    # in one array, interleaved by the leading dimension
    for _ in range(300):
        m, p_ = rng.randint(1, 6), rng.randint(1, 6)
        ldc, ldx = m + rng.choice([0, 1, m]), m + rng.choice([0, 2, m])
        off = 8 * rng.randint(-2 * p_ * ldx, 2 * p_ * ldc)
        pA, pB, pC, pX = base + (1 << 24), base + (1 << 25), base, base + off
        expect = BAD if _elements(pC, ldc, m, p_) & _elements(pX, ldx, m, p_) else CUDA
        assert lib.signtri_sylvester(m, p_, pA, m, pB, p_, pC, ldc, pX, ldx, 0) == expect, (m, p_, ldc, ldx, off)
        # the same pair as C = A B with A (m x k) in C's place
        assert lib.signtri_gemm_emulated(m, p_, p_, pC, ldc, pB, p_, pX, ldx, 0) == \
            (BAD if _elements(pC, ldc, m, p_) & _elements(pX, ldx, m, p_) else CUDA)
    # the Parlett-Sylvester reorder: Tr and Q each against T and each other
    n = 5
    assert lib.signtri_reorder_by_sign(n, base, n, base + 8 * n * n, n, base + 16 * n * n, n)[0] == CUDA
    assert lib.signtri_reorder_by_sign(n, base, n, base + 8 * n * n, n, base + 8 * (n * n + 3), n)[0] == BAD
    assert lib.signtri_reorder_by_sign(n, base, 2 * n, base + 8 * n, 2 * n, base + 16 * n * n, n)[0] == CUDA
    assert lib.signtri_reorder_by_sign(n, base, 2 * n, base + 8 * (n - 1), 2 * n, base + 16 * n * n, n)[0] == BAD


def test_batched_binding_rejects_ragged_lists(lib):
    with pytest.raises(ValueError):
        lib.sign_tri_batched([4, 4], [0], [4, 4], [0, 0], [4, 4], 1)
    # an empty batch is a no-op that needs no GPU
    assert lib.sign_tri_batched([], [], [], [], [], 1) == (lib.Status.OK, [])


def test_missing_library_fails_loudly(tmp_path):
    """Without libsigntri.so every entry point raises: there is no CPU or
    eager fallback behind the binding."""
    code = (
        "import paper_1607_06303_gb300 as p\n"
        "from paper_1607_06303_gb300 import signtri as s\n"
        "s.load.__defaults__ = (%r,)\n"
        "for call in (lambda: s.load(), lambda: p.sign_tri(4, 16, 4, 4096, 4, 1, 0),\n"
        "             lambda: p.signtri_status_string(0)):\n"
        "    try:\n"
        "        call()\n"
        "    except RuntimeError as e:\n"
        "        assert 'not built' in str(e), e\n"
        "    else:\n"
        "        raise SystemExit('no error without the library')\n"
        "print('raised')\n" % str(tmp_path / "missing" / "libsigntri.so"))
    out = subprocess.run([os.sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT)
    assert out.returncode == 0 and out.stdout.strip() == "raised", out.stdout + out.stderr
