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
    return {"signtri_variant": "int", "signtri_status": "int"}.get(base, base)


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
