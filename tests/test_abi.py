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
    names = re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\**\s*([a-z_]+)\s*\(", txt, flags=re.M)
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
