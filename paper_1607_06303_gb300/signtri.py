"""Thin ctypes binding of libsigntri.so (include/signtri.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  The functions keep the C names; the helpers at the end wrap torch
tensors (device memory and streams only).

A column-major n x n matrix M is held in a torch tensor `Mt` of shape
(n, n), contiguous, with Mt[j, i] = M[i, j] (the row-major storage of M^T);
its data pointer is then exactly the column-major array with ld = n.
"""
import ctypes
import enum
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsigntri.so")


class Variant(enum.IntEnum):
    AUTO = 0
    PH_FP64 = 1
    PS_FP64 = 2
    PH_MIXED_TF32 = 3
    PH_MIXED_BF16 = 4
    PH_FP64_EFFICIENT = 5
    PH_MIXED_FP16 = 6


class Status(enum.IntEnum):
    OK = 0
    ERR_BAD_ARG = 1
    ERR_ZERO_EIGENVALUE = 2
    ERR_NONFINITE = 3
    ERR_NO_CONVERGENCE = 4
    ERR_TIMEOUT = 5
    ERR_CUDA = 6
    ERR_NO_WORKSPACE = 7
    ERR_UNSUPPORTED = 8
    ERR_DOMAIN = 9


class Phi(enum.IntEnum):
    EXP = 1
    LOG = 2
    SQRT = 3
    SIGN = 4


class Info(ctypes.Structure):
    _fields_ = [
        ("variant", ctypes.c_int),
        ("n", ctypes.c_int),
        ("n_pos", ctypes.c_int),
        ("n_neg", ctypes.c_int),
        ("swaps", ctypes.c_longlong),
        ("work_ph", ctypes.c_double),
        ("work_ps", ctypes.c_double),
        ("cutoff", ctypes.c_int),
        ("refine_steps", ctypes.c_int),
        ("resid_commute", ctypes.c_double),
        ("resid_involution", ctypes.c_double),
        ("bad_index", ctypes.c_int),
        ("qr_sweeps", ctypes.c_longlong),
        ("qr_rotations", ctypes.c_longlong),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SignTriError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = Status(status)
        super().__init__("%s%s" % (where + ": " if where else "", self.status.name))


_lib = None
_VP = ctypes.c_void_p
_I = ctypes.c_int
_SZ = ctypes.c_size_t

# name -> (restype, argtypes)
_SIGNATURES = {
    "signtri_status_string": (ctypes.c_char_p, [_I]),
    "signtri_workspace_bytes": (_SZ, [_I, _I]),
    "signtri_set_workspace": (_I, [_VP, _SZ]),
    "signtri_set_cutoff": (_I, [_I]),
    "sign_tri": (_I, [_I, _VP, _I, _VP, _I, _I, _VP]),
    "sign_tri_host": (_I, [_I, _VP, _I, _VP, _I, _I, _VP]),
    "signtri_inertia": (_I, [_I, _VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                             ctypes.POINTER(ctypes.c_longlong), _VP]),
    "signtri_get_info": (_I, [ctypes.POINTER(Info)]),
    "signtri_profile_enable": (_I, [_I]),
    "signtri_profile_reset": (_I, []),
    "signtri_profile_read": (_I, [_I, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)]),
    "signtri_kernel_class_name": (ctypes.c_char_p, [_I]),
    "signtri_probe_fp64_peak": (_I, [ctypes.POINTER(ctypes.c_double), _VP]),
    "sign_tri_noalloc": (_I, [_I, _VP, _I, _VP, _I, _VP]),
    "signtri_reorder_by_sign": (_I, [_I, _VP, _I, _VP, _I, _VP, _I, ctypes.POINTER(ctypes.c_longlong), _VP]),
    "signtri_sylvester": (_I, [_I, _I, _VP, _I, _VP, _I, _VP, _I, _VP, _I, _VP]),
    "signtri_set_rates": (_I, [ctypes.c_double, ctypes.c_double]),
    "signtri_gemm_emulated": (_I, [_I, _I, _I, _VP, _I, _VP, _I, _VP, _I, _VP]),
    "signtri_set_refinement": (_I, [ctypes.c_double, _I]),
    "signtri_set_verification": (_I, [_I]),
    "signtri_profile_read_flops": (_I, [_I, ctypes.POINTER(ctypes.c_double)]),
    "signtri_profile_read_bytes": (_I, [_I, ctypes.POINTER(ctypes.c_double)]),
    "sign_tri_batched": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_VP), ctypes.POINTER(_I),
                              ctypes.POINTER(_VP), ctypes.POINTER(_I), _I, ctypes.POINTER(_I), _VP]),
    "signtri_set_cutoff_table": (_I, [ctypes.POINTER(_I), _I]),
    "signtri_get_cutoff_table": (_I, [ctypes.POINTER(_I), _I]),
    "signtri_autotune": (_I, [_I, _VP]),
    "signtri_get_variant_table": (_I, [ctypes.POINTER(_I), _I]),
    "signtri_set_variant_table": (_I, [ctypes.POINTER(_I), _I]),
    "signtri_batched_cache_stats": (_I, [ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    "signtri_selftest_wait": (_I, [_I, ctypes.c_longlong, _VP]),
    "signtri_sign_schur": (_I, [_I, _VP, _I, _VP, _I, _VP, _I, _I, _VP]),
    "signtri_sign_schur_workspace_bytes": (_SZ, [_I, _I]),
    "signtri_sign_tri_complex": (_I, [_I, _VP, _I, _VP, _I, _VP]),
    "signtri_sign_schur_complex": (_I, [_I, _VP, _I, _VP, _I, _VP, _I, _VP]),
    "signtri_complex_workspace_bytes": (_SZ, [_I]),
    "signtri_schur": (_I, [_I, _VP, _I, _VP, _I, _VP, _I, _VP]),
    "signtri_schur_workspace_bytes": (_SZ, [_I]),
    "signtri_sign_general": (_I, [_I, _VP, _I, _VP, _I, _VP]),
    "signtri_sign_general_workspace_bytes": (_SZ, [_I]),
    "signtri_funm": (_I, [_I, _VP, _I, _VP, _I, _I, _VP]),
}

SIGNTRI_NOALLOC_MAX_N = 1024

# kernel classes of the launch accounting (include/signtri.h)
KC_SCAN, KC_FILL, KC_DIAG_LEAF, KC_BLOCK_SUMS_F64, KC_OFFDIAG_LEAF = 0, 1, 2, 3, 4
KC_BLOCK_SUMS_TC, KC_OFFDIAG_LEAF_MIXED, KC_CONVERT, KC_RESIDUAL, KC_CORRECTION = 5, 6, 7, 8, 9
KC_GIVENS, KC_SYLV_SUMS, KC_SYLV_LEAF, KC_GEMM_F64, KC_OTHER, KC_RESIDUAL_SUM = 10, 11, 12, 13, 14, 15
KC_BATCH_GRAPH = 16
KC_SCHUR = 17
KC_HESSENBERG = 18
KC_HOST_COPY = 19
KC_COUNT = 20


def load(path: str = LIB_PATH):
    """Load libsigntri.so.  Raises if it has not been built: there is no
    fallback implementation."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libsigntri.so not built (%s); run __graft_entry__.build()" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGNATURES)


# ---- the C entry points, same names ---------------------------------------

def signtri_status_string(s: int) -> str:
    return load().signtri_status_string(int(s)).decode()


def signtri_workspace_bytes(n: int, v: int) -> int:
    return int(load().signtri_workspace_bytes(n, int(v)))


def signtri_set_workspace(dev_ptr: int, nbytes: int) -> int:
    return load().signtri_set_workspace(dev_ptr or None, nbytes)


def signtri_set_cutoff(b: int) -> int:
    return load().signtri_set_cutoff(b)


def sign_tri(n, T_ptr, ldt, U_ptr, ldu, v, stream) -> int:
    return load().sign_tri(n, T_ptr or None, ldt, U_ptr or None, ldu, int(v), stream or None)


def signtri_reorder_by_sign(n, T_ptr, ldt, Tr_ptr, ldtr, Q_ptr, ldq, stream=None):
    k = ctypes.c_longlong(0)
    st = load().signtri_reorder_by_sign(n, T_ptr or None, ldt, Tr_ptr or None, ldtr, Q_ptr or None, ldq,
                                        ctypes.byref(k), stream or None)
    return st, k.value


def signtri_sylvester(m, p, A_ptr, lda, B_ptr, ldb, C_ptr, ldc, X_ptr, ldx, stream=None) -> int:
    return load().signtri_sylvester(m, p, A_ptr or None, lda, B_ptr or None, ldb, C_ptr or None, ldc,
                                    X_ptr or None, ldx, stream or None)


def signtri_gemm_emulated(m, n, k, A_ptr, lda, B_ptr, ldb, C_ptr, ldc, stream=None) -> int:
    return load().signtri_gemm_emulated(m, n, k, A_ptr or None, lda, B_ptr or None, ldb, C_ptr or None, ldc,
                                        stream or None)


def sign_tri_batched(ns, T_ptrs, ldts, U_ptrs, ldus, v, stream=None):
    """Batched call on host lists; returns (status, per-matrix info list)."""
    cnt = len(ns)
    if not (len(T_ptrs) == len(ldts) == len(U_ptrs) == len(ldus) == cnt):
        raise ValueError("sign_tri_batched: n, T, ldt, U and ldu must have the same length")
    arr = lambda t, xs: (t * max(cnt, 1))(*xs)
    info = (_I * max(cnt, 1))()
    st = load().sign_tri_batched(cnt, arr(_I, ns), arr(_VP, T_ptrs), arr(_I, ldts), arr(_VP, U_ptrs),
                                 arr(_I, ldus), int(v), info, stream or None)
    return st, list(info)[:cnt]


def signtri_set_cutoff_table(table) -> int:
    arr = (_I * max(len(table), 1))(*table)
    return load().signtri_set_cutoff_table(arr, len(table))


def signtri_get_cutoff_table(length: int = 32):
    arr = (_I * length)()
    st = load().signtri_get_cutoff_table(arr, length)
    if st != 0:
        raise SignTriError(st, "signtri_get_cutoff_table")
    return list(arr)


def signtri_autotune(n_max: int, stream=None) -> int:
    return load().signtri_autotune(int(n_max), stream or None)


def signtri_set_variant_table(table) -> int:
    arr = (_I * max(len(table), 1))(*[int(v) for v in table])
    return load().signtri_set_variant_table(arr, len(table))


def signtri_get_variant_table(length: int = 32):
    arr = (_I * length)()
    st = load().signtri_get_variant_table(arr, length)
    if st != 0:
        raise SignTriError(st, "signtri_get_variant_table")
    return list(arr)


def signtri_batched_cache_stats():
    """(launches of a kept batch graph, graphs built) since the library was loaded."""
    h, b = ctypes.c_longlong(0), ctypes.c_longlong(0)
    st = load().signtri_batched_cache_stats(ctypes.byref(h), ctypes.byref(b))
    if st != 0:
        raise SignTriError(st, "signtri_batched_cache_stats")
    return h.value, b.value


def signtri_selftest_wait(arrive: bool, limit_cycles: int, stream=None) -> int:
    return load().signtri_selftest_wait(1 if arrive else 0, int(limit_cycles), stream or None)


def signtri_set_refinement(tol: float, max_steps: int) -> int:
    return load().signtri_set_refinement(float(tol), int(max_steps))


def signtri_set_verification(full: int) -> int:
    return load().signtri_set_verification(int(full))


def signtri_set_rates(gemm_flops_per_s: float, givens_flops_per_s: float) -> int:
    return load().signtri_set_rates(float(gemm_flops_per_s), float(givens_flops_per_s))


def sign_tri_noalloc(n, T_ptr, ldt, U_ptr, ldu, stream) -> int:
    """sign_tri with SIGNTRI_PH_FP64, scratch in a static device array (no
    allocation); n <= SIGNTRI_NOALLOC_MAX_N."""
    return load().sign_tri_noalloc(n, T_ptr or None, ldt, U_ptr or None, ldu, stream or None)


def sign_tri_host(n, T_ptr, ldt, U_ptr, ldu, v, stream) -> int:
    return load().sign_tri_host(n, T_ptr or None, ldt, U_ptr or None, ldu, int(v), stream or None)


def signtri_inertia(n, T_ptr, ldt, stream=None):
    p, m, k = _I(0), _I(0), ctypes.c_longlong(0)
    st = load().signtri_inertia(n, T_ptr or None, ldt, ctypes.byref(p), ctypes.byref(m), ctypes.byref(k),
                                stream or None)
    return st, p.value, m.value, k.value


def signtri_get_info() -> Info:
    out = Info()
    st = load().signtri_get_info(ctypes.byref(out))
    if st != 0:
        raise SignTriError(st, "signtri_get_info")
    return out


def signtri_profile_enable(on: bool) -> int:
    return load().signtri_profile_enable(1 if on else 0)


def signtri_profile_reset() -> int:
    return load().signtri_profile_reset()


def signtri_profile_read(cls: int):
    n, ms = ctypes.c_longlong(0), ctypes.c_double(0)
    st = load().signtri_profile_read(cls, ctypes.byref(n), ctypes.byref(ms))
    if st != 0:
        raise SignTriError(st, "signtri_profile_read")
    return n.value, ms.value


def signtri_profile_read_flops(cls: int) -> float:
    f = ctypes.c_double(0)
    st = load().signtri_profile_read_flops(cls, ctypes.byref(f))
    if st != 0:
        raise SignTriError(st, "signtri_profile_read_flops")
    return f.value


def signtri_profile_read_bytes(cls: int) -> float:
    b = ctypes.c_double(0)
    st = load().signtri_profile_read_bytes(cls, ctypes.byref(b))
    if st != 0:
        raise SignTriError(st, "signtri_profile_read_bytes")
    return b.value


def signtri_kernel_class_name(cls: int) -> str:
    return load().signtri_kernel_class_name(cls).decode()


def signtri_probe_fp64_peak(stream=None) -> float:
    g = ctypes.c_double(0)
    st = load().signtri_probe_fp64_peak(ctypes.byref(g), stream or None)
    if st != 0:
        raise SignTriError(st, "signtri_probe_fp64_peak")
    return g.value


# ---- torch helpers (device memory and streams only) ------------------------

def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def check_operands(Tt, Ut=None):
    """The checks sign() makes before a pointer reaches the library: T (and
    U, when given) square, contiguous float64 CUDA tensors; U with T's shape
    and device and no byte in common with T (sign_tri writes all n*n entries
    of U and reads T while it does)."""
    import torch
    for name, t in (("T", Tt), ("out", Ut)):
        if t is None:
            continue
        if t.dtype != torch.float64 or not t.is_cuda or t.dim() != 2 or t.shape[0] != t.shape[1]:
            raise ValueError("%s must be a square CUDA float64 tensor" % name)
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
    if Ut is not None:
        if tuple(Ut.shape) != tuple(Tt.shape) or Ut.device != Tt.device:
            raise ValueError("out must have T's shape and device")
        nbytes = 8 * Tt.numel()
        if nbytes and Ut.data_ptr() < Tt.data_ptr() + nbytes and Tt.data_ptr() < Ut.data_ptr() + nbytes:
            raise ValueError("out must not overlap T")


def sign(Tt, variant=Variant.AUTO, out=None, stream=None, check=True):
    """U = sign(T) for a CUDA float64 tensor holding T column-major (see the
    module docstring).  Returns the tensor holding U in the same layout.
    Runs on T's device, on `stream` (default: that device's current stream)."""
    import torch
    check_operands(Tt, out)
    n = Tt.shape[0]
    Ut = out if out is not None else torch.empty_like(Tt)
    with torch.cuda.device(Tt.device):
        st = sign_tri(n, Tt.data_ptr(), max(n, 1), Ut.data_ptr(), max(n, 1), variant, _stream_handle(stream))
    if check and st != 0:
        raise SignTriError(st, "sign_tri")
    return Ut


def signtri_sign_schur(n, Q_ptr, ldq, T_ptr, ldt, S_ptr, lds, variant=Variant.AUTO, stream=None) -> int:
    return load().signtri_sign_schur(n, Q_ptr or None, ldq, T_ptr or None, ldt, S_ptr or None, lds, int(variant),
                                     stream or None)


def signtri_sign_schur_workspace_bytes(n, variant=Variant.AUTO) -> int:
    return load().signtri_sign_schur_workspace_bytes(n, int(variant))


def sign_schur(Qt, Tt, variant=Variant.AUTO, out=None, stream=None, check=True):
    """S = Q sign(T) Q^T from a real Schur pair (CUDA float64 tensors in the
    layout above, Q orthogonal, T upper triangular).  Returns S."""
    import torch
    check_operands(Tt, out)
    check_operands(Qt, out)
    n = Tt.shape[0]
    if tuple(Qt.shape) != tuple(Tt.shape) or Qt.device != Tt.device:
        raise ValueError("Q and T must be n x n on the same device")
    St = out if out is not None else torch.empty_like(Tt)
    with torch.cuda.device(Tt.device):
        st = signtri_sign_schur(n, Qt.data_ptr(), max(n, 1), Tt.data_ptr(), max(n, 1), St.data_ptr(), max(n, 1),
                                variant, _stream_handle(stream))
    if check and st != 0:
        raise SignTriError(st, "signtri_sign_schur")
    return St


def signtri_sign_tri_complex(n, T_ptr, ldt, U_ptr, ldu, stream=None) -> int:
    return load().signtri_sign_tri_complex(n, T_ptr or None, ldt, U_ptr or None, ldu, stream or None)


def signtri_sign_schur_complex(n, Q_ptr, ldq, T_ptr, ldt, S_ptr, lds, stream=None) -> int:
    return load().signtri_sign_schur_complex(n, Q_ptr or None, ldq, T_ptr or None, ldt, S_ptr or None, lds,
                                             stream or None)


def signtri_complex_workspace_bytes(n) -> int:
    return load().signtri_complex_workspace_bytes(n)


def _check_complex(name, t):
    import torch
    if t.dtype != torch.complex128 or not t.is_cuda or t.dim() != 2 or t.shape[0] != t.shape[1]:
        raise ValueError("%s must be a square CUDA complex128 tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)


def sign_complex(Tt, out=None, stream=None, check=True):
    """U = sign(T) for a CUDA complex128 tensor holding complex upper
    triangular T column-major (to_device_complex's layout)."""
    import torch
    _check_complex("T", Tt)
    Ut = out if out is not None else torch.empty_like(Tt)
    _check_complex("out", Ut)
    n = Tt.shape[0]
    with torch.cuda.device(Tt.device):
        st = signtri_sign_tri_complex(n, Tt.data_ptr(), max(n, 1), Ut.data_ptr(), max(n, 1), _stream_handle(stream))
    if check and st != 0:
        raise SignTriError(st, "signtri_sign_tri_complex")
    return Ut


def sign_schur_complex(Qt, Tt, out=None, stream=None, check=True):
    """S = Q sign(T) Q^H from a complex Schur pair (CUDA complex128 tensors,
    column-major as to_device_complex makes them)."""
    import torch
    _check_complex("T", Tt)
    _check_complex("Q", Qt)
    if tuple(Qt.shape) != tuple(Tt.shape) or Qt.device != Tt.device:
        raise ValueError("Q and T must be n x n on the same device")
    St = out if out is not None else torch.empty_like(Tt)
    _check_complex("out", St)
    n = Tt.shape[0]
    with torch.cuda.device(Tt.device):
        st = signtri_sign_schur_complex(n, Qt.data_ptr(), max(n, 1), Tt.data_ptr(), max(n, 1), St.data_ptr(),
                                        max(n, 1), _stream_handle(stream))
    if check and st != 0:
        raise SignTriError(st, "signtri_sign_schur_complex")
    return St


def to_device_complex(M_colmajor, device="cuda"):
    """numpy complex n x n matrix -> CUDA complex128 tensor holding it
    column-major (interleaved re, im; the tensor is the transpose)."""
    import numpy as np
    import torch
    a = np.asfortranarray(np.asarray(M_colmajor, dtype=np.complex128))
    return torch.from_numpy(np.ascontiguousarray(a.T)).to(device)


def signtri_schur(n, A_ptr, lda, Q_ptr, ldq, T_ptr, ldt, stream=None) -> int:
    return load().signtri_schur(n, A_ptr or None, lda, Q_ptr or None, ldq, T_ptr or None, ldt, stream or None)


def signtri_schur_workspace_bytes(n) -> int:
    return load().signtri_schur_workspace_bytes(n)


def signtri_sign_general(n, A_ptr, lda, S_ptr, lds, stream=None) -> int:
    return load().signtri_sign_general(n, A_ptr or None, lda, S_ptr or None, lds, stream or None)


def signtri_sign_general_workspace_bytes(n) -> int:
    return load().signtri_sign_general_workspace_bytes(n)


def schur(At, stream=None, check=True):
    """Complex Schur decomposition A = Q T Q^H of a real A (a CUDA float64
    tensor in the layout above), on the GPU.  Returns (Q, T) as CUDA
    complex128 tensors in to_device_complex's layout."""
    import torch
    check_operands(At)
    n = At.shape[0]
    Qt = torch.empty((n, n), dtype=torch.complex128, device=At.device)
    Tt = torch.empty((n, n), dtype=torch.complex128, device=At.device)
    with torch.cuda.device(At.device):
        st = signtri_schur(n, At.data_ptr(), max(n, 1), Qt.data_ptr(), max(n, 1), Tt.data_ptr(), max(n, 1),
                           _stream_handle(stream))
    if check and st != 0:
        raise SignTriError(st, "signtri_schur")
    return Qt, Tt


def sign_general(At, out=None, stream=None, check=True):
    """S = sign(A) of a general real A (CUDA float64 tensor, layout above):
    the Schur decomposition, the complex sign of T and Q U Q^H, all on the
    GPU.  Returns S (real)."""
    import torch
    check_operands(At, out)
    n = At.shape[0]
    St = out if out is not None else torch.empty_like(At)
    with torch.cuda.device(At.device):
        st = signtri_sign_general(n, At.data_ptr(), max(n, 1), St.data_ptr(), max(n, 1), _stream_handle(stream))
    if check and st != 0:
        raise SignTriError(st, "signtri_sign_general")
    return St


def signtri_funm(n, T_ptr, ldt, F_ptr, ldf, phi, stream=None) -> int:
    return load().signtri_funm(n, T_ptr or None, ldt, F_ptr or None, ldf, int(phi), stream or None)


def funm(Tt, phi, out=None, stream=None, check=True):
    """F = phi(T) (Phi.EXP, LOG, SQRT, SIGN) for a CUDA float64 tensor holding
    upper triangular T column-major, by Parlett's substitution (distinct
    diagonal entries)."""
    import torch
    check_operands(Tt, out)
    n = Tt.shape[0]
    Ft = out if out is not None else torch.empty_like(Tt)
    with torch.cuda.device(Tt.device):
        st = signtri_funm(n, Tt.data_ptr(), max(n, 1), Ft.data_ptr(), max(n, 1), Phi(phi), _stream_handle(stream))
    if check and st != 0:
        raise SignTriError(st, "signtri_funm")
    return Ft


def to_device(T_colmajor, device="cuda"):
    """numpy column-major (Fortran-order) n x n float64 -> CUDA tensor in the
    layout above."""
    import numpy as np
    import torch
    a = np.asfortranarray(np.asarray(T_colmajor, dtype=np.float64))
    return torch.from_numpy(np.ascontiguousarray(a.T)).to(device)


def to_numpy(Mt):
    """Inverse of to_device: CUDA tensor -> numpy column-major array."""
    import numpy as np
    return np.asfortranarray(Mt.cpu().numpy().T)
