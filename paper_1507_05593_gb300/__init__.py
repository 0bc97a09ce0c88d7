"""Python binding of the rank-structured supernodal Cholesky library (``librsc.so``).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels (symbolic analysis in its C++ host code).  The functions carry the names
of the C ABI in ``include/rsc.h``; see that header for the meaning, layout,
ownership and error behaviour of each argument.

The shared library is loaded on first use.  If it is missing the call raises
``RuntimeError``; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librsc.so")

RSC_OK = 0
STATUS = {0: "RSC_OK", 1: "RSC_ERR_INVALID_ARG", 2: "RSC_ERR_NOT_SPD", 3: "RSC_ERR_NO_CONVERGENCE",
          4: "RSC_ERR_OOM", 5: "RSC_ERR_CUDA", 6: "RSC_ERR_TIMEOUT", 7: "RSC_ERR_STATE"}
PREC = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3}


class rsc_options(C.Structure):
    _fields_ = [("tau_O", C.c_int32), ("tau_D", C.c_int32), ("leaf_size", C.c_int32),
                ("sample_block", C.c_int32), ("power_iters", C.c_int32), ("dof_per_node", C.c_int32),
                ("max_restarts", C.c_int32), ("precision", C.c_int32), ("diag_compress", C.c_int32),
                ("ordering", C.c_int32), ("seed", C.c_uint64), ("amalgamate", C.c_int32),
                ("interior_blocks", C.c_int32)]


class rsc_stats_t(C.Structure):
    _fields_ = [("factor_bytes", C.c_double), ("factor_flops", C.c_double), ("factor_seconds", C.c_double),
                ("solve_seconds", C.c_double), ("restarts", C.c_int32), ("n_supernodes", C.c_int32),
                ("n_compressed", C.c_int32), ("n_levels", C.c_int32), ("max_rank", C.c_int32),
                ("last_iters", C.c_int32), ("last_relres", C.c_double), ("gpu_launches", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class RscError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None

_P = C.c_void_p
_SIGS = {
    "rsc_options_default": (C.c_int, [C.POINTER(rsc_options)]),
    "rsc_analyze": (C.c_int, [C.c_int64, _P, _P, _P, _P, C.POINTER(rsc_options), C.POINTER(_P)]),
    "rsc_get_ordering": (C.c_int, [_P, _P, C.POINTER(C.c_int32), _P]),
    "rsc_get_structure": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "rsc_get_coordinates": (C.c_int, [_P, _P]),
    "rsc_factor": (C.c_int, [_P, C.c_double]),
    "rsc_factor_fixed_rank": (C.c_int, [_P, C.c_double, C.c_double, C.c_int32]),
    "rsc_refactor_values": (C.c_int, [_P, _P]),
    "rsc_solve": (C.c_int, [_P, _P, _P, C.c_double, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "rsc_solve_device": (C.c_int, [_P, _P, _P, C.c_double, C.c_int32, C.POINTER(C.c_int32),
                                   C.POINTER(C.c_double), _P]),
    "rsc_apply_preconditioner_device": (C.c_int, [_P, _P, _P, _P]),
    "rsc_apply_preconditioner_device_noalloc": (C.c_int, [_P, _P, _P, _P]),
    "rsc_pattern_outer_device": (C.c_int, [_P, _P, _P, C.c_double, _P, _P]),
    "rsc_get_systems": (C.c_int, [_P, C.POINTER(C.c_int32), _P]),
    "rsc_solve_batch_device": (C.c_int, [_P, C.c_int32, _P, _P, C.c_double, C.c_int32, _P, _P, _P]),
    "rsc_get_supernode_info": (C.c_int, [_P, C.c_int32, _P]),
    "rsc_get_supernode_blocks": (C.c_int, [_P, C.c_int32, _P, _P]),
    "rsc_get_stats": (C.c_int, [_P, C.POINTER(rsc_stats_t)]),
    "rsc_profile": (C.c_int, [_P, C.c_int32, C.c_char_p]),
    "rsc_get_kernel_profile": (C.c_int, [_P, C.c_char_p, C.c_int64]),
    "rsc_get_autotune": (C.c_int, [_P, C.c_char_p, C.c_int64]),
    "rsc_set_wait_limit": (C.c_int, [_P, C.c_int64]),
    "rsc_refactor_values_device": (C.c_int, [_P, _P, _P]),
    "rsc_last_error": (C.c_char_p, [_P]),
    "rsc_destroy": (None, [_P]),
}


def lib():
    """Load ``librsc.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1507_05593_gb300._build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _check(st, h=None):
    if st != RSC_OK:
        msg = lib().rsc_last_error(h)
        raise RscError(st, msg.decode() if msg else "")


def rsc_options_default(**kw) -> rsc_options:
    o = rsc_options()
    _check(lib().rsc_options_default(C.byref(o)))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PREC[v]
        if not any(f == k for f, _ in rsc_options._fields_):
            raise TypeError(f"unknown option {k!r}")
        setattr(o, k, int(v))
    return o


class Handle:
    """Owns one ``rsc_handle*``; destroyed with the object."""

    def __init__(self, ptr, n):
        self.ptr = C.c_void_p(ptr)
        self.n = n

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.rsc_destroy(self.ptr)
            self.ptr = None


def rsc_analyze(n, row_ptr, col_idx, val, coords, opts: rsc_options | None = None) -> Handle:
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    v = np.ascontiguousarray(val, dtype=np.float64)
    xyz = None if coords is None else np.ascontiguousarray(coords, dtype=np.float64)
    out = C.c_void_p()
    st = lib().rsc_analyze(int(n), _ptr(rp), _ptr(ci), _ptr(v), _ptr(xyz),
                           C.byref(opts) if opts is not None else None, C.byref(out))
    _check(st)
    h = Handle(out.value, int(n))
    h.dof = int(opts.dof_per_node) if opts is not None else 1
    return h


def rsc_get_ordering(h: Handle):
    perm = np.empty(h.n, np.int32)
    m = C.c_int32()
    _check(lib().rsc_get_ordering(h.ptr, _ptr(perm), C.byref(m), None), h.ptr)
    sp = np.empty(m.value + 1, np.int64)
    _check(lib().rsc_get_ordering(h.ptr, None, None, _ptr(sp)), h.ptr)
    return perm, sp


def rsc_get_coordinates(h: Handle) -> np.ndarray:
    """Node positions the ordering used, (n / dof_per_node) x 3."""
    pos = np.empty((h.n // getattr(h, "dof", 1), 3), np.float64)
    _check(lib().rsc_get_coordinates(h.ptr, _ptr(pos)), h.ptr)
    return pos


def rsc_get_structure(h: Handle):
    _, sp = rsc_get_ordering(h)
    M = sp.size - 1
    rows_ptr = np.empty(M + 1, np.int64)
    _check(lib().rsc_get_structure(h.ptr, _ptr(rows_ptr), None, None, None, None), h.ptr)
    rows = np.empty(max(int(rows_ptr[-1]), 1), np.int32)
    parent = np.empty(M, np.int32)
    level = np.empty(M, np.int32)
    kind = np.empty(M, np.int32)
    _check(lib().rsc_get_structure(h.ptr, _ptr(rows_ptr), _ptr(rows), _ptr(parent), _ptr(level), _ptr(kind)),
           h.ptr)
    return rows_ptr, rows[:rows_ptr[-1]], parent, level, kind


def rsc_factor(h: Handle, tol: float) -> None:
    _check(lib().rsc_factor(h.ptr, float(tol)), h.ptr)


def rsc_factor_fixed_rank(h: Handle, alpha_O: float, alpha_D: float = 0.5, p: int = 8) -> None:
    """Fixed-rank form (Section 5.2): ranks ceil(alpha sqrt(k) log2 k) + p, k = min(m, n)."""
    _check(lib().rsc_factor_fixed_rank(h.ptr, float(alpha_O), float(alpha_D), int(p)), h.ptr)


def rsc_refactor_values(h: Handle, val) -> None:
    v = np.ascontiguousarray(val, dtype=np.float64)
    _check(lib().rsc_refactor_values(h.ptr, _ptr(v)), h.ptr)


def rsc_refactor_values_device(h: Handle, d_val, stream=None) -> None:
    """d_val: CUDA float64 tensor of the nnz values (or a raw device pointer as an int)."""
    pv = d_val.data_ptr() if hasattr(d_val, "data_ptr") else int(d_val)
    s = None if stream is None else C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().rsc_refactor_values_device(h.ptr, C.c_void_p(pv), s), h.ptr)


def rsc_solve(h: Handle, b, rtol: float = 1e-8, max_iter: int = 1000, raise_on_no_convergence: bool = True):
    """Returns (x, iters, final_relres)."""
    bb = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty_like(bb)
    it = C.c_int32()
    rr = C.c_double()
    st = lib().rsc_solve(h.ptr, _ptr(bb), _ptr(x), float(rtol), int(max_iter), C.byref(it), C.byref(rr))
    if st != RSC_OK and not (st == 3 and not raise_on_no_convergence):
        _check(st, h.ptr)
    return x, it.value, rr.value


def rsc_solve_device(h: Handle, d_b, d_x, rtol: float = 1e-8, max_iter: int = 1000, stream=None):
    """d_b, d_x: CUDA float64 tensors (or raw device pointers as ints)."""
    pb = d_b.data_ptr() if hasattr(d_b, "data_ptr") else int(d_b)
    px = d_x.data_ptr() if hasattr(d_x, "data_ptr") else int(d_x)
    s = None if stream is None else C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    it = C.c_int32()
    rr = C.c_double()
    _check(lib().rsc_solve_device(h.ptr, C.c_void_p(pb), C.c_void_p(px), float(rtol), int(max_iter), C.byref(it),
                                  C.byref(rr), s), h.ptr)
    return it.value, rr.value


def rsc_apply_preconditioner_device(h: Handle, d_r, d_z, stream=None) -> None:
    pr = d_r.data_ptr() if hasattr(d_r, "data_ptr") else int(d_r)
    pz = d_z.data_ptr() if hasattr(d_z, "data_ptr") else int(d_z)
    s = None if stream is None else C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().rsc_apply_preconditioner_device(h.ptr, C.c_void_p(pr), C.c_void_p(pz), s), h.ptr)


def rsc_apply_preconditioner_device_noalloc(h: Handle, d_r, d_z, stream=None) -> None:
    pr = d_r.data_ptr() if hasattr(d_r, "data_ptr") else int(d_r)
    pz = d_z.data_ptr() if hasattr(d_z, "data_ptr") else int(d_z)
    s = None if stream is None else C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().rsc_apply_preconditioner_device_noalloc(h.ptr, C.c_void_p(pr), C.c_void_p(pz), s), h.ptr)


def rsc_get_systems(h: Handle):
    """Returns sys_ptr (n_systems + 1 row offsets of the independent systems)."""
    m = C.c_int32()
    _check(lib().rsc_get_systems(h.ptr, C.byref(m), None), h.ptr)
    ptr = np.empty(m.value + 1, np.int64)
    _check(lib().rsc_get_systems(h.ptr, C.byref(m), _ptr(ptr)), h.ptr)
    return ptr


def rsc_solve_batch_device(h: Handle, d_B, d_X, rtol: float = 1e-8, max_iter: int = 1000, stream=None,
                           raise_on_no_convergence: bool = True):
    """d_B, d_X: CUDA float64 tensors of shape (nrhs, n) (each row one right-hand side).
    Returns (iters, relres) arrays of shape (nrhs, n_systems)."""
    nrhs = int(d_B.shape[0]) if d_B.dim() == 2 else 1
    nsys = rsc_get_systems(h).size - 1
    it = np.zeros(nrhs * nsys, np.int32)
    rr = np.zeros(nrhs * nsys, np.float64)
    s = None if stream is None else C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    st = lib().rsc_solve_batch_device(h.ptr, nrhs, C.c_void_p(d_B.data_ptr()), C.c_void_p(d_X.data_ptr()),
                                      float(rtol), int(max_iter), _ptr(it), _ptr(rr), s)
    if st != RSC_OK and not (st == 3 and not raise_on_no_convergence):
        _check(st, h.ptr)
    return it.reshape(nrhs, nsys), rr.reshape(nrhs, nsys)


def rsc_pattern_outer_device(h: Handle, d_u, d_v, alpha: float, d_out, stream=None) -> None:
    pu = d_u.data_ptr() if hasattr(d_u, "data_ptr") else int(d_u)
    pv = d_v.data_ptr() if hasattr(d_v, "data_ptr") else int(d_v)
    po = d_out.data_ptr() if hasattr(d_out, "data_ptr") else int(d_out)
    s = None if stream is None else C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().rsc_pattern_outer_device(h.ptr, C.c_void_p(pu), C.c_void_p(pv), float(alpha), C.c_void_p(po), s),
           h.ptr)


def rsc_get_supernode_info(h: Handle, j: int) -> dict:
    info = np.zeros(8, np.int32)
    _check(lib().rsc_get_supernode_info(h.ptr, int(j), _ptr(info)), h.ptr)
    keys = ["c", "r", "compressed", "rank", "hierarchical", "nblocks", "level", "kind"]
    return dict(zip(keys, info.tolist()))


def rsc_get_supernode_blocks(h: Handle, j: int):
    """Returns (LD [c x c], LO [r x c]) as FP64 arrays."""
    info = rsc_get_supernode_info(h, j)
    c, r = info["c"], info["r"]
    LD = np.zeros((c, c), order="F")
    LO = np.zeros((r, c), order="F")
    _check(lib().rsc_get_supernode_blocks(h.ptr, int(j), _ptr(LD), _ptr(LO) if r else None), h.ptr)
    return LD, LO


def rsc_get_stats(h: Handle) -> dict:
    s = rsc_stats_t()
    _check(lib().rsc_get_stats(h.ptr, C.byref(s)), h.ptr)
    return s.as_dict()


def rsc_profile(h: Handle, enable: bool = True, kernels: str | None = None) -> None:
    _check(lib().rsc_profile(h.ptr, int(bool(enable)), kernels.encode() if kernels else None), h.ptr)


def rsc_get_kernel_profile(h: Handle) -> dict:
    import json
    buf = C.create_string_buffer(1 << 16)
    _check(lib().rsc_get_kernel_profile(h.ptr, buf, len(buf)), h.ptr)
    return json.loads(buf.value.decode())


def rsc_set_wait_limit(h: Handle, polls: int) -> None:
    _check(lib().rsc_set_wait_limit(h.ptr, int(polls)), h.ptr)


def rsc_get_autotune(h: Handle) -> dict:
    """The kernel-variant choices of the BF16 / TF32 forms (see include/rsc.h)."""
    import json
    buf = C.create_string_buffer(1 << 16)
    _check(lib().rsc_get_autotune(h.ptr, buf, len(buf)), h.ptr)
    return json.loads(buf.value.decode())


def rsc_last_error(h: Handle | None = None) -> str:
    m = lib().rsc_last_error(h.ptr if h is not None else None)
    return m.decode() if m else ""


def rsc_destroy(h: Handle) -> None:
    if h.ptr:
        lib().rsc_destroy(h.ptr)
        h.ptr = None
