"""Python binding of libjjacobi (ctypes): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; this module never
computes. PyTorch tensors are accepted for device memory and streams. If the
shared library is missing it raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libjjacobi.so")

JJ_F64, JJ_C128 = 0, 1
JJ_ORDER_ROUND_ROBIN, JJ_ORDER_MODULUS = 0, 1
JJ_GEMM_FP64, JJ_GEMM_OZAKI_FP16, JJ_GEMM_OZAKI_GRAM, JJ_GEMM_AUTO = 0, 1, 2, 3
JJ_BLOCK_AUTO = -1
JJ_FULL_BLOCK, JJ_BLOCK_ORIENTED = 0, 1
JJ_PIVOT_CHOLESKY, JJ_PIVOT_SPECIAL = 0, 1
(JJ_OK, JJ_INVALID_ARG, JJ_NOT_CONVERGED, JJ_NOT_POSDEF, JJ_NONFINITE, JJ_DEVICE_TIMEOUT,
 JJ_CUDA_ERROR, JJ_NOT_SOLVED) = range(8)

# Every symbol the C headers declare (include/jjacobi.h, include/jjacobi_kernels.h).
EXPORTS = [
    "jjacobi_default_params", "jjacobi_create", "jjacobi_solve", "jjacobi_extract",
    "jjacobi_solve_host", "jjacobi_solve_batched", "jjacobi_destroy",
    "jjacobi_status_string", "jjacobi_version", "jjacobi_schedule", "jjacobi_kernel_times",
    "jjacobi_set_wait_limit", "jjacobi_factor",
    "jjk_column_norms", "jjk_plain_step", "jjk_gram", "jjk_inner", "jjk_update", "jjk_extract",
    "jjk_gram_noalloc",
]


class jj_params(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("block_width", ctypes.c_int32), ("inner_block_width", ctypes.c_int32),
                ("order", ctypes.c_int32), ("gemm", ctypes.c_int32),
                ("ozaki_slices", ctypes.c_int32), ("tol", ctypes.c_double),
                ("max_sweeps", ctypes.c_int32), ("inner_max_sweeps", ctypes.c_int32),
                ("cuda_stream", ctypes.c_void_p), ("profile", ctypes.c_int32),
                ("block_strategy", ctypes.c_int32), ("pivot_factor", ctypes.c_int32)]


class jj_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("sweeps", ctypes.c_int32),
                ("rotations", ctypes.c_int64), ("last_max_offdiag", ctypes.c_double),
                ("seconds", ctypes.c_double), ("block_width", ctypes.c_int32),
                ("nbl", ctypes.c_int32), ("steps_per_sweep", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int32), ("pairs_evaluated", ctypes.c_int64),
                ("pairs_rotated", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class JJError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


_lib = None


def load(path: Optional[str] = None) -> ctypes.CDLL:
    """Load libjjacobi.so (built by __graft_entry__.build() / _build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libjjacobi.so not found at {p}: build it first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(p)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "jjacobi_default_params": (None, [P(jj_params), i64, i64, i32]),
        "jjacobi_create": (ctypes.c_int, [P(ctypes.c_void_p), P(jj_params)]),
        "jjacobi_solve": (ctypes.c_int, [vp, vp, i64, vp, P(jj_info)]),
        "jjacobi_extract": (ctypes.c_int, [vp, vp, vp, i64, i32]),
        "jjacobi_solve_host": (ctypes.c_int, [vp, vp, i64, vp, vp, vp, i64, P(jj_info)]),
        "jjacobi_solve_batched": (ctypes.c_int, [vp, i32, vp, vp, vp, vp, vp, vp, vp]),
        "jjacobi_destroy": (None, [vp]),
        "jjacobi_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "jjacobi_version": (i32, []),
        "jjacobi_schedule": (i32, [i32, i32, i32, vp]),
        "jjacobi_kernel_times": (ctypes.c_int, [vp, vp, vp]),
        "jjacobi_set_wait_limit": (ctypes.c_int, [vp, i64]),
        "jjacobi_factor": (ctypes.c_int, [i32, vp, i64, i64, dbl, vp, i64, vp, vp, vp, vp, vp]),
        "jjk_column_norms": (ctypes.c_int, [i32, vp, i64, i64, i64, vp, vp]),
        "jjk_plain_step": (ctypes.c_int, [i32, vp, i64, i64, i64, vp, i32, vp, vp, dbl, vp, vp]),
        "jjk_gram": (ctypes.c_int, [i32, i32, vp, i64, i64, vp, i32, vp, i32, vp]),
        "jjk_inner": (ctypes.c_int, [i32, vp, vp, i32, vp, i32, vp, dbl, i32, i32, vp, vp]),
        "jjk_update": (ctypes.c_int, [i32, i32, vp, vp, i64, i64, vp, i32, vp, i32, vp]),
        "jjk_extract": (ctypes.c_int, [i32, vp, i64, i64, i64, vp, vp, vp, i64, vp]),
        "jjk_gram_noalloc": (ctypes.c_int, [i32, vp, i64, i64, vp, i32, vp, i32, i64, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().jjacobi_status_string(int(status)).decode()


def _check(rc: int, where: str, ok=(JJ_OK,)):
    if rc not in ok:
        raise JJError(rc, where)
    return rc


def _ptr(x) -> Optional[int]:
    """Raw address of a torch tensor, a numpy array or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(type(x))


def _avail_bytes(x) -> int:
    """Bytes addressable from the first element of a tensor or array onward."""
    if hasattr(x, "untyped_storage"):
        return x.untyped_storage().nbytes() - x.storage_offset() * x.element_size()
    if not x.flags["C_CONTIGUOUS"] and not x.flags["F_CONTIGUOUS"]:
        raise ValueError("host arrays passed to the library must be contiguous")
    return x.nbytes


def _check_buffer(x, what: str, count: int, elem_bytes: int, device: bool,
                  dtypes: Sequence[str] = ()) -> None:
    """Argument checks the C entry points cannot make themselves: a tensor or
    array must lie on the side the call reads it from, have the element type
    and cover `count` elements. Raw integer addresses are passed unchecked."""
    if x is None or isinstance(x, int):
        return
    is_cuda = bool(getattr(x, "is_cuda", False))
    if device and not is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    name = str(x.dtype).replace("torch.", "")
    if dtypes and name not in dtypes:
        raise ValueError(f"{what} must have dtype {' or '.join(dtypes)}, not {name}")
    if count > 0 and _avail_bytes(x) < count * elem_bytes:
        raise ValueError(f"{what} holds fewer than the {count} elements the call reads")


def _matrix_span(m: int, n: int, ld: int) -> int:
    """Elements spanned by an m x n column-major matrix with leading dimension ld."""
    return 0 if n < 1 else (n - 1) * ld + m


def _signs(J, n: int, what: str = "J") -> np.ndarray:
    Jc = np.ascontiguousarray(np.asarray(J, dtype=np.int8))
    if Jc.ndim != 1 or Jc.shape[0] != n:
        raise ValueError(f"{what} must hold exactly {n} signs, got shape {Jc.shape}")
    return Jc


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:  # pragma: no cover - torch is plumbing only
            return None
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def jjacobi_schedule(nbl: int, order: int, sweep: int = 1) -> np.ndarray:
    """Block pairs of one sweep, [steps, nbl/2, 2] (Algs. 4.1-4.3, host)."""
    lib = load()
    buf = np.zeros(2 * nbl * (nbl // 2) + 2, dtype=np.int32)
    steps = lib.jjacobi_schedule(int(nbl), int(order), int(sweep), buf.ctypes.data)
    if steps < 0:
        raise JJError(JJ_INVALID_ARG, "jjacobi_schedule")
    return buf[: steps * nbl].reshape(steps, nbl // 2, 2).copy()


def jjacobi_default_params(m: int, n: int, dtype: int) -> jj_params:
    p = jj_params()
    load().jjacobi_default_params(ctypes.byref(p), int(m), int(n), int(dtype))
    return p


class Handle:
    """Owning wrapper of a jj_handle (jjacobi_create / jjacobi_destroy)."""

    def __init__(self, m: int, n: int, dtype: int, block_width: int = 0,
                 inner_block_width: int = 0, order: int = JJ_ORDER_ROUND_ROBIN,
                 gemm: int = JJ_GEMM_FP64, tol: float = 0.0, max_sweeps: int = 0,
                 inner_max_sweeps: int = 0, ozaki_slices: int = 0, stream=None,
                 profile: bool = False, block_strategy: int = JJ_FULL_BLOCK,
                 pivot_factor: int = JJ_PIVOT_CHOLESKY):
        lib = load()
        p = jjacobi_default_params(m, n, dtype)
        p.block_width = block_width
        p.inner_block_width = inner_block_width
        p.order = order
        p.gemm = gemm
        p.ozaki_slices = ozaki_slices
        if tol > 0:
            p.tol = tol
        if max_sweeps > 0:
            p.max_sweeps = max_sweeps
        if inner_max_sweeps > 0:
            p.inner_max_sweeps = inner_max_sweeps
        sp = _stream_ptr(stream)
        p.cuda_stream = sp
        p.profile = 1 if profile else 0
        p.block_strategy = block_strategy
        p.pivot_factor = pivot_factor
        self.params = p
        self.h = ctypes.c_void_p()
        _check(lib.jjacobi_create(ctypes.byref(self.h), ctypes.byref(p)), "jjacobi_create")
        self.m, self.n, self.dtype = m, n, dtype

    def close(self):
        if self.h:
            load().jjacobi_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _elem(self):
        """(bytes, dtype names) of one matrix element of this handle."""
        return (16, ("complex128",)) if self.dtype == JJ_C128 else (8, ("float64",))

    def jjacobi_solve(self, G, ldg: int, J: Sequence[int], allow=(JJ_OK,)) -> jj_info:
        esz, names = self._elem()
        _check_buffer(G, "G", _matrix_span(self.m, self.n, int(ldg)), esz, True, names)
        Jc = _signs(J, self.n)
        info = jj_info()
        rc = load().jjacobi_solve(self.h, _ptr(G), int(ldg), Jc.ctypes.data, ctypes.byref(info))
        _check(rc, "jjacobi_solve", allow)
        return info

    def jjacobi_set_wait_limit(self, ns: int) -> None:
        """Bound (ns) of the device-side waits of this handle's kernels; <= 0: 2 s."""
        _check(load().jjacobi_set_wait_limit(self.h, int(ns)), "jjacobi_set_wait_limit")

    def jjacobi_kernel_times(self):
        """(ms, launches) per kernel family: gram, inner, update, plain step, norms."""
        t = np.zeros(8, dtype=np.float64)
        n = np.zeros(8, dtype=np.int64)
        _check(load().jjacobi_kernel_times(self.h, t.ctypes.data, n.ctypes.data),
               "jjacobi_kernel_times")
        names = ["gram", "inner", "update", "plain_step", "norms"]
        return {k: (float(t[i]), int(n[i])) for i, k in enumerate(names)}

    def jjacobi_extract(self, lam, U=None, ldu: int = 0, sort: int = 0) -> None:
        esz, names = self._elem()
        _check_buffer(lam, "lambda", self.n, 8, False, ("float64",))
        _check_buffer(U, "U", _matrix_span(self.m, self.n, int(ldu)), esz, True, names)
        _check(load().jjacobi_extract(self.h, _ptr(lam), _ptr(U), int(ldu), int(sort)),
               "jjacobi_extract")

    def jjacobi_solve_host(self, G: np.ndarray, J: Sequence[int], want_U: bool = False,
                           allow=(JJ_OK,)):
        """Host buffers in and out (column-major numpy array G)."""
        Gf = np.asfortranarray(G)
        if Gf.shape != (self.m, self.n):
            raise ValueError(f"G must be {self.m} x {self.n}, got {Gf.shape}")
        Gf = Gf.astype(np.complex128 if self.dtype == JJ_C128 else np.float64, copy=False)
        Jc = _signs(J, self.n)
        lam = np.zeros(self.n, dtype=np.float64)
        U = np.zeros_like(Gf, order="F") if want_U else None
        info = jj_info()
        rc = load().jjacobi_solve_host(self.h, Gf.ctypes.data, Gf.shape[0], Jc.ctypes.data,
                                       lam.ctypes.data, _ptr(U), Gf.shape[0] if want_U else 0,
                                       ctypes.byref(info))
        _check(rc, "jjacobi_solve_host", allow)
        return lam, U, info

    def jjacobi_solve_batched(self, Gs, Js, lam=None, allow=(JJ_OK,)):
        """Solve len(Gs) independent problems (device tensors, column-major
        m_k x n_k, leading dimension = stride(1)) in place. lam (device tensor or
        numpy array, sum n_k doubles) receives the eigenvalues, problem k at
        offset sum_{l<k} n_l. Returns the status and the per-problem infos."""
        count = len(Gs)
        ptrs = (ctypes.c_void_p * count)(*[_ptr(G) for G in Gs])
        m = np.array([G.shape[0] for G in Gs], dtype=np.int64)
        n = np.array([G.shape[1] for G in Gs], dtype=np.int64)
        ld = np.array([G.stride(1) if hasattr(G, "stride") else G.shape[0] for G in Gs],
                      dtype=np.int64)
        if len(Js) != count:
            raise ValueError(f"{count} matrices but {len(Js)} sign vectors")
        esz, names = self._elem()
        for k, G in enumerate(Gs):
            if getattr(G, "ndim", 2) != 2:
                raise ValueError(f"G[{k}] must be a matrix")
            if hasattr(G, "stride") and G.shape[1] > 1 and G.stride(0) != 1:
                raise ValueError(f"G[{k}] must be column-major (stride(0) == 1)")
            _check_buffer(G, f"G[{k}]", _matrix_span(int(m[k]), int(n[k]), int(ld[k])), esz,
                          True, names)
        Jcs = [_signs(J, int(n[k]), f"J[{k}]") for k, J in enumerate(Js)]
        _check_buffer(lam, "lambda", int(n.sum()), 8, False, ("float64",))
        jptrs = (ctypes.c_void_p * count)(*[J.ctypes.data for J in Jcs])
        infos = (jj_info * count)()
        rc = load().jjacobi_solve_batched(self.h, count, ptrs, m.ctypes.data, n.ctypes.data,
                                          ld.ctypes.data, jptrs, _ptr(lam), infos)
        _check(rc, "jjacobi_solve_batched", allow)
        return rc, list(infos)


# ---------------------------------------------------------------------------
# Building blocks (include/jjacobi_kernels.h)
# ---------------------------------------------------------------------------

def jjacobi_factor(H, rank_tol: float = 0.0, stream=None):
    """H = G J G^* (Sec. 2.2): returns (G, J, perm, pivot_size, rank) with G a
    device tensor n x r (column-major), J, perm, pivot_size numpy arrays."""
    import torch

    n = H.shape[0]
    if H.shape != (n, n) or not H.is_cuda:
        raise ValueError("H must be a square CUDA tensor")
    dt = JJ_C128 if H.is_complex() else JJ_F64
    Hc = H.t().contiguous().t()  # column-major
    G = torch.zeros((n, n), dtype=H.dtype, device=H.device).t()  # column-major n x n
    J = np.zeros(n, dtype=np.int8)
    perm = np.zeros(n, dtype=np.int32)
    psize = np.zeros(n, dtype=np.int8)
    r = ctypes.c_int64(0)
    _check(load().jjacobi_factor(dt, _ptr(Hc), n, n, float(rank_tol), _ptr(G), n, J.ctypes.data,
                                 perm.ctypes.data, psize.ctypes.data, ctypes.byref(r),
                                 _stream_ptr(stream)), "jjacobi_factor")
    rr = int(r.value)
    return G[:, :rr], J[:rr], perm, psize[:rr], rr


def jjk_column_norms(dtype, G, ld, m, n, d, stream=None):
    _check(load().jjk_column_norms(dtype, _ptr(G), ld, m, n, _ptr(d), _stream_ptr(stream)),
           "jjk_column_norms")


def jjk_plain_step(dtype, G, ld, m, n, pairs, npairs, J, d, tol, counters, stream=None):
    _check(load().jjk_plain_step(dtype, _ptr(G), ld, m, n, _ptr(pairs), npairs, _ptr(J), _ptr(d),
                                 float(tol), _ptr(counters), _stream_ptr(stream)),
           "jjk_plain_step")


def jjk_gram(dtype, gemm, G, ld, m, pairs, npairs, A, kmax, stream=None):
    _check(load().jjk_gram(dtype, gemm, _ptr(G), ld, m, _ptr(pairs), npairs, _ptr(A), kmax,
                           _stream_ptr(stream)), "jjk_gram")


def jjk_inner(dtype, A, W, kmax, pairs, npairs, J, tol, inner_max_sweeps, inner_block_width,
              counters, stream=None):
    _check(load().jjk_inner(dtype, _ptr(A), _ptr(W), kmax, _ptr(pairs), npairs, _ptr(J),
                            float(tol), inner_max_sweeps, inner_block_width, _ptr(counters),
                            _stream_ptr(stream)), "jjk_inner")


def jjk_update(dtype, gemm, Gs, Gd, ld, m, pairs, npairs, W, kmax, stream=None):
    _check(load().jjk_update(dtype, gemm, _ptr(Gs), _ptr(Gd), ld, m, _ptr(pairs), npairs,
                             _ptr(W), kmax, _stream_ptr(stream)), "jjk_update")


def jjk_extract(dtype, G, ld, m, n, J, lam, U=None, ldu=0, stream=None):
    _check(load().jjk_extract(dtype, _ptr(G), ld, m, n, _ptr(J), _ptr(lam), _ptr(U), ldu,
                              _stream_ptr(stream)), "jjk_extract")


def jjk_gram_noalloc(dtype, G, ld, m, pairs, npairs, A, kmax, ncols, stream=None):
    """Digit-product Gram without allocation (scratch in a fixed device array)."""
    _check(load().jjk_gram_noalloc(dtype, _ptr(G), ld, m, _ptr(pairs), npairs, _ptr(A), kmax,
                                   ncols, _stream_ptr(stream)), "jjk_gram_noalloc")
