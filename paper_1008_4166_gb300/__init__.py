"""GB300-native one-sided hyperbolic (J-)Jacobi eigensolver.

The method, its forms and its C ABI are described in include/jjacobi.h. This
package holds the CUDA sources (csrc/), the in-tree build (_build.py) and the
ctypes binding (jjacobi.py); `solve` below is the convenience entry for torch
tensors.
"""
from __future__ import annotations

from . import jjacobi
from .jjacobi import (JJ_C128, JJ_F64, JJ_GEMM_AUTO, JJ_GEMM_FP64, JJ_GEMM_OZAKI_FP16,
                      JJ_GEMM_OZAKI_GRAM,
                      JJ_ORDER_MODULUS, JJ_ORDER_ROUND_ROBIN, Handle, JJError)

__all__ = ["jjacobi", "Handle", "JJError", "solve", "JJ_F64", "JJ_C128", "JJ_GEMM_FP64",
           "JJ_GEMM_OZAKI_FP16", "JJ_GEMM_OZAKI_GRAM", "JJ_GEMM_AUTO", "JJ_ORDER_ROUND_ROBIN", "JJ_ORDER_MODULUS"]


def solve(G, J, block_width: int = 0, want_vectors: bool = True, **kw):
    """Eigenpairs of H = G J G^* for a column-major torch CUDA tensor G (m x n).

    G must be a column-major CUDA tensor (e.g. `X.t().contiguous().t()` or a
    transposed contiguous tensor) of dtype float64 or complex128; it is
    overwritten by G~ = G W. Returns (lambda, U, info) with lambda a float64
    CUDA tensor and U a column-major CUDA tensor (or None).
    """
    import torch

    if not G.is_cuda:
        raise ValueError("G must be a CUDA tensor")
    m, n = G.shape
    if G.stride(0) != 1:
        raise ValueError("G must be column-major (stride(0) == 1)")
    ld = G.stride(1) if n > 1 else m
    dtype = JJ_C128 if G.dtype == torch.complex128 else JJ_F64
    if G.dtype not in (torch.float64, torch.complex128):
        raise ValueError("G must be float64 or complex128")
    with Handle(m, n, dtype, block_width=block_width, **kw) as h:
        info = h.jjacobi_solve(G, ld, J, allow=(jjacobi.JJ_OK, jjacobi.JJ_NOT_CONVERGED))
        lam = torch.empty(n, dtype=torch.float64, device=G.device)
        U = None
        if want_vectors:
            U = torch.empty((n, m), dtype=G.dtype, device=G.device).t()
        h.jjacobi_extract(lam, U, m if want_vectors else 0)
        torch.cuda.current_stream().synchronize()
    return lam, U, info.as_dict()
