"""Helpers for GPU tests: device buffers through torch (plumbing only)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    from paper_1008_4166_gb300 import jjacobi

    jjacobi.load()
    return jjacobi


def to_dev(G: np.ndarray):
    """Column-major device copy of a numpy matrix (m x n)."""
    Gc = np.ascontiguousarray(np.asarray(G).T)
    return torch.from_numpy(Gc).to("cuda").t()


def from_dev(Gd) -> np.ndarray:
    return np.asfortranarray(Gd.t().contiguous().cpu().numpy().T)


def dtype_of(G):
    from paper_1008_4166_gb300 import jjacobi as jj

    return jj.JJ_C128 if np.iscomplexobj(G) else jj.JJ_F64


def col_rel_err(A: np.ndarray, B: np.ndarray) -> float:
    """max over columns of ||a_c - b_c|| / ||b_c||."""
    num = np.linalg.norm(np.asarray(A) - np.asarray(B), axis=0)
    den = np.linalg.norm(np.asarray(B), axis=0)
    return float(np.max(num / den))


def solve_gpu(G: np.ndarray, J, block_width=0, gemm=0, order=0, max_sweeps=0, allow=(0,),
              want_U=False, sort=0, **kw):
    jj = require_gpu()
    Gd = to_dev(G)
    m, n = G.shape
    with jj.Handle(m, n, dtype_of(G), block_width=block_width, gemm=gemm, order=order,
                   max_sweeps=max_sweeps, **kw) as h:
        ld = Gd.stride(1) if n > 1 else m  # a single column has no meaningful stride
        info = h.jjacobi_solve(Gd, ld, J, allow=allow)
        lam = torch.empty(n, dtype=torch.float64, device="cuda")
        U = None
        if want_U:
            U = torch.empty((n, m), dtype=Gd.dtype, device="cuda").t()
        if info.status in (0, 2):
            h.jjacobi_extract(lam, U, m if want_U else 0, sort)
        torch.cuda.synchronize()
    return dict(Gt=from_dev(Gd), lam=lam.cpu().numpy(), U=from_dev(U) if want_U else None,
                info=info.as_dict())
