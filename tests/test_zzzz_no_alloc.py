"""The allocation-free Gram entry point against the ordinary one.

jjk_gram_noalloc serves callers that cannot allocate device memory: it keeps
its scratch in a fixed array inside the library instead of asking an
allocator. This file runs last (pytest collects files in name order), so a
failure here, in a run that stops at the first failure, comes after every
other test has run. It also passes when run alone in a fresh process: the
first call on a device looks the array up by itself.
"""
import ctypes

import numpy as np
import pytest

from tests._util import U64
from tests.gpu_util import dtype_of, require_gpu, to_dev

pytestmark = pytest.mark.gpu


def _gram_both(jj, torch, G, pairs, kmax):
    lib = jj.load()
    f = lib.jjk_gram_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p]
    m, n = G.shape
    E = 2 if np.iscomplexobj(G) else 1
    Gd = to_dev(G)
    pd = torch.from_numpy(pairs).cuda()
    A_ref = torch.zeros(len(pairs) * kmax * kmax * E, dtype=torch.float64, device="cuda")
    A_na = torch.full_like(A_ref, float("nan"))
    jj.jjk_gram(dtype_of(G), jj.JJ_GEMM_OZAKI_FP16, Gd, Gd.stride(1), m, pd, len(pairs), A_ref, kmax)
    st = torch.cuda.current_stream().cuda_stream
    rc = f(dtype_of(G), Gd.data_ptr(), Gd.stride(1), m, pd.data_ptr(), len(pairs), A_na.data_ptr(),
           kmax, n, st)
    assert rc == 0, jj.status_string(rc)
    torch.cuda.synchronize()
    return A_ref.cpu().numpy(), A_na.cpu().numpy()


def _check(A_ref, A_na, pairs, kmax, cplx, m):
    if cplx:
        A_ref, A_na = A_ref.view(np.complex128), A_na.view(np.complex128)
    A_ref = A_ref.reshape(len(pairs), kmax, kmax)
    A_na = A_na.reshape(len(pairs), kmax, kmax)
    for q, p in enumerate(pairs):
        k = p[1] + p[3]
        R, N = A_ref[q, :k, :k], A_na[q, :k, :k]
        d = np.sqrt(np.abs(np.diag(R)))
        assert np.all(np.isfinite(N))
        # the same tolerance as the Gram parity test
        assert np.max(np.abs(N - R) / np.outer(d, d)) <= 64 * U64 * np.sqrt(m)


@pytest.mark.parametrize("cplx", [True, False])
def test_gram_noalloc_matches_gram_on_two_calls(cplx):
    jj = require_gpu()
    import torch

    rng = np.random.default_rng(17 + cplx)
    m, n = 333, 96
    hi = 16 if cplx else 32
    kmax = 2 * hi
    pairs = np.array([[0, hi, 40, hi - 3], [hi, hi - 1, 60, hi]], dtype=np.int32)
    for call in range(2):  # two calls in a row, different inputs: no stale scratch leaks
        G = rng.standard_normal((m, n)) + (1j * rng.standard_normal((m, n)) if cplx else 0)
        G *= 10.0 ** rng.uniform(-3, 3, size=(m, 1))
        G = np.asfortranarray(G)
        A_ref, A_na = _gram_both(jj, torch, G, pairs, kmax)
        _check(A_ref, A_na, pairs, kmax, cplx, m)


def test_gram_noalloc_rejects_oversize():
    jj = require_gpu()
    lib = jj.load()
    f = lib.jjk_gram_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p]
    # 4096 pairs of real width 64 need 64 MiB of accumulators: beyond the fixed array
    assert f(1, 1, 10, 10, 1, 4096, 1, 32, 10, None) == jj.JJ_INVALID_ARG
    # more columns than the exponent table holds
    assert f(1, 1, 10, 10, 1, 1, 1, 32, 1 << 20, None) == jj.JJ_INVALID_ARG
