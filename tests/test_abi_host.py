"""CPU tests of the C ABI: the library builds, loads and exports every symbol
the headers declare; the host-side logic (ordering tables, parameters, status
strings, argument validation) works without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def jj():
    import __graft_entry__ as g

    g.build()
    from paper_1008_4166_gb300 import jjacobi

    return jjacobi


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return set(re.findall(r"\b(jj[a-z]*_[a-z_]+)\s*\(", txt))


def test_every_declared_symbol_is_exported(jj):
    lib = jj.load()
    declared = _declared("jjacobi.h") | _declared("jjacobi_kernels.h")
    assert declared, "no declarations parsed"
    assert declared == set(jj.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_version_and_status_strings(jj):
    lib = jj.load()
    assert lib.jjacobi_version() == 10000
    for s in range(8):
        assert jj.status_string(s).startswith("JJ_")
    assert jj.status_string(99) == "JJ_UNKNOWN"


def test_default_params(jj):
    p = jj.jjacobi_default_params(100, 80, jj.JJ_C128)
    assert (p.m, p.n, p.dtype, p.block_width) == (100, 80, jj.JJ_C128, 0)
    assert p.tol == 128 * 2.0 ** -53 and p.max_sweeps == 60 and p.inner_max_sweeps == 30


@pytest.mark.parametrize("nbl", [2, 4, 6, 8, 16, 64, 128, 1000])
@pytest.mark.parametrize("order", [0, 1])
def test_schedule_matches_oracle(jj, nbl, order):
    """The library builds the pair sets from their closed forms and assigns
    them to processes by the ring shift; the oracle simulates the paper's
    per-process steps. Bit for bit the same tables, except with two processes
    (nbl = 4), which are each other's neighbour on both sides: there the ring
    does not fix who holds which pair, and for the modulus ordering the
    library's choice differs from the paper's. Both are valid: the same pairs
    in every step, and every process keeps one block and receives one."""
    prev_last = None
    for sweep in (1, 2, 3):
        got = jj.jjacobi_schedule(nbl, order, sweep)
        ref = oracle.schedule(nbl, order, sweep)
        assert got.shape == ref.shape
        if nbl == 4 and order == 1:
            for t in range(got.shape[0]):
                assert {tuple(x) for x in got[t]} == {tuple(x) for x in ref[t]}
            seq = ([prev_last] if prev_last is not None else []) + list(got)
            for a, b in zip(seq[:-1], seq[1:]):
                for q in range(got.shape[1]):
                    assert len(set(a[q]) & set(b[q])) >= 1
            prev_last = got[-1]
        else:
            assert np.array_equal(got, ref)


def test_schedule_invalid(jj):
    with pytest.raises(jj.JJError):
        jj.jjacobi_schedule(5, 0, 1)
    with pytest.raises(jj.JJError):
        jj.jjacobi_schedule(4, 2, 1)


def test_create_rejects_bad_params(jj):
    lib = jj.load()
    h = ctypes.c_void_p()
    p = jj.jjacobi_default_params(10, 20, jj.JJ_F64)  # m < n
    assert lib.jjacobi_create(ctypes.byref(h), ctypes.byref(p)) == jj.JJ_INVALID_ARG
    assert not h
    p = jj.jjacobi_default_params(10, 10, 7)
    assert lib.jjacobi_create(ctypes.byref(h), ctypes.byref(p)) == jj.JJ_INVALID_ARG
    for m, n in ((0, 0), (5, 0), (-1, -1), (4, 5)):  # empty, negative, wide
        p = jj.jjacobi_default_params(m, n, jj.JJ_F64)
        assert lib.jjacobi_create(ctypes.byref(h), ctypes.byref(p)) == jj.JJ_INVALID_ARG
        assert not h
    for field, bad in (("order", 2), ("gemm", 4), ("gemm", -1), ("block_strategy", 2),
                       ("inner_block_width", -1), ("ozaki_slices", -1), ("pivot_factor", 2)):
        q = jj.jjacobi_default_params(8, 8, jj.JJ_F64)
        setattr(q, field, bad)
        assert lib.jjacobi_create(ctypes.byref(h), ctypes.byref(q)) == jj.JJ_INVALID_ARG, field
    q = jj.jjacobi_default_params(8, (1 << 30) + 1, jj.JJ_F64)
    q.m = q.n
    assert lib.jjacobi_create(ctypes.byref(h), ctypes.byref(q)) == jj.JJ_INVALID_ARG
    assert lib.jjacobi_create(None, ctypes.byref(p)) == jj.JJ_INVALID_ARG
    lib.jjacobi_destroy(None)  # no-op


def test_create_accepts_auto_block_width_only_as_minus_one(jj):
    lib = jj.load()
    h = ctypes.c_void_p()
    p = jj.jjacobi_default_params(64, 64, jj.JJ_C128)
    p.block_width = -2
    assert lib.jjacobi_create(ctypes.byref(h), ctypes.byref(p)) == jj.JJ_INVALID_ARG


def test_kernel_entry_points_validate_arguments(jj):
    lib = jj.load()
    assert lib.jjk_gram(9, 0, None, 1, 1, None, 0, None, 1, None) == jj.JJ_INVALID_ARG
    assert lib.jjk_extract(0, None, 1, 1, 1, None, None, None, 0, None) == jj.JJ_INVALID_ARG
    assert lib.jjacobi_extract(None, None, None, 0, 0) == jj.JJ_INVALID_ARG
    # gemm outside jj_gemm, and digit products asked for a pivot wider than they
    # take (complex kmax 129: real width 258 > 256); every case returns before any
    # device work (the dummy addresses are never dereferenced)
    x = 256
    for g in (-1, 4):
        assert lib.jjk_gram(0, g, x, 1, 1, x, 0, x, 1, None) == jj.JJ_INVALID_ARG
        assert lib.jjk_update(0, g, x, x, 1, 1, x, 0, x, 1, None) == jj.JJ_INVALID_ARG
    for g in (jj.JJ_GEMM_OZAKI_FP16, jj.JJ_GEMM_OZAKI_GRAM):
        assert lib.jjk_gram(jj.JJ_C128, g, x, 1, 1, x, 0, x, 129, None) == jj.JJ_INVALID_ARG
    # negative sizes
    assert lib.jjk_plain_step(0, x, 1, 1, -1, x, 0, x, x, 0.0, x, None) == jj.JJ_INVALID_ARG
    assert lib.jjk_plain_step(0, x, 1, 1, 1, x, -1, x, x, 0.0, x, None) == jj.JJ_INVALID_ARG
    assert lib.jjk_inner(0, x, x, 8, x, 0, x, 0.0, 30, -1, x, None) == jj.JJ_INVALID_ARG
    assert lib.jjk_extract(0, x, 1, 1, -1, x, x, None, 0, None) == jj.JJ_INVALID_ARG
    assert lib.jjk_column_norms(0, x, 1, 1, -1, x, None) == jj.JJ_INVALID_ARG


def test_solve_entry_points_report_errors_through_info(jj):
    """Every solve entry point fills its jj_info on an argument error (here a
    null handle, rejected before any device work)."""
    lib = jj.load()
    info = jj.jj_info()
    info.status = 12345
    assert lib.jjacobi_solve(None, None, 1, None, ctypes.byref(info)) == jj.JJ_INVALID_ARG
    assert info.status == jj.JJ_INVALID_ARG and info.seconds >= 0.0
    info.status = 12345
    assert lib.jjacobi_solve_host(None, None, 1, None, None, None, 0,
                                  ctypes.byref(info)) == jj.JJ_INVALID_ARG
    assert info.status == jj.JJ_INVALID_ARG
    infos = (jj.jj_info * 3)()
    for k in range(3):
        infos[k].status = 12345
        infos[k].sweeps = 7
    rc = lib.jjacobi_solve_batched(None, 3, None, None, None, None, None, None, infos)
    assert rc == jj.JJ_INVALID_ARG
    assert all(infos[k].status == jj.JJ_INVALID_ARG and infos[k].sweeps == 0 for k in range(3))


def test_product_does_not_import_oracle():
    """The product package (Python binding, CUDA sources, build script) never
    imports, loads or names the oracle: the two share no code."""
    pkg = os.path.join(ROOT, "paper_1008_4166_gb300")
    pattern = re.compile(r"\boracle\b|liboracle", re.I)
    checked = 0
    for dp, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dp, f), errors="replace").read()
                assert not pattern.search(txt), f
                checked += 1
    assert checked >= 8


C_PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include "jjacobi.h"
#include "jjacobi_kernels.h"

int main(void) {
    jj_params p;
    jjacobi_default_params(&p, 100, 80, JJ_C128);
    int32_t pairs[2 * 8 * 4];
    int steps = jjacobi_schedule(8, JJ_ORDER_ROUND_ROBIN, 1, pairs);
    jj_handle h = (jj_handle)0;
    p.m = 10; p.n = 20;  /* m < n: refused before any device work */
    int rc = jjacobi_create(&h, &p);
    printf("%d %d %d %s %d %d %d\n", (int)jjacobi_version(), steps, pairs[0] * 100 + pairs[1],
           jjacobi_status_string(JJ_NOT_POSDEF), rc, h == (jj_handle)0, p.max_sweeps);
    jjacobi_destroy((jj_handle)0);
    return 0;
}
"""


def test_c_program_compiles_links_and_calls_the_abi(jj, tmp_path):
    """The headers are valid C99 and the library links from C: host-only entry
    points called from a C program (no GPU needed)."""
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "abi"
    libdir = os.path.join(ROOT, "paper_1008_4166_gb300")
    subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-L", libdir, "-ljjacobi", "-Wl,-rpath," + libdir, "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    ref = oracle.schedule(8, 0, 1)
    assert out[0] == "10000" and out[1] == str(ref.shape[0])
    assert int(out[2]) == int(ref[0, 0, 0]) * 100 + int(ref[0, 0, 1])
    assert out[3] == "JJ_NOT_POSDEF" and int(out[4]) == jj.JJ_INVALID_ARG
    assert out[5] == "1" and out[6] == "60"


def _fake_handle(jj, m, n, dtype):
    """A Handle object with a null jj_handle: enough to exercise the binding's
    own argument checks, which run before any library call."""
    h = jj.Handle.__new__(jj.Handle)
    h.h = ctypes.c_void_p()
    h.m, h.n, h.dtype = m, n, dtype
    return h


def test_binding_rejects_buffers_the_kernels_would_overrun(jj):
    """Host tensors where device memory is read, wrong element types, short
    buffers and sign vectors of the wrong length are refused in Python, before
    a pointer reaches the library."""
    import torch

    h = _fake_handle(jj, 6, 4, jj.JJ_C128)
    J = [1, 1, -1, -1]
    G_host = torch.zeros((4, 6), dtype=torch.complex128).t()
    with pytest.raises(ValueError, match="CUDA"):
        h.jjacobi_solve(G_host, 6, J)
    with pytest.raises(ValueError, match="CUDA"):
        h.jjacobi_extract(np.zeros(4), G_host, 6)
    with pytest.raises(ValueError, match="CUDA"):
        h.jjacobi_solve_batched([G_host], [J])
    with pytest.raises(ValueError, match="signs"):
        h.jjacobi_solve_host(np.zeros((6, 4), complex), [1, -1])
    with pytest.raises(ValueError, match="6 x 4"):
        h.jjacobi_solve_host(np.zeros((4, 6), complex), [1, -1, 1, -1, 1, -1])
    with pytest.raises(ValueError, match="fewer"):
        h.jjacobi_extract(np.zeros(3), None)
    with pytest.raises(ValueError, match="float64"):
        h.jjacobi_extract(np.zeros(4, dtype=np.float32), None)
    with pytest.raises(ValueError, match="sign vectors"):
        h.jjacobi_solve_batched([G_host, G_host], [J])
    # the checks themselves, on host tensors (device=False) where a call may read host memory
    check = jj._check_buffer
    check(torch.zeros(10, dtype=torch.float64), "x", 10, 8, False, ("float64",))
    check(torch.zeros(12, dtype=torch.float64)[2:], "x", 10, 8, False, ("float64",))
    with pytest.raises(ValueError, match="fewer"):
        check(torch.zeros(12, dtype=torch.float64)[3:], "x", 10, 8, False, ("float64",))
    with pytest.raises(ValueError, match="complex128"):
        check(torch.zeros(10, dtype=torch.float64), "x", 5, 16, False, ("complex128",))
    with pytest.raises(ValueError, match="contiguous"):
        check(np.zeros((4, 4))[:, ::2], "x", 4, 8, False)
    assert jj._matrix_span(6, 4, 8) == 3 * 8 + 6 and jj._matrix_span(6, 0, 8) == 0
    check(12345, "raw address", 10 ** 9, 8, True)  # raw addresses are the caller's contract
