"""Failure paths on the GPU without a fault: a device-side wait that runs out
(the bound is set so short that every wait not satisfied at its first poll
expires) is reported as JJ_DEVICE_TIMEOUT and leaves the handle usable; and a
solve capped after some sweeps and resumed from its G~ gives the bits of the
uninterrupted solve (the state between sweeps is G~ alone, Alg. 3.2)."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import eig_rel_tol, max_rel_err
from tests.gpu_util import require_gpu, solve_gpu, to_dev

pytestmark = pytest.mark.gpu


def test_device_wait_timeout_is_reported_and_the_handle_recovers():
    """The all-digit form: the update's pipeline waits (its builders, product
    issue and drain wait on one another) cannot all succeed at their first
    poll, so a 1 ns bound makes one run out."""
    jj = require_gpu()
    gemm = jj.JJ_GEMM_OZAKI_FP16
    import torch

    P = synth.make_workload("plain_c128_n128", n=96)
    ref = oracle.solve_plain(P.G, P.J)
    with jj.Handle(P.m, P.n, jj.JJ_C128, block_width=16, gemm=gemm) as h:
        h.jjacobi_set_wait_limit(1)
        Gd = to_dev(P.G)
        info = h.jjacobi_solve(Gd, Gd.stride(1), P.J, allow=(jj.JJ_DEVICE_TIMEOUT,))
        assert info.status == jj.JJ_DEVICE_TIMEOUT
        torch.cuda.synchronize()  # the kernels returned: the context is usable
        h.jjacobi_set_wait_limit(0)  # back to the default bound
        Gd = to_dev(P.G)
        info = h.jjacobi_solve(Gd, Gd.stride(1), P.J)
        lam = torch.empty(P.n, dtype=torch.float64, device="cuda")
        h.jjacobi_extract(lam)
        torch.cuda.synchronize()
    assert info.status == 0
    assert max_rel_err(lam.cpu().numpy(), ref["lam"]) <= eig_rel_tol(P.G)


@pytest.mark.parametrize("form", [(0, 0), (16, 1), (16, 2), (16, 0)])
def test_capped_then_resumed_solve_gives_the_uninterrupted_bits(form):
    """A checkpoint is a copy of G~ after a capped solve (JJ_NOT_CONVERGED);
    solving that G~ again continues where the first solve stopped: the same
    sweeps in total and the same bits (every kernel is deterministic, and the
    skip state rebuilt by the first resumed sweep only re-evaluates pairs that
    would give no rotation)."""
    require_gpu()
    from paper_1008_4166_gb300 import jjacobi as jj

    bw, gemm = form
    P = synth.make_workload("graded_c128_n4096_b64", n=192)
    kw = dict(block_width=bw, gemm=gemm, block_strategy=jj.JJ_BLOCK_ORIENTED if bw else 0)
    full = solve_gpu(P.G, P.J, **kw)
    assert full["info"]["status"] == 0 and full["info"]["sweeps"] > 3
    part = solve_gpu(P.G, P.J, max_sweeps=3, allow=(0, 2), **kw)
    assert part["info"]["status"] == jj.JJ_NOT_CONVERGED and part["info"]["sweeps"] == 3
    rest = solve_gpu(part["Gt"], P.J, **kw)
    assert rest["info"]["status"] == 0
    assert part["info"]["sweeps"] + rest["info"]["sweeps"] == full["info"]["sweeps"]
    assert np.array_equal(rest["Gt"], full["Gt"])
