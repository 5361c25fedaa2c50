"""The three-level forms at the published full size, in the launch
configuration bench.py times for the real workload of order 16384 (outer
pivots of 256 columns and inner blocks of 16, digit products at both levels:
--gemm ozaki, one capped sweep).

The workload's own recipe takes minutes to generate on the host (a Haar QR of
a 16384 x 16384 matrix), so this test takes a Gaussian G of the same shape and
the same J split: the kernels' index arithmetic, the tables and the launch
shapes depend on the sizes only, and the property checked holds for any input
and after any number of sweeps. One sweep of the method is a J-unitary
transformation W (W J W^* = J), so G~ J G~^* x = G J G^* x for every x; it is
checked on sampled vectors relative to the rounding scale of both sides. The
file runs last, so a failure under -x skips nothing else."""
import numpy as np
import pytest

from tests.gpu_util import from_dev, require_gpu, to_dev

pytestmark = pytest.mark.gpu

N = 16384


@pytest.mark.parametrize("strategy", ["oriented", "full"])
def test_three_level_one_sweep_at_full_size_is_j_unitary(strategy):
    jj = require_gpu()
    rng = np.random.default_rng(16384)
    G = np.asfortranarray(rng.standard_normal((N, N)))
    J = np.concatenate([np.ones(N // 2), -np.ones(N // 2)]).astype(np.int8)
    Gd = to_dev(G)
    strat = jj.JJ_BLOCK_ORIENTED if strategy == "oriented" else jj.JJ_FULL_BLOCK
    with jj.Handle(N, N, jj.JJ_F64, block_width=128, inner_block_width=16,
                   gemm=jj.JJ_GEMM_OZAKI_FP16, block_strategy=strat, max_sweeps=1) as h:
        info = h.jjacobi_solve(Gd, Gd.stride(1), J, allow=(jj.JJ_OK, jj.JJ_NOT_CONVERGED)).as_dict()
    assert info["status"] == jj.JJ_NOT_CONVERGED and info["sweeps"] == 1
    assert info["nbl"] == 128 and info["rotations"] > 0
    Gt = from_dev(Gd)
    del Gd
    assert np.all(np.isfinite(Gt))
    Jf = J.astype(np.float64)
    for _ in range(2):
        x = rng.standard_normal(N)
        a = G @ (Jf * (G.T @ x))
        b = Gt @ (Jf * (Gt.T @ x))
        scale = np.abs(G) @ (np.abs(G).T @ np.abs(x)) + np.abs(Gt) @ (np.abs(Gt).T @ np.abs(x))
        assert np.max(np.abs(a - b) / scale) <= 1e-10
