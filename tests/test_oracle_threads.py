"""The multithreaded CPU baseline (round-robin plain method on several host
threads) against the sequential oracle in the same order: the pairs of a
parallel step are disjoint, so every thread count gives the same bits."""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("cplx", [True, False])
@pytest.mark.parametrize("n", [37, 64])
def test_threads_bit_equal_to_sequential_round_robin(cplx, n):
    P = synth.make_problem(n, cplx, n // 2 + 3, (1e-3, 1e3), 2 * n, 2.0, seed=(77, n, cplx),
                           precision="f64", m=n + 5)
    ref = oracle.solve_plain(P.G, P.J, order=oracle.ORDER_ROUND_ROBIN)
    assert ref["status"] == 0
    for nt in (1, 2, 3, 5):
        got = oracle.solve_plain_threads(P.G, P.J, nthreads=nt)
        assert got["status"] == 0
        assert got["sweeps"] == ref["sweeps"] and got["rotations"] == ref["rotations"]
        assert got["maxoff"] == ref["maxoff"]
        assert np.array_equal(got["Gt"], ref["Gt"])


def test_threads_more_threads_than_pairs_and_sweep_cap():
    P = synth.make_problem(6, True, 3, (1e-2, 1e2), 12, 2.0, seed=5, precision="f64")
    ref = oracle.solve_plain(P.G, P.J, order=oracle.ORDER_ROUND_ROBIN, max_sweeps=2)
    got = oracle.solve_plain_threads(P.G, P.J, nthreads=8, max_sweeps=2)
    assert got["status"] == ref["status"] and got["sweeps"] == ref["sweeps"] == 2
    assert np.array_equal(got["Gt"], ref["Gt"])


def test_threads_reject_bad_arguments():
    G = np.eye(4)
    with pytest.raises(ValueError):
        oracle.solve_plain_threads(G, [1, 1, 2, -1], nthreads=2)
    with pytest.raises(ValueError):
        oracle.solve_plain_threads(G, [1, 1, -1, -1], nthreads=0)
