"""Pins for the oracle's schedules (Algs. 4.1-4.3), the uniform partition (3.3)
and the blocked full-block reference (Alg. 5.2, 2F)."""
import os
from itertools import combinations

import numpy as np
import pytest

import oracle
import synth
from tests._util import eig_rel_tol, max_rel_err, orth_residual, reconstruction_residual

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("n,nbl", [(10, 3), (4096, 64), (33, 4), (7, 7), (100, 8), (2048, 64)])
def test_uniform_partition(n, nbl):
    sizes = oracle.uniform_partition(n, nbl)
    assert sum(sizes) == n and len(sizes) == nbl
    assert max(sizes) - min(sizes) <= 1
    assert sizes == sorted(sizes, reverse=True)
    assert max(sizes) == -(-n // nbl)


def _golden_layout():
    pairs, dups = [], []
    with open(os.path.join(GOLDEN, "initial_layout_p3.txt")) as f:
        for line in f:
            line = line.split("#")[0].split()
            if not line:
                continue
            if line[0] == "dup":
                dups.append((int(line[1]), int(line[2])))
            else:
                pairs.append((int(line[0]), int(line[1]), int(line[2])))
    return pairs, dups


def test_initial_layout_matches_text():
    pairs, dups = _golden_layout()
    for strat in (oracle.STRATEGY_ROUND_ROBIN, oracle.STRATEGY_MODULUS):
        first = oracle.simulate(6, strat, 1)[0][0]["pairs"]
        for q, i, j in pairs:
            assert tuple(first[q]) == (i, j)
    tab = oracle.schedule(6, oracle.STRATEGY_MODULUS)
    seen = {}
    for step in tab:
        for i, j in step:
            seen[(i + 1, j + 1)] = seen.get((i + 1, j + 1), 0) + 1
    assert sorted(k for k, v in seen.items() if v == 2) == sorted(dups)


@pytest.mark.parametrize("nbl", [2, 4, 6, 8, 10, 16, 64, 128, 1024])
@pytest.mark.parametrize("strat", [oracle.STRATEGY_ROUND_ROBIN, oracle.STRATEGY_MODULUS])
def test_schedule_properties(nbl, strat):
    p = nbl // 2
    for sweep in (1, 2, 3):
        tab = oracle.schedule(nbl, strat, sweep)
        assert tab.shape == (oracle.steps_per_sweep(nbl, strat), p, 2)
        count = {}
        for step in tab:
            assert sorted(step.reshape(-1).tolist()) == list(range(nbl))  # a partition
            for i, j in step:
                assert i < j
                count[(i, j)] = count.get((i, j), 0) + 1
        assert set(count) == set(combinations(range(nbl), 2))  # every pair visited
        extra = sorted(k for k, v in count.items() if v > 1)
        if strat == oracle.STRATEGY_ROUND_ROBIN:
            assert extra == []  # minimal number of steps, no pair twice
        else:
            assert extra == [(i, i + p) for i in range(p)]  # p-th superdiagonal twice


@pytest.mark.parametrize("nbl", [4, 6, 8, 12, 32])
@pytest.mark.parametrize("strat", [oracle.STRATEGY_ROUND_ROBIN, oracle.STRATEGY_MODULUS])
def test_ring_exchange_is_consistent(nbl, strat):
    """Each step sends one block to snd_rnk and receives one from rcv_rnk (Sec. 4):
    the next layout equals the old pair minus snd_blk plus rcv_blk, and what a
    rank receives is what its rcv_rnk sent."""
    p = nbl // 2
    sim = oracle.simulate(nbl, strat, 3)
    flat = [rec for sw in sim for rec in sw]
    for a, b in zip(flat[:-1], flat[1:]):
        for q in range(p):
            old = set(a["pairs"][q])
            assert a["snd_blk"][q] in old
            new = (old - {a["snd_blk"][q]}) | {a["rcv_blk"][q]}
            assert new == set(b["pairs"][q])
            src = a["rcv_rnk"][q]
            assert a["snd_rnk"][src] == q
            assert a["snd_blk"][src] == a["rcv_blk"][q]


def test_column_rr_table_covers_all_pairs():
    for n in (2, 3, 8, 33, 128):
        tab = oracle.column_rr_table(n)
        npl = n + (n & 1)
        seen = set()
        for step in tab:
            for i, j in step:
                seen.add((i, j))
        assert seen == set(combinations(range(npl), 2))


@pytest.mark.parametrize("strat", [oracle.STRATEGY_ROUND_ROBIN, oracle.STRATEGY_MODULUS])
@pytest.mark.parametrize("b", [4, 8, 13])
def test_blocked_full_block_matches_construction(strat, b):
    P = synth.make_workload("plain_c128_n128", n=64)
    res = oracle.solve_blocked(P.G, P.J, b, strategy=strat)
    assert res["status"] == 0
    assert max_rel_err(res["lam"], P.lam_exact) <= eig_rel_tol(P.G)
    assert orth_residual(res["U"]) <= 8 * oracle.TOL_DEFAULT
    assert reconstruction_residual(P.G, P.J, res["lam"], res["U"]) <= 1e-12


def test_blocked_real_odd_order_and_shuffled_j():
    P = synth.make_workload("blocked_f64_n2048_b32", n=71)
    rng = np.random.default_rng(0)
    perm = rng.permutation(P.n)
    G = np.asfortranarray(P.G[:, perm])
    J = P.J[perm]
    res = oracle.solve_blocked(G, J, 6)
    assert res["status"] == 0
    assert max_rel_err(res["lam"], P.lam_exact) <= eig_rel_tol(P.G)
    plain = oracle.solve_plain(G, J)
    # column order is preserved: lambda_i belongs to column i of the input
    assert np.all(np.sign(res["lam"]) == J)
    assert max_rel_err(res["lam"], plain["lam"]) <= eig_rel_tol(P.G)
