"""The distributed sweep driver (the paper's process layout of Sec. 4 over
torch.distributed) with world_size 2 on CPU (gloo): the exchanged blocks
reproduce the sequential blocked reference bit for bit, and a rank that
leaves makes the other return an error status instead of hanging."""
import os
import socket
import time
from datetime import timedelta

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _setup(n, b):
    import oracle
    import synth

    P = synth.make_workload("blocked_f64_n2048_b32", n=n)
    perm = oracle.j_sort_permutation(np.asarray(P.J))
    Gp = np.asfortranarray(P.G[:, perm])
    Jp = np.asarray(P.J)[perm]
    nbl = 2 * ((n + 2 * b - 1) // (2 * b))
    sizes = oracle.uniform_partition(n, nbl)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return P, perm, Gp, Jp, nbl, sizes, offs


def _worker(rank, world, port, n, b, order, mode, q):
    import torch.distributed as dist

    import oracle
    from paper_1008_4166_gb300 import ring

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world, timeout=timedelta(seconds=8))
    P, perm, Gp, Jp, nbl, sizes, offs = _setup(n, b)
    if mode == "drop" and rank == 1:
        os._exit(0)  # leaves before the first exchange, between steps
    tab = ring.schedule(nbl, order, 1)
    blocks = {}
    for qq in range(nbl // 2):
        if qq % world == rank:
            for blk in tab[0][qq]:
                blocks[int(blk)] = torch.from_numpy(np.ascontiguousarray(Gp[:, offs[blk]:offs[blk + 1]]))

    def pair_fn(i, j, Xi, Xj):
        cols = np.concatenate([np.arange(offs[i], offs[i + 1]), np.arange(offs[j], offs[j + 1])])
        GP = np.asfortranarray(np.concatenate([Xi.numpy(), Xj.numpy()], axis=1))
        R = oracle.cholesky_upper(oracle.gram(GP))
        res = oracle.inner_solve(R, Jp[cols])
        out = oracle.update(GP, res["W"])
        Xi.copy_(torch.from_numpy(np.ascontiguousarray(out[:, :sizes[i]])))
        Xj.copy_(torch.from_numpy(np.ascontiguousarray(out[:, sizes[i]:])))
        return res["rotations"]

    t0 = time.time()
    status, sweeps = ring.ring_sweeps(rank, world, blocks, list(sizes), nbl, order, pair_fn)
    q.put((rank, status, sweeps, time.time() - t0,
           {k: v.numpy().copy() for k, v in blocks.items()}))
    if status == ring.RING_OK:
        dist.destroy_process_group()


def _run(world, n, b, order, mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, b, order, mode, q))
             for r in range(world)]
    for p in procs:
        p.start()
    out = []
    expect = world if mode != "drop" else 1
    for _ in range(expect):
        out.append(q.get(timeout=180))
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    return sorted(out, key=lambda x: x[0])


@pytest.mark.parametrize("order", [0, 1])
def test_ring_two_ranks_matches_sequential_blocked(order):
    import oracle
    from paper_1008_4166_gb300 import ring

    n, b = 48, 4
    res = _run(2, n, b, order, "ok")
    P, perm, Gp, Jp, nbl, sizes, offs = _setup(n, b)
    blocks = {}
    for rank, status, sweeps, _, blk in res:
        assert status == ring.RING_OK
        blocks.update(blk)
    assert sorted(blocks) == list(range(nbl))
    Gt = np.concatenate([blocks[k] for k in range(nbl)], axis=1)
    ref = oracle.solve_blocked(P.G, P.J, b, strategy=order)
    assert ref["status"] == 0
    assert res[0][2] == ref["sweeps"]
    assert np.array_equal(Gt, ref["Gt"][:, perm])


@pytest.mark.parametrize("order", [0, 1])
def test_ring_three_ranks_matches_sequential_blocked(order):
    """Three ranks for four processes (nbl = 8): processes 0 and 3 share rank 0,
    so some exchanges are moves within a rank, the others messages."""
    import oracle
    from paper_1008_4166_gb300 import ring

    n, b = 32, 4
    res = _run(3, n, b, order, "ok")
    P, perm, Gp, Jp, nbl, sizes, offs = _setup(n, b)
    assert nbl == 8
    blocks = {}
    for rank, status, sweeps, _, blk in res:
        assert status == ring.RING_OK
        assert not (set(blocks) & set(blk))  # every block on exactly one rank
        blocks.update(blk)
    Gt = np.concatenate([blocks[k] for k in range(nbl)], axis=1)
    ref = oracle.solve_blocked(P.G, P.J, b, strategy=order)
    assert res[0][2] == ref["sweeps"]
    assert np.array_equal(Gt, ref["Gt"][:, perm])


def test_ring_rank_leaves_other_returns_error():
    from paper_1008_4166_gb300 import ring

    res = _run(2, 48, 4, 0, "drop")
    rank, status, sweeps, secs, _ = res[0]
    assert rank == 0
    assert status == ring.RING_PEER_LOST
    assert secs < 60


def test_transitions_move_one_block_per_process():
    """Host logic alone: applying the transitions to the layout of step t gives
    the layout of step t + 1, and every sent block is received by its new holder."""
    from paper_1008_4166_gb300 import ring

    for nbl in (4, 6, 10, 16):
        for order in (0, 1):
            t1, t2 = ring.schedule(nbl, order, 1), ring.schedule(nbl, order, 2)
            for tab, nxt in ((t1, t2), (t2, t1)):
                tr = ring.transitions(tab, nxt)
                for t in range(tab.shape[0]):
                    nlay = tab[t + 1] if t + 1 < tab.shape[0] else nxt[0]
                    for q in range(tab.shape[1]):
                        x = tr[t][q]
                        have = set(int(v) for v in tab[t][q])
                        if x.send >= 0:
                            have = (have - {x.send}) | {x.recv}
                            assert tr[t][x.send_to].recv == x.send
                            assert tr[t][x.send_to].recv_from == q
                        assert have == set(int(v) for v in nlay[q])


class _DroppingDist:
    """torch.distributed with the first point-to-point send of this rank dropped
    (the message never leaves: a lost message on the host side)."""

    def __init__(self, dist):
        self._d = dist
        self.dropped = False

    def isend(self, tensor, dst, tag=0):
        if not self.dropped:
            self.dropped = True

            class _Done:
                def wait(self):
                    return True
            return _Done()
        return self._d.isend(tensor, dst, tag=tag)

    def __getattr__(self, name):
        return getattr(self._d, name)


def _worker_fault(rank, world, port, mode, q):
    import time as _t

    import torch.distributed as dist

    import oracle
    from paper_1008_4166_gb300 import ring

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world, timeout=timedelta(seconds=5))
    P, perm, Gp, Jp, nbl, sizes, offs = _setup(32, 4)
    tab = ring.schedule(nbl, 0, 1)
    blocks = {}
    for qq in range(nbl // 2):
        if qq % world == rank:
            for blk in tab[0][qq]:
                blocks[int(blk)] = torch.from_numpy(np.ascontiguousarray(Gp[:, offs[blk]:offs[blk + 1]]))
    late = {"done": False}

    def pair_fn(i, j, Xi, Xj):
        if mode == "late" and rank == 1 and not late["done"]:
            late["done"] = True
            _t.sleep(12)  # beyond the group's 5 s timeout, before its first exchange
        cols = np.concatenate([np.arange(offs[i], offs[i + 1]), np.arange(offs[j], offs[j + 1])])
        GP = np.asfortranarray(np.concatenate([Xi.numpy(), Xj.numpy()], axis=1))
        res = oracle.inner_solve(oracle.cholesky_upper(oracle.gram(GP)), Jp[cols])
        out = oracle.update(GP, res["W"])
        Xi.copy_(torch.from_numpy(np.ascontiguousarray(out[:, :sizes[i]])))
        Xj.copy_(torch.from_numpy(np.ascontiguousarray(out[:, sizes[i]:])))
        return res["rotations"]

    d = _DroppingDist(dist) if (mode == "drop_message" and rank == 1) else dist
    t0 = _t.time()
    status, sweeps = ring.ring_sweeps(rank, world, blocks, list(sizes), nbl, 0, pair_fn, dist=d)
    q.put((rank, status, _t.time() - t0))


def _run_fault(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_fault, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = []
    for _ in range(2):
        try:
            out.append(q.get(timeout=120))
        except Exception:
            break
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    return sorted(out)


@pytest.mark.parametrize("mode", ["drop_message", "late"])
def test_ring_lost_message_or_late_rank_returns_error(mode):
    """A block that never arrives (rank 1 drops its first send), or a rank that
    is late beyond the group timeout: the waiting rank's exchange fails within
    the timeout and ring_sweeps returns RING_PEER_LOST instead of hanging."""
    from paper_1008_4166_gb300 import ring

    res = _run_fault(mode)
    assert res, "no rank reported"
    waiting = [r for r in res if r[0] == 0]
    assert waiting and waiting[0][1] == ring.RING_PEER_LOST
    assert waiting[0][2] < 60
