"""Distributed sweeps of the blocked method: the paper's process layout
(Sec. 4) over torch.distributed ranks.

The paper runs p = nbl/2 processes; process q holds one block pair and, after
every parallel step, keeps one block and sends the other to the process that
needs it next (Initialize/MMStep/RLStep, Algs. 4.1-4.3); at the end of a sweep
the processes agree on the number of rotations applied (convergence, Sec. 5).
Here the processes are spread over the ranks of a process group (process q
on rank q mod world); the exchange between two processes on different ranks
is a point-to-point send/receive of the block's columns, between processes on
the same rank a move. Who sends what to whom follows from two consecutive
steps of the ordering table (`jjacobi_schedule`): process q keeps the block
its next pair shares with its current one, and receives the other from the
process holding it now.

The pivot-pair work itself (Gram, Cholesky, inner J-Jacobi, update) is a
`pair_fn(i, j, block_i, block_j) -> rotations` that transforms the two blocks
in place; `library_pair_fn` builds one that runs the library's kernels on the
GPU (the blocks may live on the host between steps, as the gloo transport
needs, or on the device).

Failure handling is on the host: every receive and every reduction is
bounded by the process group's timeout; a rank that never joins, leaves, or
drops a message makes the others' next exchange fail, and `ring_sweeps`
returns RING_PEER_LOST instead of hanging.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Dict, List, Tuple

import numpy as np

RING_OK = 0
RING_NOT_CONVERGED = 2
RING_PEER_LOST = 5


@dataclasses.dataclass
class Transition:
    """What process q does between two parallel steps."""

    keep: int       # block kept
    send: int       # block sent
    send_to: int    # process that receives it
    recv: int       # block received
    recv_from: int  # process that sends it


def schedule(nbl: int, order: int, sweep: int = 1) -> np.ndarray:
    """[steps, nbl/2, 2] block pairs of one sweep (the library's ordering table;
    the assignment of pairs to processes has period two in the sweep number)."""
    from . import jjacobi

    return jjacobi.jjacobi_schedule(nbl, order, sweep)


def transitions(tab: np.ndarray, tab_next: np.ndarray) -> List[List[Transition]]:
    """Exchanges after each step t of a sweep with table `tab` (into step t + 1;
    after the last step into the first step of the next sweep, `tab_next`): the
    layout of the next step is reached by moving one block per process (Sec. 4)."""
    steps, P, _ = tab.shape
    out = []
    for t in range(steps):
        cur = tab[t]
        nxt = tab[t + 1] if t + 1 < steps else tab_next[0]
        holder, nxt_holder = {}, {}
        for q in range(P):
            for b in cur[q]:
                holder[int(b)] = q
            for b in nxt[q]:
                nxt_holder[int(b)] = q
        row = []
        for q in range(P):
            a, b = set(int(x) for x in cur[q]), set(int(x) for x in nxt[q])
            common = a & b
            if len(common) == 2:  # the same pair again: nothing moves
                row.append(Transition(keep=min(a), send=-1, send_to=-1, recv=-1, recv_from=-1))
                continue
            if len(common) != 1:
                raise ValueError("the ordering moves more than one block per process")
            keep = common.pop()
            send = (a - {keep}).pop()
            recv = (b - {keep}).pop()
            row.append(Transition(keep=keep, send=send, send_to=nxt_holder[send], recv=recv,
                                  recv_from=holder[recv]))
        out.append(row)
    return out


def library_pair_fn(J, offs, sizes, gemm: int = 0, device="cuda", tol: float = 0.0,
                    inner_max_sweeps: int = 30):
    """A pair_fn running one pivot pair through the library's kernels: the Gram
    (3.6), the Cholesky factor and the inner J-Jacobi with W accumulated (3.12)
    (full block, Sec. 3.3), and the update (2.9), on one device.

    J: the signs of the work columns (J-sorted order); offs/sizes: the block
    partition (3.3); gemm: jj_gemm of the contractions. The pivot [X_i X_j] is
    copied to the device in column-major order, transformed there, and copied
    back into the caller's blocks (host or device tensors)."""
    import torch

    from . import jjacobi as jj

    Jv = np.asarray(J, dtype=np.int8)
    g_gram = jj.JJ_GEMM_FP64 if gemm == jj.JJ_GEMM_FP64 else jj.JJ_GEMM_OZAKI_FP16
    g_upd = jj.JJ_GEMM_OZAKI_FP16 if gemm == jj.JJ_GEMM_OZAKI_FP16 else jj.JJ_GEMM_FP64

    def fn(i, j, Xi, Xj):
        ni, nj = int(sizes[i]), int(sizes[j])
        k = ni + nj
        X = torch.cat([Xi, Xj], dim=1).to(device)
        m = X.shape[0]
        cplx = X.is_complex()
        G = X.t().contiguous().t()  # m x k, column-major (ld = m)
        dt = jj.JJ_C128 if cplx else jj.JJ_F64
        E = 2 if cplx else 1
        pairs = torch.tensor([[0, ni, ni, nj]], dtype=torch.int32, device=device)
        A = torch.zeros(k * k * E, dtype=torch.float64, device=device)
        W = torch.zeros_like(A)
        cols = np.r_[offs[i]:offs[i] + ni, offs[j]:offs[j] + nj]
        Jd = torch.from_numpy(np.ascontiguousarray(Jv[cols])).to(device)
        cnt = torch.zeros(8, dtype=torch.int64, device=device)
        jj.jjk_gram(dt, g_gram, G, m, m, pairs, 1, A, k)
        jj.jjk_inner(dt, A, W, k, pairs, 1, Jd, tol, inner_max_sweeps, 0, cnt)
        jj.jjk_update(dt, g_upd, G, G, m, m, pairs, 1, W, k)
        c = cnt.cpu()
        if int(c[2]) != 0:
            raise RuntimeError(f"pair ({i}, {j}): device error flags {int(c[2])}")
        Xi.copy_(G[:, :ni])
        Xj.copy_(G[:, ni:])
        return int(c[0])

    return fn


def ring_sweeps(pg_rank: int, world: int, blocks: Dict[int, "object"], sizes: List[int],
                nbl: int, order: int, pair_fn: Callable[[int, int, object, object], int],
                max_sweeps: int = 60, dist=None) -> Tuple[int, int]:
    """Run parallel-ordered sweeps until one applies no rotation.

    blocks: the blocks this rank's processes hold at the start (the first pairs
    of sweep 1), torch tensors (rows x sizes[b]) keyed by block id; they are
    transformed and exchanged in this dict. Returns (status, sweeps)."""
    import torch

    if dist is None:
        import torch.distributed as dist
    tabs = [schedule(nbl, order, 1), schedule(nbl, order, 2)]
    trans = [transitions(tabs[0], tabs[1]), transitions(tabs[1], tabs[0])]
    steps, P, _ = tabs[0].shape
    mine = [q for q in range(P) if q % world == pg_rank]
    proto = next(iter(blocks.values()))
    for sweep in range(1, max_sweeps + 1):
        tab, tr_s = tabs[(sweep - 1) % 2], trans[(sweep - 1) % 2]
        rot = 0
        for t in range(steps):
            for q in mine:
                i, j = (int(x) for x in tab[t][q])
                rot += int(pair_fn(i, j, blocks[i], blocks[j]))
            # exchange into the next step's layout
            reqs, incoming, gone = [], {}, []
            try:
                for q in mine:
                    tr = tr_s[t][q]
                    if tr.send >= 0 and tr.send_to % world != pg_rank:
                        reqs.append(dist.isend(blocks[tr.send].contiguous(), tr.send_to % world,
                                               tag=tr.send))
                        gone.append(tr.send)
                for q in mine:
                    tr = tr_s[t][q]
                    if tr.recv >= 0 and tr.recv_from % world != pg_rank:
                        buf = torch.empty((proto.shape[0], sizes[tr.recv]), dtype=proto.dtype,
                                          device=proto.device)
                        reqs.append(dist.irecv(buf, tr.recv_from % world, tag=tr.recv))
                        incoming[tr.recv] = buf
                for r in reqs:
                    r.wait()
            except RuntimeError:
                return RING_PEER_LOST, sweep
            for b in gone:
                del blocks[b]
            blocks.update(incoming)
        total = torch.tensor([rot], dtype=torch.int64, device=proto.device)
        try:
            dist.all_reduce(total)
        except RuntimeError:
            return RING_PEER_LOST, sweep
        if int(total.item()) == 0:
            return RING_OK, sweep
    return RING_NOT_CONVERGED, max_sweeps
