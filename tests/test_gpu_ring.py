"""The distributed sweep driver with the library's own pair function: two
gloo ranks (two processes sharing this GPU, each launching its own kernels;
no kernel waits on another) run the parallel-ordered sweeps of Sec. 4 with
the Gram, inner J-Jacobi and update of every pair on the GPU, exchanging
block columns between steps. The result equals, bit for bit, the same driver
in one process, and its eigenvalues match the oracle's."""
import socket
from datetime import timedelta

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _setup(recipe, n, b):
    import oracle
    import synth

    P = synth.make_workload(recipe, n=n)
    perm = oracle.j_sort_permutation(np.asarray(P.J))
    Gp = np.asfortranarray(P.G[:, perm])
    Jp = np.asarray(P.J)[perm]
    nbl = 2 * ((n + 2 * b - 1) // (2 * b))
    sizes = oracle.uniform_partition(n, nbl)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return P, perm, Gp, Jp, nbl, sizes, offs


def _worker(rank, world, port, recipe, n, b, order, gemm, q):
    import torch.distributed as dist

    from paper_1008_4166_gb300 import jjacobi, ring

    jjacobi.load()
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world, timeout=timedelta(seconds=60))
    P, perm, Gp, Jp, nbl, sizes, offs = _setup(recipe, n, b)
    tab = ring.schedule(nbl, order, 1)
    blocks = {}
    for qq in range(nbl // 2):
        if qq % world == rank:
            for blk in tab[0][qq]:
                blocks[int(blk)] = torch.from_numpy(np.ascontiguousarray(Gp[:, offs[blk]:offs[blk + 1]]))
    fn = ring.library_pair_fn(Jp, offs, sizes, gemm=gemm)
    status, sweeps = ring.ring_sweeps(rank, world, blocks, list(sizes), nbl, order, fn)
    q.put((rank, status, sweeps, {k: v.numpy().copy() for k, v in blocks.items()}))
    dist.destroy_process_group()


def _run(world, *args):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port) + args + (q,)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    blocks, statuses, sweeps = {}, set(), set()
    for rank, st, sw, blk in out:
        statuses.add(st)
        sweeps.add(sw)
        blocks.update(blk)
    return statuses, sweeps, blocks


@pytest.mark.parametrize("recipe,gemm", [("blocked_f64_n2048_b32", 0),
                                         ("plain_c128_n128", 1)])
def test_ring_with_library_kernels_two_ranks_on_one_gpu(recipe, gemm):
    from tests.gpu_util import require_gpu
    from tests._util import eig_rel_tol, max_rel_err

    require_gpu()
    import oracle
    from paper_1008_4166_gb300 import ring

    n, b, order = 64, 8, 1
    st2, sw2, blk2 = _run(2, recipe, n, b, order, gemm)
    st1, sw1, blk1 = _run(1, recipe, n, b, order, gemm)
    assert st2 == {ring.RING_OK} and st1 == {ring.RING_OK} and sw2 == sw1
    P, perm, Gp, Jp, nbl, sizes, offs = _setup(recipe, n, b)
    assert sorted(blk2) == list(range(nbl))
    for k in range(nbl):
        assert np.array_equal(blk2[k], blk1[k]), k
    Gt = np.concatenate([blk2[k] for k in range(nbl)], axis=1)
    lam = Jp * np.linalg.norm(Gt, axis=0) ** 2
    ref = oracle.solve_plain(P.G, P.J)
    assert max_rel_err(lam, ref["lam"]) <= eig_rel_tol(P.G)
