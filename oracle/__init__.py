"""CPU oracle for the one-sided hyperbolic (J-)Jacobi method.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
CPU-baseline leg import this package. The product library (the CUDA path)
never imports, links or calls it, and the two share no code. The oracle is
plain and slow on purpose: every function follows one passage of the paper
("Three-Level Parallel J-Jacobi Algorithms for Hermitian Matrices", Singer et
al.) in the paper's order and notation.

Contents
  rotation(...)        Alg. 3.1 rotation parameters (C, jj_oracle_body.h).
  solve_plain(...)     Alg. 3.2 + Alg. 3.1, non-blocked, float64 or long double,
                       row-cyclic / column-cyclic / round-robin order (C).
  eigenpairs(...)      lambda_i = J_ii ||g_i||^2, u_i = g_i/||g_i|| (Alg. 5.2 end).
  uniform_partition    block sizes of the uniform partition (3.3).
  schedule(...)        per-step block pairs of Initialize/MMStep/RLStep
                       (Algs. 4.1-4.3), simulated rank by rank.
  column_rr_table(n)   the round-robin order of Alg. 4.3 over single columns.
  gram, cholesky_upper, inner_solve, update
                       the four steps of one pivot of the blocked form.
  solve_blocked(...)   the two-level full-block algorithm (2F) of Alg. 5.2 on one
                       address space: Gram (3.6), Cholesky, inner Alg. 3.2 on R
                       with explicit accumulation of W (3.12), update (2.9).
  solve_block_oriented(...)  the two-level block-oriented algorithm (2B: one
                       pass per pivot, Alg. 3.4 / Sec. 5.3).
  solve_three_level(...)     the three-level algorithms (3F, 3B: the inner
                       method on R blocked, Algs. 3.3 and 5.1).
  cholesky_special, solve_blocked_special
                       the Cholesky factor of a pivot with diagonal diagonal
                       blocks (3.9)-(3.11), and 2F built on it (Sec. 3.3).
  solve_plain_threads  the plain method in round-robin order on several host
                       threads (jj_threads.c): the multithreaded CPU baseline,
                       bit-equal to solve_plain in round-robin order.
  frontend             (module) H -> (G, J) by Bunch-Parlett factorization
                       and block diagonalization (Sec. 2.2, (2.5)), the
                       zero-eigenvalue completion by QR, and the whole method
                       on a Hermitian H.

Every function is pinned by tests/test_oracle_*.py against closed forms,
invariants, constructions with known eigenvalues, LAPACK special cases and
brute force; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_NAME = "liboracle_jj.so"
_lib = None

# Convergence threshold of the published workloads: 128 * eps with
# eps = 2^-53 (unit roundoff of float64).
TOL_DEFAULT = 128.0 * 2.0 ** -53

ORDER_ROW_CYCLIC = 0
ORDER_COLUMN_CYCLIC = 1
ORDER_ROUND_ROBIN = 2

STRATEGY_ROUND_ROBIN = 0
STRATEGY_MODULUS = 1


def build(outdir: Optional[str] = None, force: bool = False) -> str:
    """Compile jj_oracle.c (the oracle) and jj_threads.c (the multithreaded CPU
    baseline) into one shared library with gcc (plain C11, -O2, pthreads)."""
    outdir = outdir or _HERE
    out = os.path.join(outdir, _LIB_NAME)
    srcs = [os.path.join(_HERE, f) for f in ("jj_oracle.c", "jj_threads.c")]
    body = os.path.join(_HERE, "jj_oracle_body.h")
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= max(os.path.getmtime(f) for f in srcs + [body])):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp]
                          + srcs + ["-lm"])
    os.replace(tmp, out)
    return out


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = build()
    lib = ctypes.CDLL(path)
    i64 = ctypes.c_int64
    vp = ctypes.c_void_p
    for sfx, R in (("z", ctypes.c_double), ("d", ctypes.c_double),
                   ("zl", ctypes.c_longdouble), ("dl", ctypes.c_longdouble)):
        f = getattr(lib, "jjo_solve_" + sfx)
        f.restype = ctypes.c_int
        f.argtypes = [i64, i64, vp, i64, vp, R, ctypes.c_int, ctypes.c_int, vp, i64,
                      vp, vp, vp, ctypes.c_int, vp, ctypes.c_int]
        g = getattr(lib, "jjo_eig_" + sfx)
        g.restype = None
        g.argtypes = [i64, i64, vp, i64, vp, vp, vp, i64]
        h = getattr(lib, "jjo_rotation_" + sfx)
        h.restype = ctypes.c_int
        h.argtypes = [R, R, R, R, ctypes.c_int, ctypes.c_int, vp]
    lib.jjo_long_double_mantissa_bits.restype = ctypes.c_int
    lib.jjt_solve_rr.restype = ctypes.c_int
    lib.jjt_solve_rr.argtypes = [ctypes.c_int, i64, i64, vp, i64, vp, ctypes.c_double,
                                 ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, vp, vp, vp]
    _lib = lib
    return lib


def long_double_bits() -> int:
    """Mantissa bits of this host's C long double (64 on x86-64, 113 on aarch64)."""
    return _load().jjo_long_double_mantissa_bits()


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _suffix(cplx: bool, precision: str) -> str:
    return ("z" if cplx else "d") + ("l" if precision == "ld" else "")


def rotation(arr: float, ass: float, ars: complex, hyp: int, cplx: bool = True,
             precision: str = "f64", mutation: int = 0) -> Optional[Dict[str, float]]:
    """Rotation parameters of Alg. 3.1 for one pivot (a_rr, a_ss, a_rs), hyp = J_rr J_ss.

    Returns c, s, e^{i alpha}, t, eta and the updated d_rr, d_ss, or None if the
    hyperbolic case has theta^2 < 1 (pivot not positive definite).
    """
    lib = _load()
    sfx = _suffix(cplx, precision)
    R = np.longdouble if precision == "ld" else np.float64
    out = np.zeros(8, dtype=R)
    ars = complex(ars)
    rc = getattr(lib, "jjo_rotation_" + sfx)(arr, ass, ars.real, ars.imag, int(hyp),
                                             int(mutation), _ptr(out))
    if rc:
        return None
    return dict(c=out[0], s=out[1], e=complex(float(out[2]), float(out[3])), t=out[4],
                eta=out[5], d_r=out[6], d_s=out[7])


def _as_work(G: np.ndarray, precision: str) -> np.ndarray:
    cplx = np.iscomplexobj(G)
    if precision == "ld":
        dt = np.clongdouble if cplx else np.longdouble
    else:
        dt = np.complex128 if cplx else np.float64
    return np.asfortranarray(np.array(G, dtype=dt, copy=True))


def solve_plain(G: np.ndarray, J: Sequence[int], tol: float = TOL_DEFAULT,
                max_sweeps: int = 60, order: int = ORDER_ROW_CYCLIC,
                accumulate: bool = False, precision: str = "f64",
                mutation: int = 0, table: Optional[np.ndarray] = None) -> Dict[str, object]:
    """Non-blocked one-sided J-Jacobi (Alg. 3.2 with Alg. 3.1 as the sweep).

    G is m x n (m >= n, full column rank), J a vector of +-1. Returns a dict with
    the final Gt = G W, the eigenpairs (lam, U), the accumulated W (if asked),
    the number of sweeps, applied rotations, the status (0 converged,
    2 not converged, 3 loss of positive definiteness) and the largest scaled
    off-diagonal |a_rs|/sqrt(a_rr a_ss) seen in the last sweep.
    """
    lib = _load()
    cplx = np.iscomplexobj(G)
    sfx = _suffix(cplx, precision)
    Gw = _as_work(G, precision)
    m, n = Gw.shape
    Jc = np.ascontiguousarray(np.asarray(J, dtype=np.int32))
    W = None
    if accumulate:
        W = np.asfortranarray(np.zeros((n, n), dtype=Gw.dtype))
    sweeps = np.zeros(1, dtype=np.int32)
    rots = np.zeros(1, dtype=np.int64)
    R = np.longdouble if precision == "ld" else np.float64
    maxoff = np.zeros(1, dtype=R)
    nsteps = 0
    if table is not None:
        # an explicit sweep: [steps][n_pad/2][2] column pairs, entries >= n skipped
        order = ORDER_ROUND_ROBIN
        nsteps = int(table.shape[0])
        table = np.ascontiguousarray(np.asarray(table, dtype=np.int32))
    elif order == ORDER_ROUND_ROBIN:
        tab = column_rr_table(n)
        nsteps = tab.shape[0]
        table = np.ascontiguousarray(tab.astype(np.int32))
    st = getattr(lib, "jjo_solve_" + sfx)(m, n, _ptr(Gw), m, _ptr(Jc), tol, max_sweeps,
                                          order, _ptr(W), n, _ptr(sweeps), _ptr(rots),
                                          _ptr(maxoff), int(mutation), _ptr(table), nsteps)
    lam, U = eigenpairs(Gw, Jc, precision=precision)
    return dict(Gt=Gw, lam=lam, U=U, W=W, sweeps=int(sweeps[0]), rotations=int(rots[0]),
                status=int(st), maxoff=float(maxoff[0]))


def solve_plain_threads(G: np.ndarray, J: Sequence[int], nthreads: int,
                        tol: float = TOL_DEFAULT, max_sweeps: int = 60) -> Dict[str, object]:
    """The plain method in round-robin order on nthreads host threads (the
    multithreaded CPU baseline, jj_threads.c): the pairs of a parallel step are
    disjoint, so it returns the bits of solve_plain(order=ORDER_ROUND_ROBIN)."""
    lib = _load()
    cplx = np.iscomplexobj(G)
    Gw = _as_work(G, "f64")
    m, n = Gw.shape
    Jc = np.ascontiguousarray(np.asarray(J, dtype=np.int32))
    tab = np.ascontiguousarray(column_rr_table(n).astype(np.int32))
    sweeps = np.zeros(1, dtype=np.int32)
    rots = np.zeros(1, dtype=np.int64)
    maxoff = np.zeros(1, dtype=np.float64)
    st = lib.jjt_solve_rr(int(cplx), m, n, _ptr(Gw), m, _ptr(Jc), tol, max_sweeps, _ptr(tab),
                          int(tab.shape[0]), int(nthreads), _ptr(sweeps), _ptr(rots),
                          _ptr(maxoff))
    if st == 1:
        raise ValueError("jjt_solve_rr: invalid argument or no resources")
    return dict(Gt=Gw, sweeps=int(sweeps[0]), rotations=int(rots[0]), status=int(st),
                maxoff=float(maxoff[0]))


def eigenpairs(Gt: np.ndarray, J: Sequence[int], precision: Optional[str] = None
               ) -> Tuple[np.ndarray, np.ndarray]:
    """lambda_i = J_ii ||g_i||^2 and u_i = g_i/||g_i|| from the final factor (Alg. 5.2)."""
    lib = _load()
    cplx = np.iscomplexobj(Gt)
    if precision is None:
        precision = "ld" if Gt.dtype in (np.longdouble, np.clongdouble) else "f64"
    Gw = _as_work(Gt, precision)
    m, n = Gw.shape
    Jc = np.ascontiguousarray(np.asarray(J, dtype=np.int32))
    R = np.longdouble if precision == "ld" else np.float64
    lam = np.zeros(n, dtype=R)
    U = np.asfortranarray(np.zeros_like(Gw))
    getattr(lib, "jjo_eig_" + _suffix(cplx, precision))(m, n, _ptr(Gw), m, _ptr(Jc),
                                                        _ptr(lam), _ptr(U), m)
    return lam, U


# ---------------------------------------------------------------------------
# Block partition and parallel orderings (Secs. 3.1, 4.1, 4.2)
# ---------------------------------------------------------------------------

def uniform_partition(n: int, nbl: int) -> List[int]:
    """Block sizes of the uniform partition (3.3): the first n mod nbl blocks get
    floor(n/nbl)+1 columns, the rest floor(n/nbl)."""
    assert 1 <= nbl <= n
    br = n % nbl
    nmin = n // nbl
    return [nmin + 1 if l < br else nmin for l in range(nbl)]


def _initialize(rank: int, nbl: int):
    """Alg. 4.1: starting pivot of process `rank` (1-based block indices)."""
    ip = rank + 1
    i_blk = ip
    jp = nbl - rank
    j_blk = jp
    return [ip, jp, i_blk, j_blk]


def _ring(rank: int, nproc: int, nsweep: int) -> Tuple[int, int]:
    """Neighbour ranks of Algs. 4.2/4.3 (their last if/else): (snd_rnk, rcv_rnk)."""
    if nsweep % 2 > 0:
        return (nproc + rank - 1) % nproc, (nproc + rank + 1) % nproc
    return (nproc + rank + 1) % nproc, (nproc + rank - 1) % nproc


def _mm_step(rank, nbl, nproc, nsweep, state):
    """Alg. 4.2 (modified modulus), one step for one process."""
    ip, jp, i_blk, j_blk = state
    if ip + jp > nbl:
        snd_blk = i_blk
        ip = ip + 1
        if ip == jp:
            ip = ip - nbl // 2
            jp = ip
        i_blk = ip
        rcv_blk = i_blk
    else:
        snd_blk = j_blk
        jp = jp + 1
        j_blk = jp
        rcv_blk = j_blk
    snd_rnk, rcv_rnk = _ring(rank, nproc, nsweep)
    return [ip, jp, i_blk, j_blk], snd_blk, rcv_blk, snd_rnk, rcv_rnk, 0


def _rl_step(rank, nbl, nproc, nsweep, state):
    """Alg. 4.3 (modified round-robin), one step for one process."""
    ip, jp, i_blk, j_blk = state
    swflag = 0
    if ip + jp > nbl:
        if jp < nbl:
            snd_blk = i_blk
            ip = ip + 1
            if ip < jp:
                i_blk = ip
                rcv_blk = i_blk
            else:
                ip = jp
                i_blk = j_blk
                swflag = 1
                jp = nbl
                j_blk = jp
                rcv_blk = j_blk
        else:
            if ip > nbl // 2:
                snd_blk = i_blk
                ip = ip - nbl // 2 + 1
                i_blk = ip
                rcv_blk = i_blk
            else:
                snd_blk = j_blk
                jp = ip + 1
                j_blk = jp
                rcv_blk = j_blk
    else:
        snd_blk = j_blk
        jp = jp + 1
        j_blk = jp
        rcv_blk = j_blk
    snd_rnk, rcv_rnk = _ring(rank, nproc, nsweep)
    return [ip, jp, i_blk, j_blk], snd_blk, rcv_blk, snd_rnk, rcv_rnk, swflag


def steps_per_sweep(nbl: int, strategy: int) -> int:
    """2p steps for modulus, 2p - 1 for round-robin (Sec. 5.3), nbl = 2p."""
    return nbl if strategy == STRATEGY_MODULUS else nbl - 1


def simulate(nbl: int, strategy: int, sweeps: int = 1) -> List[List[dict]]:
    """Run Initialize and then MMStep/RLStep for every process for `sweeps` sweeps.

    Returns, per sweep, per step, a dict with the per-rank pivot blocks
    `pairs[q] = (i_blk, j_blk)` (1-based, as held by process q at that step,
    before the step's exchange) and the exchange that follows the step:
    `snd_blk[q]`, `rcv_blk[q]`, `snd_rnk[q]`, `rcv_rnk[q]`.
    """
    assert nbl >= 2 and nbl % 2 == 0
    p = nbl // 2
    st = [_initialize(q, nbl) for q in range(p)]
    stepfn = _mm_step if strategy == STRATEGY_MODULUS else _rl_step
    out = []
    for nsweep in range(1, sweeps + 1):
        tab = []
        for _ in range(steps_per_sweep(nbl, strategy)):
            rec = dict(pairs=[(s[2], s[3]) for s in st], snd_blk=[], rcv_blk=[],
                       snd_rnk=[], rcv_rnk=[])
            new = []
            for q in range(p):
                ns, sb, rb, sr, rr, _ = stepfn(q, nbl, p, nsweep, st[q])
                new.append(ns)
                rec["snd_blk"].append(sb)
                rec["rcv_blk"].append(rb)
                rec["snd_rnk"].append(sr)
                rec["rcv_rnk"].append(rr)
            st = new
            tab.append(rec)
        out.append(tab)
    return out


def schedule(nbl: int, strategy: int, sweep: int = 1) -> np.ndarray:
    """Block pairs of one sweep as an int array [steps, nbl/2, 2], 0-based, i < j.

    Pair q of a step is the pivot held by process q (Sec. 5.3)."""
    tab = simulate(nbl, strategy, sweep)[sweep - 1]
    arr = np.zeros((len(tab), nbl // 2, 2), dtype=np.int64)
    for s, rec in enumerate(tab):
        for q, (a, b) in enumerate(rec["pairs"]):
            arr[s, q] = (min(a, b) - 1, max(a, b) - 1)
    return arr


def column_rr_table(n: int) -> np.ndarray:
    """Round-robin order over single columns for the plain parallel sweep:
    the pairs of Alg. 4.3 with every 'block' one column (n padded to even;
    index n is the dummy column, skipped)."""
    npl = n + (n & 1)
    if npl < 2:
        return np.zeros((0, 1, 2), dtype=np.int64)
    return schedule(npl, STRATEGY_ROUND_ROBIN, 1)


# ---------------------------------------------------------------------------
# Blocked two-level full-block algorithm (Alg. 5.2, case 2F) on one process
# ---------------------------------------------------------------------------

def j_sort_permutation(J: Sequence[int]) -> np.ndarray:
    """Column permutation P1 that orders J as diag(I_nu, -I_{n-nu}) (Sec. 2.3), stable."""
    J = np.asarray(J)
    return np.concatenate([np.nonzero(J > 0)[0], np.nonzero(J < 0)[0]])


def gram(GP: np.ndarray) -> np.ndarray:
    """Pivot Gram A_P = G_P^* G_P of (3.6) (a library matmul as the step)."""
    GP = np.asarray(GP)
    return GP.conj().T @ GP


def cholesky_upper(AP: np.ndarray) -> np.ndarray:
    """Cholesky factor R (upper, positive diagonal) with A_P = R^* R, (3.8).

    Uses LAPACK's lower Cholesky, R = L^*; raises LinAlgError if A_P is not
    positive definite (G_P not of full column rank, Sec. 3.2)."""
    L = np.linalg.cholesky(np.asarray(AP))
    return np.asfortranarray(L.conj().T)


def inner_solve(R: np.ndarray, JP: Sequence[int], tol: float = TOL_DEFAULT,
                max_sweeps: int = 30) -> Dict[str, object]:
    """HSVD of the pivot factor, R W = U Sigma (3.12), by Alg. 3.2 applied to
    the columns of R with the transformations accumulated explicitly in W."""
    res = solve_plain(R, JP, tol=tol, max_sweeps=max_sweeps, order=ORDER_ROW_CYCLIC,
                      accumulate=True)
    return dict(Rt=res["Gt"], W=res["W"], status=res["status"], rotations=res["rotations"],
                lam=res["lam"])


def update(GP: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Block update [G_i G_j] <- [G_i G_j] W of (2.9) (a library matmul)."""
    return np.asarray(GP) @ np.asarray(W)


def solve_blocked(G: np.ndarray, J: Sequence[int], block_width: int,
                  strategy: int = STRATEGY_ROUND_ROBIN, tol: float = TOL_DEFAULT,
                  max_sweeps: int = 60, inner_max_sweeps: int = 30,
                  max_steps: Optional[int] = None) -> Dict[str, object]:
    """Two-level full-block one-sided J-Jacobi (Alg. 5.2, 2F), sequentially.

    Steps of one parallel step, for every pivot pair (i, j) of the schedule:
      A_P = [G_i G_j]^* [G_i G_j]                       (3.6), (4.1)
      A_P = R^* R (Cholesky, R upper triangular)        (3.8)
      R W = U Sigma by Alg. 3.2 on R with J_P, W accumulated explicitly (3.12)
      [G_i G_j] <- [G_i G_j] W                          (2.9)
    J is first sorted as diag(I, -I) by P1 (Sec. 2.3); the blocks are the
    uniform partition (3.3) with nbl = 2 ceil(n / (2 b)) blocks. A sweep with no
    inner rotation ends the iteration (Sec. 5.3). The returned Gt is in the
    caller's original column order. `max_steps` stops after that many parallel
    steps (for step-by-step comparisons).
    """
    G = np.asarray(G)
    m, n = G.shape
    Jv = np.asarray(J, dtype=np.int64)
    perm = j_sort_permutation(Jv)
    Gp = np.asfortranarray(G[:, perm].astype(np.complex128 if np.iscomplexobj(G) else np.float64))
    Jp = Jv[perm]
    nbl = 2 * ((n + 2 * block_width - 1) // (2 * block_width))
    nbl = max(2, min(nbl, n - (n & 1)))
    sizes = uniform_partition(n, nbl)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    status = 2
    sweeps = 0
    total_rot = 0
    steps_done = 0
    for sweep in range(1, max_sweeps + 1):
        sweeps = sweep
        tab = schedule(nbl, strategy, sweep)
        rot_sweep = 0
        for step in range(tab.shape[0]):
            if max_steps is not None and steps_done >= max_steps:
                break
            for q in range(tab.shape[1]):
                i, j = tab[step, q]
                cols = np.concatenate([np.arange(offs[i], offs[i + 1]),
                                       np.arange(offs[j], offs[j + 1])])
                GP = Gp[:, cols]
                AP = gram(GP)
                try:
                    Rm = cholesky_upper(AP)
                except np.linalg.LinAlgError:
                    return dict(Gt=None, status=3, sweeps=sweeps, rotations=total_rot)
                res = inner_solve(Rm, Jp[cols], tol=tol, max_sweeps=inner_max_sweeps)
                if res["status"] == 3:
                    return dict(Gt=None, status=3, sweeps=sweeps, rotations=total_rot)
                rot_sweep += res["rotations"]
                Gp[:, cols] = update(GP, res["W"])
            steps_done += 1
        total_rot += rot_sweep
        if max_steps is not None and steps_done >= max_steps:
            status = 2
            break
        if rot_sweep == 0:
            status = 0
            break
    Gt = np.empty_like(Gp)
    Gt[:, perm] = Gp
    lam, U = eigenpairs(Gt, Jv)
    return dict(Gt=Gt, lam=lam, U=U, status=status, sweeps=sweeps, rotations=total_rot,
                nbl=nbl, sizes=sizes)


# ---------------------------------------------------------------------------
# Block-oriented strategy (Alg. 3.4, Sec. 5.3 case B) and the three-level
# forms (Sec. 5.1-5.2, Algs. 3.3 and 5.1), sequentially
# ---------------------------------------------------------------------------

def pass_table(n: int, pairs: Sequence[Tuple[int, int]]) -> np.ndarray:
    """A sweep table for solve_plain that visits `pairs` once, in the given
    order (one pair per table step, the other slots dummies >= n)."""
    npl = n + (n & 1)
    tab = np.full((max(len(pairs), 1), npl // 2, 2), n, dtype=np.int32)
    for t, (r, s) in enumerate(pairs):
        tab[t, 0] = (r, s)
    return tab


def block_oriented_pairs(ni: int, nj: int, whole: bool) -> List[Tuple[int, int]]:
    """Column pairs of one block-oriented pass over the pivot [G_i G_j] (Alg. 3.4):
    whole = True (the first step of a sweep): the pairs inside block i, inside
    block j (each row-cyclic), then the off-diagonal block; whole = False: the
    off-diagonal block only, columns s of block j outer, r of block i inner."""
    out = []
    if whole:
        for base, w in ((0, ni), (ni, nj)):
            for r in range(w - 1):
                for q in range(r + 1, w):
                    out.append((base + r, base + q))
    for q in range(nj):
        for r in range(ni):
            out.append((r, ni + q))
    return out


def _inner_pass(R: np.ndarray, JP, pairs, tol: float) -> Dict[str, object]:
    """One pass of Alg. 3.1 rotations over the given column pairs of R, with the
    transformation accumulated explicitly (3.12)."""
    n = R.shape[1]
    res = solve_plain(R, JP, tol=tol, max_sweeps=1, accumulate=True, table=pass_table(n, pairs))
    return dict(Rt=res["Gt"], W=res["W"], status=res["status"], rotations=res["rotations"])


def solve_block_oriented(G: np.ndarray, J: Sequence[int], block_width: int,
                         strategy: int = STRATEGY_ROUND_ROBIN, tol: float = TOL_DEFAULT,
                         max_sweeps: int = 60, whole_first: bool = True) -> Dict[str, object]:
    """Two-level block-oriented algorithm (Sec. 5.3 case B, the sweeps of
    Alg. 3.4 distributed over the parallel steps of Sec. 4): for every pivot pair
    (i, j) of a step, A_P = [G_i G_j]^*[G_i G_j] (3.6), A_P = R^*R, then ONE pass
    of rotations on the columns of R (the whole pivot in the first step of a
    sweep, the off-diagonal block in the others), W accumulated (3.12), and
    [G_i G_j] <- [G_i G_j] W (2.9). A sweep with no rotation ends it.
    whole_first=False plants a mistake for the pin tests (no whole-pivot pass:
    column pairs inside one block are never rotated)."""
    G = np.asarray(G)
    m, n = G.shape
    Jv = np.asarray(J, dtype=np.int64)
    perm = j_sort_permutation(Jv)
    Gp = np.asfortranarray(G[:, perm].astype(np.complex128 if np.iscomplexobj(G) else np.float64))
    Jp = Jv[perm]
    nbl = 2 * ((n + 2 * block_width - 1) // (2 * block_width))
    nbl = max(2, min(nbl, n - (n & 1)))
    sizes = uniform_partition(n, nbl)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    status, sweeps, total = 2, 0, 0
    for sweep in range(1, max_sweeps + 1):
        sweeps = sweep
        tab = schedule(nbl, strategy, sweep)
        rot = 0
        for step in range(tab.shape[0]):
            for q in range(tab.shape[1]):
                i, j = tab[step, q]
                cols = np.concatenate([np.arange(offs[i], offs[i + 1]), np.arange(offs[j], offs[j + 1])])
                GP = Gp[:, cols]
                try:
                    R = cholesky_upper(gram(GP))
                except np.linalg.LinAlgError:
                    return dict(Gt=None, status=3, sweeps=sweeps, rotations=total)
                res = _inner_pass(R, Jp[cols],
                                  block_oriented_pairs(sizes[i], sizes[j], whole_first and step == 0), tol)
                if res["status"] == 3:
                    return dict(Gt=None, status=3, sweeps=sweeps, rotations=total)
                rot += res["rotations"]
                Gp[:, cols] = update(GP, res["W"])
        total += rot
        if rot == 0:
            status = 0
            break
    Gt = np.empty_like(Gp)
    Gt[:, perm] = Gp
    lam, U = eigenpairs(Gt, Jv)
    return dict(Gt=Gt, lam=lam, U=U, status=status, sweeps=sweeps, rotations=total, nbl=nbl,
                sizes=sizes)


def _inner_blocks(ni: int, nj: int, ib: int) -> List[int]:
    """Inner partition of a pivot that respects the boundary of its two blocks
    (Sec. 5.2, Alg. 5.1): nb blocks of each, uniform partitions (3.3)."""
    nb = max((ni + ib - 1) // ib, (nj + ib - 1) // ib)
    nb = max(1, min(nb, ni, nj))
    return uniform_partition(ni, nb) + uniform_partition(nj, nb)


def _inner_blocked(R: np.ndarray, JP, ib: int, ni: int, nj: int, variant: str, first: bool,
                   tol: float, inner_max_sweeps: int) -> Dict[str, object]:
    """The inner problem of a three-level step on the Cholesky factor R of one
    pivot: the blocked one-sided method on the columns of R (Alg. 3.3), with W
    accumulated by applying every inner transformation to [R; W] too.
    variant 'F': sweeps over all inner block pairs, each inner pivot solved to
    convergence, until a sweep applies no rotation. variant 'B': one pass --
    in the first outer step of a sweep over every inner block pair (each inner
    pivot: its whole pass in the first inner step, its off-diagonal block in
    the others), in the other outer steps over the pairs of an inner block of
    block i with one of block j, each inner pivot's off-diagonal block once
    (Alg. 5.1)."""
    k = R.shape[1]
    X = np.concatenate([R, np.eye(k, dtype=R.dtype)], axis=0)
    isz = _inner_blocks(ni, nj, ib)
    nb = len(isz) // 2
    ioff = np.concatenate([[0], np.cumsum(isz)]).astype(np.int64)
    total = 0

    def pivot(a, b, whole_or_converge):
        nonlocal total
        cols = np.concatenate([np.arange(ioff[a], ioff[a + 1]), np.arange(ioff[b], ioff[b + 1])])
        XP = X[:, cols]
        Rin = cholesky_upper(gram(XP[:k]))
        if variant == "F":
            res = inner_solve(Rin, JP[cols], tol=tol, max_sweeps=inner_max_sweeps)
        else:
            res = _inner_pass(Rin, JP[cols], block_oriented_pairs(isz[a], isz[b], whole_or_converge), tol)
        if res["status"] == 3:
            raise np.linalg.LinAlgError("inner pivot not positive definite")
        total += res["rotations"]
        X[:, cols] = update(XP, res["W"])
        return res["rotations"]

    if variant == "F":
        for sweep in range(1, inner_max_sweeps + 1):
            tab = schedule(2 * nb, STRATEGY_ROUND_ROBIN, sweep)
            rot = 0
            for step in range(tab.shape[0]):
                for a, b in tab[step]:
                    rot += pivot(a, b, True)
            if rot == 0:
                break
    elif first:
        tab = schedule(2 * nb, STRATEGY_ROUND_ROBIN, 1)
        for step in range(tab.shape[0]):
            for a, b in tab[step]:
                pivot(a, b, step == 0)
    else:
        for b in range(nb, 2 * nb):
            for a in range(nb):
                pivot(a, b, False)
    return dict(W=X[k:], rotations=total)


def solve_three_level(G: np.ndarray, J: Sequence[int], block_width: int, inner_width: int,
                      variant: str = "F", strategy: int = STRATEGY_ROUND_ROBIN,
                      tol: float = TOL_DEFAULT, max_sweeps: int = 60,
                      inner_max_sweeps: int = 30) -> Dict[str, object]:
    """Three-level algorithm (Sec. 5.1 case 3F, Sec. 5.2 case 3B): the two-level
    step of Alg. 5.2 with the inner J-Jacobi on R itself blocked
    (_inner_blocked), sequentially. A sweep with no rotation ends it."""
    G = np.asarray(G)
    m, n = G.shape
    Jv = np.asarray(J, dtype=np.int64)
    perm = j_sort_permutation(Jv)
    Gp = np.asfortranarray(G[:, perm].astype(np.complex128 if np.iscomplexobj(G) else np.float64))
    Jp = Jv[perm]
    nbl = 2 * ((n + 2 * block_width - 1) // (2 * block_width))
    nbl = max(2, min(nbl, n - (n & 1)))
    sizes = uniform_partition(n, nbl)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    status, sweeps, total = 2, 0, 0
    for sweep in range(1, max_sweeps + 1):
        sweeps = sweep
        tab = schedule(nbl, strategy, sweep)
        rot = 0
        for step in range(tab.shape[0]):
            for q in range(tab.shape[1]):
                i, j = tab[step, q]
                cols = np.concatenate([np.arange(offs[i], offs[i + 1]), np.arange(offs[j], offs[j + 1])])
                GP = Gp[:, cols]
                try:
                    R = cholesky_upper(gram(GP))
                    res = _inner_blocked(R, Jp[cols], inner_width, sizes[i], sizes[j], variant,
                                         step == 0, tol, inner_max_sweeps)
                except np.linalg.LinAlgError:
                    return dict(Gt=None, status=3, sweeps=sweeps, rotations=total)
                rot += res["rotations"]
                Gp[:, cols] = update(GP, res["W"])
        total += rot
        if rot == 0:
            status = 0
            break
    Gt = np.empty_like(Gp)
    Gt[:, perm] = Gp
    lam, U = eigenpairs(Gt, Jv)
    return dict(Gt=Gt, lam=lam, U=U, status=status, sweeps=sweeps, rotations=total, nbl=nbl,
                sizes=sizes)


# ---------------------------------------------------------------------------
# Full block with diagonalized diagonal blocks: the special Cholesky (3.9)-(3.11)
# ---------------------------------------------------------------------------

def cholesky_special(lam_i: np.ndarray, lam_j: np.ndarray, Aij: np.ndarray,
                     mutation: int = 0) -> np.ndarray:
    """Cholesky factor R of a pivot with diagonal diagonal blocks (3.7):
    R_ii = sqrt(Lambda_ii) (3.9), R_ij = R_ii^{-1} A_ij (3.10), and R_jj the
    Cholesky factor of Lambda_jj - R_ij^* R_ij (3.11). Raises LinAlgError when
    that block is not positive definite. mutation=1 plants a mistake for the
    pins (A_ij scaled from the wrong side)."""
    lam_i = np.asarray(lam_i, dtype=np.float64)
    lam_j = np.asarray(lam_j, dtype=np.float64)
    Aij = np.asarray(Aij)
    ni, nj = len(lam_i), len(lam_j)
    rii = np.sqrt(lam_i)
    if mutation == 1:
        Rij = Aij / rii[None, :nj] if nj <= ni else Aij / rii.mean()
    else:
        Rij = Aij / rii[:, None]
    Rjj = cholesky_upper(np.diag(lam_j).astype(Aij.dtype) - Rij.conj().T @ Rij)
    R = np.zeros((ni + nj, ni + nj), dtype=np.result_type(Aij.dtype, np.float64))
    R[:ni, :ni] = np.diag(rii)
    R[:ni, ni:] = Rij
    R[ni:, ni:] = Rjj
    return np.asfortranarray(R)


def solve_blocked_special(G: np.ndarray, J: Sequence[int], block_width: int,
                          strategy: int = STRATEGY_ROUND_ROBIN, tol: float = TOL_DEFAULT,
                          max_sweeps: int = 60, inner_max_sweeps: int = 30) -> Dict[str, object]:
    """Two-level full block (2F) with the structure of Sec. 3.3: at the start of
    every sweep the diagonal block A_ii of every block is diagonalized (the
    re-diagonalization of Sec. 5.3), so that each pivot has the form (3.7) and
    its factor R comes from the special Cholesky (3.9)-(3.11) (the diagonal
    blocks' off-diagonal entries, at most tol sqrt(a_rr a_ss) after a full
    block solve, are taken as zero); then the inner J-Jacobi on R with W
    accumulated (3.12) and the update (2.9), as in solve_blocked."""
    G = np.asarray(G)
    m, n = G.shape
    Jv = np.asarray(J, dtype=np.int64)
    perm = j_sort_permutation(Jv)
    Gp = np.asfortranarray(G[:, perm].astype(np.complex128 if np.iscomplexobj(G) else np.float64))
    Jp = Jv[perm]
    nbl = 2 * ((n + 2 * block_width - 1) // (2 * block_width))
    nbl = max(2, min(nbl, n - (n & 1)))
    sizes = uniform_partition(n, nbl)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    status, sweeps, total = 2, 0, 0
    for sweep in range(1, max_sweeps + 1):
        sweeps = sweep
        rot = 0
        # diagonalize every diagonal block A_ii (one-sided, on the block's columns)
        for i in range(nbl):
            cols = np.arange(offs[i], offs[i + 1])
            res = solve_plain(Gp[:, cols], Jp[cols], tol=tol, max_sweeps=inner_max_sweeps)
            if res["status"] == 3:
                return dict(Gt=None, status=3, sweeps=sweeps, rotations=total)
            rot += res["rotations"]
            Gp[:, cols] = res["Gt"]
        tab = schedule(nbl, strategy, sweep)
        for step in range(tab.shape[0]):
            for q in range(tab.shape[1]):
                i, j = tab[step, q]
                ci = np.arange(offs[i], offs[i + 1])
                cj = np.arange(offs[j], offs[j + 1])
                cols = np.concatenate([ci, cj])
                GP = Gp[:, cols]
                lam_i = np.sum(np.abs(Gp[:, ci]) ** 2, axis=0)
                lam_j = np.sum(np.abs(Gp[:, cj]) ** 2, axis=0)
                Aij = Gp[:, ci].conj().T @ Gp[:, cj]
                try:
                    R = cholesky_special(lam_i, lam_j, Aij)
                except np.linalg.LinAlgError:
                    return dict(Gt=None, status=3, sweeps=sweeps, rotations=total)
                res = inner_solve(R, Jp[cols], tol=tol, max_sweeps=inner_max_sweeps)
                if res["status"] == 3:
                    return dict(Gt=None, status=3, sweeps=sweeps, rotations=total)
                rot += res["rotations"]
                Gp[:, cols] = update(GP, res["W"])
        total += rot
        if rot == 0:
            status = 0
            break
    Gt = np.empty_like(Gp)
    Gt[:, perm] = Gp
    lam, U = eigenpairs(Gt, Jv)
    return dict(Gt=Gt, lam=lam, U=U, status=status, sweeps=sweeps, rotations=total, nbl=nbl,
                sizes=sizes)
