#!/usr/bin/env python3
"""Benchmark of the GB300 one-sided J-Jacobi solver (one JSON line on stdout).

A step is one complete solve of the hot path on one synthetic input: J sort,
parallel-ordered sweeps of the blocked full-block method (Gram, Cholesky +
inner J-Jacobi with accumulated W, update, convergence count) until a sweep
applies no rotation, then eigenpair extraction. The headline workload is the
graded complex128 problem of order 4096 (G = D1 B D2, B = Q |Lambda|^{1/2} W,
J = diag(+I_2560, -I_1536)).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--block-width B] [--gemm hybrid|ozaki|fp64] [--strategy oriented|full]
                  [--no-plain] [--no-cpu]
                  [--one-step]

--impl reference times the CPU oracle (the plain one-sided J-Jacobi, in C,
single-threaded) on a bounded sample of the same workload. The default run
reports it as cpu_baseline, and beside it cpu_baseline_threads: the same
method in round-robin order on all host cores (pthreads, bit-equal to the
sequential oracle in that order), on a bounded sample too.
--one-step runs only the first parallel step of the sweep (column exponents,
Gram, inner solve, update of every block pair) through the building-block
entry points, K times: the small case for kernel profiles.
--study orders,crossover times round-robin against modulus ordering and the
plain form against the blocked forms over n (graded complex recipe).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "graded_c128_n4096_b64"
METRIC = "time-to-solution & GFLOP/s, blocked J-Jacobi n=4096 c128, vs plain form at rel-err≤1e-12"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2070e6 / 1e12  # SMs x FP64 FMA/clk/SM x 2 flops x max SM clock


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def blocked_flops(n: int, m: int, cplx: bool, info: dict) -> float:
    """FP64-equivalent flops of the work one blocked solve executed.

    The Gram's Hermitian half, k(k+1)/2 * m MACs, for every pair whose Gram and
    inner solve ran (pairs_evaluated: the solver skips pairs unchanged since
    they were last found diagonal); the update's m k^2 MACs for every pair whose
    inner solve applied a rotation (pairs_rotated: the others are left as they
    are); 5 k MACs per applied inner rotation (dot, R and W column pairs). A
    complex MAC is 8 real flops, a real MAC 2."""
    mac = 8.0 if cplx else 2.0
    k = 2.0 * n / info["nbl"]
    gram = info["pairs_evaluated"] * k * (k + 1) / 2 * m
    update = info["pairs_rotated"] * m * k * k
    inner = info["rotations"] * 5.0 * k
    return mac * (gram + update + inner)


def blocked_flops_all_pairs(n: int, m: int, cplx: bool, info: dict) -> float:
    """The same conventions charged for every pair of every step of every sweep
    (as if no pair were skipped): context for comparisons with implementations
    that always recompute."""
    mac = 8.0 if cplx else 2.0
    nbl = info["nbl"]
    k = 2.0 * n / nbl
    pair_steps = info["sweeps"] * info["steps_per_sweep"] * (nbl // 2)
    return mac * (pair_steps * (k * (k + 1) / 2 * m + m * k * k) + info["rotations"] * 5.0 * k)


def plain_flops(n: int, m: int, cplx: bool, sweeps: int) -> float:
    """Algorithmic flops of the plain method: per pair and sweep one dot product
    and one column-pair rotation (3 m MACs)."""
    mac = 8.0 if cplx else 2.0
    return mac * sweeps * n * (n - 1) / 2 * 3.0 * m


def cpu_baseline(P, budget_s: float = 15.0):
    """The oracle on a bounded sample: one row-cyclic sweep of the plain method on
    the leading ncol columns of G (all m rows), ncol grown until about budget_s
    of CPU time. Returns GFLOP/s of plain-method work, and the sample."""
    import numpy as np

    import oracle

    ncol = 32
    best = None
    while True:
        Gs = np.asfortranarray(P.G[:, :ncol])
        t0 = time.perf_counter()
        oracle.solve_plain(Gs, P.J[:ncol], max_sweeps=1)
        dt = time.perf_counter() - t0
        fl = plain_flops(ncol, P.m, P.is_complex, 1) * 1.0
        best = (fl / dt / 1e9, ncol, dt)
        if dt > budget_s / 3 or ncol >= P.n:
            break
        ncol = min(P.n, ncol * 2)
    return best


def cpu_model() -> str:
    """The host CPU's model name (lscpu), with the architecture."""
    import platform

    name = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return f"{name or 'unknown model'} ({platform.machine()})"


def cpu_baseline_threads(P, budget_s: float = 10.0):
    """The multithreaded CPU baseline on a bounded sample: one round-robin sweep
    of the plain method on all host cores (oracle.solve_plain_threads), on the
    leading ncol columns of G (all m rows), ncol grown until about budget_s.
    Returns GFLOP/s of plain-method work, the sample and the thread count."""
    import numpy as np

    import oracle

    nt = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    ncol = 64
    while True:
        Gs = np.asfortranarray(P.G[:, :ncol])
        t0 = time.perf_counter()
        oracle.solve_plain_threads(Gs, P.J[:ncol], nthreads=nt, max_sweeps=1)
        dt = time.perf_counter() - t0
        best = (plain_flops(ncol, P.m, P.is_complex, 1) / dt / 1e9, ncol, dt, nt)
        if dt > budget_s / 3 or ncol >= P.n:
            return best
        ncol = min(P.n, ncol * 2)


def bench_config(args, P, world: int = 1) -> dict:
    """The workload and launch configuration both arms report."""
    name = re.sub(r"_b\d+$", f"_b{args.block_width}", args.workload)
    return {"workload": name, "recipe": args.workload, "m": P.m, "n": P.n,
            "block_width": args.block_width, "gemm": args.gemm,
            **({"inner_block_width": args.inner_block_width} if getattr(args, "inner_block_width", 0) else {}),
            "update_digits": (args.digits or 11) if args.gemm == "ozaki" and args.block_width else None,
            "strategy": args.strategy, "order": "round_robin",
            "pivot_factor": getattr(args, "pivot_factor", "cholesky"),
            "l2": "inputs larger than L2 (G = 256 MiB; every step reads and writes it)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def run_reference(args):
    rank, world, local = _dist()
    if rank != 0:
        return
    import synth

    P = synth.make_workload(args.workload, precision="f64")
    vals = []
    for i in range(args.warmup + args.steps):
        g, ncol, dt = cpu_baseline(P, budget_s=args.ref_budget)
        if i >= args.warmup:
            vals.append((g, ncol, dt))
    v = statistics.median(x[0] for x in vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "GFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.median(x[2] for x in vals) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(args, P, world),
        "cpu_baseline": {"value": v, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                         "cpu": cpu_model(),
                         "sample": f"one row-cyclic plain sweep on the leading {vals[0][1]} "
                                   f"columns (all {P.m} rows) of the n={P.n} input"},
        "e2e": {"value": v, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def captured_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from profiles/traffic.txt, if the
    kernel's source files are unchanged since the capture (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.txt")) as f:
            for line in f:
                parts = line.split()
                if len(parts) != 4 or line.startswith("#") or parts[0] != kernel:
                    continue
                h = hashlib.sha256()
                for name in parts[2].split(","):
                    with open(os.path.join(ROOT, "paper_1008_4166_gb300", "csrc", name), "rb") as fh:
                        h.update(fh.read())
                return int(parts[1]) if h.hexdigest()[:16] == parts[3] else None
    except OSError:
        return None
    return None


def gram_products(s: int) -> int:
    """Digit products of the split-precision Gram (t + u <= s + 1)."""
    return sum(1 for d in range(2, s + 2) for t in range(1, s + 1) if 1 <= d - t <= s)


def update_products(s: int) -> int:
    return sum(1 for d in range(2, s + 2) for t in range(1, s + 1) if 1 <= d - t <= s)


def kernel_roofline(jj, P, times, info, gemm_gram_digits, gemm_upd_digits, peaks):
    """Achieved rate of the dominant kernel family over a profiled solve.

    Work counted (algorithmic, per family, summed over the solve):
      gram   digit form: products x 2 K2^2 m tensor flops per evaluated pair;
             FP64 form: Hermitian half k(k+1)/2 m MACs per evaluated pair;
      inner  5 k MACs per applied rotation plus k^3/3 MACs (Cholesky) per pair;
      update digit form: products x 2 m K2^2 tensor flops per rotated pair;
             FP64 form: m k^2 MACs per rotated pair.
    """
    cplx = P.is_complex
    mac = 8.0 if cplx else 2.0
    m = P.m
    if not info["nbl"]:
        # plain form: one dot product and one column-pair rotation (3 m MACs)
        # for every column pair of every sweep, on the FP64 pipe
        ms, launches = times["plain_step"]
        work = info["sweeps"] * P.n * (P.n - 1) / 2 * 3.0 * m * mac
        achieved = work / (ms * 1e-3) / 1e12
        return {"kernel": "plain_step_kernel", "bound": "alu", "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "peak_source": "FP64: 152 SMs x 2 FMA/clk/SM x 2 flops x 2070 MHz (derived; 1.19 measured)",
                "ms_per_launch": ms / max(launches, 1), "launches": launches,
                "family_ms": {"plain_step": ms}}
    k = 2.0 * P.n / info["nbl"]
    K2 = 2 * k if cplx else k
    upd_digits = info.get("update_digits", 11)
    fam = {f: times[f] for f in ("gram", "inner", "update")}
    dom = max(fam, key=lambda f: fam[f][0])
    ms, launches = fam[dom]
    if dom == "gram":
        if gemm_gram_digits:
            work = info["pairs_evaluated"] * gram_products(8) * 2.0 * K2 * K2 * m
            bound, peak, unit, name = "tensor", peaks.get("bf16_tflops", 1900.0), "TFLOP/s", "gram_ozaki_kernel"
        else:
            work = info["pairs_evaluated"] * k * (k + 1) / 2 * m * mac
            bound, peak, unit, name = "alu", FP64_PEAK_TFLOPS, "TFLOP/s", "gram_fp64_kernel"
    elif dom == "inner":
        work = info["rotations"] * 5.0 * k * mac + info["pairs_evaluated"] * k ** 3 / 3 * mac
        bound, peak, unit, name = "alu", FP64_PEAK_TFLOPS, "TFLOP/s", "inner_smem_kernel"
    else:
        if gemm_upd_digits:
            # the kernel contracts all 64 real-form positions of a pivot
            work = info["pairs_rotated"] * update_products(upd_digits) * 2.0 * m * 64 * 64
            # narrow pivots with the full digit count run the TMA-fed kernel
            name = "update_narrow_kernel" if K2 <= 64 and upd_digits == 11 else "update_digits_kernel"
            bound, peak, unit = "tensor", peaks.get("bf16_tflops", 1900.0), "TFLOP/s"
        else:
            work = info["pairs_rotated"] * m * k * k * mac
            bound, peak, unit, name = "alu", FP64_PEAK_TFLOPS, "TFLOP/s", "update_fp64_kernel"
    achieved = work / (ms * 1e-3) / 1e12
    if bound == "tensor":
        src = ("measured bf16 burst of MEASURED_PEAKS.json (fp16 has the same dense rate)"
               if "bf16_tflops" in peaks else "fallback bf16 burst figure, 1.9 PFLOP/s (no measured peaks)")
    else:
        src = "FP64: 152 SMs x 2 FMA/clk/SM x 2 flops x 2070 MHz (derived; 1.19 measured)"
    roof = {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "peak_source": src,
            "ms_per_launch": ms / max(launches, 1), "launches": launches,
            "family_ms": {f: fam[f][0] for f in fam}}
    return roof


def run_ours(args):
    import numpy as np
    import torch

    import __graft_entry__
    import synth

    rank, world, local = _dist()
    __graft_entry__.build()
    from paper_1008_4166_gb300 import jjacobi as jj

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    P = synth.make_workload(args.workload, precision="f64")
    n, m = P.n, P.m
    cplx = P.is_complex
    dt_code = jj.JJ_C128 if cplx else jj.JJ_F64
    gemm = {"ozaki": jj.JJ_GEMM_OZAKI_FP16, "hybrid": jj.JJ_GEMM_OZAKI_GRAM,
            "fp64": jj.JJ_GEMM_FP64}[args.gemm]
    g_gram = jj.JJ_GEMM_FP64 if gemm == jj.JJ_GEMM_FP64 else jj.JJ_GEMM_OZAKI_FP16
    g_upd = jj.JJ_GEMM_OZAKI_FP16 if gemm == jj.JJ_GEMM_OZAKI_FP16 else jj.JJ_GEMM_FP64
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        G0 = torch.from_numpy(np.ascontiguousarray(P.G.T)).to("cuda").t()  # column-major
        Gw = torch.empty_like(G0)
        lam = torch.empty(n, dtype=torch.float64, device="cuda")
    strat = {"full": jj.JJ_FULL_BLOCK, "oriented": jj.JJ_BLOCK_ORIENTED}[args.strategy]
    pf = jj.JJ_PIVOT_SPECIAL if args.pivot_factor == "special" else jj.JJ_PIVOT_CHOLESKY
    h = jj.Handle(m, n, dt_code, block_width=args.block_width, gemm=gemm, stream=stream,
                  block_strategy=strat, max_sweeps=args.max_sweeps, ozaki_slices=args.digits,
                  pivot_factor=pf, inner_block_width=args.inner_block_width)
    ok = (jj.JJ_OK, jj.JJ_NOT_CONVERGED) if args.max_sweeps else (jj.JJ_OK,)

    def step():
        Gw.copy_(G0)
        info = h.jjacobi_solve(Gw, Gw.stride(1), P.J, allow=ok)
        h.jjacobi_extract(lam, None, 0, 0)
        return info

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            info = step()
    stream.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = ClockSampler(local)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    with torch.cuda.stream(stream):
        stream.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            infos.append(step().as_dict())
        e1.record(stream)
    stream.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    info = infos[-1]
    if info["nbl"]:
        flops = blocked_flops(n, m, cplx, info)
        flops_all = blocked_flops_all_pairs(n, m, cplx, info)
    else:  # plain form
        flops = flops_all = plain_flops(n, m, cplx, info["sweeps"])
    value = flops * world / (ms * 1e-3) / 1e9
    launches = sum(x["kernel_launches"] + 1 for x in infos)  # + extraction kernel
    lam_blocked = lam.cpu().numpy().copy()

    # end to end through the C ABI with host buffers (pinned), copies timed
    Gh = torch.from_numpy(np.ascontiguousarray(P.G.T)).pin_memory().numpy().T
    esz = 16 if cplx else 8
    t0 = time.perf_counter()
    e2e_steps = 1
    for _ in range(e2e_steps):
        lam_h, _, _ = h.jjacobi_solve_host(Gh, P.J, want_U=False, allow=ok)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": flops / e2e_s / 1e9, "unit": "GFLOP/s",
           "h2d_bytes_per_step": int(m * n * esz), "d2h_bytes_per_step": int(n * 8)}

    # per-kernel device times from a profiled solve of the first sweeps (events
    # around every kernel family of every step, on the solve's stream) and the
    # dominant kernel's roofline
    hp_ = jj.Handle(m, n, dt_code, block_width=args.block_width, gemm=gemm, stream=stream,
                    profile=True, max_sweeps=args.profile_sweeps, block_strategy=strat,
                    ozaki_slices=args.digits, pivot_factor=pf, inner_block_width=args.inner_block_width)
    with torch.cuda.stream(stream):
        Gw.copy_(G0)
        pinfo_ = hp_.jjacobi_solve(Gw, Gw.stride(1), P.J, allow=(jj.JJ_OK, jj.JJ_NOT_CONVERGED))
    stream.synchronize()
    times = hp_.jjacobi_kernel_times()
    hp_.close()
    roof = kernel_roofline(jj, P, times, dict(pinfo_.as_dict(), update_digits=args.digits or 11),
                           g_gram == jj.JJ_GEMM_OZAKI_FP16,
                           g_upd == jj.JJ_GEMM_OZAKI_FP16, _peaks())
    # DRAM bytes per launch from the ncu capture of the same kernel (one step of
    # this workload; per launch, like `achieved`), null once the kernel changed
    roof["traffic"] = captured_traffic(roof["kernel"])

    # the plain form on the same input, same accuracy target
    plain = None
    if args.plain and rank == 0:
        hp = jj.Handle(m, n, dt_code, block_width=0, stream=stream)
        with torch.cuda.stream(stream):
            Gw.copy_(G0)
            ep0, ep1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ep0.record(stream)
            pinfo = hp.jjacobi_solve(Gw, Gw.stride(1), P.J)
            ep1.record(stream)
            hp.jjacobi_extract(lam, None, 0, 0)
        stream.synchronize()
        lam_plain = lam.cpu().numpy()
        pi = pinfo.as_dict()
        rel = float(np.max(np.abs(np.sort(lam_blocked) - np.sort(lam_plain)) / np.abs(np.sort(lam_plain))))
        plain = {"time_to_solution_s": ep0.elapsed_time(ep1) / 1e3, "sweeps": pi["sweeps"],
                 "gflops": plain_flops(n, m, cplx, pi["sweeps"]) / (ep0.elapsed_time(ep1) * 1e-3) / 1e9,
                 "speedup_blocked_vs_plain": (ep0.elapsed_time(ep1)) / ms,
                 "max_rel_eig_diff_blocked_vs_plain": rel}
        hp.close()
    h.close()

    cpu = cpu_threads = None
    if rank == 0 and world == 1 and not args.no_cpu:
        g, ncol, dt = cpu_baseline(P, budget_s=15.0)
        cpu = {"value": g, "unit": "GFLOP/s", "cores": 1, "kind": "oracle", "cpu": cpu_model(),
               "sample": f"one row-cyclic plain sweep on the leading {ncol} columns (all {m} rows) "
                         f"of the n={n} input, {dt:.1f} s"}
        g, ncol, dt, nt = cpu_baseline_threads(P, budget_s=10.0)
        cpu_threads = {"value": g, "unit": "GFLOP/s", "cores": nt, "cpu": cpu_model(),
                       "kind": "round-robin plain method on all host cores (pthreads)",
                       "sample": f"one round-robin plain sweep on the leading {ncol} columns "
                                 f"(all {m} rows) of the n={n} input, {dt:.1f} s"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": dict(bench_config(args, P, world), sweeps=info["sweeps"],
                           steps_per_sweep=info["steps_per_sweep"], time_to_solution_s=ms / 1e3,
                           max_sweeps=args.max_sweeps or None,
                           flops="executed work: Gram per evaluated pair, update per rotated pair",
                           pairs_evaluated=info["pairs_evaluated"],
                           pairs_rotated=info["pairs_rotated"],
                           gflops_if_every_pair_were_recomputed=flops_all * world / (ms * 1e-3) / 1e9),
            "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clocks, "plain": plain, "cpu_baseline_threads": cpu_threads,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_one_step(args):
    """One parallel step (every block pair of step 1 of the round-robin order)
    through the building-block entry points, repeated --steps times."""
    import numpy as np
    import torch

    import __graft_entry__
    import synth

    __graft_entry__.build()
    from paper_1008_4166_gb300 import jjacobi as jj

    P = synth.make_workload(args.workload, precision="f64")
    n, m, cplx = P.n, P.m, P.is_complex
    dt_code = jj.JJ_C128 if cplx else jj.JJ_F64
    g_gram = jj.JJ_GEMM_FP64 if args.gemm == "fp64" else jj.JJ_GEMM_OZAKI_FP16
    g_upd = jj.JJ_GEMM_OZAKI_FP16 if args.gemm == "ozaki" else jj.JJ_GEMM_FP64
    b = args.block_width
    nbl = 2 * ((n + 2 * b - 1) // (2 * b))
    sizes = [n // nbl + (1 if l < n % nbl else 0) for l in range(nbl)]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    tab = jj.jjacobi_schedule(nbl, 0, 1)
    pairs = np.array([[offs[i], sizes[i], offs[j], sizes[j]] for i, j in tab[0]], dtype=np.int32)
    kmax = 2 * max(sizes)
    E = 2 if cplx else 1
    G = torch.from_numpy(np.ascontiguousarray(P.G.T)).to("cuda").t()
    Gd = torch.empty_like(G)
    pd = torch.from_numpy(pairs).cuda()
    A = torch.zeros(len(pairs) * kmax * kmax * E, dtype=torch.float64, device="cuda")
    W = torch.zeros_like(A)
    Jd = torch.from_numpy(P.J.astype(np.int8)).cuda()
    cnt = torch.zeros(8, dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for it in range(args.warmup + args.steps):
        if it == args.warmup:
            e0.record(st)
        jj.jjk_gram(dt_code, g_gram, G, G.stride(1), m, pd, len(pairs), A, kmax)
        jj.jjk_inner(dt_code, A, W, kmax, pd, len(pairs), Jd, 0.0, 30, 0, cnt)
        jj.jjk_update(dt_code, g_upd, G, Gd, G.stride(1), m, pd, len(pairs), W, kmax)
    e1.record(st)
    torch.cuda.synchronize()
    print(json.dumps({"one_step": args.workload, "block_width": b, "gemm": args.gemm,
                      "pairs": len(pairs), "kmax": kmax,
                      "ms_per_step": e0.elapsed_time(e1) / max(args.steps, 1),
                      "rotations": int(cnt[0]), "err_flags": int(cnt[2])}), flush=True)


def run_batched(args):
    """The batched workload: every step solves all problems (copies of the
    resident inputs) in one jjacobi_solve_batched call."""
    import numpy as np
    import torch

    import __graft_entry__
    import synth

    __graft_entry__.build()
    from paper_1008_4166_gb300 import jjacobi as jj

    probs = synth.make_batched(count=args.batch_count, precision="f64")
    gemm = {"ozaki": jj.JJ_GEMM_OZAKI_FP16, "hybrid": jj.JJ_GEMM_OZAKI_GRAM,
            "fp64": jj.JJ_GEMM_FP64}[args.gemm]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        G0 = [torch.from_numpy(np.ascontiguousarray(P.G.T)).to("cuda").t() for P in probs]
        Gw = [torch.empty_like(g) for g in G0]
        lam = torch.empty(sum(P.n for P in probs), dtype=torch.float64, device="cuda")
    mmax = max(P.m for P in probs)
    nmax = max(P.n for P in probs)
    bw = args.block_width if args.block_width_set else 0
    strat = {"full": jj.JJ_FULL_BLOCK, "oriented": jj.JJ_BLOCK_ORIENTED}[args.strategy]
    h = jj.Handle(mmax, nmax, jj.JJ_C128, block_width=bw, gemm=gemm, stream=stream,
                  block_strategy=strat)

    def step():
        for a, b in zip(Gw, G0):
            a.copy_(b)
        return h.jjacobi_solve_batched(Gw, [P.J for P in probs], lam)[1]

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()
    clk = ClockSampler(0)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(args.steps):
            infos = step()
        e1.record(stream)
    stream.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / args.steps
    # per-problem pair counters of a batch are batch totals: every pair of every
    # step of each problem's sweeps is charged here
    flops = sum(blocked_flops_all_pairs(P.n, P.m, True, i.as_dict()) for P, i in zip(probs, infos)
                if i.nbl > 0)
    sweeps = [i.sweeps for i in infos]
    line = {
        "metric": "batched J-Jacobi GFLOP/s and problems/s", "value": flops / (ms * 1e-3) / 1e9,
        "unit": "GFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "batched_c128_512x", "problems": len(probs),
                   "n_range": [min(P.n for P in probs), nmax], "gemm": args.gemm,
                   "strategy": args.strategy,
                   "block_widths": sorted(set(i.block_width for i in infos)),
                   "problems_per_s": len(probs) / (ms * 1e-3),
                   "sweeps_min_max": [min(sweeps), max(sweeps)],
                   "launches_per_solve": infos[0].kernel_launches},
        "clocks": clocks,
    }
    h.close()
    print(json.dumps(line), flush=True)


def make_threelevel_on_gpu(torch, synth):
    """The 16384-column real recipe (synth's "threelevel_f64_n16384_b128": the
    same seed, the same draws in the same order) with its two expensive steps
    on the GPU: the QR of the Ginibre matrix (cuSOLVER through torch) and the
    65536 column rotations. The exact eigenvalues are J |Lambda| as in the host
    recipe; the bits of G differ from the host recipe's by rounding only."""
    import math
    import numpy as np
    w = synth.WORKLOADS["threelevel_f64_n16384_b128"]
    n, npos = w["n"], w["npos"]
    rng = np.random.Generator(np.random.PCG64(w["seed"]))
    Z = torch.from_numpy(rng.standard_normal((n, n))).cuda()
    Q, R = torch.linalg.qr(Z)
    del Z
    Q = Q * torch.sign(torch.diagonal(R))[None, :]
    del R
    mag = np.exp(rng.uniform(math.log(w["lam"][0]), math.log(w["lam"][1]), n))
    J = np.ones(n, dtype=np.int8)
    J[npos:] = -1
    draws = synth.random_rotation_draws(n, J, w["rots"], w["smax"], rng, False)
    G = Q * torch.from_numpy(np.sqrt(mag)).cuda()[None, :]
    del Q
    for (r, s_, hyper, par, ph) in draws:
        if hyper:
            a, b = math.sqrt(1.0 + par * par), par
            gr, gs = G[:, r].clone(), G[:, s_].clone()
            G[:, r] = a * gr + b * gs
            G[:, s_] = b * gr + a * gs
        else:
            a, b = math.cos(par), math.sin(par)
            gr, gs = G[:, r].clone(), G[:, s_].clone()
            G[:, r] = a * gr - b * gs
            G[:, s_] = b * gr + a * gs
    G = G.t().contiguous().t()  # column-major
    torch.cuda.synchronize()
    return G, J, J.astype(np.float64) * mag


def run_threelevel(args):
    """The three-level workload (real, n = 16384, b = 128, inner blocks of 16):
    one solve (or --max-sweeps sweeps of it), against the plain form's sweeps."""
    import numpy as np
    import torch

    import __graft_entry__
    import synth

    __graft_entry__.build()
    from paper_1008_4166_gb300 import jjacobi as jj

    t0 = time.time()
    if args.gpu_input:
        Gsrc, Jv, lam_exact = make_threelevel_on_gpu(torch, synth)
        P = synth.Problem(G=None, J=Jv, lam_exact=lam_exact, name="threelevel_gpu_input", seed=1004,
                          graded=False)
    else:
        P = synth.make_workload("threelevel_f64_n16384_b128", precision="f64")
        Gsrc = None
    gen_s = time.time() - t0
    # progress on stderr: generation and every form as it finishes (a long run
    # that is stopped still leaves its finished forms)
    print(json.dumps({"generation_s": gen_s}), file=sys.stderr, flush=True)
    n, m = (Gsrc.shape[1], Gsrc.shape[0]) if Gsrc is not None else (P.n, P.m)
    gemm = {"ozaki": jj.JJ_GEMM_OZAKI_FP16, "hybrid": jj.JJ_GEMM_OZAKI_GRAM,
            "fp64": jj.JJ_GEMM_FP64}[args.gemm]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        G0 = Gsrc if Gsrc is not None else torch.from_numpy(np.ascontiguousarray(P.G.T)).to("cuda").t()
        Gw = torch.empty_like(G0)
    out = {}
    lam = torch.empty(n, dtype=torch.float64, device="cuda")
    for name, kw in (("three_level", dict(block_width=128, inner_block_width=16, gemm=gemm)),
                     ("three_level_oriented", dict(block_width=128, inner_block_width=16, gemm=gemm,
                                                   block_strategy=jj.JJ_BLOCK_ORIENTED)),
                     ("two_level", dict(block_width=128, gemm=jj.JJ_GEMM_FP64)),
                     ("plain", dict(block_width=0))):
        if name not in args.forms.split(","):
            continue
        h = jj.Handle(m, n, jj.JJ_F64, stream=stream, max_sweeps=args.max_sweeps, **kw)
        with torch.cuda.stream(stream):
            Gw.copy_(G0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = h.jjacobi_solve(Gw, Gw.stride(1), P.J, allow=(jj.JJ_OK, jj.JJ_NOT_CONVERGED))
            e1.record(stream)
        stream.synchronize()
        d = info.as_dict()
        s = e0.elapsed_time(e1) / 1e3
        out[name] = {"seconds": s, "sweeps": d["sweeps"], "s_per_sweep": s / max(d["sweeps"], 1),
                     "status": d["status"], "rotations": d["rotations"]}
        if d["status"] == jj.JJ_OK and P.lam_exact is not None:
            # eigenvalues against the construction J |Lambda| (sorted: lambda comes
            # out in column order)
            with torch.cuda.stream(stream):
                h.jjacobi_extract(lam, None, 0, 1)
            stream.synchronize()
            got = np.sort(lam.cpu().numpy())
            ref = np.sort(np.asarray(P.lam_exact, dtype=np.float64))
            out[name]["max_rel_err_vs_construction"] = float(np.max(np.abs(got - ref) / np.abs(ref)))
        print(json.dumps({name: out[name]}), file=sys.stderr, flush=True)
        h.close()
    print(json.dumps({"workload": "threelevel_f64_n16384_b128", "gemm": args.gemm,
                      "generation_s": gen_s, "max_sweeps": args.max_sweeps, "forms": out}),
          flush=True)


def run_study(args):
    """Two studies on the graded complex recipe (one solve per point, CUDA events):
    round-robin against modulus ordering at the headline size, and the plain
    form against the blocked forms over n (the crossover; time / n^3)."""
    import numpy as np
    import torch

    import __graft_entry__
    import synth

    __graft_entry__.build()
    from paper_1008_4166_gb300 import jjacobi as jj

    def solve(P, **kw):
        G = torch.from_numpy(np.ascontiguousarray(P.G.T)).to("cuda").t()
        with jj.Handle(P.m, P.n, jj.JJ_C128, **kw) as h:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            info = h.jjacobi_solve(G, G.stride(1), P.J)
            e1.record()
            torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, info.sweeps

    out = {"orders": {}, "crossover": {}}
    hyb = dict(block_width=16, gemm=jj.JJ_GEMM_OZAKI_GRAM, block_strategy=jj.JJ_BLOCK_ORIENTED)
    dig = dict(block_width=16, gemm=jj.JJ_GEMM_OZAKI_FP16, block_strategy=jj.JJ_BLOCK_ORIENTED)
    if "orders" in args.study:
        P = synth.make_workload("graded_c128_n4096_b64", precision="f64")
        for name, order in (("round_robin", jj.JJ_ORDER_ROUND_ROBIN), ("modulus", jj.JJ_ORDER_MODULUS)):
            t, sw = solve(P, order=order, **hyb)
            out["orders"][name] = {"seconds": t, "sweeps": sw}
        print(json.dumps(out), flush=True)
    if "crossover" in args.study:
        for n in (256, 512, 1024, 2048):
            P = synth.make_workload("graded_c128_n4096_b64", n=n, precision="f64")
            row = {}
            for name, kw in (("plain", dict(block_width=0)), ("blocked_hybrid", hyb), ("blocked_digit", dig)):
                t, sw = solve(P, **kw)
                row[name] = {"seconds": t, "sweeps": sw, "c_ns_per_n3": t / n ** 3 * 1e9}
            out["crossover"][n] = row
            print(json.dumps({"n": n, **row}), flush=True)
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--block-width", type=int, default=16)
    ap.add_argument("--inner-block-width", type=int, default=0,
                    help="inner block width: the three-level form (e.g. --block-width 64 --inner-block-width 16)")
    ap.add_argument("--gemm", default="ozaki", choices=["hybrid", "ozaki", "fp64"])
    ap.add_argument("--pivot-factor", default="cholesky", choices=["cholesky", "special"],
                    help="full-block pivot factor: Cholesky of the pivot, or (3.9)-(3.11)")
    ap.add_argument("--digits", type=int, default=0,
                    help="digits per operand of the split-precision update (0: 11)")
    ap.add_argument("--strategy", default="oriented", choices=["oriented", "full"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-plain", dest="plain", action="store_false")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ref-budget", type=float, default=6.0)
    ap.add_argument("--profile-sweeps", type=int, default=3)
    ap.add_argument("--one-step", action="store_true")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--max-sweeps", type=int, default=0,
                    help="cap the sweeps of each solve (0: to convergence; for short profiling runs)")
    ap.add_argument("--forms", default="three_level,three_level_oriented,two_level,plain")
    ap.add_argument("--gpu-input", action="store_true",
                    help="three-level workload: build the input's QR and rotations on the GPU")
    ap.add_argument("--study", default="", help="orders,crossover: ordering and crossover studies")
    args = ap.parse_args()
    args.block_width_set = any(a.startswith("--block-width") for a in sys.argv[1:])
    if args.study:
        run_study(args)
    elif args.one_step:
        run_one_step(args)
    elif args.workload == "batched_c128_512x":
        run_batched(args)
    elif args.workload == "threelevel_f64_n16384_b128":
        run_threelevel(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
