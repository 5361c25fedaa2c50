"""Host-side logic of bench.py (no GPU): the algorithmic flop conventions, the
traffic lookup keyed to kernel sources, the clock sampler's parsing, the
reference arm's JSON line (the oracle on a bounded sample) and the
multithreaded CPU baseline's sampler."""
import json
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_blocked_flop_convention():
    # executed work: Gram k(k+1)/2 m MACs per evaluated pair, update m k^2 MACs
    # per rotated pair, 5 k MACs per inner rotation; complex MAC = 8 flops
    info = {"nbl": 2, "sweeps": 4, "steps_per_sweep": 1, "rotations": 3,
            "pairs_evaluated": 3, "pairs_rotated": 2}
    n, m = 8, 10
    k = 2.0 * n / 2
    expect = 8.0 * (3 * k * (k + 1) / 2 * m + 2 * m * k * k + 3 * 5.0 * k)
    assert bench.blocked_flops(n, m, True, info) == pytest.approx(expect)
    assert bench.blocked_flops(n, m, False, info) == pytest.approx(expect / 4.0)
    # every pair of every step of every sweep: 4 sweeps x 1 step x 1 pair
    every = 8.0 * (4 * (k * (k + 1) / 2 * m + m * k * k) + 3 * 5.0 * k)
    assert bench.blocked_flops_all_pairs(n, m, True, info) == pytest.approx(every)


def test_plain_flop_convention():
    # n(n-1)/2 pairs per sweep, 3 m MACs each (dot + two rotated columns)
    assert bench.plain_flops(4, 10, True, 2) == pytest.approx(8.0 * 2 * 6 * 3 * 10)


def test_captured_traffic_is_void_once_the_kernel_source_changes(tmp_path, monkeypatch):
    fake = tmp_path / "repo"
    (fake / "profiles").mkdir(parents=True)
    csrc = fake / "paper_1008_4166_gb300" / "csrc"
    csrc.mkdir(parents=True)
    import hashlib
    h = hashlib.sha256()
    for f in ("jj_update.cu", "jj_common.cuh"):
        shutil.copy(os.path.join(ROOT, "paper_1008_4166_gb300", "csrc", f), csrc / f)
        h.update(open(csrc / f, "rb").read())
    with open(fake / "profiles" / "traffic.txt", "w") as fh:
        fh.write("# kernel bytes files hash\n")
        fh.write(f"update_fp64_kernel 123456 jj_update.cu,jj_common.cuh {h.hexdigest()[:16]}\n")
    monkeypatch.setattr(bench, "ROOT", str(fake))
    assert bench.captured_traffic("update_fp64_kernel") == 123456
    assert bench.captured_traffic("no_such_kernel") is None
    with open(csrc / "jj_update.cu", "a") as fh:
        fh.write("// edited\n")
    assert bench.captured_traffic("update_fp64_kernel") is None


def test_clock_sampler_parses_reasons():
    s = bench.ClockSampler(0)

    class _P:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s.proc = _P()
    s.lines = ["2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
               "2055, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
               "garbage line"]
    out = s.stop()
    assert out["sm_max_mhz"] == 2070.0
    assert out["sm_mhz"] == pytest.approx((2070 + 2055) / 2)
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 2


def test_reference_arm_line_matches_the_measured_arm_config():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--ref-budget", "1.5"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["unit"] == "GFLOP/s" and line["higher_is_better"] is True and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"] == {"value": line["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}

    class _A:
        workload = bench.WORKLOAD
        block_width = 16
        gemm = "ozaki"
        digits = 0
        strategy = "oriented"
        pivot_factor = "cholesky"

    class _P:
        m = n = 4096

    assert line["config"] == bench.bench_config(_A, _P)
    assert line["metric"] == bench.METRIC


def test_threaded_cpu_baseline_sampler_grows_to_the_budget():
    import synth

    P = synth.make_workload("plain_c128_n128", precision="f64")
    g, ncol, dt, nt = bench.cpu_baseline_threads(P, budget_s=0.01)
    assert g > 0 and nt >= 1 and ncol == 64 and dt > 0  # the first sample already exceeds it
    g, ncol, dt, nt = bench.cpu_baseline_threads(P, budget_s=1e9)
    assert ncol == P.n  # grown to the whole input, then stopped


def test_measured_arm_line_carries_every_contract_key():
    """The JSON line of the default run (run_ours) is built from one dict
    literal; it names every key the benchmark contract asks for. (Checked on the
    source: the run itself needs a GPU.)"""
    import ast

    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    fn = next(n for n in tree.body if isinstance(n, ast.FunctionDef) and n.name == "run_ours")
    keys = set()
    for node in ast.walk(fn):
        if (isinstance(node, ast.Assign) and any(getattr(t, "id", None) == "line"
                                                 for t in node.targets)
                and isinstance(node.value, ast.Dict)):
            keys |= {k.value for k in node.value.keys if isinstance(k, ast.Constant)}
    required = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "roofline", "cpu_baseline", "e2e", "clocks", "gpu_launches"}
    assert required <= keys, required - keys


def test_kernel_roofline_picks_the_dominant_family_and_its_peak():
    class _P:
        is_complex = True
        m = n = 4096

    info = {"nbl": 256, "pairs_evaluated": 1000, "pairs_rotated": 800, "rotations": 5000}
    times = {"gram": (10.0, 5), "inner": (2.0, 5), "update": (50.0, 5)}
    r = bench.kernel_roofline(None, _P, times, info, True, False, {"bf16_tflops": 1919.0})
    k = 2.0 * 4096 / 256
    assert r["kernel"] == "update_fp64_kernel" and r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(800 * 4096 * k * k * 8.0 / 50e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"]) and r["unit"] == "TFLOP/s"
    assert r["ms_per_launch"] == pytest.approx(10.0)
    times = {"gram": (60.0, 5), "inner": (2.0, 5), "update": (50.0, 5)}
    r = bench.kernel_roofline(None, _P, times, info, True, False, {"bf16_tflops": 1919.0})
    assert r["kernel"] == "gram_ozaki_kernel" and r["bound"] == "tensor" and r["peak"] == 1919.0
    assert "measured" in r["peak_source"]
    r = bench.kernel_roofline(None, _P, times, info, True, False, {})
    assert r["peak"] == 1900.0 and "fallback" in r["peak_source"]
