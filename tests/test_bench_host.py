"""Host-side legs of bench.py (no GPU): the CPU-oracle baselines and the
reference arm's JSON line.

The reference arm times the FP64 oracle's closed loop (plain joint
bisection, Alg. 1 on all scenarios) on the host cores and prints one JSON
line with the contract's keys; the CPU baselines of the batched and sweep
workloads report the threaded oracle and the sequential one beside it.
"""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["steps"] == 1 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_sweep_cpu_baseline_reports_threaded_and_one_core():
    from paper_2510_08288_gb300 import inputs
    c = bench.sweep_cpu(inputs.fc3_params(), 0.01, 2)
    assert c["kind"] == "oracle" and c["cores"] == 2 and c["value"] > 0
    assert c["one_core"]["cores"] == 1 and c["one_core"]["value"] > 0
    assert c["unit"] == c["one_core"]["unit"] == "trajectory-steps/s"
    json.dumps(c)


def test_batch_cpu_baseline_reports_threaded_and_one_core():
    from oracle import oracle as O
    from paper_2510_08288_gb300 import inputs
    p = inputs.fc3_params()
    b = inputs.batched_instances(bench.BATCH_S, bench.BATCH_SEED)
    x0 = np.array([O.equilibrium(p, v) for v in b["v_prev"]]) * b["xfac"]
    c = bench.batch_cpu(p, b, x0, b["r"], 0.01, 2)
    assert c["kind"] == "oracle" and c["cores"] == 2 and c["value"] > 0
    one = c["one_core"]
    assert one["cores"] == 1 and one["value"] > 0 and one["threaded_same_instances"] > 0
    json.dumps(c)


def test_closed_loop_cpu_legs_agree_and_serialise():
    from oracle import oracle as O
    from paper_2510_08288_gb300 import inputs
    x0 = O.equilibrium(inputs.fc3_params(), bench.V0)
    r = inputs.staircase(1000, 8, 125, bench.SEED)
    val, n, secs, kaps, first = bench.cpu_oracle_closed_loop(x0, r, 0.01, 2)
    assert n == 1 and val > 0 and first > 0
    v1, k1 = bench.cpu_oracle_one_core(x0, r)
    assert v1 > 0 and k1 == float(kaps[0])  # thread count does not change the oracle's result
    json.dumps({"value": val, "one_core": v1, "kappa": k1})


def test_adjoint_cpu_baseline_runs_whole_gradients():
    from oracle import oracle as O
    from paper_2510_08288_gb300 import inputs
    p = inputs.fc3_params()
    w = inputs.WORKLOADS["adjoint"]
    x_t = O.equilibrium(p, 100.0)
    c = bench.adjoint_cpu(p, x_t, 100.0, 250.0, w["N"], w["H"], 0.01, [-1, -1])
    assert c["kind"] == "oracle" and c["cores"] == 1 and c["value"] > 0
    assert c["argmin_equal_to_gpu_fp64"] is False  # no scenario has index -1
    json.dumps(c)


def test_traffic_guard_drops_figures_of_changed_sources():
    """A profiled DRAM figure is reported only while the hashed source regions
    are the ones profiled."""
    assert bench.measured_traffic((("bench.py", None, None, "0" * 40),), 123) is None
    assert bench.measured_traffic((("bench.py", "no such marker", "x", "0" * 40),), 123) is None
    import hashlib
    sha = hashlib.sha1(bench.source_region("bench.py", None, None).encode("utf-8")).hexdigest()
    assert bench.measured_traffic((("bench.py", None, None, sha),), 123) == 123


def test_closed_loop_window_crosses_the_first_level_change():
    """The timed window opens at update 115 (the staircase's first level change
    is at 125) unless the W warm-up updates or the K timed ones do not fit."""
    assert bench.window_start(5, 20) == 115
    assert bench.window_start(3, 100) == 115
    assert bench.window_start(200, 20) == 200          # the warm-up comes first
    assert bench.window_start(5, 990) == 10             # the window stays inside the run
    c = bench.workload_config(115, 5, 20)
    assert "timed updates [115, 135)" in c["workload"] and "[110, 115) warm up" in c["workload"]


def test_sweep_issue_ceiling_follows_the_kernel_that_ran():
    """The sweep line's issue ceiling is the one of the kernel that fed most of
    the top row's steps: the TMA ring (110 instructions per trajectory-step)
    or the register ring (114)."""
    tma = bench.sweep_ceiling({"tma_step_fraction": 1.0})
    regs = bench.sweep_ceiling({"tma_step_fraction": 0.0})
    assert abs(tma - bench.FLOPS_PER_STEP / (2.0 * bench.TMA_INSTR_PER_STEP)) < 1e-12
    assert abs(regs - bench.ISSUE_CEILING) < 1e-12
    assert tma > regs


def test_batch_kernel_names():
    assert bench.batch_kernel_name((bench.BATCH_PAIR_VARIANT, 32, 8)).startswith("batch_rollout_warp_pair_kernel<8>")
    assert bench.batch_kernel_name((7, 32, 16)) == "batch_rollout_warp_kernel<16>"
    assert bench.batch_kernel_name((3, 128, 16)) == "batch_rollout_kernel<128, 16>"
    assert bench.batch_kernel_name((bench.BATCH_SPLIT_VARIANT, 16, 8)).startswith("batch_rollout_split_kernel<8>")
    assert bench.batch_ceiling((bench.BATCH_SPLIT_VARIANT, 16, 8)) is None
    assert bench.batch_ceiling((7, 32, 16)) == bench.ISSUE_CEILING


def test_apply_tma_leaves_handles_without_a_tma_ring_alone():
    """--tma auto|always on a handle that has no TMA ring (n_scenarios not a
    multiple of 4) keeps it off instead of failing; never is always set."""
    class FakeR:
        TMA_NEVER, TMA_AUTO, TMA_ALWAYS = 0, 1, 2

    class FakeGov:
        def __init__(self, available):
            self.mode = FakeR.TMA_AUTO if available else FakeR.TMA_NEVER
            self.calls = []

        def get_tma(self):
            return self.mode

        def set_tma(self, mode):
            self.calls.append(mode)
            self.mode = mode

    g = FakeGov(available=False)
    bench.apply_tma(FakeR, g, FakeR.TMA_ALWAYS)
    assert g.calls == [] and g.get_tma() == FakeR.TMA_NEVER
    bench.apply_tma(FakeR, g, FakeR.TMA_NEVER)
    assert g.calls == [FakeR.TMA_NEVER]
    g = FakeGov(available=True)
    bench.apply_tma(FakeR, g, FakeR.TMA_ALWAYS)
    assert g.calls == [FakeR.TMA_ALWAYS]
    assert bench.TMA_MODES == ("never", "auto", "always") and len(bench.TMA_NAMES) == 3
