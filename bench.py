#!/usr/bin/env python
"""Benchmark of the robust reference governor on one GB300 (or N replicas).

Workload: the closed-loop RG run with 1,024 disturbance scenarios and a
2,000-step RK4 horizon (dt = 0.01 s) on the FC3 fuel-cell air-path model, the
reference a seeded 8-level staircase over 50..300 A held 125 updates per
level.  One benchmark step is one closed-loop update: redraw the scenarios,
run the robust RG search (speculative bisection, N_kappa = 12, binary32
rollouts with a binary64 recheck of near-zero slacks), move the simulated
plant one step.  W warm-up updates run first; the K timed updates are the
next K of the same run, each a replay of the library's one-update CUDA graph
(rrg_closed_loop_dev with the graph on; the rounds after the pipelined pair
sit in a conditional node).

Printed (rank 0): one JSON line.  value = RG updates/s over all ranks, device
time (CUDA events on the library's stream, inputs resident in HBM, L2 flushed
between timed steps).  direct_launches = the same K updates with every kernel
launched directly; its CUDA events around each rollout launch give the
roofline's kernel duration.  e2e = the same through the host-buffer C-ABI calls
(rrg_sample_scenarios + rrg_step + rrg_plant_step, host copies included).
roofline = the binary32 rollout kernel's achieved FP32 rate vs the FP32 FMA
peak derived from the device's SM count x 128 lanes x 2 flop x the SM clock
sampled during the timed region.  cpu_baseline = the
FP64 CPU oracle (plain joint bisection) on a bounded prefix of the same run.

--impl reference times that oracle alone (the CPU arm) on the same workload.

--workload sweep: the large-sweep workload instead, one RG update per step
(k-section with 16 kappa candidates per round, 3 rounds, binary32 rollouts
with the binary64 recheck) over N_sim = 1,024 ... 65,536 scenarios, each with
per-step disturbances and per-scenario parametric uncertainty (+-10 % on the
uncertain FC3 parameters), horizon 5,000 steps; one JSON line with
trajectory-steps/s per N.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RG updates/s & trajectory-steps/s at stated kappa tol; FP32+adjoint vs plain FP64 bisect"
UNIT = "RG updates/s"
N_SCEN, HORIZON, N_BISECT, M_CAND = 1024, 2000, 12, 64
SEED, V0 = 1, 100.0
RECHECK_EPS_REL = 1e-6
RUN_UPDATES = 1000
# The timed window of the closed loop opens at update 115, ten updates before
# the staircase's first level change (update 125): the timed updates include
# the large kappas and the binary64 rechecks of a reference step.  The
# updates before it run untimed (the last W of them are the warm-up).
WINDOW_START = 115
PROBE_STEPS = 128
# algorithmic binary32 flops of one trajectory step, counted from the source
# of the rollout's right-hand side with its constants multiplied out: 4
# right-hand sides of 24 (3 MUFU operations counted as one flop each), 3
# stage points of 6, the RK4 combination of 18, the disturbance add of 3, and
# output, slack, running min and the finiteness accumulator of 6
FLOPS_PER_STEP = 141
# MUFU operations per binary32 trajectory step: per right-hand side the power
# term's lg2 and ex2 and the torque term's reciprocal, 4 evaluations per step
MUFU_PER_STEP = 12
# instructions a warp issues per trajectory step in the register-ring loop
# (ncu: instructions executed by the 65,536-scenario sweep's rollout launches
# at 32,768 scenarios over their lane-steps / 32, parametric and nominal
# model alike): an issue-bound step reaches at most 141 / (2 x 114) of the
# derived FP32 peak, which counts every instruction as an FMA
INSTR_PER_STEP = 114
ISSUE_CEILING = FLOPS_PER_STEP / (2.0 * INSTR_PER_STEP)
FP32_LANES_PER_SM = 128


def fp32_peak(clk):
    """FP32 FMA peak in TFLOP/s from unit counts and clocks: the device's SM
    count (queried) x 128 FP32 lanes x 2 flop per FMA x the median SM clock
    sampled during the timed region (the maximum SM clock nvidia-smi reports
    when no sample fell inside it); returns (peak, source)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz, how = clk.get("sm_mhz"), "median sampled SM clock"
    if not mhz:
        mhz, how = clk.get("sm_max_mhz"), "maximum SM clock (no sample in the timed region)"
    if not mhz:
        return None, "no SM clock available from nvidia-smi"
    peak = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    return peak, "derived: %d SMs x %d FP32 lanes x 2 flop/FMA x %.0f MHz (%s)" % (
        sms, FP32_LANES_PER_SM, mhz, how)


def frac_of(a, b):
    return (a / b) if (a is not None and b) else None
L2_FLUSH_BYTES = 256 << 20
# large sweep: N_sim 1K..64K, 16 candidates, horizon 5,000, parametric uncertainty
SWEEP_N = (1024, 2048, 4096, 8192, 16384, 32768, 65536)
SWEEP_H, SWEEP_M, SWEEP_ROUNDS = 5000, 16, 3
SWEEP_CASE = (100.0, 150.0)     # v_prev, r_t: x_t at the equilibrium of v_prev
# DRAM bytes per rollout launch on this workload (ncu, one pass over one
# update's four launches with the tuned shape 64 nodes / 32-step probe:
# probe, continuation + round 2, two no-op rounds), valid while the
# rollout's sources are the ones profiled: the trajectory loops and model
# (rrg_lane.cuh, rrg_device.cuh), the rollout kernels and their dispatch in
# rrg_kernels.cu, and the Launch struct (sha1 of each region)
TRAFFIC_PER_LAUNCH = (433664 + 24614656 + 35840 + 35584) / 4
TRAFFIC_SOURCES = (
    ("paper_2510_08288_gb300/csrc/rrg_lane.cuh", None, None, "bb86588f91e49ec177d60d8ba804f8f0da51ccab"),
    ("paper_2510_08288_gb300/csrc/rrg_device.cuh", None, None, "1ef24ed4a16f67f78ee586ee6229fd831974dc8e"),
    ("paper_2510_08288_gb300/csrc/rrg_kernels.cu", "// Where a rollout lane takes its disturbances from.",
     "// Binary64 re-run of the trajectories", "69650da0e7a4601cab97766b63f3c5ad23e6b113"),
    ("paper_2510_08288_gb300/csrc/rrg_internal.h", "struct Launch {", "\n};\n",
     "fb4621135eb51875cc90e855eb357a809ab05b13"),
)


def source_region(rel, begin, end):
    """The text of a source file, or of its region from `begin` up to the
    first `end` after it."""
    with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
        text = f.read()
    if begin is None:
        return text
    i = text.index(begin)
    return text[i:text.index(end, i) + len(end)]


# The sweep's rollout launches at 65,536 scenarios (parametric model, TMA
# ring): DRAM bytes per launch of one update's three k-section rounds (ncu,
# one pass over the three launches of the first timed update).  Each round
# reads the array once per candidate that is still running (tile-major order;
# the 3.9 GB array does not fit in L2), up to 16 times the algorithmic bytes.
SWEEP_TRAFFIC_64K = (7911768832 + 3319040 + 19845668096 + 436992 + 51305741824 + 906496) / 3
# warp instructions per trajectory-step of the TMA-ring kernel there (22.50 G
# over 6.56 G lane-steps in the same capture)
TMA_INSTR_PER_STEP = 110


# DRAM bytes of one adjoint_forward_kernel<float, float> launch on the adjoint
# workload (4,096 x 1,000, checkpoint 50; ncu, one pass over one launch of the
# bench's adjoint workload: the 49 MB binary32 disturbance array read once;
# the 3.8 MB of checkpoints and lane minima stay in L2 during the launch),
# valid while the forward kernel, its launch, the step and the Launch struct
# are the ones profiled
ADJ_TRAFFIC_PER_LAUNCH = 49196288 + 3328
ADJ_TRAFFIC_SOURCES = (
    ('paper_2510_08288_gb300/csrc/rrg_adjoint.cu', 'constexpr int kFwdRing = 8;', '__global__ void adjoint_argmin_kernel', 'dd5593761eb2e7fa9699a30371ebecad854ba470'),
    ('paper_2510_08288_gb300/csrc/rrg_adjoint.cu', 'cudaError_t launch_adjoint_forward(', 'adjoint_argmin_kernel<<<', 'a97cb6582368d4a124a1b7416784f62ca4ea66c5'),
    ('paper_2510_08288_gb300/csrc/rrg_device.cuh', None, None, '1ef24ed4a16f67f78ee586ee6229fd831974dc8e'),
    ('paper_2510_08288_gb300/csrc/rrg_lane.cuh', None, None, 'bb86588f91e49ec177d60d8ba804f8f0da51ccab'),
    ('paper_2510_08288_gb300/csrc/rrg_internal.h', 'struct Launch {', '\n};\n', 'fb4621135eb51875cc90e855eb357a809ab05b13'),
)


def measured_traffic(sources=TRAFFIC_SOURCES, per_launch=TRAFFIC_PER_LAUNCH):
    """The profiled DRAM bytes per launch, or None if the kernel changed."""
    import hashlib
    for rel, begin, end, sha in sources:
        try:
            region = source_region(rel, begin, end)
        except (OSError, ValueError):
            return None
        if hashlib.sha1(region.encode("utf-8")).hexdigest() != sha:
            return None
    return per_launch


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("gpu", "reference"), default="gpu")
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="updates of the plain FP64 bisection comparator (default: all timed updates)")
    ap.add_argument("--window-start", type=int, default=WINDOW_START,
                    help="closed loop: first timed update (the updates before it run untimed)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU-oracle baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-spec", action="store_true", help="batch: skip the speculative-bisection leg")
    ap.add_argument("--pairing", choices=("never", "filled", "always", "autotune"), default="filled",
                    help="sweep: candidates per thread of the rollouts (rrg_set_pairing); autotune times "
                         "every mode on the first warm-up update and keeps the fastest")
    ap.add_argument("--scenarios", type=int, default=N_SCEN, help="smaller cases for profiling only")
    ap.add_argument("--horizon", type=int, default=HORIZON, help="smaller cases for profiling only")
    ap.add_argument("--probe-steps", type=int, default=PROBE_STEPS,
                    help="steps of the probe that pipelines the first two bisection rounds (0: off)")
    ap.add_argument("--shape", type=str, default=None,
                    help="closed loop: 'm,probe' sets the speculative bisection's shape instead of autotuning it")
    ap.add_argument("--tma", choices=("never", "auto", "always"), default="auto",
                    help="closed loop, sweep: which binary32 ring launches take their disturbances through the "
                         "TMA (rrg_set_tma; auto: the library's default rule)")
    ap.add_argument("--workload", choices=("closed_loop", "sweep", "batch", "single", "adjoint"),
                    default="closed_loop")
    ap.add_argument("--instances", type=int, default=BATCH_S, help="batch: number of RG instances")
    ap.add_argument("--variant", type=int, default=None,
                    help="batch: use this rollout variant instead of autotuning it")
    ap.add_argument("--sweep-n", type=str, default=",".join(str(n) for n in SWEEP_N),
                    help="scenario counts of the sweep")
    ap.add_argument("--param-unc-rel", type=float, default=None,
                    help="sweep: half-range of the parameter multipliers (default 0.1; 0 = nominal model)")
    return ap.parse_args()


def window_start(W, K, start=WINDOW_START):
    """First timed update of the closed loop: `start`, moved so that the W
    warm-up updates fit before it and the K timed ones inside the run."""
    return max(W, min(start, RUN_UPDATES - K))


def apply_tma(R, g, mode):
    """rrg_set_tma where the handle has a TMA ring (otherwise it stays off)."""
    if mode == R.TMA_NEVER or g.get_tma() != R.TMA_NEVER:
        g.set_tma(mode)


def shape_seconds(g, shape, states, seed, reps=3):
    """Host time of `reps` synchronous updates at each state (update index,
    x_t, r_t, v_prev) with the speculative bisection's shape (m, probe)."""
    g.set_tuning(*shape)
    total = 0.0
    for t, x, r, v in states:
        g.sample_scenarios(seed, t)
        g.step(x, r, v)
        t0 = time.perf_counter()
        for _ in range(reps):
            g.step(x, r, v)
        total += time.perf_counter() - t0
    return total


def workload_config(S0, W, K, N=N_SCEN, H=HORIZON, probe=PROBE_STEPS, m=M_CAND, given=False):
    return {
        "workload": "closed-loop robust RG on FC3: N_sim=%d scenarios, horizon %d RK4 steps "
                    "(dt=0.01 s), staircase r (8 levels over 50..300 A, seed 1, 125 updates/level), "
                    "timed updates [%d, %d) of the 1000-update run (updates [%d, %d) warm up, the ones "
                    "before them position the loop; the level change at update 125 falls in the window "
                    "when it is long enough)" % (N, H, S0, S0 + K, S0 - W, S0),
        "search": "speculative bisection (Alg. 1 result), N_kappa=12, %d candidates/round, "
                  "first two rounds pipelined after a %d-step probe (0: not pipelined); shape %s"
                  % (m, probe, "given" if given else
                     "chosen by rrg_autotune on update 0 and on update %d (the first warm-up update); "
                     "when the two differ, the one with the smaller time over both" % (S0 - W)),
        "kappa_tol": 2.0 ** -11,
        "precision": "binary32 rollouts, binary64 recheck of |slack| < 1e-6*1.9",
        "l2": "256 MB written between timed steps",
        "launch": "one CUDA graph replay per update (rrg_closed_loop_dev, graph on)",
    }


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi's SM clock, throttle reasons, power draw (and, where the
    driver answers them, memory clock and enforced power limit) every
    PERIOD_MS, read by a thread that stamps each line with the host clock.  begin()/end() bracket
    a timed region (host times taken after a device synchronize, so the
    region's kernels ran between them); stop() keeps the samples inside the
    regions widened by one period on each side, so that a region shorter than
    the period still gets the samples that bracket it."""
    PERIOD_MS = 100
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    EXTRA = ",clocks.mem,enforced.power.limit"

    def __init__(self, gpu_index=None):
        self.lines, self.windows, self._t0 = [], [], None
        self.p = None
        # the extra fields first; the required ones alone if that query is refused
        for fields in (self.FIELDS + self.EXTRA, self.FIELDS):
            if self._start(fields, gpu_index):
                return

    def _start(self, fields, gpu_index):
        import threading
        cmd = ["nvidia-smi", "--query-gpu=" + fields, "--format=csv,noheader,nounits",
               "-lms", str(self.PERIOD_MS)]
        if gpu_index is not None:
            cmd += ["-i", str(gpu_index)]
        self._first = threading.Event()
        try:
            self.p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
            return True                     # no nvidia-smi at all: nothing to retry
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()
        self._first.wait(5.0)               # nvidia-smi is up before any region starts
        if any(len(x.split(",")) >= 9 for _, x in self.lines):
            return True
        try:
            self.p.wait(timeout=1.0)
        except subprocess.TimeoutExpired:
            return True                     # still running: keep it
        self.th.join(timeout=5)             # refused (an unknown field): try the next query
        self.lines, self.p = [], None
        return False

    def _read(self):
        for line in self.p.stdout:
            self.lines.append((time.monotonic(), line))
            if len(line.split(",")) >= 9:
                self._first.set()
        self._first.set()                   # the query ended (refused, or stop())

    def begin(self):
        self._t0 = time.monotonic()

    def end(self):
        if self._t0 is not None:
            self.windows.append((self._t0, time.monotonic()))
            self._t0 = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            self.p.wait()
        self.th.join(timeout=5)
        pad = self.PERIOD_MS / 1e3
        keep = [line for t, line in self.lines
                if not self.windows or any(a - pad <= t <= b + pad for a, b in self.windows)]
        sm, smax, mem, plim, power, reasons = [], [], [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

        def num(v, into):
            try:
                into.append(float(v))
            except ValueError:
                pass
        for line in keep:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            num(f[3], power)
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
            if len(f) >= 11:
                num(f[9], mem)
                num(f[10], plim)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "timed_ms": round(1e3 * sum(b - a for a, b in self.windows), 1),
                "period_ms": self.PERIOD_MS,
                "mem_mhz": statistics.median(mem) if mem else None,
                "power_w": statistics.median(power) if power else None,
                "power_limit_w": statistics.median(plim) if plim else None}


# -------------------------------------------------------------- CPU side --
def cpu_oracle_closed_loop(x0, r_seq, seconds, cores):
    """Times the FP64 oracle's closed loop (plain joint bisection) on a
    bounded prefix of the run; returns (updates/s, updates, seconds, kappas,
    seconds of the first update)."""
    from oracle import oracle as O
    from paper_2510_08288_gb300 import inputs
    p = inputs.fc3_params()
    c = O.cfg(H=HORIZON, N=N_SCEN)
    t0 = time.perf_counter()
    v, kap, fl, xs = O.closed_loop(p, c, x0, V0, r_seq[:1], SEED, 0, inputs.DIST_AMP, inputs.DIST_AMP,
                                   search=0, n_kappa=N_BISECT, nthreads=cores)
    one = time.perf_counter() - t0
    more = max(0, min(len(r_seq) - 1, int(seconds / max(one, 1e-3)) - 1))
    kaps = list(kap)
    if more:
        t1 = time.perf_counter()
        v2, kap2, fl2, xs2 = O.closed_loop(p, c, xs[1], v[0], r_seq[1:1 + more], SEED, 1, inputs.DIST_AMP,
                                           inputs.DIST_AMP, search=0, n_kappa=N_BISECT, nthreads=cores)
        kaps += list(kap2)
        total = one + (time.perf_counter() - t1)
    else:
        total = one
    n = 1 + more
    return n / total, n, total, kaps, one


def cpu_oracle_one_core(x0, r_seq):
    """The first update of the same closed loop on one host thread: the
    sequential FP64 oracle beside the threaded one; returns (updates/s, kappa)."""
    from oracle import oracle as O
    from paper_2510_08288_gb300 import inputs
    p = inputs.fc3_params()
    c = O.cfg(H=HORIZON, N=N_SCEN)
    t0 = time.perf_counter()
    v, kap, fl, xs = O.closed_loop(p, c, x0, V0, r_seq[:1], SEED, 0, inputs.DIST_AMP, inputs.DIST_AMP,
                                   search=0, n_kappa=N_BISECT, nthreads=1)
    return 1.0 / (time.perf_counter() - t0), float(kap[0])


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_2510_08288_gb300 import inputs
    p = inputs.fc3_params()
    W, K = args.warmup, args.steps
    S0 = window_start(W, K, args.window_start)
    r_seq = inputs.staircase(S0 + K, 8, 125, SEED)
    x0 = O.equilibrium(p, V0)
    cores = os.cpu_count() or 1
    c = O.cfg(H=HORIZON, N=N_SCEN)
    amp = inputs.DIST_AMP
    # untimed: the updates before the window (the last W of them the warm-up)
    v, kap, fl, xs = O.closed_loop(p, c, x0, V0, r_seq[:S0], SEED, 0, amp, amp, search=0, n_kappa=N_BISECT,
                                   nthreads=cores) if S0 else (None, None, None, [x0])
    xw, vw = (xs[-1], v[-1]) if S0 else (x0, V0)
    t0 = time.perf_counter()
    O.closed_loop(p, c, xw, vw, r_seq[S0:S0 + K], SEED, S0, amp, amp, search=0, n_kappa=N_BISECT,
                  nthreads=cores)
    dt = time.perf_counter() - t0
    val = K / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": K, "warmup": W, "ms_per_step": 1e3 * dt / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(S0, W, K), search="plain joint bisection (Alg. 1 on all scenarios)",
                       precision="binary64", l2="n/a (CPU)"),
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "updates [%d, %d) of the closed loop, FP64 CPU oracle, %d threads"
                                   % (S0, S0 + K, cores)},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------- GPU side --
def e2e_loop_run(R, p, cfg, stream, x0, r_seq, seed, amp, W, T, flush, kap_dev, tuning, tma=1):
    """The timed updates [W, T) as one rrg_closed_loop_dev call each (plant
    state on the device, as in the timed value) on a fresh handle: every
    update copies its r_t in from pinned host memory, and its v_t, kappa,
    flags and x_{t+1} out to pinned host memory, and waits for them."""
    import numpy as np
    import torch
    g2 = R.Governor(p, cfg, stream)
    g2.set_tuning(*tuning)
    apply_tma(R, g2, tma)
    dev = torch.device("cuda", torch.cuda.current_device())
    d_r = torch.zeros(T, dtype=torch.float64, device=dev)
    d_v, d_k = torch.zeros_like(d_r), torch.zeros_like(d_r)
    d_f = torch.zeros(T, dtype=torch.int32, device=dev)
    d_x = torch.zeros(3 * (T + 1), dtype=torch.float64, device=dev)
    h_r = torch.tensor(r_seq[:T], dtype=torch.float64).pin_memory()
    h_out = torch.zeros(6, dtype=torch.float64).pin_memory()   # v, kappa, x_{t+1}[3], flags
    h_f = torch.zeros(1, dtype=torch.int32).pin_memory()
    d_r[:W].copy_(h_r[:W])
    R.rrg_closed_loop_dev(g2.h, x0, V0, d_r, W, seed, 0, amp, True, d_v, d_k, d_f, d_x)
    torch.cuda.synchronize()
    e2e_s, kap = 0.0, []
    with torch.cuda.stream(stream):
        for t in range(W, T):
            flush.fill_(float(t))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            d_r[t:t + 1].copy_(h_r[t:t + 1], non_blocking=True)
            R.rrg_closed_loop_dev(g2.h, None, 0.0, d_r, 1, seed, 0, amp, True, d_v, d_k, d_f, d_x)
            h_out[0:1].copy_(d_v[t:t + 1], non_blocking=True)
            h_out[1:2].copy_(d_k[t:t + 1], non_blocking=True)
            h_out[2:5].copy_(d_x[3 * (t + 1):3 * (t + 2)], non_blocking=True)
            h_f.copy_(d_f[t:t + 1], non_blocking=True)
            stream.synchronize()
            e2e_s += time.perf_counter() - t0
            kap.append(float(h_out[1]))
    g2.close()
    K = T - W
    return {"value": K / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8, "d2h_bytes_per_step": 8 + 8 + 24 + 4,
            "call": "rrg_closed_loop_dev, one update per call, plant state on the device",
            "kappa_equal_to_device_run": bool(np.all(np.array(kap) == kap_dev[W:T]))}


def e2e_run(R, p, cfg, stream, x0, r_seq, seed, amp, W, T, flush, kap_dev, tuning, tma=1):
    """The timed updates [W, T) again through the host-buffer entry points
    (rrg_sample_scenarios, rrg_step, rrg_plant_step) on a fresh handle, after
    the updates before them untimed; every call copies its inputs from and its
    results to host memory."""
    import numpy as np
    import torch
    g2 = R.Governor(p, cfg, stream)
    g2.set_tuning(*tuning)
    apply_tma(R, g2, tma)
    x, v = x0.copy(), V0
    for t in range(W):
        g2.sample_scenarios(seed, t)
        v, _, _ = g2.step(x, r_seq[t], v)
        x = g2.plant_step(x, v, seed, t, amp)
    e2e_s, kap_e2e = 0.0, []
    for t in range(W, T):
        flush.fill_(float(t))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g2.sample_scenarios(seed, t)
        v, kk, _ = g2.step(x, r_seq[t], v)
        x = g2.plant_step(x, v, seed, t, amp)
        e2e_s += time.perf_counter() - t0
        kap_e2e.append(kk)
    g2.close()
    K = T - W
    # bytes copied per update: rrg_step sends x_t, r_t, v_prev (40 B) and
    # returns v_t, kappa, flags (20 B); rrg_plant_step sends its 12-double
    # staging block (96 B) and returns x_{t+1} (24 B)
    return {"value": K / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 40 + 96, "d2h_bytes_per_step": 20 + 24,
            "kappa_equal_to_device_run": bool(np.all(np.array(kap_e2e) == kap_dev[W:T]))}


def fp64_comparator(R, torch, p, stream, flush, H, N, seed, amp, d_r, S0, n, x_start, v_start, kap32, dev):
    """Plain FP64 bisection (Alg. 1, 12 rounds) on the same closed loop over
    updates [S0, S0 + n), through rrg_closed_loop_dev from the given state,
    with CUDA events around every update on the launching stream."""
    import numpy as np
    if n <= 0:
        return None
    cfg64 = R.rrg_config_default(horizon=H, n_scenarios=N, max_candidates=M_CAND, n_bisect=N_BISECT,
                                 search=R.SEARCH_BISECT, precision=R.FP64, early_exit=R.EXIT_CANDIDATE)
    g3 = R.Governor(p, cfg64, stream)
    o_v = torch.zeros(n, dtype=torch.float64, device=dev)
    o_k = torch.zeros(n, dtype=torch.float64, device=dev)
    o_f = torch.zeros(n, dtype=torch.int32, device=dev)
    o_x = torch.zeros(3 * (n + 1), dtype=torch.float64, device=dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for i in range(n):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            if i == 0:
                R.rrg_closed_loop_dev(g3.h, np.asarray(x_start, dtype=np.float64), float(v_start), d_r[S0:], 1,
                                      seed, S0, amp, False, o_v, o_k, o_f, o_x)
            else:
                R.rrg_closed_loop_dev(g3.h, None, 0.0, d_r[S0:], 1, seed, S0, amp, False, o_v, o_k, o_f, o_x)
            evs[i][1].record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in evs]
    g3.close()
    k64 = o_k.cpu().numpy()
    diff = np.abs(k64 - np.asarray(kap32[:n]))
    return {"value": n / (sum(ms) / 1e3), "unit": UNIT, "ms_per_update": sum(ms) / n, "updates": n,
            "window": [S0, S0 + n],
            "timing": "CUDA events around each update (rrg_closed_loop_dev, direct launches), L2 flushed "
                      "between updates, same closed loop and updates as the timed binary32 window",
            "kappa_equal_to_fp32_recheck": bool(np.all(diff == 0.0)),
            "kappa_max_abs_diff": float(diff.max())}


def merge_fp32_errors(parts, where):
    """One fp32_error object from several probes (the worst of each figure)."""
    if not parts:
        return None
    out = dict(parts[0])
    out["updates"] = where
    out["scenarios"] = [q["scenarios"] for q in parts]
    out["trajectories"] = sum(q["trajectories"] for q in parts)
    out["steps_per_trajectory"] = [q["steps_per_trajectory"] for q in parts]
    for key in ("max_abs_slack_error", "median_trajectory_max_error", "max_error_over_band_or_slack"):
        out[key] = max(q[key] for q in parts)
    out["unsafe_steps"] = sum(q["unsafe_steps"] for q in parts)
    return out


def fp32_error_probe(R, p, stream, H, N, seed, probes, m_grid=16, m_near=16, param_unc=0.0, n_cap=None):
    """The binary32 rollouts' slack error against binary64 on sampled updates
    (rrg_slack_error: every trajectory in both precisions over the full
    horizon, no early exit): per update (t, x_t, v_prev, r_t, kappa_t), the
    candidates are m_grid points on [0, 1] and m_near dyadic points spaced
    2^-11 around the update's kappa.  n_cap: only the first n_cap scenarios
    (the Philox draws are nested in N, so they are the run's own)."""
    import numpy as np
    from paper_2510_08288_gb300 import inputs
    n = N if n_cap is None else min(N, n_cap)
    band = RECHECK_EPS_REL * inputs.Y_MIN
    kw = {}
    if param_unc > 0:
        kw = dict(param_unc_rel=param_unc, param_unc_mask=inputs.FC3_UNCERTAIN_MASK)
    cfg = R.rrg_config_default(horizon=H, n_scenarios=n, max_candidates=m_grid + m_near,
                               precision=R.FP32_RECHECK, recheck_eps_rel=RECHECK_EPS_REL, **kw)
    g = R.Governor(p, cfg, stream)
    emax, rmax, bad, lanes, meds, ts = 0.0, 0.0, 0, 0, [], []
    for (t, x, vp, r, kap) in probes:
        near = np.clip(kap + (np.arange(m_near) - (m_near // 2 - 1)) * 2.0 ** -11, 0.0, 1.0)
        kappas = np.unique(np.concatenate([np.linspace(0.0, 1.0, m_grid), near]))
        g.sample_scenarios(seed, t)
        out = g.slack_error(np.asarray(x, dtype=np.float64), float(vp), float(r), kappas, band)
        emax = max(emax, float(out["err"].max()))
        rmax = max(rmax, float(out["ratio"].max()))
        bad += int(out["unsafe"].sum())
        lanes += out["err"].size
        meds.append(float(np.median(out["err"])))
        ts.append(int(t))
    g.close()
    return {"band": band, "updates": ts, "trajectories": lanes, "steps_per_trajectory": H + 1,
            "scenarios": n if n == N else "%d of %d" % (n, N),
            "kappas": "%d grid points on [0, 1] and %d dyadic points spaced 2^-11 around the update's kappa"
                      % (m_grid, m_near),
            "max_abs_slack_error": emax,
            "median_trajectory_max_error": float(np.median(meds)),
            "max_error_over_band_or_slack": rmax,
            "unsafe_steps": bad,
            "basis": "rrg_slack_error: binary32 and binary64 slacks of every trajectory at every step "
                     "j = 0..H, no early exit; unsafe = steps the band rule would decide wrongly; "
                     "max_error_over_band_or_slack = max |s32 - s64| / max(band, |s64|) (below 1: exact)"}


def run_gpu(args):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2510_08288_gb300 import build as B
    B.build()
    from paper_2510_08288_gb300 import inputs
    from paper_2510_08288_gb300 import rrg as R

    p = inputs.fc3_params()
    W, K = args.warmup, args.steps
    S0 = window_start(W, K, args.window_start)   # first timed update
    T = S0 + K
    seed = SEED + 1000 * rank          # replicas run independent closed loops
    r_seq = inputs.staircase(T, 8, 125, SEED)
    amp = np.array(inputs.DIST_AMP)
    stream = torch.cuda.Stream()
    NS, HZ = args.scenarios, args.horizon
    cfg = R.rrg_config_default(horizon=HZ, n_scenarios=NS, max_candidates=M_CAND,
                               n_bisect=N_BISECT, search=R.SEARCH_SPEC_BISECT,
                               precision=R.FP32_RECHECK, early_exit=R.EXIT_CANDIDATE,
                               recheck_eps_rel=RECHECK_EPS_REL, probe_steps=args.probe_steps)
    g = R.Governor(p, cfg, stream)
    apply_tma(R, g, TMA_MODES.index(args.tma))
    x0, _ = g.equilibrium(V0)
    # the speculative bisection's shape (tree width, probe length) by the
    # library's autotuner; every shape gives Alg. 1's kappa
    shapes = []
    if args.shape:
        tune_m, tune_probe = (int(v) for v in args.shape.split(","))
        g.set_tuning(tune_m, tune_probe)
    else:
        g.sample_scenarios(seed, 0)
        tune_m, tune_probe, _ = g.autotune(x0, r_seq[0], V0, repeats=2)
        shapes.append((tune_m, tune_probe))
    dev = torch.device("cuda", local)
    d_r = torch.tensor(r_seq, dtype=torch.float64, device=dev)
    d_v = torch.zeros(T, dtype=torch.float64, device=dev)
    d_k = torch.zeros(T, dtype=torch.float64, device=dev)
    d_f = torch.zeros(T, dtype=torch.int32, device=dev)
    d_x = torch.zeros(3 * (T + 1), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()

    # the updates before the window, the last W of them the warm-up (they
    # also initialise the loop state on the device and capture the one-update
    # CUDA graph the timed updates replay); the shape is tuned a second time
    # on the first warm-up update, an operating point of the run itself
    tw = S0 - W
    R.rrg_closed_loop_dev(g.h, x0, V0, d_r, tw, seed, 0, amp, True, d_v, d_k, d_f, d_x)
    torch.cuda.synchronize()
    if not args.shape and tw > 0:
        xw = d_x[3 * tw:3 * tw + 3].cpu().numpy()
        vw = float(d_v[tw - 1].item())
        g.sample_scenarios(seed, tw)
        m2, p2, _ = g.autotune(xw, r_seq[tw], vw, repeats=2)
        shapes.append((m2, p2))
        if shapes[1] != shapes[0]:
            states = [(0, x0, r_seq[0], V0), (tw, xw, r_seq[tw], vw)]
            tune_m, tune_probe = min(shapes, key=lambda sh: shape_seconds(g, sh, states, seed))
        else:
            tune_m, tune_probe = m2, p2
        g.set_tuning(tune_m, tune_probe)
    R.rrg_closed_loop_dev(g.h, None, 0.0, d_r, W, seed, 0, amp, True, d_v, d_k, d_f, d_x)
    torch.cuda.synchronize()
    g.reset_stats()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    clocks = ClockSampler()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.begin()
    with torch.cuda.stream(stream):
        for i in range(K):
            flush.fill_(float(i))                       # L2 flush, outside the timed window
            evs[i][0].record(stream)
            R.rrg_closed_loop_dev(g.h, None, 0.0, d_r, 1, seed, 0, amp, True, d_v, d_k, d_f, d_x)
            evs[i][1].record(stream)
    torch.cuda.synchronize()
    clocks.end()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_s = sum(step_ms) / 1e3
    st = g.stats()
    if dist:
        t = torch.tensor([total_s], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    # graph replays cannot time single kernels: the same K updates again by
    # direct launches, on a fresh handle from the same start, with CUDA
    # events around every rollout launch (the roofline's kernel duration)
    gd = R.Governor(p, cfg, stream)
    gd.set_tuning(tune_m, tune_probe)
    apply_tma(R, gd, TMA_MODES.index(args.tma))
    dd_v, dd_k = torch.zeros_like(d_v), torch.zeros_like(d_k)
    dd_f, dd_x = torch.zeros_like(d_f), torch.zeros_like(d_x)
    R.rrg_closed_loop_dev(gd.h, x0, V0, d_r, S0, seed, 0, amp, False, dd_v, dd_k, dd_f, dd_x)
    torch.cuda.synchronize()
    gd.reset_stats()
    gd.set_profiling(True)
    devs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for i in range(K):
            flush.fill_(float(i))
            devs[i][0].record(stream)
            R.rrg_closed_loop_dev(gd.h, None, 0.0, d_r, 1, seed, 0, amp, False, dd_v, dd_k, dd_f, dd_x)
            devs[i][1].record(stream)
    torch.cuda.synchronize()
    direct_s = sum(a.elapsed_time(b) for a, b in devs) / 1e3
    std = gd.stats()
    gd.set_profiling(False)
    direct_same = bool(torch.equal(dd_k, d_k))
    gd.close()
    # and once more with the disturbances drawn inside the trajectory loop
    # (no stored scenario array, no sampler pass)
    cfg_gen = R.rrg_config_default(horizon=HZ, n_scenarios=NS, max_candidates=M_CAND,
                                   n_bisect=N_BISECT, search=R.SEARCH_SPEC_BISECT,
                                   precision=R.FP32_RECHECK, early_exit=R.EXIT_CANDIDATE,
                                   recheck_eps_rel=RECHECK_EPS_REL, probe_steps=args.probe_steps,
                                   scenarios_in_register=1)
    gr = R.Governor(p, cfg_gen, stream)
    gr.set_tuning(tune_m, tune_probe)
    rd_v, rd_k = torch.zeros_like(d_v), torch.zeros_like(d_k)
    rd_f, rd_x = torch.zeros_like(d_f), torch.zeros_like(d_x)
    R.rrg_closed_loop_dev(gr.h, x0, V0, d_r, S0, seed, 0, amp, True, rd_v, rd_k, rd_f, rd_x)
    revs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for i in range(K):
            flush.fill_(float(i))
            revs[i][0].record(stream)
            R.rrg_closed_loop_dev(gr.h, None, 0.0, d_r, 1, seed, 0, amp, True, rd_v, rd_k, rd_f, rd_x)
            revs[i][1].record(stream)
    torch.cuda.synchronize()
    reg_s = sum(a.elapsed_time(b) for a, b in revs) / 1e3
    reg_same = bool(torch.equal(rd_k, d_k))
    gr.close()

    kap_dev = d_k.cpu().numpy()
    flags_dev = d_f.cpu().numpy()
    x_dev = d_x.cpu().numpy().reshape(T + 1, 3)
    value = world * K / total_s

    # executed trajectory-steps of the timed updates; the rollout kernel's
    # duration and work per launch from the direct-launch run
    exec_steps = st["lane_steps"]
    fp32_steps = std["lane_steps"] - std["lane_steps_fp64"]
    avg_roll_ms = std["rollout_ms"] / max(1, std["timed_rollouts"])
    roll_launches = max(1, std["timed_rollouts"])
    achieved = (fp32_steps / roll_launches) * FLOPS_PER_STEP / (avg_roll_ms * 1e-3) / 1e12

    # the FP32 FMA, FP64 FMA and MUFU throughput measured on this GPU, next to
    # the derived peak the roofline fraction is reported against
    peaks = R.rrg_alu_peaks()
    # the latency bound of the launches whose surviving lanes run alone on a
    # scheduler: one warp's cycles per trajectory step against the rollout
    # time per update spread over the horizon those lanes integrate
    chain_cycles = g.step_latency(V0, HZ)
    roll_ms_per_update = std["rollout_ms"] / max(1, K)
    peak, peak_src = fp32_peak(clk)
    sm_mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz")
    step_cycles = roll_ms_per_update * 1e-3 * sm_mhz * 1e6 / HZ if sm_mhz else None
    out = None
    if rank == 0:
        # e2e: the same updates through the host-buffer C ABI, on a fresh handle
        e2e = e2e_loop = None
        if not args.no_e2e:
            e2e = e2e_run(R, p, cfg, stream, x0, r_seq, seed, amp, S0, T, flush, kap_dev, (tune_m, tune_probe),
                          TMA_MODES.index(args.tma))
            e2e_loop = e2e_loop_run(R, p, cfg, stream, x0, r_seq, seed, amp, S0, T, flush, kap_dev,
                                    (tune_m, tune_probe), TMA_MODES.index(args.tma))

        # plain FP64 bisection on the same GPU over the same timed updates,
        # timed the same way (CUDA events around each update, L2 flushed in
        # between): the same closed loop through rrg_closed_loop_dev, started
        # from the binary32 run's state at the window (its kappas, and so its
        # states, must then agree update by update)
        v_dev = d_v.cpu().numpy()
        nf = K if args.fp64_steps is None else min(args.fp64_steps, K)
        fp64 = fp64_comparator(R, torch, p, stream, flush, HZ, NS, seed, amp, d_r, S0, nf,
                               x_dev[S0], v_dev[S0 - 1] if S0 else V0, kap_dev[S0:S0 + nf], dev)
        # binary32 slack error against binary64 on sampled timed updates
        probe_ts = sorted({S0, min(max(125, S0), T - 1), S0 + K // 2, T - 1})
        fp32_err = fp32_error_probe(R, p, stream, HZ, NS, seed,
                                    [(t, x_dev[t], v_dev[t - 1] if t else V0, r_seq[t], kap_dev[t])
                                     for t in probe_ts])
        if fp64 is not None:
            fp32_err["kappa_max_abs_diff_fp64"] = fp64["kappa_max_abs_diff"]

        cpu = None
        if not args.no_cpu_baseline and (NS, HZ) == (N_SCEN, HORIZON):
            cores = os.cpu_count() or 1
            from oracle import oracle as O
            x0o = O.equilibrium(p, V0)
            cval, cn, cs, ckap, cone = cpu_oracle_closed_loop(x0o, inputs.staircase(1000, 8, 125, SEED),
                                                        args.cpu_seconds, cores)
            cpu = {"value": cval, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": "first %d updates of the same closed loop (seed %d), FP64 plain joint "
                             "bisection, %.1f s" % (cn, SEED, cs)}
            # rank 0's replica starts from the same state and scenarios: kappas must agree
            nk = min(cn, T)
            cpu["kappa_equal_to_gpu"] = bool(np.all(np.array(ckap[:nk]) == kap_dev[:nk]))
            v1, k1 = cpu_oracle_one_core(x0o, inputs.staircase(1000, 8, 125, SEED))
            cpu["one_core"] = {"value": v1, "unit": UNIT, "cores": 1,
                               "threaded_same_update": 1.0 / cone,
                               "sample": "first update of the same closed loop, one host thread",
                               "kappa_equal_to_threaded": bool(k1 == float(ckap[0]))}

        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": 1e3 * total_s / K, "ms_per_step_median": statistics.median(step_ms),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(S0, W, K, NS, HZ, tune_probe, tune_m, bool(args.shape)),
                           rollout_ring=TMA_NAMES[g.get_tma()]),
            "trajectory_steps_per_s": {"executed": world * exec_steps / total_s,
                                       "executed_per_update": exec_steps / K},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": frac_of(achieved, peak),
                         "traffic": measured_traffic() if (NS, HZ) == (N_SCEN, HORIZON) else None,
                         "kernel": "rollout_kernel<float>",
                         "avg_launch_ms": avg_roll_ms, "launches": std["timed_rollouts"],
                         "timing": "CUDA events around each rollout launch of the same K updates run by "
                                   "direct launches (graph replays cannot time single kernels)",
                         "flops_per_traj_step": FLOPS_PER_STEP,
                         "peak_source": peak_src,
                         "issue_ceiling": ISSUE_CEILING,
                         "frac_of_issue_ceiling": frac_of(frac_of(achieved, peak), ISSUE_CEILING),
                         "measured_units": {"fp32_fma_tflops": peaks[0], "fp64_fma_tflops": peaks[1],
                                            "mufu_ex2_tops": peaks[2],
                                            "frac_of_measured_fp32": achieved / peaks[0],
                                            "mufu_per_traj_step": MUFU_PER_STEP,
                                            "frac_of_measured_mufu": achieved / FLOPS_PER_STEP * MUFU_PER_STEP
                                            / peaks[2]},
                         "latency": {"cycles_per_step": step_cycles, "chain_cycles_per_step": chain_cycles,
                                     "frac": frac_of(chain_cycles, step_cycles),
                                     "basis": "rollout time per update (direct launches) over the %d-step "
                                              "horizon its surviving lanes integrate, at the sampled SM clock; "
                                              "chain: rrg_step_latency, one warp, same right-hand side" % HZ}},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "e2e_device_loop": e2e_loop,
            "direct_launches": {"value": world * K / direct_s, "unit": UNIT, "ms_per_step": 1e3 * direct_s / K,
                                "gpu_launches": std["launches"], "kappa_equal_to_graph_replay": direct_same},
            "scenarios_in_register": {"value": world * K / reg_s, "unit": UNIT, "ms_per_step": 1e3 * reg_s / K,
                                      "mode": "graph replay, disturbances drawn in the trajectory loop",
                                      "kappa_equal_to_stored_scenarios": reg_same},
            "gpu_launches": st["launches"],
            "clocks": clk,
            "fp64_bisect_gpu": fp64,
            "fp32_error": fp32_err,
            "rechecked_trajectories": st["rechecked"],
            "pipeline_repairs": st["repairs"],
            "no_admissible_updates": int(np.sum(flags_dev[S0:T] & 1)),
            "kappa_mean": float(np.mean(kap_dev[S0:T])),
            "kappa_max": float(np.max(kap_dev[S0:T])),
        }
    g.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)
    return 0


# ------------------------------------------------------------------ batch --
BATCH_S, BATCH_M, BATCH_ROUNDS, BATCH_SEED = 256, 32, 3, 2
BATCH_METRIC = "RG updates/s (instance updates, batched) & trajectory-steps/s; FP32 + FP64 recheck"


BATCH_PAIR_VARIANT = 8   # warp tiles of two candidates per thread
BATCH_SPLIT_VARIANT = 9  # warp tiles of 16 scenarios, two lanes per trajectory


def batch_kernel_name(variant):
    """The rollout kernel of a batch variant (index, lanes per tile, prefetch)."""
    if variant[0] == BATCH_PAIR_VARIANT:
        return "batch_rollout_warp_pair_kernel<%d> (two candidates per thread)" % variant[2]
    if variant[0] == BATCH_SPLIT_VARIANT:
        return "batch_rollout_split_kernel<%d> (two lanes per trajectory)" % variant[2]
    if variant[1] == 32:
        return "batch_rollout_warp_kernel<%d>" % variant[2]
    return "batch_rollout_kernel<%d, %d>" % (variant[1], variant[2])


def batch_ceiling(variant):
    """Issue ceiling of a batch variant's rollout (fraction of the FP32 peak), or None."""
    return None if variant[0] == BATCH_SPLIT_VARIANT else ISSUE_CEILING


def batch_config(S, W, K, variant):
    return {"workload": "batched instances on FC3: %d independent RG problems advanced together per step "
                        "(closed loop with plants), scenario counts log-uniform on [64, 8192], horizons "
                        "uniform on {200..4000} (seed %d), x_0 = equilibrium of v_prev x U[0.9, 1.1] per "
                        "state, v_prev and r per instance uniform on 50..300 A; k-section with %d candidates "
                        "per round, %d rounds; one persistent rollout launch per round" %
                        (S, BATCH_SEED, BATCH_M, BATCH_ROUNDS),
            "precision": "binary32 rollouts, binary64 recheck of |slack| < 1e-6*1.9",
            "timed": "updates [%d, %d) of the graph-replayed closed loop" % (W, W + K),
            "rollout_variant": variant, "l2": "256 MB written between timed steps"}


def batch_inputs(R, p, S):
    import numpy as np
    from paper_2510_08288_gb300 import inputs
    b = inputs.batched_instances(S, BATCH_SEED)
    with R.Governor(p, R.rrg_config_default(horizon=1, n_scenarios=1, max_candidates=2)) as g1:
        x0 = np.array([g1.equilibrium(v)[0] for v in b["v_prev"]]) * b["xfac"]
    return b, x0


def batch_cpu(p, b, x0, r, seconds, cores):
    """The FP64 oracle's k-section on a bounded sample: whole instances (the
    shortest first) for one update each, until about `seconds` are spent; then
    the sequential oracle on one thread over the first of those instances, for
    about a quarter of that time."""
    from oracle import oracle as O
    from paper_2510_08288_gb300 import inputs
    order = sorted(range(len(b["N"])), key=lambda s: int(b["N"][s]) * int(b["H"][s]))

    def one(s, threads):
        N, H = int(b["N"][s]), int(b["H"][s])
        d = O.sample_disturbances(SEED + s, 0, N, H, inputs.DIST_AMP)
        t0 = time.perf_counter()
        O.ksection(p, O.cfg(H=H, N=N), x0[s], b["v_prev"][s], r[s], BATCH_M, BATCH_ROUNDS, d, nthreads=threads)
        return time.perf_counter() - t0

    per = []
    for s in order:
        per.append(one(s, cores))
        if sum(per) > seconds:
            break
    t1 = []
    for s in order[:len(per)]:
        t1.append(one(s, 1))
        if sum(t1) > seconds / 4:
            break
    n1 = len(t1)
    return {"value": len(per) / sum(per), "unit": "RG updates/s (instance updates)", "cores": cores,
            "kind": "oracle",
            "sample": "%d of %d instances (smallest N*H first: biased towards cheap ones), one update each, "
                      "FP64 k-section, %.1f s" % (len(per), len(b["N"]), sum(per)),
            "one_core": {"value": n1 / sum(t1), "unit": "RG updates/s (instance updates)", "cores": 1,
                         "threaded_same_instances": n1 / sum(per[:n1]),
                         "sample": "the first %d of those instances on one host thread, %.1f s" % (n1, sum(t1))}}


def run_batch(args):
    import numpy as np
    import torch
    from paper_2510_08288_gb300 import build as B
    B.build()
    from paper_2510_08288_gb300 import inputs
    from paper_2510_08288_gb300 import rrg as R
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    p = inputs.fc3_params()
    S, W, K = args.instances, args.warmup, args.steps
    K2 = min(K, 5)        # extra updates without the graph, for the kernel timing
    T = W + K + K2
    b, x0 = batch_inputs(R, p, S)
    r = b["r"]
    r_seq = np.tile(r, (T, 1))
    amp = np.array(inputs.DIST_AMP)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream()
    cfg = R.rrg_config_default(max_candidates=BATCH_M, n_rounds=BATCH_ROUNDS, search=R.SEARCH_KSECTION,
                               precision=R.FP32_RECHECK, early_exit=R.EXIT_CANDIDATE,
                               recheck_eps_rel=RECHECK_EPS_REL)
    g = R.BatchGovernor(p, cfg, b["N"], b["H"], stream)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    dx0, dv0, dr = d(x0.reshape(-1)), d(b["v_prev"]), d(r_seq.reshape(-1))
    torch.cuda.synchronize()
    # the rollout variant: by the library's autotuner on the first update, or
    # given (results never depend on it)
    if args.variant is not None:
        g.set_variant(args.variant)
        tune_ms = None
    else:
        best, tune_ms = R.rrg_batch_autotune(g.h, dx0, d(r), dv0, SEED, 0, 1)
    dv = torch.zeros(T * S, dtype=torch.float64, device=dev)
    dk = torch.zeros_like(dv)
    df = torch.zeros(T * S, dtype=torch.int32, device=dev)
    dxo = torch.zeros((T + 1) * S * 3, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    R.rrg_batch_closed_loop_dev(g.h, dx0, dv0, dr, W, SEED, 0, amp, True, dv, dk, df, dxo)
    torch.cuda.synchronize()
    g.reset_stats()
    g.set_profiling(True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    clocks = ClockSampler()
    torch.cuda.synchronize()
    clocks.begin()
    with torch.cuda.stream(stream):
        for i in range(K):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            R.rrg_batch_closed_loop_dev(g.h, None, None, dr, 1, SEED, 0, amp, True, dv, dk, df, dxo)
            evs[i][1].record(stream)
    torch.cuda.synchronize()
    clocks.end()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(c) for a, c in evs]
    secs = sum(step_ms) / 1e3
    st = g.stats()
    # graph replays cannot time single kernels: K2 more updates with direct
    # launches give the rollout kernel's duration (CUDA events in the library)
    g.reset_stats()
    R.rrg_batch_closed_loop_dev(g.h, None, None, dr, K2, SEED, 0, amp, False, dv, dk, df, dxo)
    st2 = g.stats()
    g.set_profiling(False)
    kap = dk.cpu().numpy().reshape(T, S)
    flags = df.cpu().numpy().reshape(T, S)
    fp32_steps = st2["lane_steps"] - st2["lane_steps_fp64"]
    avg_roll_ms = st2["rollout_ms"] / max(1, st2["timed_rollouts"])
    achieved = (fp32_steps / max(1, st2["timed_rollouts"])) * FLOPS_PER_STEP / (avg_roll_ms * 1e-3) / 1e12
    variant = R.rrg_batch_get_variant(g.h)
    # e2e: the same K updates through the host-array call (copies included),
    # on a fresh handle that first replays the warm-up updates
    e2e = None
    if not args.no_e2e:
        g2 = R.BatchGovernor(p, cfg, b["N"], b["H"], stream)
        g2.set_variant(variant[0])
        xw = dxo.cpu().numpy().reshape(T + 1, S, 3)[W]
        vw = dv.cpu().numpy().reshape(T, S)[W - 1] if W else b["v_prev"]
        t0 = time.perf_counter()
        v2, k2, f2, x2 = g2.closed_loop(xw, vw, r_seq[W:W + K], SEED, W, amp)
        e2e_s = time.perf_counter() - t0
        g2.close()
        e2e = {"value": S * K / e2e_s, "unit": "RG updates/s (instance updates)",
               # per call: x_0, v_0 and the K x S references in; v, kappa,
               # flags and the K + 1 states out
               "h2d_bytes_per_step": (4 * S * 8) // K + S * 8,
               "d2h_bytes_per_step": S * (8 + 8 + 4) + ((K + 1) * S * 3 * 8) // K,
               "kappa_equal_to_device_run": bool(np.array_equal(k2, kap[W:W + K]))}
    cpu = None
    if not args.no_cpu_baseline:
        cpu = batch_cpu(p, b, x0, r, args.cpu_seconds, os.cpu_count() or 1)
    # binary32 slack error against binary64 at the first timed update, on the
    # two longest-horizon instances (each with its own scenarios, seed + s)
    xs_all = dxo.cpu().numpy().reshape(T + 1, S, 3)
    vs_all = dv.cpu().numpy().reshape(T, S)
    parts = []
    for s_i in np.argsort(-b["H"])[:2]:
        s_i = int(s_i)
        parts.append(fp32_error_probe(R, p, stream, int(b["H"][s_i]), int(b["N"][s_i]), SEED + s_i,
                                      [(W, xs_all[W, s_i], vs_all[W - 1, s_i] if W else b["v_prev"][s_i],
                                        r_seq[W][s_i], kap[W, s_i])],
                                      m_grid=BATCH_M, m_near=16))
    fp32_err = merge_fp32_errors(parts, "update %d of the two longest-horizon instances (%s)"
                                 % (W, ", ".join("H=%d, N=%d" % (b["H"][i], b["N"][i])
                                                 for i in np.argsort(-b["H"])[:2])))
    g.close()
    # the speculative-bisection batch (Alg. 1's kappa per instance for every
    # tree width): the library's autotuner picks the width (the candidate
    # count) on the first update, then the same K updates are timed
    spec = None
    if not args.no_spec:
        cfg_s = R.rrg_config_default(max_candidates=64, n_bisect=N_BISECT, search=R.SEARCH_SPEC_BISECT,
                                     precision=R.FP32_RECHECK, early_exit=R.EXIT_CANDIDATE,
                                     recheck_eps_rel=RECHECK_EPS_REL)
        gs = R.BatchGovernor(p, cfg_s, b["N"], b["H"], stream)
        gs.set_variant(variant[0])
        w_best, ws, wms = R.rrg_batch_autotune_width(gs.h, dx0, d(r), dv0, SEED, 0, 1)
        sv, sk = torch.zeros_like(dv), torch.zeros_like(dk)
        sf, sx = torch.zeros_like(df), torch.zeros_like(dxo)
        R.rrg_batch_closed_loop_dev(gs.h, dx0, dv0, dr, W, SEED, 0, amp, True, sv, sk, sf, sx)
        sevs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for i in range(K):
                flush.fill_(float(i))
                sevs[i][0].record(stream)
                R.rrg_batch_closed_loop_dev(gs.h, None, None, dr, 1, SEED, 0, amp, True, sv, sk, sf, sx)
                sevs[i][1].record(stream)
        torch.cuda.synchronize()
        ssecs = sum(a.elapsed_time(c) for a, c in sevs) / 1e3
        gs.close()
        spec = {"value": S * K / ssecs, "unit": "RG updates/s (instance updates)", "ms_per_step": 1e3 * ssecs / K,
                "search": "speculative bisection, N_kappa = %d (Alg. 1's kappa per instance for every width)"
                          % N_BISECT,
                "width_chosen": int(w_best),
                "autotune": {"widths": [int(x) for x in ws], "ms_per_update": [float(x) for x in wms]},
                "kappa_mean": float(np.mean(sk.cpu().numpy().reshape(T, S)[W:W + K]))}
    peak, peak_src = fp32_peak(clk)
    out = {
        "metric": BATCH_METRIC, "value": S * K / secs, "unit": "RG updates/s (instance updates)", "n_gpus": 1,
        "steps": K, "warmup": W, "ms_per_step": 1e3 * secs / K, "ms_per_step_median": statistics.median(step_ms),
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": batch_config(S, W, K, {"index": variant[0], "tile_lanes": variant[1], "prefetch": variant[2]}),
        "trajectory_steps_per_s": {"executed": st["lane_steps"] / secs, "executed_per_step": st["lane_steps"] / K},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": frac_of(achieved, peak), "traffic": None,
                     "kernel": batch_kernel_name(variant),
                     "avg_launch_ms": avg_roll_ms, "launches": st2["timed_rollouts"],
                     "timing": "%d direct-launch updates after the timed ones" % K2,
                     "flops_per_traj_step": FLOPS_PER_STEP,
                     "peak_source": peak_src,
                     # the one-lane loop's ceiling (its instructions per step were
                     # counted); none for the two-lane split, whose were not
                     "issue_ceiling": batch_ceiling(variant),
                     "frac_of_issue_ceiling": frac_of(frac_of(achieved, peak), batch_ceiling(variant))},
        "autotune_rollout_ms": [float(x) for x in tune_ms] if tune_ms is not None else None,
        "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": st["launches"],
        "rechecked_trajectories": st["rechecked"],
        "no_admissible_fraction": float(np.mean(flags[W:W + K] & 1)),
        "kappa_mean": float(np.mean(kap[W:W + K])),
        "fp32_error": fp32_err,
        "spec_bisect_autotuned_width": spec,
    }
    print(json.dumps(out), flush=True)
    return 0


# ----------------------------------------------------- single update (cfg 1) --
SINGLE_METRIC = "RG update latency (single robust update, 32 scenarios x 500 steps, N_kappa = 12)"


def timed_updates(R, torch, g, x_t, r, v_prev, W, K, seed, flush, stream):
    """W + K updates (sample + search) through the host-buffer calls; device
    time of each of the last K from CUDA events on the library's stream."""
    kap = None
    ms = []
    for i in range(W + K):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        a.record(stream)
        g.sample_scenarios(seed, 0)
        _, kap, fl = g.step(x_t, r, v_prev)
        b.record(stream)
        torch.cuda.synchronize()
        if i >= W:
            ms.append((a.elapsed_time(b), 1e3 * (time.perf_counter() - t0)))
    return kap, fl, ms


def run_single(args):
    import numpy as np
    import torch
    from paper_2510_08288_gb300 import build as B
    B.build()
    from paper_2510_08288_gb300 import inputs
    from paper_2510_08288_gb300 import rrg as R
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    w = inputs.WORKLOADS["single"]
    p = inputs.fc3_params()
    W, K = args.warmup, args.steps
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    legs = {}
    clocks = ClockSampler()
    torch.cuda.synchronize()
    clocks.begin()
    for name, search, prec, M in (("fp64_bisect", R.SEARCH_BISECT, R.FP64, 2),
                                  ("fp32_recheck_spec", R.SEARCH_SPEC_BISECT, R.FP32_RECHECK, 64)):
        cfg = R.rrg_config_default(horizon=w["H"], n_scenarios=w["N"], max_candidates=M, n_bisect=w["n_bisect"],
                                   search=search, precision=prec, early_exit=R.EXIT_CANDIDATE,
                                   recheck_eps_rel=RECHECK_EPS_REL)
        with R.Governor(p, cfg, stream) as g:
            x_t, _ = g.equilibrium(w["v_prev"])
            shape = None
            if search == R.SEARCH_SPEC_BISECT:
                # the tree width and probe by the library's autotuner on this
                # update (every shape gives Alg. 1's kappa)
                g.sample_scenarios(w["seed"], 0)
                shape = g.autotune(x_t, w["r"], w["v_prev"], repeats=2)[:2]
            g.reset_stats()
            kap, fl, ms = timed_updates(R, torch, g, x_t, w["r"], w["v_prev"], W, K, w["seed"], flush, stream)
            st = g.stats()
        dev = [a for a, _ in ms]
        legs[name] = {"ms_per_update": statistics.median(dev), "host_ms_per_update": statistics.median([b for _, b in ms]),
                      "kappa": kap, "flags": fl, "gpu_launches_per_update": st["launches"] // (W + K)}
        if shape is not None:
            legs[name]["shape"] = {"candidates_per_round": shape[0], "probe_steps": shape[1]}
    torch.cuda.synchronize()
    clocks.end()
    clk = clocks.stop()
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import oracle as O
        x_o = O.equilibrium(p, w["v_prev"])
        d = O.sample_disturbances(w["seed"], 0, w["N"], w["H"], inputs.DIST_AMP)
        c = O.cfg(H=w["H"], N=w["N"])
        cores = os.cpu_count() or 1
        reps, t_all = 0, 0.0
        while t_all < min(args.cpu_seconds, 5.0):
            t0 = time.perf_counter()
            k_o, f_o = O.bisect_joint(p, c, x_o, w["v_prev"], w["r"], w["n_bisect"], d, nthreads=1)
            t_all += time.perf_counter() - t0
            reps += 1
        t1 = time.perf_counter()
        O.bisect_joint(p, c, x_o, w["v_prev"], w["r"], w["n_bisect"], d, nthreads=cores)
        t_thr = time.perf_counter() - t1
        cpu = {"value": reps / t_all, "unit": "RG updates/s", "cores": 1, "kind": "oracle",
               "sample": "the same update, FP64 joint bisection, %d repetitions on 1 core" % reps,
               "ms_per_update_1core": 1e3 * t_all / reps, "ms_per_update_%dcores" % cores: 1e3 * t_thr,
               "kappa": k_o, "kappa_equal_to_gpu": bool(k_o == legs["fp64_bisect"]["kappa"] ==
                                                        legs["fp32_recheck_spec"]["kappa"])}
    main = legs["fp64_bisect"]
    # binary32 slack error against binary64 on this update, at the kappa the
    # binary32 + recheck search chose
    k32 = float(legs["fp32_recheck_spec"]["kappa"])
    fp32_err = fp32_error_probe(R, p, stream, w["H"], w["N"], w["seed"], [(0, x_t, w["v_prev"], w["r"], k32)])
    fp32_err["kappa_max_abs_diff_fp64"] = abs(k32 - float(legs["fp64_bisect"]["kappa"]))
    out = {"metric": SINGLE_METRIC, "value": 1e3 / main["ms_per_update"], "unit": "RG updates/s", "n_gpus": 1,
           "steps": K, "warmup": W, "ms_per_step": main["ms_per_update"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "single robust RG update on FC3: x_t at the 100 A equilibrium, r_t = 250 A, "
                                  "32 scenarios (seed 0), horizon 500 RK4 steps (dt=0.01 s), N_kappa = 12",
                      "timing": "median device time of sample + search (CUDA events), host time beside it",
                      "l2": "256 MB written between timed steps"},
           "legs": legs, "cpu_baseline": cpu, "clocks": clk, "fp32_error": fp32_err}
    print(json.dumps(out), flush=True)
    return 0


# ----------------------------------------------------------- adjoint (cfg 4) --
ADJ_METRIC = "adjoint gradient latency (4,096 scenarios x 1,000 steps) and Newton kappa search vs 20-step bisection"


def run_adjoint(args):
    import numpy as np
    import torch
    from paper_2510_08288_gb300 import build as B
    B.build()
    from paper_2510_08288_gb300 import inputs
    from paper_2510_08288_gb300 import rrg as R
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    w = inputs.WORKLOADS["adjoint"]
    p = inputs.fc3_params()
    W, K = args.warmup, args.steps
    N, H, C = w["N"], w["H"], w["checkpoint"]
    v_prev, r = 100.0, 250.0
    stream = torch.cuda.Stream()
    out_legs = {}
    clocks = ClockSampler()
    torch.cuda.synchronize()
    clocks.begin()
    cfg = R.rrg_config_default(horizon=H, n_scenarios=N, max_candidates=16, precision=R.FP32_RECHECK,
                               recheck_eps_rel=RECHECK_EPS_REL)
    with R.Governor(p, cfg, stream) as g:
        x_t, _ = g.equilibrium(v_prev)
        g.sample_scenarios(3, 0)
        for name, prec in (("gradient_fp64", R.FP64), ("gradient_fp32", R.FP32)):
            ts = []
            for i in range(W + K):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                gv, grad, ks, js = g.slack_gradient(x_t, v_prev, r, 0.1, C, prec)
                if i >= W:
                    ts.append(1e3 * (time.perf_counter() - t0))
            out_legs[name] = {"ms": statistics.median(ts), "g": gv, "argmin": [ks, js],
                              "dg_dkappa": float(grad[0])}
        # the forward pass's device time per launch (CUDA events on the
        # handle's stream around it), over K more binary32 gradients
        g.reset_stats()
        g.set_profiling(True)
        for i in range(K):
            g.slack_gradient(x_t, v_prev, r, 0.1, C, R.FP32)
        stp = g.stats()
        g.set_profiling(False)
        fwd_ms = stp["rollout_ms"] / max(1, stp["timed_rollouts"])
        launches_per_gradient = stp["launches"] / max(1, K)
        chain_cycles = g.step_latency(v_prev + 0.1 * (r - v_prev), H)
        tol = 2.0 ** -19
        for name, prec in (("newton_fp32_recheck_eval", R.FP32),):
            ts, res = [], None
            for i in range(W + K):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                res = g.newton_search(x_t, r, v_prev, tol=tol, max_iter=40, checkpoint=C, precision=prec)
                if i >= W:
                    ts.append(1e3 * (time.perf_counter() - t0))
            out_legs[name] = {"ms": statistics.median(ts), "kappa": res[0], "flags": res[1], "gradients": res[2]}
    # the comparator: plain bisection with 20 iterations on the same scenarios
    for name, prec, search, M in (("bisect20_fp64", R.FP64, R.SEARCH_BISECT, 2),
                                  ("bisect20_fp32_recheck_spec", R.FP32_RECHECK, R.SEARCH_SPEC_BISECT, 64)):
        cfgb = R.rrg_config_default(horizon=H, n_scenarios=N, max_candidates=M, n_bisect=20, search=search,
                                    precision=prec, recheck_eps_rel=RECHECK_EPS_REL)
        with R.Governor(p, cfgb, stream) as g:
            g.sample_scenarios(3, 0)
            ts, kap = [], None
            for i in range(W + K):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, kap, fl = g.step(x_t, r, v_prev)
                if i >= W:
                    ts.append(1e3 * (time.perf_counter() - t0))
            out_legs[name] = {"ms": statistics.median(ts), "kappa": kap, "flags": fl}
    torch.cuda.synchronize()
    clocks.end()
    clk = clocks.stop()
    kb = out_legs["bisect20_fp64"]["kappa"]
    out_legs["newton_fp32_recheck_eval"]["within_one_bracket_of_bisect20"] = bool(
        abs(out_legs["newton_fp32_recheck_eval"]["kappa"] - kb) <= 2 * tol)
    main = out_legs["gradient_fp32"]
    peak, peak_src = fp32_peak(clk)
    sm_mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz")
    achieved = N * H * FLOPS_PER_STEP / (fwd_ms * 1e-3) / 1e12
    step_cycles = fwd_ms * 1e-3 * sm_mhz * 1e6 / H if sm_mhz else None
    cpu = None if args.no_cpu_baseline else adjoint_cpu(p, x_t, v_prev, r, N, H, args.cpu_seconds,
                                                        out_legs["gradient_fp64"]["argmin"])
    value = 1e3 / main["ms"]
    out = {"metric": ADJ_METRIC, "value": value, "unit": "gradients/s", "n_gpus": 1, "steps": K,
           "warmup": W, "ms_per_step": main["ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "discrete adjoint of min slack on FC3: 4,096 scenarios (seed 3) x 1,000 RK4 "
                                  "steps, checkpoint every 50 steps, x_t at the 100 A equilibrium, r_t = 250 A, "
                                  "kappa = 0.1; Newton search to 2^-19 vs 20-iteration bisection",
                      "timing": "median host time per synchronous call (x_t in from and the gradient out to "
                                "host memory: value and e2e are the same measurement)",
                      "l2": "scenarios (49 MB binary32) re-read by every call; no flush"},
           "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": frac_of(achieved, peak),
                        "traffic": measured_traffic(ADJ_TRAFFIC_SOURCES, ADJ_TRAFFIC_PER_LAUNCH),
                        "algorithmic_bytes_per_launch": N * H * 3 * 4,
                        "kernel": "adjoint_forward_kernel<float>", "avg_launch_ms": fwd_ms,
                        "launches": stp["timed_rollouts"],
                        "timing": "CUDA events around the forward pass of %d more binary32 gradients" % K,
                        "flops_per_traj_step": FLOPS_PER_STEP, "traj_steps_per_launch": N * H,
                        "peak_source": peak_src,
                        "issue_ceiling": ISSUE_CEILING,
                        "frac_of_issue_ceiling": frac_of(frac_of(achieved, peak), ISSUE_CEILING),
                        "latency": {"cycles_per_step": step_cycles, "chain_cycles_per_step": chain_cycles,
                                    "frac": frac_of(chain_cycles, step_cycles),
                                    "basis": "forward pass time over its %d dependent steps at the sampled SM "
                                             "clock (4,096 scenarios: 128 warps, one per SM); chain: "
                                             "rrg_step_latency, one warp, the rollout kernel's step" % H}},
           "cpu_baseline": cpu,
           "e2e": {"value": value, "unit": "gradients/s", "h2d_bytes_per_step": 3 * 8,
                   "d2h_bytes_per_step": (3 + 4 + 27) * 8},
           "gpu_launches": int(round(launches_per_gradient * K)),
           "legs": out_legs, "clocks": clk}
    print(json.dumps(out), flush=True)
    return 0


def adjoint_cpu(p, x_t, v_prev, r, N, H, seconds, gpu_argmin):
    """The FP64 oracle's gradient of the same workload, whole: min slack and
    its argmin over every scenario and step, then the complex-step gradient
    at the argmin; repeated while the time stays under `seconds`."""
    from oracle import oracle as O
    from paper_2510_08288_gb300 import inputs
    c = O.cfg(H=H, N=N, early_exit=0)
    d = O.sample_disturbances(3, 0, N, H, inputs.DIST_AMP)
    I = O.governed(v_prev, r, 0.1)
    n, t, kj = 0, 0.0, None
    while n == 0 or t + t / n < seconds:
        t0 = time.perf_counter()
        g, k, j = O.min_slack_argmin(p, c, x_t, I, d)
        O.slack_grad(p, c, x_t, v_prev, r, 0.1, d, k, j)
        t += time.perf_counter() - t0
        n += 1
        kj = [k, j]
    return {"value": n / t, "unit": "gradients/s", "cores": 1, "kind": "oracle",
            "sample": "%d whole gradient(s) of the same workload (4,096 x 1,000 forward, complex-step "
                      "gradient at the argmin), FP64, one host thread, %.1f s" % (n, t),
            "argmin_equal_to_gpu_fp64": kj == list(gpu_argmin)}


# ------------------------------------------------------------------ sweep --
SWEEP_METRIC = "trajectory-steps/s vs scenario count (large sweep, FP32 + FP64 recheck)"
PAIRING_NAMES = ("never", "filled", "always")
TMA_MODES = ("never", "auto", "always")
TMA_NAMES = ("per-lane cp.async", "TMA for ring launches of >= 24 warps per SM, per-lane cp.async below",
             "TMA for every ring launch")


def sweep_ceiling(row):
    """Issue ceiling of the kernel that ran the row: FLOPS_PER_STEP over two
    flops per issued FMA slot times its instructions per trajectory-step."""
    instr = TMA_INSTR_PER_STEP if row["tma_step_fraction"] > 0.5 else INSTR_PER_STEP
    return FLOPS_PER_STEP / (2.0 * instr)


def sweep_config(ns, W, K):
    return {"workload": "large sweep on FC3: one robust RG update per step, N_sim in %s, k-section "
                        "with %d kappa candidates per round, %d rounds, horizon %d RK4 steps (dt=0.01 s), "
                        "per-step disturbances plus per-scenario parametric uncertainty +-10%% on k_ca, "
                        "eta_cp, J_cp, eta_cm, R_cm, a_w, a_p; x_t at the %g A equilibrium, r_t = %g A; "
                        "scenarios redrawn every step (update index = step)"
                        % (list(ns), SWEEP_M, SWEEP_ROUNDS, SWEEP_H, SWEEP_CASE[0], SWEEP_CASE[1]),
            "precision": "binary32 rollouts, binary64 recheck of |slack| < 1e-6*1.9",
            "timed": "steps [%d, %d) per N" % (W, W + K), "l2": "256 MB written between timed steps"}


def sweep_cpu(p, seconds, cores):
    """The FP64 oracle on a bounded sample of the sweep workload: the 16
    candidates of a k-section round on the first n scenarios (n sized to
    ~seconds), full horizon with early exit at a trajectory's first
    violation; trajectory-steps/s."""
    import numpy as np
    from oracle import oracle as O
    from paper_2510_08288_gb300 import inputs
    v_prev, r = SWEEP_CASE
    x_t = O.equilibrium(p, v_prev)
    kappas = np.linspace(0.0, 1.0, SWEEP_M)
    n = 16
    while True:
        c = O.cfg(H=SWEEP_H, N=n)
        d = O.sample_disturbances(SEED, 0, n, SWEEP_H, inputs.DIST_AMP)
        m = O.sample_param_multipliers(SEED, 0, n, inputs.PARAM_UNC_REL, inputs.FC3_UNCERTAIN_MASK)
        t0 = time.perf_counter()
        with O.param_multipliers(m):
            _, _, _, steps = O.eval_candidates(p, c, x_t, v_prev, r, kappas, d, nthreads=cores)
        dt = time.perf_counter() - t0
        if dt > seconds / 4 or n >= 4096:
            break
        n *= 2
    # the sequential oracle on one thread, over the first n / cores scenarios
    n1 = max(16, n // max(cores, 1))
    with O.param_multipliers(m[:n1]):
        t1 = time.perf_counter()
        _, _, _, steps1 = O.eval_candidates(p, O.cfg(H=SWEEP_H, N=n1), x_t, v_prev, r, kappas, d[:, :, :n1],
                                            nthreads=1)
        dt1 = time.perf_counter() - t1
    return {"value": steps / dt, "unit": "trajectory-steps/s", "cores": cores, "kind": "oracle",
            "sample": "%d scenarios x %d candidates x horizon %d, FP64, %.1f s" % (n, SWEEP_M, SWEEP_H, dt),
            "one_core": {"value": steps1 / dt1, "unit": "trajectory-steps/s", "cores": 1,
                         "sample": "%d scenarios x %d candidates x horizon %d, FP64, one host thread, %.1f s"
                                   % (n1, SWEEP_M, SWEEP_H, dt1)}}


def run_sweep(args):
    import numpy as np
    import torch
    from paper_2510_08288_gb300 import build as B
    B.build()
    from paper_2510_08288_gb300 import inputs
    from paper_2510_08288_gb300 import rrg as R
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    p = inputs.fc3_params()
    W, K = args.warmup, args.steps
    ns = [int(x) for x in args.sweep_n.split(",") if x]
    rho = inputs.PARAM_UNC_REL if args.param_unc_rel is None else args.param_unc_rel
    v_prev, r = SWEEP_CASE
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    rows = []
    clocks = ClockSampler()
    for N in ns:
        cfg = R.rrg_config_default(horizon=SWEEP_H, n_scenarios=N, max_candidates=SWEEP_M,
                                   n_rounds=SWEEP_ROUNDS, search=R.SEARCH_KSECTION,
                                   precision=R.FP32_RECHECK,
                                   early_exit=R.EXIT_CANDIDATE, recheck_eps_rel=RECHECK_EPS_REL,
                                   param_unc_rel=rho, param_unc_mask=inputs.FC3_UNCERTAIN_MASK)
        g = R.Governor(p, cfg, stream)
        x_t, _ = g.equilibrium(v_prev)
        pairing_ms = None
        if args.pairing == "autotune":
            g.sample_scenarios(SEED, 0)
            _, ms_modes = g.autotune_pairing(x_t, r, v_prev, repeats=3)
            pairing_ms = dict(zip(PAIRING_NAMES, ms_modes))
        else:
            g.set_pairing(PAIRING_NAMES.index(args.pairing))
        apply_tma(R, g, TMA_MODES.index(args.tma))
        d_x = torch.tensor(x_t, dtype=torch.float64, device=dev)
        d_r = torch.tensor([r], dtype=torch.float64, device=dev)
        d_vp = torch.tensor([v_prev], dtype=torch.float64, device=dev)
        d_out = torch.zeros(2 * (W + K), dtype=torch.float64, device=dev)
        d_fl = torch.zeros(W + K, dtype=torch.int32, device=dev)
        for t in range(W):
            g.sample_scenarios(SEED, t)
            R.rrg_step_dev(g.h, d_x, d_r, d_vp, d_out[2 * t:2 * t + 1], d_out[2 * t + 1:2 * t + 2], d_fl[t:t + 1])
        torch.cuda.synchronize()
        g.reset_stats()
        g.set_profiling(True)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        clocks.begin()
        with torch.cuda.stream(stream):
            for i in range(K):
                t = W + i
                flush.fill_(float(t))
                evs[i][0].record(stream)
                g.sample_scenarios(SEED, t)
                R.rrg_step_dev(g.h, d_x, d_r, d_vp, d_out[2 * t:2 * t + 1], d_out[2 * t + 1:2 * t + 2],
                               d_fl[t:t + 1])
                evs[i][1].record(stream)
        torch.cuda.synchronize()
        clocks.end()
        secs = sum(a.elapsed_time(b) for a, b in evs) / 1e3
        st = g.stats()
        g.set_profiling(False)
        fp32_steps = st["lane_steps"] - st["lane_steps_fp64"]
        avg_roll_ms = st["rollout_ms"] / max(1, st["timed_rollouts"])
        achieved = (fp32_steps / max(1, st["timed_rollouts"])) * FLOPS_PER_STEP / (avg_roll_ms * 1e-3) / 1e12
        kap = d_out.cpu().numpy()[1::2][W:]
        flags = d_fl.cpu().numpy()[W:]
        # the same first timed update in plain binary64 (same search), small N only
        fp64 = None
        if N <= 8192:
            cfg64 = R.rrg_config_default(horizon=SWEEP_H, n_scenarios=N, max_candidates=SWEEP_M,
                                         n_rounds=SWEEP_ROUNDS, search=R.SEARCH_KSECTION, precision=R.FP64,
                                         early_exit=R.EXIT_CANDIDATE, param_unc_rel=rho,
                                         param_unc_mask=inputs.FC3_UNCERTAIN_MASK)
            g64 = R.Governor(p, cfg64, stream)
            g64.sample_scenarios(SEED, W)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, k64, _ = g64.step(x_t, r, v_prev)
            fp64 = {"ms_per_update": 1e3 * (time.perf_counter() - t0), "kappa_equal": bool(k64 == kap[0])}
            g64.close()
        # the same updates with the disturbances drawn inside the trajectory
        # loop (no stored array, no sampler pass), at the largest N only
        gen_leg = None
        if N == ns[-1]:
            cfg_g = R.rrg_config_default(horizon=SWEEP_H, n_scenarios=N, max_candidates=SWEEP_M,
                                         n_rounds=SWEEP_ROUNDS, search=R.SEARCH_KSECTION,
                                         precision=R.FP32_RECHECK, early_exit=R.EXIT_CANDIDATE,
                                         recheck_eps_rel=RECHECK_EPS_REL, param_unc_rel=rho,
                                         param_unc_mask=inputs.FC3_UNCERTAIN_MASK, scenarios_in_register=1)
            gg = R.Governor(p, cfg_g, stream)
            kg, gms = [], []
            for t in range(W + K):
                flush.fill_(float(t))
                torch.cuda.synchronize()
                a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(stream):
                    a_ev.record(stream)
                    gg.sample_scenarios(SEED, t)
                    R.rrg_step_dev(gg.h, d_x, d_r, d_vp, d_out[2 * t:2 * t + 1], d_out[2 * t + 1:2 * t + 2],
                                   d_fl[t:t + 1])
                    b_ev.record(stream)
                torch.cuda.synchronize()
                if t >= W:
                    gms.append(a_ev.elapsed_time(b_ev))
                    kg.append(float(d_out[2 * t + 1].item()))
            gg.close()
            gen_leg = {"ms_per_update": statistics.mean(gms), "kappa_equal_to_stored": kg == [float(x) for x in kap]}
        rows.append({"n_scenarios": N, "updates_per_s": K / secs, "ms_per_update": 1e3 * secs / K,
                     "trajectory_steps_per_s": st["lane_steps"] / secs,
                     "nominal_trajectory_steps_per_update": SWEEP_ROUNDS * SWEEP_M * N * SWEEP_H,
                     "executed_trajectory_steps_per_update": st["lane_steps"] / K,
                     "rollout_tflops": achieved,
                     "rollout_avg_launch_ms": avg_roll_ms, "rechecked": st["rechecked"],
                     "pairing": PAIRING_NAMES[g.get_pairing()], "pairing_autotune_ms": pairing_ms,
                     "rollout_ring": TMA_NAMES[g.get_tma()],
                     "paired_step_fraction": st["lane_steps_paired"] / max(1, st["lane_steps"]),
                     "tma_step_fraction": st["lane_steps_tma"] / max(1, st["lane_steps"]),
                     "gpu_launches": st["launches"], "kappa": [float(x) for x in kap],
                     "no_admissible_updates": int(np.sum(flags & 1)), "fp64_same_search": fp64,
                     "scenarios_in_register": gen_leg})
        g.close()
        del d_x, d_r, d_vp, d_out, d_fl
        torch.cuda.empty_cache()
    clk = clocks.stop()
    peak, peak_src = fp32_peak(clk)
    unit_peaks = R.rrg_alu_peaks()   # measured FP32 FMA, FP64 FMA, MUFU throughput
    for row in rows:
        row["rollout_frac"] = frac_of(row["rollout_tflops"], peak)
    top = rows[-1]
    # binary32 slack error against binary64 at the first timed update of the
    # largest N, on its first 8,192 scenarios (nested draws: the run's own)
    fp32_err = fp32_error_probe(R, p, stream, SWEEP_H, top["n_scenarios"], SEED,
                                [(W, x_t, v_prev, r, top["kappa"][0])], m_grid=SWEEP_M, m_near=16,
                                param_unc=rho, n_cap=8192)
    fp32_err["kappa_equal_fp64_same_search"] = {str(row["n_scenarios"]): row["fp64_same_search"]["kappa_equal"]
                                                for row in rows if row["fp64_same_search"]}
    cpu = None if args.no_cpu_baseline else sweep_cpu(p, args.cpu_seconds, os.cpu_count() or 1)
    out = {
        "metric": SWEEP_METRIC, "value": top["trajectory_steps_per_s"], "unit": "trajectory-steps/s",
        "n_gpus": 1, "steps": K, "warmup": W, "ms_per_step": top["ms_per_update"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(sweep_config(ns, W, K), param_unc_rel=rho,
                       pairing="%s (two candidates per thread where the paired grid fills the SMs 6 times "
                               "over)" % args.pairing if args.pairing == "filled" else args.pairing),
        "roofline": {"bound": "alu", "achieved": top["rollout_tflops"], "peak": peak,
                     "unit": "TFLOP/s", "frac": top["rollout_frac"],
                     "traffic": (SWEEP_TRAFFIC_64K if top["n_scenarios"] == 65536 and rho == inputs.PARAM_UNC_REL
                                 and top["tma_step_fraction"] > 0.5 and measured_traffic() is not None
                                 else None),
                     "traffic_basis": "ncu DRAM bytes per rollout launch at 65,536 scenarios (one update's "
                                      "3 rounds, TMA ring)",
                     "kernel": ("rollout_tma_kernel<parametric> (TMA ring)" if top["tma_step_fraction"] > 0.5
                                else "rollout_pair_kernel<parametric> (two candidates per thread)"
                                if top["paired_step_fraction"] > 0.5 else "rollout_kernel<float, parametric>"),
                     "n_scenarios": top["n_scenarios"],
                     "peak_source": peak_src,
                     "issue_ceiling": sweep_ceiling(top),
                     "frac_of_issue_ceiling": frac_of(top["rollout_frac"], sweep_ceiling(top)),
                     "measured_units": {"fp32_fma_tflops": unit_peaks[0], "mufu_ex2_tops": unit_peaks[2],
                                        "frac_of_measured_fp32": top["rollout_tflops"] / unit_peaks[0],
                                        "mufu_per_traj_step": MUFU_PER_STEP,
                                        "frac_of_measured_mufu": top["rollout_tflops"] / FLOPS_PER_STEP
                                        * MUFU_PER_STEP / unit_peaks[2]}},
        "cpu_baseline": cpu, "sweep": rows, "clocks": clk,
        "gpu_launches": top["gpu_launches"],
        "fp32_error": fp32_err,
    }
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "single":
        return run_single(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
