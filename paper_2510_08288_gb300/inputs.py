"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle calls.

This module holds numbers and random draws only: the FC3 parameter values,
workload sizes and seeded generators for references, initial-state
perturbations and explicit disturbance arrays.  It contains none of the
method's arithmetic (no model equations, no integration, no search), so both
the CUDA path and the CPU oracle can be fed from it without sharing code.

Workloads follow the fuel-cell experiment of Sec. IV (dt = 0.01 s, disturbance
ranges +-50, +-10, +-50 on [p_ca, w_cp, p_sm], OER >= 1.9, 381 cells, up to
300 A).  The paper's own model equations and its benchmark data are not
available; FC3 is this library's declared third-order stand-in.
"""
from __future__ import annotations

import numpy as np

# FC3 parameter vector, in the order the C interfaces expect (SI units).
FC3_PARAM_NAMES = (
    "p_atm", "T_atm", "T_st", "R_a", "V_sm", "V_ca", "k_sm", "k_ca",
    "n_cell", "faraday", "M_O2", "x_O2", "gamma", "c_p", "eta_cp", "J_cp",
    "eta_cm", "k_t", "k_v", "R_cm", "a_w", "a_p", "lam_ref", "K_p",
    "c0", "c1", "c2",
)

FC3_DEFAULTS = {
    "p_atm": 101325.0,      # Pa, ambient pressure
    "T_atm": 298.15,        # K, ambient temperature (compressor inlet)
    "T_st": 353.15,         # K, stack / manifold temperature
    "R_a": 286.9,           # J/(kg K), gas constant of air
    "V_sm": 0.02,           # m^3, supply manifold volume
    "V_ca": 0.01,           # m^3, cathode volume
    "k_sm": 3.629e-6,       # kg/(s Pa), supply manifold -> cathode orifice
    "k_ca": 2.177e-6,       # kg/(s Pa), cathode -> ambient outlet
    "n_cell": 381.0,        # cells in the stack (Sec. IV-A)
    "faraday": 96485.0,     # C/mol
    "M_O2": 0.032,          # kg/mol
    "x_O2": 0.233,          # O2 mass fraction of dry air
    "gamma": 1.4,           # ratio of specific heats of air
    "c_p": 1004.0,          # J/(kg K)
    "eta_cp": 0.8,          # compressor isentropic efficiency
    "J_cp": 5.0e-5,         # kg m^2, compressor + motor inertia
    "eta_cm": 0.98,         # motor mechanical efficiency
    "k_t": 0.0153,          # N m/A, motor torque constant
    "k_v": 0.0153,          # V s/rad, motor back-EMF constant
    "R_cm": 0.82,           # Ohm, motor armature resistance
    "a_w": 1.2e-5,          # kg/(s rad/s), compressor flow per unit speed
    "a_p": 5.0e-7,          # kg/(s Pa), compressor flow loss per unit boost
    "lam_ref": 2.2,         # OER the low-level controller aims for
    "K_p": 500.0,           # V/(kg/s), proportional gain on the air-flow error
    # Static feed-forward motor voltage v_ff(I) = c0 + c1 I + c2 I^2, a
    # least-squares fit over 50..300 A of the voltage that holds OER = lam_ref
    # at steady state.
    "c0": 0.1669,
    "c1": 0.6123,
    "c2": -4.589e-5,
}

# Parameters perturbed per scenario in the parametric-uncertainty workload:
# the ones that set the air path's dynamics (cathode outlet, compressor map
# and efficiency, shaft inertia, motor).  k_sm is left nominal: it also scales
# the OER output map itself, so a +-10 % draw of it shifts the constrained
# output by up to 10 % at j = 0, and with 65,536 scenarios the hold (kappa =
# 0) at an equilibrium with OER 2.2 is then no longer admissible.
FC3_UNCERTAIN = ("k_ca", "eta_cp", "J_cp", "a_w", "a_p", "eta_cm", "R_cm")
FC3_UNCERTAIN_MASK = sum(1 << FC3_PARAM_NAMES.index(n) for n in FC3_UNCERTAIN)
PARAM_UNC_REL = 0.10            # +-10 % per uncertain parameter

DIST_AMP = (50.0, 10.0, 50.0)   # +-50 Pa, +-10 rad/s, +-50 Pa (Sec. IV-A)
DT = 0.01                       # s (Sec. IV-A)
Y_MIN = 1.9                     # OER lower bound (Sec. IV-A)
I_MIN, I_MAX = 50.0, 300.0      # operating range of the governed stack current, A


def fc3_params(**overrides) -> np.ndarray:
    """FC3 parameter vector (float64) with optional named overrides."""
    d = dict(FC3_DEFAULTS)
    for k, v in overrides.items():
        if k not in d:
            raise KeyError(k)
        d[k] = float(v)
    return np.array([d[n] for n in FC3_PARAM_NAMES], dtype=np.float64)


# Workload sizes.  "single" is the small update the oracle finishes in
# seconds; "closed_loop" is the 1,000-update run with 1,024 scenarios and a
# 2,000-step horizon; "batched", "adjoint" and "sweep" size the wider rows.
WORKLOADS = {
    "single": dict(N=32, H=500, n_bisect=12, v_prev=100.0, r=250.0, seed=0, update=0),
    "closed_loop": dict(N=1024, H=2000, n_bisect=12, T=1000, levels=8, hold=125, seed=1,
                        recheck_eps_rel=1e-6, v0=100.0),
    "batched": dict(instances=256, N_lo=64, N_hi=8192, H_lo=200, H_hi=4000, M=32, seed=2),
    "adjoint": dict(N=4096, H=1000, checkpoint=50, fd_h=1e-6),
    "sweep": dict(N_list=tuple(1024 * i for i in (1, 2, 4, 8, 16, 32, 64)), M=16, H=5000,
                  param_unc_rel=0.1),
}


def staircase(T: int, levels: int, hold: int, seed: int, lo: float = I_MIN, hi: float = I_MAX):
    """Piecewise-constant reference: `levels` values uniform on [lo, hi], each
    held for `hold` steps, repeated/truncated to length T (seeded)."""
    rng = np.random.default_rng(seed)
    vals = rng.uniform(lo, hi, size=levels)
    out = np.repeat(vals, hold)
    if out.shape[0] < T:
        out = np.resize(out, T)
    return np.ascontiguousarray(out[:T], dtype=np.float64)


def uniform_disturbances(N: int, H: int, seed: int, amp=DIST_AMP) -> np.ndarray:
    """Explicit disturbance array d[3][H][N], i.i.d. uniform on [-a_i, a_i)."""
    rng = np.random.default_rng(seed)
    a = np.asarray(amp, dtype=np.float64).reshape(3, 1, 1)
    return np.ascontiguousarray(a * rng.uniform(-1.0, 1.0, size=(3, H, N)))


def state_perturbation(n: int, seed: int, rel: float = 0.1) -> np.ndarray:
    """Multiplicative factors (n, 3) uniform on [1 - rel, 1 + rel]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(1.0 - rel, 1.0 + rel, size=(n, 3))


def batched_instances(S: int, seed: int, N_lo: int = 64, N_hi: int = 8192, H_lo: int = 200,
                      H_hi: int = 4000, rel: float = 0.1):
    """S independent RG problems (seeded): scenario counts log-uniform on
    [N_lo, N_hi], horizons uniform on {H_lo..H_hi}, (v_prev, r) uniform over
    the operating range, and per-state factors uniform on [1 - rel, 1 + rel]
    that the caller applies to the equilibrium of v_prev to get x_0."""
    rng = np.random.default_rng(seed)
    N = np.rint(np.exp(rng.uniform(np.log(N_lo), np.log(N_hi), size=S))).astype(np.int32)
    H = rng.integers(H_lo, H_hi + 1, size=S).astype(np.int32)
    v_prev = rng.uniform(I_MIN, I_MAX, size=S)
    r = rng.uniform(I_MIN, I_MAX, size=S)
    xfac = rng.uniform(1.0 - rel, 1.0 + rel, size=(S, 3))
    return {"N": np.clip(N, N_lo, N_hi), "H": H, "v_prev": v_prev, "r": r, "xfac": xfac}


def random_problems(n: int, seed: int):
    """(v_prev, r) pairs drawn uniformly over the operating range."""
    rng = np.random.default_rng(seed)
    return rng.uniform(I_MIN, I_MAX, size=n), rng.uniform(I_MIN, I_MAX, size=n)
