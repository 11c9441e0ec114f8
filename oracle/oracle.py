"""ctypes binding of the FP64 CPU oracle (rrg_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check of
the build entry point and by the CPU-baseline / reference legs of the
benchmark.  The CUDA product path never imports this module, and this module
imports nothing from the product package.

Every wrapper names the passage of the paper (arXiv 2510.08288) that the C
function it calls follows.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rrg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.%s.so" % platform.machine())
_lock = threading.Lock()
_lib = None

_d = ctypes.c_double
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_int = ctypes.c_int
_p = ctypes.c_void_p


class OrcCfg(ctypes.Structure):
    """Mirror of orc_cfg in rrg_oracle.c."""

    _fields_ = [
        ("dt", _d), ("H", _i64), ("N", _i64), ("y_min", _d), ("ss_check", _int),
        ("eps_ss", _d), ("y_c", _d), ("early_exit", _int),
    ]


def build(force: bool = False) -> str:
    """Compile rrg_oracle.c with the host C compiler (no fused multiply-add)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + ".tmp%d" % os.getpid()
            cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                   "-shared", "-pthread", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_nparam.restype = _int
        L.orc_fc3_rhs.argtypes = [_p, _p, _d, _p]
        L.orc_fc3_output.argtypes = [_p, _p, _d]
        L.orc_fc3_output.restype = _d
        L.orc_rk4_step.argtypes = [_p, _p, _d, _d, _p]
        L.orc_rk4_linear.argtypes = [_int, _p, _p, _d, _p, _d, _p]
        L.orc_philox4x64_10.argtypes = [_p, _p, _p]
        L.orc_sample_disturbances.argtypes = [_u64, _u64, _i64, _i64, _p, _p]
        L.orc_plant_disturbance.argtypes = [_u64, _u64, _p, _p]
        L.orc_equilibrium.argtypes = [_p, _d, _p]
        L.orc_equilibrium.restype = _int
        L.orc_ss_ok.argtypes = [_p, ctypes.POINTER(OrcCfg), _d]
        L.orc_ss_ok.restype = _int
        L.orc_rollout.argtypes = [_p, ctypes.POINTER(OrcCfg), _p, _d, _p, _i64, ctypes.POINTER(_i64)]
        L.orc_rollout.restype = _d
        L.orc_governed.argtypes = [_d, _d, _d]
        L.orc_governed.restype = _d
        L.orc_eval_candidates.argtypes = [_p, ctypes.POINTER(OrcCfg), _p, _d, _d, _p, _int, _p,
                                          _p, _p, _p, _int]
        L.orc_eval_candidates.restype = _i64
        L.orc_alg1.argtypes = [_p, ctypes.POINTER(OrcCfg), _p, _d, _d, _int, ctypes.POINTER(_int)]
        L.orc_alg1.restype = _d
        L.orc_alg2.argtypes = [_p, ctypes.POINTER(OrcCfg), _p, _d, _d, _int, _p, ctypes.POINTER(_int)]
        L.orc_alg2.restype = _d
        L.orc_bisect_joint.argtypes = [_p, ctypes.POINTER(OrcCfg), _p, _d, _d, _int, _p,
                                       ctypes.POINTER(_int), _int]
        L.orc_bisect_joint.restype = _d
        L.orc_alg3.argtypes = [_p, ctypes.POINTER(OrcCfg), _p, _d, _d, _int, _p,
                               ctypes.POINTER(_int), _int]
        L.orc_alg3.restype = _d
        L.orc_ksection.argtypes = [_p, ctypes.POINTER(OrcCfg), _p, _d, _d, _int, _int, _p,
                                   ctypes.POINTER(_int), _int]
        L.orc_ksection.restype = _d
        L.orc_closed_loop.argtypes = [_p, ctypes.POINTER(OrcCfg), _p, _d, _p, _int, _u64, _u64,
                                      _p, _p, _int, _int, _int, _int, _int, _d, ctypes.c_uint32,
                                      _p, _p, _p, _p]
        L.orc_closed_loop.restype = _i64
        L.orc_min_slack_argmin.argtypes = [_p, ctypes.POINTER(OrcCfg), _p, _d, _p, ctypes.POINTER(_i64),
                                           ctypes.POINTER(_i64)]
        L.orc_min_slack_argmin.restype = _d
        L.orc_slack_grad.argtypes = [_p, ctypes.POINTER(OrcCfg), _p, _d, _d, _d, _p, _i64, _i64, _p, _p]
        L.orc_sample_param_multipliers.argtypes = [_u64, _u64, _i64, _d, ctypes.c_uint32, _p]
        L.orc_set_param_multipliers.argtypes = [_p]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def cfg(dt=0.01, H=500, N=32, y_min=1.9, ss_check=1, eps_ss=0.05, y_c=2.2, early_exit=1) -> OrcCfg:
    """Problem configuration (Sec. II and IV-A: j*, dt, Y, epsilon)."""
    return OrcCfg(dt, int(H), int(N), y_min, int(ss_check), eps_ss, y_c, int(early_exit))


def nparam() -> int:
    return lib().orc_nparam()


def rhs(p, x, I):
    """FC3 right-hand side f_c(x, v) (the model stand-in for Sec. IV-A)."""
    p, x = _f64(p), _f64(x)
    out = np.zeros(3)
    lib().orc_fc3_rhs(_ptr(p), _ptr(x), float(I), _ptr(out))
    return out


def output(p, x, I) -> float:
    """FC3 output h(x, v) = oxygen excess ratio (Sec. IV-A)."""
    p, x = _f64(p), _f64(x)
    return lib().orc_fc3_output(_ptr(p), _ptr(x), float(I))


def rk4_step(p, x, I, dt):
    """One RK4 step of FC3 (Sec. IV-A, fixed step)."""
    p, x = _f64(p), _f64(x)
    out = np.zeros(3)
    lib().orc_rk4_step(_ptr(p), _ptr(x), float(I), float(dt), _ptr(out))
    return out


def rk4_linear(A, B, u, x, dt):
    """One RK4 step of dx/dt = A x + B u (pin of the integrator)."""
    A, B, x = _f64(A), _f64(B), _f64(x)
    n = x.shape[0]
    out = np.zeros(n)
    lib().orc_rk4_linear(n, _ptr(A), _ptr(B), float(u), _ptr(x), float(dt), _ptr(out))
    return out


def philox4x64_10(ctr, key):
    """Philox4x64-10 block (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint64))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64))
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def sample_disturbances(seed, update, N, H, amp):
    """d_j^k of one RG update (Sec. II-C; Alg. 3 step 2), layout [3][H][N]."""
    amp = _f64(amp)
    d = np.zeros((3, H, N))
    lib().orc_sample_disturbances(int(seed), int(update), int(N), int(H), _ptr(amp), _ptr(d))
    return d


def plant_disturbance(seed, t, amp):
    amp = _f64(amp)
    out = np.zeros(3)
    lib().orc_plant_disturbance(int(seed), int(t), _ptr(amp), _ptr(out))
    return out


def equilibrium(p, I):
    """Equilibrium x_eq(v) of the closed loop (Sec. II-A, equilibrium manifold)."""
    p = _f64(p)
    x = np.zeros(3)
    rc = lib().orc_equilibrium(_ptr(p), float(I), _ptr(x))
    if rc != 0:
        raise ValueError("no equilibrium for I=%r (code %d)" % (I, rc))
    return x


def ss_ok(p, c: OrcCfg, I) -> bool:
    p = _f64(p)
    return bool(lib().orc_ss_ok(_ptr(p), ctypes.byref(c), float(I)))


def rollout(p, c: OrcCfg, x0, I, d=None, k=0):
    """min_j slack of one scenario rollout (Alg. 3 steps 2-3); returns (smin, steps)."""
    p, x0 = _f64(p), _f64(x0)
    st = _i64(0)
    dd = _f64(d) if d is not None else None
    dp = _ptr(dd) if dd is not None else None
    s = lib().orc_rollout(_ptr(p), ctypes.byref(c), _ptr(x0), float(I), dp, int(k), ctypes.byref(st))
    return s, st.value


def governed(v_prev, r, kappa) -> float:
    """Eq. 2."""
    return lib().orc_governed(float(v_prev), float(r), float(kappa))


def eval_candidates(p, c: OrcCfg, x_t, v_prev, r, kappas, d, want_P=False, nthreads=1):
    """Alg. 3 parallel steps over given kappas: (adm[m], min_slack[m], P[m,N] or None, steps)."""
    p, x_t, kap, d = _f64(p), _f64(x_t), _f64(kappas), _f64(d)
    m = kap.shape[0]
    adm = np.zeros(m, dtype=np.uint8)
    ms = np.zeros(m)
    P = np.zeros((m, c.N), dtype=np.uint8) if want_P else None
    steps = lib().orc_eval_candidates(_ptr(p), ctypes.byref(c), _ptr(x_t), float(v_prev), float(r),
                                      _ptr(kap), m, _ptr(d), _ptr(adm), _ptr(ms),
                                      _ptr(P) if P is not None else None, int(nthreads))
    return adm, ms, P, steps


def alg1(p, c, x_t, v_prev, r, n_kappa):
    """Alg. 1 (nominal bisection); returns (kappa, flags)."""
    p, x_t = _f64(p), _f64(x_t)
    f = _int(0)
    k = lib().orc_alg1(_ptr(p), ctypes.byref(c), _ptr(x_t), float(v_prev), float(r), int(n_kappa),
                       ctypes.byref(f))
    return k, f.value


def alg2(p, c, x_t, v_prev, r, n_kappa, d):
    """Alg. 2 (min over scenarios of per-scenario bisection); returns (kappa, flags)."""
    p, x_t, d = _f64(p), _f64(x_t), _f64(d)
    f = _int(0)
    k = lib().orc_alg2(_ptr(p), ctypes.byref(c), _ptr(x_t), float(v_prev), float(r), int(n_kappa),
                       _ptr(d), ctypes.byref(f))
    return k, f.value


def bisect_joint(p, c, x_t, v_prev, r, n_kappa, d, nthreads=1):
    """Alg. 1 on the joint all-scenario predicate; returns (kappa, flags)."""
    p, x_t, d = _f64(p), _f64(x_t), _f64(d)
    f = _int(0)
    k = lib().orc_bisect_joint(_ptr(p), ctypes.byref(c), _ptr(x_t), float(v_prev), float(r),
                               int(n_kappa), _ptr(d), ctypes.byref(f), int(nthreads))
    return k, f.value


def alg3(p, c, x_t, v_prev, r, M, d, nthreads=1):
    """Alg. 3 / Eq. 5 grid search; returns (kappa, flags)."""
    p, x_t, d = _f64(p), _f64(x_t), _f64(d)
    f = _int(0)
    k = lib().orc_alg3(_ptr(p), ctypes.byref(c), _ptr(x_t), float(v_prev), float(r), int(M),
                       _ptr(d), ctypes.byref(f), int(nthreads))
    return k, f.value


def ksection(p, c, x_t, v_prev, r, M, rounds, d, nthreads=1):
    """Multi-round grid (k-section) built on Alg. 3; returns (kappa, flags)."""
    p, x_t, d = _f64(p), _f64(x_t), _f64(d)
    f = _int(0)
    k = lib().orc_ksection(_ptr(p), ctypes.byref(c), _ptr(x_t), float(v_prev), float(r), int(M),
                           int(rounds), _ptr(d), ctypes.byref(f), int(nthreads))
    return k, f.value


def closed_loop(p, c, x0, v0, r_seq, seed, t0, amp, plant_amp, search=0, n_kappa=12, M=32,
                rounds=2, nthreads=1, param_unc_rel=0.0, param_unc_mask=0):
    """Closed loop of Fig. 1 under the robust RG; returns (v[T], kappa[T], flags[T], x[T+1,3]).
    param_unc_rel > 0: each update's scenarios also draw parameter multipliers."""
    p, x0, r_seq, amp, plant_amp = _f64(p), _f64(x0), _f64(r_seq), _f64(amp), _f64(plant_amp)
    T = r_seq.shape[0]
    v = np.zeros(T)
    kap = np.zeros(T)
    fl = np.zeros(T, dtype=np.int32)
    xs = np.zeros((T + 1, 3))
    lib().orc_closed_loop(_ptr(p), ctypes.byref(c), _ptr(x0), float(v0), _ptr(r_seq), T, int(seed),
                          int(t0), _ptr(amp), _ptr(plant_amp), int(search), int(n_kappa), int(M),
                          int(rounds), int(nthreads), float(param_unc_rel), int(param_unc_mask),
                          _ptr(v), _ptr(kap), _ptr(fl), _ptr(xs))
    return v, kap, fl, xs


def min_slack_argmin(p, c, x0, I, d=None):
    """min over scenarios and steps of the slack (full horizon) and its argmin (k, j)."""
    p, x0 = _f64(p), _f64(x0)
    dd = _f64(d) if d is not None else None
    kk, jj = _i64(0), _i64(0)
    g = lib().orc_min_slack_argmin(_ptr(p), ctypes.byref(c), _ptr(x0), float(I),
                                   _ptr(dd) if dd is not None else None, ctypes.byref(kk), ctypes.byref(jj))
    return g, kk.value, jj.value


def slack_grad(p, c, x_t, v_prev, r, kappa, d, k, jstar):
    """Complex-step gradient of s_jstar^k w.r.t. (kappa, x_t[3], theta[27]); returns (s, grad[31])."""
    p, x_t = _f64(p), _f64(x_t)
    dd = _f64(d) if d is not None else None
    grad = np.zeros(4 + p.shape[0])
    s = ctypes.c_double(0.0)
    lib().orc_slack_grad(_ptr(p), ctypes.byref(c), _ptr(x_t), float(v_prev), float(r), float(kappa),
                         _ptr(dd) if dd is not None else None, int(k), int(jstar), _ptr(grad), ctypes.byref(s))
    return s.value, grad


def sample_param_multipliers(seed, update, N, rho, mask):
    """Per-scenario parameter multipliers m[k, p] (parametric uncertainty workload)."""
    m = np.zeros((N, nparam()))
    lib().orc_sample_param_multipliers(int(seed), int(update), int(N), float(rho), int(mask), _ptr(m))
    return m


class param_multipliers:
    """Context manager: evaluations inside use scenario k's parameters p * m[k]."""

    def __init__(self, m):
        self.m = None if m is None else np.ascontiguousarray(np.asarray(m, dtype=np.float64))

    def __enter__(self):
        lib().orc_set_param_multipliers(_ptr(self.m) if self.m is not None else None)
        return self

    def __exit__(self, *exc):
        lib().orc_set_param_multipliers(None)
