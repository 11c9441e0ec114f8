"""Python binding of librrg (include/rrg.h): argument marshalling only.

Every function here forwards to the C entry point of the same name; all
computation runs in the library's CUDA kernels.  There is no CPU fallback:
if librrg.so is missing or fails to load, importing this module raises.

PyTorch is used only as a provider of device memory and streams for the
``*_dev`` entry points (tensors are passed by ``data_ptr()``).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("RRG_LIBRARY") or os.path.join(_HERE, "librrg.so")

RRG_OK, RRG_EINVAL, RRG_ENOMEM, RRG_ECUDA, RRG_ETIMEOUT, RRG_ENOTIMPL = range(6)
SEARCH_BISECT, SEARCH_GRID, SEARCH_KSECTION, SEARCH_SPEC_BISECT = range(4)
FP64, FP32, FP32_RECHECK = range(3)
EXIT_NONE, EXIT_LANE, EXIT_CANDIDATE = range(3)
PAIR_NEVER, PAIR_FILLED, PAIR_ALWAYS = range(3)
TMA_NEVER, TMA_AUTO, TMA_ALWAYS = range(3)
INJECT_TMA_NO_COPY = 1
NPARAM = 27
MAX_CANDIDATES = 1024
FLAG_NONE_ADMISSIBLE = 1
FLAG_INVALID_INPUT = 2

_d, _i32, _u64, _p = ctypes.c_double, ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p


class RrgConfig(ctypes.Structure):
    """Mirror of rrg_config."""

    _fields_ = [
        ("dt", _d), ("horizon", _i32), ("n_scenarios", _i32), ("max_candidates", _i32),
        ("n_bisect", _i32), ("n_rounds", _i32), ("search", _i32), ("precision", _i32),
        ("early_exit", _i32), ("ss_check", _i32), ("y_min", _d), ("eps_ss", _d), ("y_c", _d),
        ("recheck_eps_rel", _d), ("dist_amp", _d * 3), ("probe_steps", _i32),
        ("param_unc_rel", _d), ("param_unc_mask", ctypes.c_uint32), ("scenarios_in_register", _i32),
        ("scenario_base", ctypes.c_int64),
    ]


class RrgBisectState(ctypes.Structure):
    """Mirror of rrg_bisect_state."""

    _fields_ = [
        ("lo", _d), ("hi", _d), ("kappa", _d), ("kappa_opt", _d), ("iter", _i32), ("n_bisect", _i32),
        ("any", _i32), ("done", _i32),
    ]


class RrgStats(ctypes.Structure):
    """Mirror of rrg_stats."""

    _fields_ = [
        ("launches", _u64), ("rollout_launches", _u64), ("lane_steps", _u64),
        ("lane_steps_fp64", _u64), ("rechecked", _u64), ("rounds", _u64),
        ("rollout_ms", _d), ("recheck_ms", _d), ("timed_rollouts", _u64), ("repairs", _u64),
        ("graph_conditional", _u64), ("lane_steps_paired", _u64), ("wait_timeouts", _u64),
        ("lane_steps_tma", _u64),
    ]


class RrgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("librrg error %d: %s" % (code, msg))
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("librrg.so not built (%s); run paper_2510_08288_gb300.build.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    sig = {
        "rrg_config_default": (None, [P(RrgConfig)]),
        "rrg_create": (ctypes.c_int, [_p, ctypes.c_int, P(RrgConfig), _p, P(_p)]),
        "rrg_destroy": (ctypes.c_int, [_p]),
        "rrg_last_error": (ctypes.c_char_p, [_p]),
        "rrg_sample_scenarios": (ctypes.c_int, [_p, _u64, _u64]),
        "rrg_set_scenarios": (ctypes.c_int, [_p, _p]),
        "rrg_get_scenarios": (ctypes.c_int, [_p, _p]),
        "rrg_get_param_multipliers": (ctypes.c_int, [_p, _p]),
        "rrg_set_param_multipliers": (ctypes.c_int, [_p, _p]),
        "rrg_eval_candidates": (ctypes.c_int, [_p, _p, _d, _d, _p, ctypes.c_int, _p, _p, _p]),
        "rrg_bisect_init": (ctypes.c_int, [P(RrgBisectState), ctypes.c_int]),
        "rrg_bisect_plan": (ctypes.c_int, [P(RrgBisectState), ctypes.c_int, _p, P(_i32)]),
        "rrg_bisect_decide": (ctypes.c_int, [P(RrgBisectState), _p, ctypes.c_int]),
        "rrg_slack_error": (ctypes.c_int, [_p, _p, _d, _d, _p, ctypes.c_int, _d, _p, _p, _p, _p, _p, _p]),
        "rrg_step": (ctypes.c_int, [_p, _p, _d, _d, _p, _p, _p]),
        "rrg_step_dev": (ctypes.c_int, [_p, _p, _p, _p, _p, _p, _p]),
        "rrg_equilibrium": (ctypes.c_int, [_p, _d, _p, _p]),
        "rrg_closed_loop": (ctypes.c_int, [_p, _p, _d, _p, ctypes.c_int, _u64, _u64, _p, ctypes.c_int,
                                           _p, _p, _p, _p]),
        "rrg_closed_loop_dev": (ctypes.c_int, [_p, _p, _d, _p, ctypes.c_int, _u64, _u64, _p,
                                               ctypes.c_int, _p, _p, _p, _p]),
        "rrg_plant_step": (ctypes.c_int, [_p, _p, _d, _u64, _u64, _p, _p]),
        "rrg_set_profiling": (ctypes.c_int, [_p, ctypes.c_int]),
        "rrg_set_tuning": (ctypes.c_int, [_p, ctypes.c_int, ctypes.c_int]),
        "rrg_get_tuning": (ctypes.c_int, [_p, _p, _p]),
        "rrg_autotune": (ctypes.c_int, [_p, _p, _d, _d, ctypes.c_int, _p, _p, _p]),
        "rrg_set_pairing": (ctypes.c_int, [_p, ctypes.c_int]),
        "rrg_set_tma": (ctypes.c_int, [_p, ctypes.c_int]),
        "rrg_get_tma": (ctypes.c_int, [_p, _p]),
        "rrg_set_injection": (ctypes.c_int, [_p, ctypes.c_int]),
        "rrg_get_pairing": (ctypes.c_int, [_p, _p]),
        "rrg_autotune_pairing": (ctypes.c_int, [_p, _p, _d, _d, ctypes.c_int, _p, _p]),
        "rrg_get_stats": (ctypes.c_int, [_p, P(RrgStats)]),
        "rrg_reset_stats": (ctypes.c_int, [_p]),
        "rrg_slack_gradient": (ctypes.c_int, [_p, _p, _d, _d, _d, ctypes.c_int, ctypes.c_int, _p, _p,
                                              P(ctypes.c_int64), P(ctypes.c_int64)]),
        "rrg_slack_gradients": (ctypes.c_int, [_p, _p, _d, _d, _p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               _p, _p, _p, _p, _p]),
        "rrg_newton_search": (ctypes.c_int, [_p, _p, _d, _d, _d, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             _p, _p, _p]),
        "rrg_eval_candidates_static": (ctypes.c_int, [_p, ctypes.c_int, P(RrgConfig), _p, _p, _p, _p, _d,
                                                      _d, _p, ctypes.c_int, _p, _p]),
        "rrg_alu_peaks": (ctypes.c_int, [_p, _p, _p]),
        "rrg_step_latency": (ctypes.c_int, [_p, ctypes.c_double, ctypes.c_int, _p]),
        "rrg_batch_create": (ctypes.c_int, [_p, ctypes.c_int, P(RrgConfig), ctypes.c_int, _p, _p, _p, P(_p)]),
        "rrg_batch_destroy": (ctypes.c_int, [_p]),
        "rrg_batch_last_error": (ctypes.c_char_p, [_p]),
        "rrg_batch_step_dev": (ctypes.c_int, [_p, _p, _p, _p, _u64, _u64, _p, _p, _p]),
        "rrg_batch_closed_loop_dev": (ctypes.c_int, [_p, _p, _p, _p, ctypes.c_int, _u64, _u64, _p, ctypes.c_int,
                                                     _p, _p, _p, _p]),
        "rrg_batch_autotune": (ctypes.c_int, [_p, _p, _p, _p, _u64, _u64, ctypes.c_int, P(ctypes.c_int), _p]),
        "rrg_batch_set_width": (ctypes.c_int, [_p, ctypes.c_int]),
        "rrg_batch_get_width": (ctypes.c_int, [_p, P(ctypes.c_int)]),
        "rrg_batch_autotune_width": (ctypes.c_int, [_p, _p, _p, _p, _u64, _u64, ctypes.c_int, P(ctypes.c_int), _p,
                                                    _p, P(ctypes.c_int)]),
        "rrg_batch_set_variant": (ctypes.c_int, [_p, ctypes.c_int]),
        "rrg_batch_get_variant": (ctypes.c_int, [_p, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int)]),
        "rrg_batch_set_profiling": (ctypes.c_int, [_p, ctypes.c_int]),
        "rrg_batch_get_stats": (ctypes.c_int, [_p, P(RrgStats)]),
        "rrg_batch_reset_stats": (ctypes.c_int, [_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def rrg_config_default(**overrides) -> RrgConfig:
    """rrg_config_default, then named field overrides (dist_amp as a 3-sequence)."""
    c = RrgConfig()
    lib.rrg_config_default(ctypes.byref(c))
    for k, v in overrides.items():
        if k == "dist_amp":
            c.dist_amp = (_d * 3)(*[float(x) for x in v])
        elif hasattr(c, k):
            setattr(c, k, v)
        else:
            raise KeyError(k)
    return c


def rrg_last_error(h=None) -> str:
    s = lib.rrg_last_error(h)
    return s.decode() if s else ""


def _check(rc, h=None):
    if rc != RRG_OK:
        raise RrgError(rc, rrg_last_error(h))


def _tensor_ptr(t):
    """Device address of a torch tensor (or an int address)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def rrg_create(params, cfg: RrgConfig, stream=None):
    p = _f64(params)
    h = _p()
    rc = lib.rrg_create(_ptr(p), int(p.shape[0]), ctypes.byref(cfg), _stream_ptr(stream), ctypes.byref(h))
    _check(rc, None)
    return h


def rrg_destroy(h):
    _check(lib.rrg_destroy(h))


def rrg_sample_scenarios(h, seed, update_index):
    _check(lib.rrg_sample_scenarios(h, int(seed), int(update_index)), h)


def rrg_set_scenarios(h, d):
    d = _f64(d)
    _check(lib.rrg_set_scenarios(h, _ptr(d)), h)


def rrg_get_scenarios(h, n_scenarios, horizon):
    d = np.zeros((3, horizon, n_scenarios))
    _check(lib.rrg_get_scenarios(h, _ptr(d)), h)
    return d


def rrg_get_param_multipliers(h, n_scenarios):
    m = np.zeros((n_scenarios, NPARAM))
    _check(lib.rrg_get_param_multipliers(h, _ptr(m)), h)
    return m


def rrg_set_param_multipliers(h, m):
    m = _f64(m)
    _check(lib.rrg_set_param_multipliers(h, _ptr(m)), h)


def rrg_eval_candidates(h, x_t, v_prev, r_t, kappas, want_P=False, n_scenarios=None):
    x, k = _f64(x_t), _f64(kappas)
    m = k.shape[0]
    adm = np.zeros(m, dtype=np.uint8)
    ms = np.zeros(m)
    P = np.zeros((m, n_scenarios), dtype=np.uint8) if want_P else None
    rc = lib.rrg_eval_candidates(h, _ptr(x), float(v_prev), float(r_t), _ptr(k), m, _ptr(adm), _ptr(ms),
                                 _ptr(P) if P is not None else None)
    _check(rc, h)
    return adm, ms, P


def rrg_slack_error(h, x_t, v_prev, r_t, kappas, band, n_scenarios):
    """Per-trajectory binary32-vs-binary64 slack error (all arrays [m, N]):
    returns dict err, j_err, smin32, smin64, unsafe, ratio."""
    x, k = _f64(x_t), _f64(kappas)
    m = k.shape[0]
    out = dict(err=np.zeros((m, n_scenarios)), j_err=np.zeros((m, n_scenarios), dtype=np.int32),
               smin32=np.zeros((m, n_scenarios)), smin64=np.zeros((m, n_scenarios)),
               unsafe=np.zeros((m, n_scenarios), dtype=np.int32), ratio=np.zeros((m, n_scenarios)))
    rc = lib.rrg_slack_error(h, _ptr(x), float(v_prev), float(r_t), _ptr(k), m, float(band),
                             _ptr(out["err"]), _ptr(out["j_err"]), _ptr(out["smin32"]),
                             _ptr(out["smin64"]), _ptr(out["unsafe"]), _ptr(out["ratio"]))
    _check(rc, h)
    return out


def rrg_bisect_init(n_bisect) -> RrgBisectState:
    s = RrgBisectState()
    _check(lib.rrg_bisect_init(ctypes.byref(s), int(n_bisect)))
    return s


def rrg_bisect_plan(s: RrgBisectState, m_max):
    """The next round's kappas (empty once the search is done)."""
    k = np.zeros(max(1, int(m_max)))
    m = _i32(0)
    _check(lib.rrg_bisect_plan(ctypes.byref(s), int(m_max), _ptr(k), ctypes.byref(m)))
    return k[:m.value].copy()


def rrg_bisect_decide(s: RrgBisectState, admissible):
    a = np.ascontiguousarray(np.asarray(admissible, dtype=np.uint8))
    _check(lib.rrg_bisect_decide(ctypes.byref(s), _ptr(a), int(a.shape[0])))


def rrg_step(h, x_t, r_t, v_prev):
    x = _f64(x_t)
    v, kap, fl = _d(0.0), _d(0.0), _i32(0)
    _check(lib.rrg_step(h, _ptr(x), float(r_t), float(v_prev), ctypes.byref(v), ctypes.byref(kap),
                        ctypes.byref(fl)), h)
    return v.value, kap.value, fl.value


def rrg_step_dev(h, d_x_t, d_r_t, d_v_prev, d_v_t, d_kappa, d_flags):
    _check(lib.rrg_step_dev(h, _tensor_ptr(d_x_t), _tensor_ptr(d_r_t), _tensor_ptr(d_v_prev),
                            _tensor_ptr(d_v_t), _tensor_ptr(d_kappa), _tensor_ptr(d_flags)), h)


def rrg_equilibrium(h, v):
    x = np.zeros(3)
    y = _d(0.0)
    _check(lib.rrg_equilibrium(h, float(v), _ptr(x), ctypes.byref(y)), h)
    return x, y.value


def rrg_step_latency(h, v, steps=2000):
    """Cycles per binary32 trajectory step for one warp on the current GPU."""
    c = _d(0.0)
    _check(lib.rrg_step_latency(h, float(v), int(steps), ctypes.byref(c)), h)
    return c.value


def rrg_closed_loop(h, x0, v0, r_seq, seed, t0, plant_amp, use_graph=True):
    x0, r, amp = _f64(x0), _f64(r_seq), _f64(plant_amp)
    T = r.shape[0]
    v = np.zeros(T)
    kap = np.zeros(T)
    fl = np.zeros(T, dtype=np.int32)
    xs = np.zeros((T + 1, 3))
    _check(lib.rrg_closed_loop(h, _ptr(x0), float(v0), _ptr(r), T, int(seed), int(t0), _ptr(amp),
                               int(bool(use_graph)), _ptr(v), _ptr(kap), _ptr(fl), _ptr(xs)), h)
    return v, kap, fl, xs


def rrg_closed_loop_dev(h, x0, v0, d_r_seq, T, seed, t0, plant_amp, use_graph, d_v_out, d_kappa_out,
                        d_flags_out, d_x_out):
    amp = _f64(plant_amp)
    x0 = _f64(x0) if x0 is not None else None      # None: continue the previous loop
    _check(lib.rrg_closed_loop_dev(h, _ptr(x0) if x0 is not None else None, float(v0),
                                   _tensor_ptr(d_r_seq), int(T), int(seed),
                                   int(t0), _ptr(amp), int(bool(use_graph)), _tensor_ptr(d_v_out),
                                   _tensor_ptr(d_kappa_out), _tensor_ptr(d_flags_out),
                                   _tensor_ptr(d_x_out)), h)


def rrg_plant_step(h, x_t, v_t, seed, t, plant_amp):
    x, amp = _f64(x_t), _f64(plant_amp)
    out = np.zeros(3)
    _check(lib.rrg_plant_step(h, _ptr(x), float(v_t), int(seed), int(t), _ptr(amp), _ptr(out)), h)
    return out


def rrg_slack_gradient(h, x_t, v_prev, r_t, kappa, checkpoint=50, precision=FP64):
    """(g, grad[31], k*, j*): min slack over scenarios and steps and its
    gradient w.r.t. (kappa, x_t[3], theta[27]) by the discrete adjoint."""
    x = _f64(x_t)
    g = _d(0.0)
    grad = np.zeros(4 + NPARAM)
    ks, js = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib.rrg_slack_gradient(h, _ptr(x), float(v_prev), float(r_t), float(kappa), int(checkpoint),
                                  int(precision), ctypes.byref(g), _ptr(grad), ctypes.byref(ks),
                                  ctypes.byref(js)), h)
    return g.value, grad, ks.value, js.value


def rrg_slack_gradients(h, x_t, v_prev, r_t, kappas, checkpoint=50, precision=FP64):
    """Gradients at m kappas in one call: (g[m], grad[m, 31], k*[m], j*[m],
    ss_ok[m])."""
    x, k = _f64(x_t), _f64(kappas)
    m = k.shape[0]
    g, grad = np.zeros(m), np.zeros((m, 4 + NPARAM))
    ks, js = np.zeros(m, dtype=np.int64), np.zeros(m, dtype=np.int64)
    ss = np.zeros(m, dtype=np.uint8)
    _check(lib.rrg_slack_gradients(h, _ptr(x), float(v_prev), float(r_t), _ptr(k), m, int(checkpoint),
                                   int(precision), _ptr(g), _ptr(grad), _ptr(ks), _ptr(js), _ptr(ss)), h)
    return g, grad, ks, js, ss


def rrg_newton_search(h, x_t, r_t, v_prev, tol=2.0 ** -19, max_iter=40, checkpoint=50, precision=FP64):
    """(kappa, flags, iterations) of the adjoint-driven Newton search."""
    x = _f64(x_t)
    k, fl, it = _d(0.0), _i32(0), _i32(0)
    _check(lib.rrg_newton_search(h, _ptr(x), float(r_t), float(v_prev), float(tol), int(max_iter),
                                 int(checkpoint), int(precision), ctypes.byref(k), ctypes.byref(fl),
                                 ctypes.byref(it)), h)
    return k.value, fl.value, it.value


def rrg_set_tuning(h, m, probe_steps):
    _check(lib.rrg_set_tuning(h, int(m), int(probe_steps)), h)


def rrg_get_tuning(h):
    """(tree nodes per round, probe steps) of the speculative bisection."""
    m, p = _i32(0), _i32(0)
    _check(lib.rrg_get_tuning(h, ctypes.byref(m), ctypes.byref(p)), h)
    return m.value, p.value


def rrg_autotune(h, x_t, r_t, v_prev, repeats=2):
    """(m, probe_steps, mean ms per update) chosen by the autotuner."""
    x = _f64(x_t)
    m, p, ms = _i32(0), _i32(0), _d(0.0)
    _check(lib.rrg_autotune(h, _ptr(x), float(r_t), float(v_prev), int(repeats), ctypes.byref(m),
                            ctypes.byref(p), ctypes.byref(ms)), h)
    return m.value, p.value, ms.value


def rrg_set_pairing(h, mode):
    _check(lib.rrg_set_pairing(h, int(mode)), h)


def rrg_set_tma(h, mode):
    _check(lib.rrg_set_tma(h, int(mode)), h)


def rrg_set_injection(h, flags):
    _check(lib.rrg_set_injection(h, int(flags)), h)


def rrg_get_tma(h):
    """TMA_NEVER, TMA_AUTO or TMA_ALWAYS (TMA_NEVER where the TMA ring is unavailable)."""
    m = _i32(0)
    _check(lib.rrg_get_tma(h, ctypes.byref(m)), h)
    return m.value


def rrg_get_pairing(h):
    """PAIR_NEVER, PAIR_FILLED or PAIR_ALWAYS."""
    m = _i32(0)
    _check(lib.rrg_get_pairing(h, ctypes.byref(m)), h)
    return m.value


def rrg_autotune_pairing(h, x_t, r_t, v_prev, repeats=2):
    """(chosen pairing mode, mean ms per update of each mode)."""
    x = _f64(x_t)
    m = _i32(0)
    ms = (ctypes.c_double * 3)()
    _check(lib.rrg_autotune_pairing(h, _ptr(x), float(r_t), float(v_prev), int(repeats), ctypes.byref(m),
                                    ms), h)
    return m.value, list(ms)


def rrg_set_profiling(h, on):
    _check(lib.rrg_set_profiling(h, int(bool(on))), h)


def rrg_get_stats(h) -> dict:
    s = RrgStats()
    _check(lib.rrg_get_stats(h, ctypes.byref(s)), h)
    return {name: getattr(s, name) for name, _ in RrgStats._fields_}


def rrg_reset_stats(h):
    _check(lib.rrg_reset_stats(h), h)


def rrg_eval_candidates_static(params, cfg: RrgConfig, stream, d_scen64, d_scen32, d_x_t, v_prev, r_t,
                               d_kappas, m, d_admissible, d_min_slack=None):
    """Allocation-free evaluation on caller-owned device buffers (see rrg.h);
    asynchronous on `stream` (None: the legacy default stream)."""
    p = _f64(params)
    _check(lib.rrg_eval_candidates_static(_ptr(p), int(p.shape[0]), ctypes.byref(cfg), _stream_ptr(stream),
                                          _tensor_ptr(d_scen64), _tensor_ptr(d_scen32), _tensor_ptr(d_x_t),
                                          float(v_prev), float(r_t), _tensor_ptr(d_kappas), int(m),
                                          _tensor_ptr(d_admissible), _tensor_ptr(d_min_slack)), None)


@dataclass
class Governor:
    """Owning wrapper of one rrg handle (create on construction, destroy on close)."""

    params: np.ndarray
    cfg: RrgConfig
    stream: object = None

    def __post_init__(self):
        self.h = rrg_create(self.params, self.cfg, self.stream)

    def close(self):
        if getattr(self, "h", None):
            rrg_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sample_scenarios(self, seed, update_index):
        rrg_sample_scenarios(self.h, seed, update_index)

    def set_scenarios(self, d):
        rrg_set_scenarios(self.h, d)

    def get_scenarios(self):
        return rrg_get_scenarios(self.h, self.cfg.n_scenarios, self.cfg.horizon)

    def get_param_multipliers(self):
        return rrg_get_param_multipliers(self.h, self.cfg.n_scenarios)

    def set_param_multipliers(self, m):
        rrg_set_param_multipliers(self.h, m)

    def eval_candidates(self, x_t, v_prev, r_t, kappas, want_P=False):
        return rrg_eval_candidates(self.h, x_t, v_prev, r_t, kappas, want_P, self.cfg.n_scenarios)

    def slack_error(self, x_t, v_prev, r_t, kappas, band=None):
        if band is None:
            band = self.cfg.recheck_eps_rel * abs(self.cfg.y_min)
        return rrg_slack_error(self.h, x_t, v_prev, r_t, kappas, band, self.cfg.n_scenarios)

    def step(self, x_t, r_t, v_prev):
        return rrg_step(self.h, x_t, r_t, v_prev)

    def equilibrium(self, v):
        return rrg_equilibrium(self.h, v)

    def step_latency(self, v, steps=2000):
        return rrg_step_latency(self.h, v, steps)

    def closed_loop(self, x0, v0, r_seq, seed, t0, plant_amp, use_graph=True):
        return rrg_closed_loop(self.h, x0, v0, r_seq, seed, t0, plant_amp, use_graph)

    def plant_step(self, x_t, v_t, seed, t, plant_amp):
        return rrg_plant_step(self.h, x_t, v_t, seed, t, plant_amp)

    def slack_gradient(self, x_t, v_prev, r_t, kappa, checkpoint=50, precision=FP64):
        return rrg_slack_gradient(self.h, x_t, v_prev, r_t, kappa, checkpoint, precision)

    def slack_gradients(self, x_t, v_prev, r_t, kappas, checkpoint=50, precision=FP64):
        return rrg_slack_gradients(self.h, x_t, v_prev, r_t, kappas, checkpoint, precision)

    def newton_search(self, x_t, r_t, v_prev, tol=2.0 ** -19, max_iter=40, checkpoint=50, precision=FP64):
        return rrg_newton_search(self.h, x_t, r_t, v_prev, tol, max_iter, checkpoint, precision)

    def stats(self):
        return rrg_get_stats(self.h)

    def reset_stats(self):
        rrg_reset_stats(self.h)

    def set_profiling(self, on):
        rrg_set_profiling(self.h, on)

    def autotune(self, x_t, r_t, v_prev, repeats=2):
        return rrg_autotune(self.h, x_t, r_t, v_prev, repeats)

    def set_tuning(self, m, probe_steps):
        rrg_set_tuning(self.h, m, probe_steps)

    def get_tuning(self):
        return rrg_get_tuning(self.h)

    def set_pairing(self, mode):
        rrg_set_pairing(self.h, mode)

    def set_tma(self, mode):
        rrg_set_tma(self.h, mode)

    def get_tma(self):
        return rrg_get_tma(self.h)

    def set_injection(self, flags):
        rrg_set_injection(self.h, flags)

    def get_pairing(self):
        return rrg_get_pairing(self.h)

    def autotune_pairing(self, x_t, r_t, v_prev, repeats=2):
        return rrg_autotune_pairing(self.h, x_t, r_t, v_prev, repeats)


def rrg_alu_peaks():
    """Measured (binary32 FMA TFLOP/s, binary64 FMA TFLOP/s, MUFU exp2 Top/s)."""
    a, b, c = _d(0.0), _d(0.0), _d(0.0)
    _check(lib.rrg_alu_peaks(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), None)
    return a.value, b.value, c.value


# ---------------------------------------------------------------- batched --
BATCH_VARIANTS = 10
BATCH_MAX_WIDTHS = 24


def rrg_batch_last_error(h=None) -> str:
    e = lib.rrg_batch_last_error(h)
    return e.decode() if e else ""


def _bcheck(rc, h=None):
    if rc != RRG_OK:
        raise RrgError(rc, rrg_batch_last_error(h))


def rrg_batch_create(params, cfg: RrgConfig, n_scenarios, horizons, stream=None):
    p = _f64(params)
    ns = np.ascontiguousarray(np.asarray(n_scenarios, dtype=np.int32))
    hz = np.ascontiguousarray(np.asarray(horizons, dtype=np.int32))
    if ns.shape != hz.shape:
        raise ValueError("n_scenarios and horizons differ in length")
    h = _p()
    _bcheck(lib.rrg_batch_create(_ptr(p), int(p.shape[0]), ctypes.byref(cfg), int(ns.shape[0]), _ptr(ns),
                                 _ptr(hz), _stream_ptr(stream), ctypes.byref(h)), None)
    return h


def rrg_batch_destroy(h):
    _bcheck(lib.rrg_batch_destroy(h))


def rrg_batch_step_dev(h, d_x, d_r, d_v_prev, seed, update_index, d_v_t=None, d_kappa=None, d_flags=None):
    _bcheck(lib.rrg_batch_step_dev(h, _tensor_ptr(d_x), _tensor_ptr(d_r), _tensor_ptr(d_v_prev), int(seed),
                                   int(update_index), _tensor_ptr(d_v_t), _tensor_ptr(d_kappa),
                                   _tensor_ptr(d_flags)), h)


def rrg_batch_closed_loop_dev(h, d_x0, d_v0, d_r_seq, T, seed, t0, plant_amp, use_graph, d_v_out=None,
                              d_kappa_out=None, d_flags_out=None, d_x_out=None):
    amp = _f64(plant_amp)
    _bcheck(lib.rrg_batch_closed_loop_dev(h, _tensor_ptr(d_x0), _tensor_ptr(d_v0), _tensor_ptr(d_r_seq), int(T),
                                          int(seed), int(t0), _ptr(amp), int(bool(use_graph)),
                                          _tensor_ptr(d_v_out), _tensor_ptr(d_kappa_out),
                                          _tensor_ptr(d_flags_out), _tensor_ptr(d_x_out)), h)


def rrg_batch_autotune(h, d_x, d_r, d_v_prev, seed, update_index, repeats=2):
    """(chosen variant, mean rollout ms per update of each variant)."""
    v = ctypes.c_int(0)
    ms = np.zeros(BATCH_VARIANTS)
    _bcheck(lib.rrg_batch_autotune(h, _tensor_ptr(d_x), _tensor_ptr(d_r), _tensor_ptr(d_v_prev), int(seed),
                                   int(update_index), int(repeats), ctypes.byref(v), _ptr(ms)), h)
    return v.value, ms


def rrg_batch_set_width(h, width):
    _bcheck(lib.rrg_batch_set_width(h, int(width)), h)


def rrg_batch_get_width(h):
    w = ctypes.c_int(0)
    _bcheck(lib.rrg_batch_get_width(h, ctypes.byref(w)), h)
    return w.value


def rrg_batch_autotune_width(h, d_x, d_r, d_v_prev, seed, update_index, repeats=2):
    """(chosen width, widths tried, mean ms per update of each)."""
    w, n = ctypes.c_int(0), ctypes.c_int(0)
    ws = np.zeros(BATCH_MAX_WIDTHS, dtype=np.int32)
    ms = np.zeros(BATCH_MAX_WIDTHS)
    _bcheck(lib.rrg_batch_autotune_width(h, _tensor_ptr(d_x), _tensor_ptr(d_r), _tensor_ptr(d_v_prev), int(seed),
                                         int(update_index), int(repeats), ctypes.byref(w), _ptr(ws), _ptr(ms),
                                         ctypes.byref(n)), h)
    return w.value, ws[:n.value].copy(), ms[:n.value].copy()


def rrg_batch_set_variant(h, variant):
    _bcheck(lib.rrg_batch_set_variant(h, int(variant)), h)


def rrg_batch_get_variant(h):
    """(variant, lanes per tile, prefetch depth)."""
    v, t, f = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _bcheck(lib.rrg_batch_get_variant(h, ctypes.byref(v), ctypes.byref(t), ctypes.byref(f)), h)
    return v.value, t.value, f.value


def rrg_batch_set_profiling(h, on):
    _bcheck(lib.rrg_batch_set_profiling(h, int(bool(on))), h)


def rrg_batch_get_stats(h) -> dict:
    st = RrgStats()
    _bcheck(lib.rrg_batch_get_stats(h, ctypes.byref(st)), h)
    return {name: getattr(st, name) for name, _ in RrgStats._fields_}


def rrg_batch_reset_stats(h):
    _bcheck(lib.rrg_batch_reset_stats(h), h)


class BatchGovernor:
    """Owning wrapper of a batched handle; the host-array methods stage
    through torch device tensors (argument marshalling only)."""

    def __init__(self, params, cfg: RrgConfig, n_scenarios, horizons, stream=None):
        self.params = _f64(params)
        self.cfg = cfg
        self.n_scenarios = np.asarray(n_scenarios, dtype=np.int32)
        self.horizons = np.asarray(horizons, dtype=np.int32)
        self.S = int(self.n_scenarios.shape[0])
        self.stream = stream
        self.h = rrg_batch_create(self.params, cfg, self.n_scenarios, self.horizons, stream)

    def close(self):
        if getattr(self, "h", None):
            rrg_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, a, dtype=None):
        import torch
        if dtype is None:
            dtype = torch.float64
        return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")

    def _sync(self):
        import torch
        if self.stream is not None:
            self.stream.synchronize()
        torch.cuda.synchronize()

    def step(self, x, r, v_prev, seed, update_index):
        """One update from host arrays x[S, 3], r[S], v_prev[S]: (v_t, kappa, flags)."""
        import torch
        dx, dr, dv = self._dev(np.asarray(x).reshape(-1)), self._dev(r), self._dev(v_prev)
        ov = torch.zeros(self.S, dtype=torch.float64, device="cuda")
        ok = torch.zeros_like(ov)
        of = torch.zeros(self.S, dtype=torch.int32, device="cuda")
        self._sync()
        rrg_batch_step_dev(self.h, dx, dr, dv, seed, update_index, ov, ok, of)
        self._sync()
        return ov.cpu().numpy(), ok.cpu().numpy(), of.cpu().numpy()

    def closed_loop(self, x0, v0, r_seq, seed, t0, plant_amp, use_graph=True):
        """T updates from host arrays: x0[S, 3], v0[S], r_seq[T, S]; returns
        (v[T, S], kappa[T, S], flags[T, S], x[T + 1, S, 3])."""
        import torch
        r_seq = np.asarray(r_seq, dtype=np.float64)
        T = int(r_seq.shape[0])
        dx0, dv0, dr = self._dev(np.asarray(x0).reshape(-1)), self._dev(v0), self._dev(r_seq.reshape(-1))
        ov = torch.zeros(T * self.S, dtype=torch.float64, device="cuda")
        ok = torch.zeros_like(ov)
        of = torch.zeros(T * self.S, dtype=torch.int32, device="cuda")
        ox = torch.zeros((T + 1) * self.S * 3, dtype=torch.float64, device="cuda")
        self._sync()
        rrg_batch_closed_loop_dev(self.h, dx0, dv0, dr, T, seed, t0, plant_amp, use_graph, ov, ok, of, ox)
        self._sync()
        return (ov.cpu().numpy().reshape(T, self.S), ok.cpu().numpy().reshape(T, self.S),
                of.cpu().numpy().reshape(T, self.S), ox.cpu().numpy().reshape(T + 1, self.S, 3))

    def autotune(self, x, r, v_prev, seed, update_index, repeats=2):
        dx, dr, dv = self._dev(np.asarray(x).reshape(-1)), self._dev(r), self._dev(v_prev)
        self._sync()
        return rrg_batch_autotune(self.h, dx, dr, dv, seed, update_index, repeats)

    def set_variant(self, v):
        rrg_batch_set_variant(self.h, v)

    def set_width(self, w):
        rrg_batch_set_width(self.h, w)

    def get_width(self):
        return rrg_batch_get_width(self.h)

    def autotune_width(self, x, r, v_prev, seed, update_index, repeats=2):
        dx, dr, dv = self._dev(np.asarray(x).reshape(-1)), self._dev(r), self._dev(v_prev)
        self._sync()
        return rrg_batch_autotune_width(self.h, dx, dr, dv, seed, update_index, repeats)

    def get_variant(self):
        return rrg_batch_get_variant(self.h)

    def stats(self):
        return rrg_batch_get_stats(self.h)

    def reset_stats(self):
        rrg_batch_reset_stats(self.h)

    def set_profiling(self, on):
        rrg_batch_set_profiling(self.h, on)
