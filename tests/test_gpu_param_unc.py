"""Parametric uncertainty on the GPU against the oracle, through the C ABI.

Each scenario k of an update scales the uncertain FC3 parameters by its own
multipliers m_p^k = 1 + rho (2u - 1) (Philox stream 2), on top of its
disturbance sequence (Eq. 4); the steady-state check and the simulated plant
keep the nominal parameters.  Both sides draw the multipliers from the same
counters; the oracle applies them with `param_multipliers`.  Tolerances are
those of the nominal parity tests: identical decisions, P and kappa; binary64
slacks to 1e-9 relative.
"""
import numpy as np
import pytest

from paper_2510_08288_gb300 import inputs

pytestmark = pytest.mark.gpu

RHO = inputs.PARAM_UNC_REL
MASK = inputs.FC3_UNCERTAIN_MASK
SLACK32_TOL = 2e-4
BENCH_BAND = 1e-6 * inputs.Y_MIN   # the recheck band the benchmark runs with


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_08288_gb300 import build as B
    B.build()
    from paper_2510_08288_gb300 import rrg
    return rrg


def _cfg(R, N, H, **kw):
    base = dict(horizon=H, n_scenarios=N, max_candidates=32, n_bisect=12, n_rounds=3,
                search=R.SEARCH_SPEC_BISECT, precision=R.FP64, early_exit=R.EXIT_CANDIDATE,
                param_unc_rel=RHO, param_unc_mask=MASK, recheck_eps_rel=SLACK32_TOL / 1.9)
    base.update(kw)
    return R.rrg_config_default(**base)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_recheck"])
def test_multipliers_bit_exact(R, orc, params, prec):
    """The sampler draws exactly the oracle's multipliers (all precisions:
    multipliers are always binary64)."""
    p = {"fp64": R.FP64, "fp32": R.FP32, "fp32_recheck": R.FP32_RECHECK}[prec]
    for N, seed, upd, rho, mask in ((64, 0, 0, RHO, MASK), (37, 2**63 + 5, 99, 0.3, (1 << 27) - 1),
                                    (1, 7, 3, 0.05, 1)):
        with R.Governor(params, _cfg(R, N, 5, precision=p, param_unc_rel=rho, param_unc_mask=mask)) as g:
            np.testing.assert_array_equal(g.get_param_multipliers(), 1.0)
            g.sample_scenarios(seed, upd)
            got = g.get_param_multipliers()
        np.testing.assert_array_equal(got, orc.sample_param_multipliers(seed, upd, N, rho, mask))


def test_multiplier_io_and_validation(R, params):
    N = 9
    m = np.random.default_rng(0).uniform(0.8, 1.2, size=(N, 27))
    with R.Governor(params, _cfg(R, N, 5)) as g:
        g.set_param_multipliers(m)
        np.testing.assert_array_equal(g.get_param_multipliers(), m)
        for bad in (0.0, -1.0, np.nan, np.inf):
            mb = m.copy()
            mb[3, 4] = bad
            with pytest.raises(R.RrgError) as e:
                g.set_param_multipliers(mb)
            assert e.value.code == R.RRG_EINVAL
        np.testing.assert_array_equal(g.get_param_multipliers(), m)
    with R.Governor(params, _cfg(R, N, 5, param_unc_rel=0.0)) as g:
        np.testing.assert_array_equal(g.get_param_multipliers(), 1.0)
        with pytest.raises(R.RrgError) as e:
            g.set_param_multipliers(m)
        assert e.value.code == R.RRG_EINVAL


def _eval_both(R, orc, params, N, H, kappas, prec, early, v_prev=100.0, r=250.0, seed=3, upd=1, **kw):
    x_t = orc.equilibrium(params, v_prev)
    with R.Governor(params, _cfg(R, N, H, precision=prec, early_exit=early,
                                 max_candidates=max(len(kappas), 2), **kw)) as g:
        g.sample_scenarios(seed, upd)
        adm, ms, P = g.eval_candidates(x_t, v_prev, r, kappas, want_P=True)
        st = g.stats()
    d = orc.sample_disturbances(seed, upd, N, H, inputs.DIST_AMP)
    m = orc.sample_param_multipliers(seed, upd, N, RHO, MASK)
    with orc.param_multipliers(m):
        a_o, ms_o, P_o, _ = orc.eval_candidates(params, orc.cfg(H=H, N=N, early_exit=0), x_t, v_prev,
                                                r, kappas, d, want_P=True)
    return (adm, ms, P, st), (a_o, ms_o, P_o)


@pytest.mark.parametrize("N,H", [(64, 400), (129, 150), (1, 30)])
@pytest.mark.parametrize("early", [0, 2])
def test_eval_fp64_matches_oracle(R, orc, params, N, H, early):
    kappas = np.array([0.0, 0.01, 0.02, 0.04, 0.06, 0.1, 0.3, 1.0])
    (adm, ms, P, _), (a_o, ms_o, P_o) = _eval_both(R, orc, params, N, H, kappas, R.FP64, early)
    np.testing.assert_array_equal(adm, a_o)
    np.testing.assert_array_equal(P, P_o)
    ok = a_o == 1
    np.testing.assert_allclose(ms[ok], ms_o[ok], rtol=1e-9, atol=1e-12)
    if early == 0:
        np.testing.assert_allclose(ms, ms_o, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("N,H", [(257, 300), (1000, 120)])
def test_eval_fp32_recheck_is_exact(R, orc, params, N, H):
    kappas = np.linspace(0.0, 0.06, 25)
    (adm, ms, P, st), (a_o, ms_o, P_o) = _eval_both(R, orc, params, N, H, kappas, R.FP32_RECHECK, 1)
    np.testing.assert_array_equal(adm, a_o)
    np.testing.assert_array_equal(P, P_o)
    # and at the benchmark's band
    (adm, ms, P, st), (a_o, ms_o, P_o) = _eval_both(R, orc, params, N, H, kappas, R.FP32_RECHECK, 1,
                                                    recheck_eps_rel=1e-6)
    np.testing.assert_array_equal(adm, a_o)
    np.testing.assert_array_equal(P, P_o)


def test_fp32_error_band_with_uncertain_parameters(R, orc, params):
    """Per-scenario binary32 constants keep the binary32 error of each
    candidate's min slack inside the benchmark's recheck band 1.9e-6 (full
    horizon, no early exit); the per-step statement is in
    test_gpu_fp32_error.py."""
    N, H = 1024, 2000
    kappas = np.array([0.0, 0.02, 0.04, 0.1])
    x_t = orc.equilibrium(params, 100.0)
    out = []
    for prec in (R.FP32, R.FP64):
        with R.Governor(params, _cfg(R, N, H, precision=prec, early_exit=0, max_candidates=4)) as g:
            g.sample_scenarios(1, 0)
            out.append(g.eval_candidates(x_t, 100.0, 250.0, kappas)[1])
    err = np.max(np.abs(out[0] - out[1]))
    print("param-unc max |s32 - s64| = %.3e" % err)
    assert err < BENCH_BAND


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_unit_multipliers_equal_the_nominal_model(R, orc, params, prec):
    """Multipliers of exactly one reproduce the nominal handle bit for bit
    (the per-trajectory fold is the host fold)."""
    N, H = 96, 300
    p = R.FP64 if prec == "fp64" else R.FP32
    kappas = np.linspace(0.0, 0.2, 9)
    x_t = orc.equilibrium(params, 100.0)
    with R.Governor(params, _cfg(R, N, H, precision=p, early_exit=0, param_unc_rel=0.0)) as g:
        g.sample_scenarios(5, 2)
        nominal = g.eval_candidates(x_t, 100.0, 250.0, kappas, want_P=True)
    with R.Governor(params, _cfg(R, N, H, precision=p, early_exit=0)) as g:
        g.sample_scenarios(5, 2)
        g.set_param_multipliers(np.ones((N, 27)))
        ones = g.eval_candidates(x_t, 100.0, 250.0, kappas, want_P=True)
    for a, b in zip(nominal, ones):
        np.testing.assert_array_equal(a, b)


def _oracle_search(orc, params, kind, x_t, v_prev, r, d, m, N, H, M):
    c = orc.cfg(H=H, N=N)
    with orc.param_multipliers(m):
        if kind in ("bisect", "spec"):
            return orc.bisect_joint(params, c, x_t, v_prev, r, 12, d)
        if kind == "grid":
            return orc.alg3(params, c, x_t, v_prev, r, M, d)
        return orc.ksection(params, c, x_t, v_prev, r, M, 3, d)


@pytest.mark.parametrize("kind", ["bisect", "spec", "grid", "ksection"])
@pytest.mark.parametrize("prec", ["fp64", "fp32_recheck"])
@pytest.mark.parametrize("case", [(100.0, 250.0), (200.0, 60.0), (55.0, 300.0)])
def test_step_matches_oracle(R, orc, params, kind, prec, case):
    v_prev, r = case
    N, H, M = 48, 500, 16
    x_t = orc.equilibrium(params, v_prev)
    search = {"bisect": R.SEARCH_BISECT, "spec": R.SEARCH_SPEC_BISECT, "grid": R.SEARCH_GRID,
              "ksection": R.SEARCH_KSECTION}[kind]
    p = R.FP64 if prec == "fp64" else R.FP32_RECHECK
    with R.Governor(params, _cfg(R, N, H, search=search, precision=p, max_candidates=M)) as g:
        g.sample_scenarios(4, 6)
        v_t, kap, fl = g.step(x_t, r, v_prev)
    d = orc.sample_disturbances(4, 6, N, H, inputs.DIST_AMP)
    m = orc.sample_param_multipliers(4, 6, N, RHO, MASK)
    k_o, f_o = _oracle_search(orc, params, kind, x_t, v_prev, r, d, m, N, H, M)
    assert kap == k_o and fl == f_o
    assert v_t == v_prev + kap * (r - v_prev)


@pytest.mark.parametrize("probe", [1, 8, 128])
def test_pipelined_spec_bisect_matches_oracle(R, orc, params, probe):
    """The pipelined first rounds (probe, provisional tree, validation) with
    per-scenario models still give Alg. 1's kappa, also off equilibrium."""
    N, H = 64, 600
    x_eq = orc.equilibrium(params, 120.0)
    for x_t in (x_eq, x_eq * np.array([1.0, 1.08, 1.03])):
        with R.Governor(params, _cfg(R, N, H, precision=R.FP32_RECHECK, max_candidates=16,
                                     probe_steps=probe)) as g:
            g.sample_scenarios(8, 2)
            _, kap, fl = g.step(x_t, 280.0, 120.0)
        d = orc.sample_disturbances(8, 2, N, H, inputs.DIST_AMP)
        m = orc.sample_param_multipliers(8, 2, N, RHO, MASK)
        with orc.param_multipliers(m):
            k_o, f_o = orc.bisect_joint(params, orc.cfg(H=H, N=N), x_t, 120.0, 280.0, 12, d)
        assert (kap, fl) == (k_o, f_o)


@pytest.mark.parametrize("use_graph", [False, True])
def test_closed_loop_matches_oracle(R, orc, params, use_graph):
    """Closed loop with both scenario pairs (multipliers redrawn every update,
    the next update's drawn on the side stream): kappa, v_t and flags equal
    the oracle's; the nominal plant states agree to 1e-10."""
    N, H, T = 16, 150, 6
    r_seq = inputs.staircase(T, 3, 2, seed=1)
    x0 = orc.equilibrium(params, 100.0)
    amp = inputs.DIST_AMP
    cfg = _cfg(R, N, H, precision=R.FP32_RECHECK, max_candidates=16)
    with R.Governor(params, cfg) as g:
        v, kap, fl, xs = g.closed_loop(x0, 100.0, r_seq, 11, 5, amp, use_graph=use_graph)
    vo, ko, fo, xo = orc.closed_loop(params, orc.cfg(H=H, N=N), x0, 100.0, r_seq, 11, 5, amp, amp,
                                     search=0, param_unc_rel=RHO, param_unc_mask=MASK)
    np.testing.assert_array_equal(kap, ko)
    np.testing.assert_array_equal(fl, fo)
    np.testing.assert_array_equal(v, vo)
    np.testing.assert_allclose(xs, xo, rtol=1e-10)


@pytest.mark.parametrize("checkpoint", [1, 50])
def test_adjoint_matches_complex_step(R, orc, params, checkpoint):
    """Discrete adjoint with per-scenario parameters: value, argmin and the
    gradient with respect to kappa, x_t and the NOMINAL parameters equal the
    oracle's complex-step derivative."""
    N, H = 40, 300
    x_t = orc.equilibrium(params, 100.0) * np.array([1.0, 1.02, 1.01])
    with R.Governor(params, _cfg(R, N, H, max_candidates=16)) as g:
        g.sample_scenarios(2, 9)
        d = orc.sample_disturbances(2, 9, N, H, inputs.DIST_AMP)
        m = orc.sample_param_multipliers(2, 9, N, RHO, MASK)
        for kappa in (0.03, 0.1):
            gv, grad, ks, js = g.slack_gradient(x_t, 100.0, 250.0, kappa, checkpoint, R.FP64)
            c = orc.cfg(H=H, N=N, early_exit=0)
            with orc.param_multipliers(m):
                go, ko, jo = orc.min_slack_argmin(params, c, x_t, orc.governed(100.0, 250.0, kappa), d)
                _, gro = orc.slack_grad(params, c, x_t, 100.0, 250.0, kappa, d, ko, jo)
            assert (ks, js) == (ko, jo)
            assert gv == pytest.approx(go, rel=1e-10, abs=1e-12)
            scale = np.maximum(np.abs(gro), 1e-12 * np.max(np.abs(gro)))
            assert np.all(np.abs(grad - gro) <= 1e-7 * scale + 1e-14)


def test_full_size_sweep_update_matches_fp64_and_oracle(R, orc, params):
    """The large sweep's configuration at its largest size (65,536 scenarios x
    5,000 steps, k-section with 16 candidates x 3 rounds, +-10 % on the
    uncertain parameters, FP32 rollouts with the FP64 recheck, in the
    launch shape the benchmark times): kappa equals the plain FP64 search on
    the same draws, and sampled trajectories' decisions at the chosen and the
    next grid point equal the oracle's."""
    N, H, M = 65536, 5000, 16
    v_prev, r = 100.0, 150.0
    seed, upd = 1, 3
    x_t = orc.equilibrium(params, v_prev)
    kw = dict(max_candidates=M, n_rounds=3, search=R.SEARCH_KSECTION, recheck_eps_rel=1e-6)
    with R.Governor(params, _cfg(R, N, H, precision=R.FP32_RECHECK, **kw)) as g:
        g.sample_scenarios(seed, upd)
        v32, k32, f32 = g.step(x_t, r, v_prev)
        probe = np.array([k32, min(1.0, k32 + 1.0 / (M - 1))])
        adm, ms, P = g.eval_candidates(x_t, v_prev, r, probe, want_P=True)
    with R.Governor(params, _cfg(R, N, H, precision=R.FP64, **kw)) as g:
        g.sample_scenarios(seed, upd)
        v64, k64, f64 = g.step(x_t, r, v_prev)
    assert (k32, f32) == (k64, f64)
    assert adm[0] == 1
    # the oracle on scenarios k < 1,024 (Philox counters do not depend on N)
    n = 1024
    d = orc.sample_disturbances(seed, upd, n, H, inputs.DIST_AMP)
    mult = orc.sample_param_multipliers(seed, upd, n, RHO, MASK)
    c = orc.cfg(H=H, N=n, early_exit=1)
    rng = np.random.default_rng(11)
    with orc.param_multipliers(mult):
        for k in rng.choice(n, size=12, replace=False):
            for i, kk in enumerate(probe):
                s, _ = orc.rollout(params, c, x_t, orc.governed(v_prev, r, kk), d, k)
                assert P[i, k] == (1 if s >= 0 else 0), (k, i, s)
