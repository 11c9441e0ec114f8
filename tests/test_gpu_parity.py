"""GPU-vs-oracle parity of the robust reference governor, through the C ABI.

Every test here needs a GB300 and the built librrg.so.  The oracle is the
sequential FP64 C implementation under oracle/; both sides get the same seeded
inputs (the same Philox counters, or explicit arrays from the inputs module).

Tolerances:
  - integer results (admissibility flags, P entries, kappa on the dyadic or
    grid points, v_t) must be identical;
  - binary64 slacks agree to 1e-9 relative (the two sides round in different
    orders; over 2,000 contractive RK4 steps the drift stays ~1e-13);
  - binary32 slacks agree with binary64 to the band SLACK32_TOL, and
    admissibility decisions of the plain FP32 path may differ only where the
    binary64 slack is inside that band; with FP32_RECHECK they are identical
    whenever the band covers the measured binary32 error.
"""
import numpy as np
import pytest

from paper_2510_08288_gb300 import inputs

pytestmark = pytest.mark.gpu

SLACK64_RTOL = 1e-9
SLACK32_TOL = 2e-4        # absolute OER units: the plain binary32 tests' loose band
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
                search=R.SEARCH_SPEC_BISECT, precision=R.FP64, early_exit=R.EXIT_CANDIDATE)
    base.update(kw)
    return R.rrg_config_default(**base)


def _ocfg(orc, N, H, early_exit=1, **kw):
    return orc.cfg(H=H, N=N, early_exit=early_exit, **kw)


# ------------------------------------------------------------------ pieces --
def test_scenarios_bit_exact(R, orc, params):
    """Philox4x64-10 on the device draws exactly the oracle's d_j^k."""
    for N, H, seed, upd in ((32, 500, 0, 0), (37, 61, 5, 123456789), (1, 1, 2**63 + 1, 7)):
        with R.Governor(params, _cfg(R, N, H)) as g:
            g.sample_scenarios(seed, upd)
            got = g.get_scenarios()
        want = orc.sample_disturbances(seed, upd, N, H, inputs.DIST_AMP)
        np.testing.assert_array_equal(got, want)


def test_lazily_sampled_scenarios_materialize_bit_exact(R, orc, params):
    """In the binary32 modes the sampler writes only the binary32 copy; the
    binary64 values rrg_get_scenarios returns are regenerated from the same
    Philox counters and equal the oracle's draw bit for bit."""
    for prec in (R.FP32, R.FP32_RECHECK):
        with R.Governor(params, _cfg(R, 40, 33, precision=prec)) as g:
            g.sample_scenarios(77, 5)
            got = g.get_scenarios()
        np.testing.assert_array_equal(got, orc.sample_disturbances(77, 5, 40, 33, inputs.DIST_AMP))


def test_set_scenarios_roundtrip(R, params):
    d = inputs.uniform_disturbances(29, 17, seed=3)
    with R.Governor(params, _cfg(R, 29, 17)) as g:
        g.set_scenarios(d)
        np.testing.assert_array_equal(g.get_scenarios(), d)


@pytest.mark.parametrize("I", [50.0, 77.7, 100.0, 175.0, 250.0, 300.0])
def test_equilibrium(R, orc, params, I):
    """Equilibrium manifold (Sec. II-A): device Illinois solve vs oracle bisection."""
    with R.Governor(params, _cfg(R, 4, 4)) as g:
        x, y = g.equilibrium(I)
    xo = orc.equilibrium(params, I)
    np.testing.assert_allclose(x, xo, rtol=1e-11)
    assert y == pytest.approx(orc.output(params, xo, I), rel=1e-11)


def test_equilibrium_rejects_bad_setpoint(R, params):
    with R.Governor(params, _cfg(R, 4, 4)) as g:
        for v in (0.0, -5.0, float("nan"), float("inf")):
            with pytest.raises(R.RrgError):
                g.equilibrium(v)


# --------------------------------------------------------- candidate eval --
def _eval_both(R, orc, params, N, H, kappas, prec, early, v_prev=100.0, r=250.0, seed=0,
               want_P=True, x_t=None, **ckw):
    if x_t is None:
        x_t = orc.equilibrium(params, v_prev)
    with R.Governor(params, _cfg(R, N, H, precision=prec, early_exit=early,
                                 max_candidates=max(len(kappas), 2), **ckw)) as g:
        g.sample_scenarios(seed, 0)
        adm, ms, P = g.eval_candidates(x_t, v_prev, r, kappas, want_P=want_P)
        st = g.stats()
    d = orc.sample_disturbances(seed, 0, N, H, inputs.DIST_AMP)
    oc = _ocfg(orc, N, H, early_exit=0, **{k: v for k, v in ckw.items() if k in ("y_min", "ss_check", "eps_ss", "y_c")})
    a_o, ms_o, P_o, _ = orc.eval_candidates(params, oc, x_t, v_prev, r, kappas, d, want_P=True)
    return (adm, ms, P, st), (a_o, ms_o, P_o)


@pytest.mark.parametrize("N,H", [(32, 500), (37, 200), (129, 64), (1, 1), (300, 33)])
@pytest.mark.parametrize("early", [0, 1, 2])
def test_eval_fp64_matches_oracle(R, orc, params, N, H, early):
    """Alg. 3 steps 1-3 in binary64: identical P and decisions, slacks to 1e-9."""
    kappas = np.array([0.0, 0.03, 0.08, 0.1, 0.1025, 0.11, 0.3, 1.0])
    (adm, ms, P, _), (a_o, ms_o, P_o) = _eval_both(R, orc, params, N, H, kappas, R.FP64, early,
                                                   want_P=True)
    np.testing.assert_array_equal(adm, a_o)
    np.testing.assert_array_equal(P, P_o)
    ok = a_o == 1
    np.testing.assert_allclose(ms[ok], ms_o[ok], rtol=SLACK64_RTOL, atol=1e-12)
    if early == 0:
        np.testing.assert_allclose(ms, ms_o, rtol=SLACK64_RTOL, atol=1e-12)


@pytest.mark.parametrize("N,H", [(32, 500), (129, 300), (1, 1), (37, 31), (5, 32), (70, 33), (9, 65)])
def test_eval_fp32_within_band(R, orc, params, N, H):
    """Plain binary32: slack error inside the band; decisions differ only
    where the binary64 slack is inside it.  Horizons around the shared
    ring's depth and exit block (32 steps) included."""
    kappas = np.linspace(0.0, 0.2, 21)
    (adm, ms, P, _), (a_o, ms_o, P_o) = _eval_both(R, orc, params, N, H, kappas, R.FP32, 0)
    assert np.max(np.abs(ms - ms_o)) < SLACK32_TOL
    differ = adm != a_o
    assert np.all(np.abs(ms_o[differ]) < SLACK32_TOL)


@pytest.mark.parametrize("N,H", [(32, 500), (129, 300), (1000, 120), (64, 31), (64, 33)])
@pytest.mark.parametrize("eps_rel", [SLACK32_TOL / 1.9, 1e-6])
def test_eval_fp32_recheck_is_exact(R, orc, params, N, H, eps_rel):
    """Binary32 bulk + binary64 recheck of the near-zero lanes decides exactly
    like the binary64 oracle, with a wide band (many lanes rechecked) and with
    the benchmark's 1e-6 relative band."""
    kappas = np.linspace(0.09, 0.115, 26)
    (adm, ms, P, st), (a_o, ms_o, P_o) = _eval_both(
        R, orc, params, N, H, kappas, R.FP32_RECHECK, 1, recheck_eps_rel=eps_rel)
    np.testing.assert_array_equal(adm, a_o)
    np.testing.assert_array_equal(P, P_o)
    if eps_rel > 1e-5:
        assert st["rechecked"] >= 1


def test_steady_state_failure_rows(R, orc, params):
    """Candidates failing the steady-state check (Eq. 3) get an all-zero P row
    and a NaN min slack; the oracle agrees on the row."""
    kappas = np.array([0.0, 0.5, 1.0])
    ckw = dict(eps_ss=0.9, y_c=2.23378)  # threshold 2.2004: OER_ss(60 A) passes, (170, 280 A) fail
    (adm, ms, P, _), (a_o, ms_o, P_o) = _eval_both(R, orc, params, 16, 50, kappas, R.FP64, 1,
                                                   v_prev=60.0, r=280.0, **ckw)
    np.testing.assert_array_equal(adm, a_o)
    np.testing.assert_array_equal(P, P_o)
    for i in range(3):
        ss = orc.ss_ok(params, orc.cfg(eps_ss=0.9, y_c=2.23378), orc.governed(60.0, 280.0, kappas[i]))
        if not ss:
            assert np.isnan(ms[i]) and not P[i].any()
    assert not all(orc.ss_ok(params, orc.cfg(eps_ss=0.9, y_c=2.23378), orc.governed(60.0, 280.0, k))
                   for k in kappas)


def test_fp32_error_band(R, orc, params):
    """max |s32 - s64| of each candidate's min slack over full-horizon
    trajectories (no early exit) of the 1,024 x 2,000 closed-loop workload at
    kappas near the boundary, inside the benchmark's recheck band 1.9e-6 (the
    per-step, per-trajectory statement is in test_gpu_fp32_error.py)."""
    N, H = 1024, 2000
    kappas = np.array([0.0, 0.1, 0.102, 0.104, 0.2])
    x_t = orc.equilibrium(params, 100.0)
    errs = []
    for prec in (R.FP32, R.FP64):
        with R.Governor(params, _cfg(R, N, H, precision=prec, early_exit=0, max_candidates=8)) as g:
            g.sample_scenarios(1, 0)
            errs.append(g.eval_candidates(x_t, 100.0, 250.0, kappas)[1])
    err = np.max(np.abs(errs[0] - errs[1]))
    print("max |s32 - s64| (min over scenarios) = %.3e" % err)
    assert err < BENCH_BAND


# ------------------------------------------------------------- searches ----
SEARCHES = ("bisect", "spec", "grid", "ksection")


def _oracle_search(orc, params, kind, x_t, v_prev, r, d, N, H, M, n_bisect=12, rounds=3, **kw):
    c = orc.cfg(H=H, N=N, **kw)
    if kind in ("bisect", "spec"):
        return orc.bisect_joint(params, c, x_t, v_prev, r, n_bisect, d)
    if kind == "grid":
        return orc.alg3(params, c, x_t, v_prev, r, M, d)
    return orc.ksection(params, c, x_t, v_prev, r, M, rounds, d)


def _gpu_search(R, kind):
    return {"bisect": R.SEARCH_BISECT, "spec": R.SEARCH_SPEC_BISECT, "grid": R.SEARCH_GRID,
            "ksection": R.SEARCH_KSECTION}[kind]


@pytest.mark.parametrize("kind", SEARCHES)
@pytest.mark.parametrize("prec", ["fp64", "fp32_recheck"])
@pytest.mark.parametrize("case", [(100.0, 250.0), (100.0, 112.0), (200.0, 60.0), (150.0, 150.0),
                                  (55.0, 300.0)])
def test_step_matches_oracle(R, orc, params, kind, prec, case):
    """One robust RG update: kappa, v_t and flags equal the oracle's Alg. 1
    (joint predicate), Alg. 3 or k-section on the same scenarios."""
    v_prev, r = case
    N, H, M = 32, 500, 16
    x_t = orc.equilibrium(params, v_prev)
    p = R.FP64 if prec == "fp64" else R.FP32_RECHECK
    cfg = _cfg(R, N, H, search=_gpu_search(R, kind), precision=p, max_candidates=M,
               recheck_eps_rel=SLACK32_TOL / 1.9)
    with R.Governor(params, cfg) as g:
        g.sample_scenarios(0, 0)
        v_t, kap, fl = g.step(x_t, r, v_prev)
    d = orc.sample_disturbances(0, 0, N, H, inputs.DIST_AMP)
    k_o, f_o = _oracle_search(orc, params, kind, x_t, v_prev, r, d, N, H, M)
    assert kap == k_o and fl == f_o
    assert v_t == v_prev + kap * (r - v_prev)
    assert 0.0 <= kap <= 1.0
    if r == v_prev:
        assert kap == 1.0


@pytest.mark.parametrize("m_cap", [1, 2, 3, 7, 64, 1024])
def test_spec_bisect_equals_bisect_for_any_width(R, orc, params, m_cap):
    """Evaluating several levels of Alg. 1's tree per round changes nothing:
    the result equals plain bisection for every candidate budget."""
    N, H = 24, 300
    x_t = orc.equilibrium(params, 120.0)
    d = orc.sample_disturbances(9, 4, N, H, inputs.DIST_AMP)
    for r in (290.0, 140.0, 130.0):
        k_o, f_o = orc.bisect_joint(params, orc.cfg(H=H, N=N), x_t, 120.0, r, 14, d)
        cfg = _cfg(R, N, H, search=R.SEARCH_SPEC_BISECT, max_candidates=m_cap, n_bisect=14)
        with R.Governor(params, cfg) as g:
            g.sample_scenarios(9, 4)
            _, kap, fl = g.step(x_t, r, 120.0)
        assert kap == k_o and fl == f_o


def test_nothing_admissible_holds(R, orc, params):
    """y_min above every reachable OER: kappa = 0, v_t = v_prev, flag bit 0."""
    x_t = orc.equilibrium(params, 100.0)
    for kind in SEARCHES:
        cfg = _cfg(R, 8, 30, search=_gpu_search(R, kind), y_min=5.0, max_candidates=9)
        with R.Governor(params, cfg) as g:
            g.sample_scenarios(1, 0)
            v_t, kap, fl = g.step(x_t, 200.0, 100.0)
        assert (v_t, kap, fl) == (100.0, 0.0, 1)


def test_host_input_validation(R, orc, params):
    x_t = orc.equilibrium(params, 100.0)
    with R.Governor(params, _cfg(R, 8, 30)) as g:
        g.sample_scenarios(1, 0)
        for bad in ((np.array([np.nan, 1, 1]), 200.0, 100.0), (x_t, np.inf, 100.0), (x_t, 200.0, -1.0)):
            with pytest.raises(R.RrgError) as e:
                g.step(*bad)
            assert e.value.code == R.RRG_EINVAL
        with pytest.raises(R.RrgError):
            g.eval_candidates(x_t, 100.0, 200.0, [1.5])
        with pytest.raises(R.RrgError):
            g.eval_candidates(x_t, 100.0, 200.0, np.zeros(33))


def test_step_dev_flags_invalid_input_on_device(R, orc, params):
    """The device-pointer update rejects a non-finite x_t on the device:
    kappa = 0, v_t = v_prev, flag bit 1, and the handle stays usable."""
    import torch
    x_t = orc.equilibrium(params, 100.0)
    with R.Governor(params, _cfg(R, 8, 30)) as g:
        g.sample_scenarios(1, 0)
        dx = torch.tensor([np.nan, x_t[1], x_t[2]], dtype=torch.float64, device="cuda")
        dr = torch.tensor([200.0], dtype=torch.float64, device="cuda")
        dv = torch.tensor([100.0], dtype=torch.float64, device="cuda")
        out = torch.zeros(2, dtype=torch.float64, device="cuda")
        fl = torch.zeros(1, dtype=torch.int32, device="cuda")
        R.rrg_step_dev(g.h, dx, dr, dv, out[0:1], out[1:2], fl)
        torch.cuda.synchronize()
        assert out[0].item() == 100.0 and out[1].item() == 0.0 and fl.item() & 2
        v_t, kap, f = g.step(x_t, 200.0, 100.0)
        assert f == 0 and 0 < kap < 1


# --------------------------------------------------------- closed loop -----
@pytest.mark.parametrize("use_graph", [False, True])
@pytest.mark.parametrize("kind", ["spec", "ksection"])
def test_closed_loop_matches_oracle(R, orc, params, use_graph, kind):
    """Fig. 1 closed loop for 6 updates on a staircase reference: every
    kappa, v_t and flag equal the oracle's; states agree to 1e-10."""
    N, H, T = 16, 150, 6
    r_seq = inputs.staircase(T, 3, 2, seed=1)
    x0 = orc.equilibrium(params, 100.0)
    amp = inputs.DIST_AMP
    cfg = _cfg(R, N, H, search=_gpu_search(R, kind), precision=R.FP32_RECHECK, max_candidates=16,
               recheck_eps_rel=SLACK32_TOL / 1.9)
    with R.Governor(params, cfg) as g:
        v, kap, fl, xs = g.closed_loop(x0, 100.0, r_seq, 11, 5, amp, use_graph=use_graph)
    search = 0 if kind == "spec" else 2
    vo, ko, fo, xo = orc.closed_loop(params, orc.cfg(H=H, N=N), x0, 100.0, r_seq, 11, 5, amp, amp,
                                     search=search, n_kappa=12, M=16, rounds=3)
    np.testing.assert_array_equal(kap, ko)
    np.testing.assert_array_equal(v, vo)
    np.testing.assert_array_equal(fl, fo)
    np.testing.assert_allclose(xs, xo, rtol=1e-10)


def test_plant_step_matches_oracle(R, orc, params):
    x = orc.equilibrium(params, 120.0)
    with R.Governor(params, _cfg(R, 4, 4)) as g:
        got = g.plant_step(x, 180.0, 3, 9, inputs.DIST_AMP)
    want = orc.rk4_step(params, x, 180.0, 0.01) + orc.plant_disturbance(3, 9, inputs.DIST_AMP)
    np.testing.assert_allclose(got, want, rtol=1e-12)


# ------------------------------------------- full-size closed-loop workload --
def test_full_size_update_matches_oracle(R, orc, params):
    """The benchmark's configuration (N = 1,024 scenarios, horizon 2,000,
    FP32 + FP64 recheck, speculative bisection, 64 candidates per round):
    the GPU update equals the oracle's joint bisection on the same scenarios,
    and sampled P entries equal the oracle's per-trajectory decisions."""
    w = inputs.WORKLOADS["closed_loop"]
    N, H = w["N"], w["H"]
    x_t = orc.equilibrium(params, 100.0)
    cfg = _cfg(R, N, H, search=R.SEARCH_SPEC_BISECT, precision=R.FP32_RECHECK, max_candidates=64,
               recheck_eps_rel=w["recheck_eps_rel"])
    with R.Governor(params, cfg) as g:
        g.sample_scenarios(w["seed"], 0)
        v_t, kap, fl = g.step(x_t, 250.0, 100.0)
        kap_probe = np.array([kap, min(1.0, kap + 2.0 ** -11), 0.05])
        adm, ms, P = g.eval_candidates(x_t, 100.0, 250.0, kap_probe, want_P=True)
    d = orc.sample_disturbances(w["seed"], 0, N, H, inputs.DIST_AMP)
    k_o, f_o = orc.bisect_joint(params, orc.cfg(H=H, N=N), x_t, 100.0, 250.0, 12, d, nthreads=8)
    assert kap == k_o and fl == f_o
    rng = np.random.default_rng(0)
    for k in rng.choice(N, size=48, replace=False):
        for i, kk in enumerate(kap_probe):
            s, _ = orc.rollout(params, orc.cfg(H=H, N=N, early_exit=1), x_t, orc.governed(100.0, 250.0, kk), d, k)
            assert P[i, k] == (1 if s >= 0 else 0)


def test_closed_loop_continuation_equals_one_run(R, orc, params):
    """rrg_closed_loop_dev with x0 = NULL continues the previous run: 2 + 1 + 1
    updates, and 2 + 2 with other draws in between, give exactly the same
    trajectory as one call of 4 updates."""
    import torch
    N, H, T = 16, 100, 4
    r_seq = inputs.staircase(T, 2, 2, seed=4)
    x0 = orc.equilibrium(params, 90.0)
    amp = np.array(inputs.DIST_AMP)
    cfg = _cfg(R, N, H, search=R.SEARCH_SPEC_BISECT, precision=R.FP32_RECHECK, max_candidates=16,
               recheck_eps_rel=SLACK32_TOL / 1.9)
    outs = []
    for pieces in ((4,), (2, 1, 1), (2, "draw", 2)):
        with R.Governor(params, cfg) as g:
            dev = torch.device("cuda")
            d_r = torch.tensor(r_seq, dtype=torch.float64, device=dev)
            d_v = torch.zeros(T, dtype=torch.float64, device=dev)
            d_k = torch.zeros(T, dtype=torch.float64, device=dev)
            d_f = torch.zeros(T, dtype=torch.int32, device=dev)
            d_x = torch.zeros(3 * (T + 1), dtype=torch.float64, device=dev)
            first = True
            for n in pieces:
                if n == "draw":
                    # an unrelated draw between the calls (it may overwrite
                    # the pair holding the loop's next update)
                    g.sample_scenarios(99, 0)
                    g.sample_scenarios(99, 1)
                    continue
                R.rrg_closed_loop_dev(g.h, x0 if first else None, 90.0, d_r, n, 7, 3, amp, not first,
                                      d_v, d_k, d_f, d_x)
                first = False
            torch.cuda.synchronize()
            outs.append((d_v.cpu().numpy(), d_k.cpu().numpy(), d_x.cpu().numpy()))
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            np.testing.assert_array_equal(a, b)
    vo, ko, fo, xo = orc.closed_loop(params, orc.cfg(H=H, N=N), x0, 90.0, r_seq, 7, 3, amp, amp, search=0)
    np.testing.assert_array_equal(outs[0][1], ko)


@pytest.mark.parametrize("probe", [0, 1, 8, 128, 499, 500])
@pytest.mark.parametrize("prec", ["fp64", "fp32_recheck"])
def test_pipelined_spec_bisect_equals_bisect(R, orc, params, probe, prec):
    """Pipelining the first two speculative-bisection rounds (round 2 built
    from round 1's first `probe` steps) never changes the result: a wrong
    provisional outcome is detected and round 2 redone.  probe = 1 forces
    such repairs; probe >= H switches pipelining off."""
    N, H = 48, 500
    p = R.FP64 if prec == "fp64" else R.FP32_RECHECK
    repairs = 0
    # the last two start off equilibrium (compressor over-sped), so the OER
    # violations come several steps in and a 1-step probe guesses wrong
    cases = ((100.0, 250.0, (1, 1, 1)), (100.0, 112.0, (1, 1, 1)), (220.0, 290.0, (1, 1, 1)),
             (180.0, 60.0, (1, 1, 1)), (100.0, 250.0, (1.0, 1.08, 1.03)), (150.0, 220.0, (0.99, 1.1, 1.02)))
    for v_prev, r, scale in cases:
        x_t = orc.equilibrium(params, v_prev) * np.array(scale)
        d = orc.sample_disturbances(2, 1, N, H, inputs.DIST_AMP)
        k_o, f_o = orc.bisect_joint(params, orc.cfg(H=H, N=N), x_t, v_prev, r, 12, d)
        cfg = _cfg(R, N, H, search=R.SEARCH_SPEC_BISECT, precision=p, max_candidates=64,
                   probe_steps=probe, recheck_eps_rel=SLACK32_TOL / 1.9)
        with R.Governor(params, cfg) as g:
            g.sample_scenarios(2, 1)
            v_t, kap, fl = g.step(x_t, r, v_prev)
            repairs += g.stats()["repairs"]
        assert kap == k_o and fl == f_o, (v_prev, r, kap, k_o)
    if probe == 1:
        assert repairs > 0


def test_recheck_runs_only_to_the_last_uncertain_step(R, orc, params):
    """A lane whose binary32 slack is inside the band only at j = 0 (here y_min
    sits 1e-7 below the candidate's initial output, disturbance-free, and the
    OER rises by more than 0.01 at once and stays there) is rechecked in binary64 over step 0 alone: every
    lane is rechecked, no binary64 step runs, and the decisions equal the
    oracle's."""
    N, H = 300, 500
    x_t = orc.equilibrium(params, 100.0) * np.array([1.0, 1.0, 0.999])
    y_min = orc.output(params, x_t, 100.0) - 1e-7
    kappas = np.array([0.0, 0.001])
    cfg = _cfg(R, N, H, precision=R.FP32_RECHECK, early_exit=R.EXIT_LANE, max_candidates=2,
               y_min=y_min, ss_check=0, dist_amp=(0.0, 0.0, 0.0), recheck_eps_rel=1e-6)
    with R.Governor(params, cfg) as g:
        g.sample_scenarios(0, 0)
        adm, ms, P = g.eval_candidates(x_t, 100.0, 150.0, kappas, want_P=True)
        st = g.stats()
    d = np.zeros((3, H, N))
    a_o, ms_o, P_o, _ = orc.eval_candidates(params, orc.cfg(H=H, N=N, y_min=y_min, ss_check=0, early_exit=0),
                                            x_t, 100.0, 150.0, kappas, d, want_P=True)
    np.testing.assert_array_equal(adm, a_o)
    np.testing.assert_array_equal(P, P_o)
    assert list(adm) == [1, 0]
    assert st["rechecked"] == N and st["lane_steps_fp64"] == 0


@pytest.mark.parametrize("p_sm_rel", [0.97, 1.02, 1.9, 2.05])
def test_fp64_rollouts_across_the_power_series_domain(R, orc, params, p_sm_rel):
    """Binary64 rollouts from supply-manifold pressures inside and outside
    [1, 2] p_atm (the range of the binary64 x^e series; outside it pow is
    used) match the oracle's slacks to 1e-9 with identical decisions."""
    N, H = 40, 120
    names = inputs.FC3_PARAM_NAMES
    p_atm = params[names.index("p_atm")]
    x_eq = orc.equilibrium(params, 120.0)
    x_t = np.array([x_eq[0], x_eq[1], p_sm_rel * p_atm])
    if x_t[2] <= x_t[0]:
        x_t[0] = 0.99 * x_t[2]
    kappas = np.array([0.0, 0.05, 0.2, 1.0])
    (adm, ms, P, _), (a_o, ms_o, P_o) = _eval_both(R, orc, params, N, H, kappas, R.FP64, 0, v_prev=120.0,
                                                   r=200.0, x_t=x_t, ss_check=0)
    np.testing.assert_array_equal(adm, a_o)
    np.testing.assert_array_equal(P, P_o)
    fin = np.isfinite(ms_o)
    np.testing.assert_array_equal(np.isfinite(ms), fin)
    np.testing.assert_allclose(ms[fin], ms_o[fin], rtol=1e-9, atol=1e-12)


def test_autotune_and_tuning_keep_alg1_result(R, orc, params):
    """The autotuner and every tree width / probe length give Alg. 1's kappa."""
    N, H = 256, 400
    x_t = orc.equilibrium(params, 100.0)
    cfg = _cfg(R, N, H, search=R.SEARCH_SPEC_BISECT, precision=R.FP32_RECHECK, max_candidates=64,
               probe_steps=128, recheck_eps_rel=SLACK32_TOL / 1.9)
    d = orc.sample_disturbances(3, 1, N, H, inputs.DIST_AMP)
    k_o, f_o = orc.bisect_joint(params, orc.cfg(H=H, N=N), x_t, 100.0, 250.0, 12, d)
    with R.Governor(params, cfg) as g:
        g.sample_scenarios(3, 1)
        before = g.step(x_t, 250.0, 100.0)
        m, p, ms = g.autotune(x_t, 250.0, 100.0, repeats=1)
        assert 4 <= m <= 64 and p in (0, 32, 128) and ms > 0
        assert g.get_tuning() == (m, p)
        assert g.step(x_t, 250.0, 100.0) == before
        for mm, pp in ((1, 0), (3, 0), (7, 32), (64, 1), (64, 399)):
            g.set_tuning(mm, pp)
            assert g.step(x_t, 250.0, 100.0) == before, (mm, pp)
        for bad in ((0, 0), (65, 0), (8, -1)):
            with pytest.raises(R.RrgError):
                g.set_tuning(*bad)
    assert before[1:] == (k_o, f_o)
    with R.Governor(params, _cfg(R, N, H, search=R.SEARCH_SPEC_BISECT, probe_steps=0)) as g:
        with pytest.raises(R.RrgError):
            g.set_tuning(8, 32)
    with R.Governor(params, _cfg(R, N, H, search=R.SEARCH_GRID)) as g:
        with pytest.raises(R.RrgError):
            g.autotune(x_t, 250.0, 100.0)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_recheck"])
def test_in_register_scenarios_equal_stored_ones(R, orc, params, prec):
    """Drawing each step's disturbances from its Philox counters inside the
    trajectory loop gives exactly the stored-array results (same values), also
    under parametric uncertainty and through the pipelined search."""
    N, H = 300, 333
    p = {"fp64": R.FP64, "fp32": R.FP32, "fp32_recheck": R.FP32_RECHECK}[prec]
    x_t = orc.equilibrium(params, 100.0) * np.array([1.0, 1.02, 1.0])
    kappas = np.linspace(0.0, 0.3, 13)
    for unc in (0.0, 0.1):
        outs = []
        for gen in (0, 1):
            cfg = _cfg(R, N, H, precision=p, early_exit=R.EXIT_NONE, max_candidates=16,
                       scenarios_in_register=gen, param_unc_rel=unc, recheck_eps_rel=SLACK32_TOL / 1.9)
            with R.Governor(params, cfg) as g:
                g.sample_scenarios(4, 9)
                adm, ms, P = g.eval_candidates(x_t, 100.0, 250.0, kappas, want_P=True)
                step = g.step(x_t, 250.0, 100.0)
                if gen:
                    with pytest.raises(R.RrgError):
                        g.set_scenarios(np.zeros((3, H, N)))
            outs.append((adm, ms, P, np.array(step)))
        for a, b in zip(*outs):
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("unc,N", [(0.0, 8192), (0.1, 32768)])
def test_register_and_shared_rings_agree(R, orc, params, unc, N):
    """Binary32 lanes read the stored scenarios through a shared-memory ring
    when a launch leaves most warp slots empty (at most 16 warps per SM, 64
    with parametric uncertainty) and through a register ring when it fills
    the SMs.  12 candidates in one launch (3,072 / 12,288 warps: register
    ring) and each candidate alone (256 / 1,024 warps: shared ring) give the
    same min slack and the same P bit for bit; sampled lanes match the
    oracle's per-trajectory decisions."""
    H = 200
    x_t = orc.equilibrium(params, 100.0) * np.array([1.0, 1.03, 1.0])
    kappas = np.linspace(0.0, 1.0, 12)
    cfg = _cfg(R, N, H, precision=R.FP32, early_exit=R.EXIT_NONE, max_candidates=16, param_unc_rel=unc)
    with R.Governor(params, cfg) as g:
        g.sample_scenarios(5, 2)
        adm, ms, P = g.eval_candidates(x_t, 100.0, 250.0, kappas, want_P=True)
        for i, k in enumerate(kappas):
            a1, m1, P1 = g.eval_candidates(x_t, 100.0, 250.0, [k], want_P=True)
            assert a1[0] == adm[i] and m1[0] == ms[i]
            np.testing.assert_array_equal(P1[0], P[i])
    d = orc.sample_disturbances(5, 2, N, H, inputs.DIST_AMP)
    mult = orc.sample_param_multipliers(5, 2, N, unc, inputs.FC3_UNCERTAIN_MASK) if unc else None
    assert 0 < int(P.sum()) < P.size
    c = orc.cfg(H=H, N=N, early_exit=0)
    rng = np.random.default_rng(7)
    with orc.param_multipliers(mult):
        for k in rng.choice(N, size=12, replace=False):
            for i in (0, 5, 11):
                s, _ = orc.rollout(params, c, x_t, orc.governed(100.0, 250.0, kappas[i]), d, k)
                if abs(s) > SLACK32_TOL:
                    assert P[i, k] == (1 if s >= 0 else 0)


def test_in_register_scenarios_closed_loop(R, orc, params):
    N, H, T = 32, 200, 5
    r_seq = inputs.staircase(T, 3, 2, seed=8)
    x0 = orc.equilibrium(params, 100.0)
    amp = inputs.DIST_AMP
    runs = []
    for gen in (0, 1):
        cfg = _cfg(R, N, H, precision=R.FP32_RECHECK, max_candidates=16, scenarios_in_register=gen,
                   recheck_eps_rel=SLACK32_TOL / 1.9)
        with R.Governor(params, cfg) as g:
            runs.append(g.closed_loop(x0, 100.0, r_seq, 3, 1, amp, use_graph=True))
    for a, b in zip(*runs):
        np.testing.assert_array_equal(a, b)


def test_step_latency(R, orc, params):
    """One warp's cycles per binary32 trajectory step: positive, stable over
    horizons, argument errors reported, and the handle's results unchanged."""
    cfg = _cfg(R, 64, 300, precision=R.FP32_RECHECK, recheck_eps_rel=SLACK32_TOL / 1.9)
    x_t = orc.equilibrium(params, 100.0)
    with R.Governor(params, cfg) as g:
        g.sample_scenarios(3, 1)
        before = g.step(x_t, 250.0, 100.0)
        c2000 = g.step_latency(100.0, 2000)
        c500 = g.step_latency(180.0, 500)
        assert 50.0 < c2000 < 5000.0 and 50.0 < c500 < 5000.0
        assert abs(c500 - c2000) < 0.3 * c2000
        with pytest.raises(R.RrgError):
            g.step_latency(-1.0)
        with pytest.raises(R.RrgError):
            g.step_latency(100.0, 0)
        assert g.step(x_t, 250.0, 100.0) == before


def test_alu_peaks_are_plausible(R):
    """The unit throughput measured on this GPU: binary32 FMA near the
    derived 80.5 TFLOP/s, binary64 FMA far below it, MUFU exp2 in between."""
    f32, f64, mufu = R.rrg_alu_peaks()
    print("measured: fp32 FMA %.1f TFLOP/s, fp64 FMA %.2f TFLOP/s, MUFU ex2 %.2f Top/s" % (f32, f64, mufu))
    assert 20.0 < f32 < 100.0
    assert 0.05 < f64 < f32 / 8
    assert 0.5 < mufu < f32


@pytest.mark.parametrize("m,probe", [(4, 1), (64, 1), (64, 32)])
def test_closed_loop_graph_runs_remaining_rounds_when_needed(R, orc, params, m, probe):
    """In the replayed graph the rounds after the pipelined pair sit in a
    conditional node that runs only when the search is unfinished (a wrong
    provisional outcome, or more levels than the pair covers, as with 4
    candidates per round): the kappas equal direct launches and the oracle."""
    N, H, T = 24, 150, 6
    r_seq = inputs.staircase(T, 3, 2, seed=12)
    x0 = orc.equilibrium(params, 100.0) * np.array([1.0, 1.04, 1.02])
    amp = inputs.DIST_AMP
    cfg = _cfg(R, N, H, search=R.SEARCH_SPEC_BISECT, precision=R.FP32_RECHECK, max_candidates=m,
               probe_steps=probe, recheck_eps_rel=SLACK32_TOL / 1.9)
    runs, stats = [], []
    for use_graph in (False, True):
        with R.Governor(params, cfg) as g:
            runs.append(g.closed_loop(x0, 100.0, r_seq, 2, 0, amp, use_graph=use_graph))
            stats.append(g.stats())
            assert stats[-1]["graph_conditional"] == (1 if use_graph else 0)
    for a, b in zip(*runs):
        np.testing.assert_array_equal(a, b)
    # launch counts: direct launches enqueue every round of every update (the
    # pair, then `extra` rounds that are no-ops once the search is done); the
    # replays count the conditional body's rounds only on the updates where
    # it ran (rollout + recheck + search kernel per round)
    direct, graph = stats
    extra = direct["rounds"] // T - 1
    assert extra >= 1 and direct["rounds"] == T * (1 + extra)
    assert (graph["rounds"] - T) % extra == 0
    body_runs = (graph["rounds"] - T) // extra
    assert 0 <= body_runs <= T
    skipped = T - body_runs
    assert graph["rollout_launches"] == direct["rollout_launches"] - skipped * extra
    assert graph["launches"] == direct["launches"] - skipped * extra * 3
    if m == 4:      # the pair covers 5 of the 12 levels: unfinished unless kappa = 1 passes
        assert body_runs >= 1
    vo, ko, fo, xo = orc.closed_loop(params, orc.cfg(H=H, N=N), x0, 100.0, r_seq, 2, 0, amp, amp, search=0)
    np.testing.assert_array_equal(runs[1][1], ko)
    np.testing.assert_array_equal(runs[1][2], fo)


@pytest.mark.parametrize("kind,probe", [("spec", 0), ("spec", 32), ("spec", 128), ("ksection", 0), ("bisect", 0)])
def test_step_graph_equals_direct_launches(R, orc, params, kind, probe):
    """rrg_step replays its search as a captured graph (with a pipelined search
    the rounds after the pipelined pair sit in a conditional node); with the
    library's rollout timing on it launches directly.  Both give the same
    results on a sequence of inputs, the graph is rebuilt after a shape
    change, and each equals the oracle's joint bisection (Alg. 1)."""
    N, H, seed = 512, 300, 4
    search = {"spec": R.SEARCH_SPEC_BISECT, "ksection": R.SEARCH_KSECTION, "bisect": R.SEARCH_BISECT}[kind]
    cases = [(100.0, 250.0, orc.equilibrium(params, 100.0)),
             (180.0, 90.0, orc.equilibrium(params, 180.0) * np.array([1.02, 0.99, 1.01])),
             (60.0, 280.0, orc.equilibrium(params, 60.0)),
             (250.0, 260.0, orc.equilibrium(params, 250.0))]
    cfg = _cfg(R, N, H, search=search, precision=R.FP32_RECHECK, max_candidates=64, probe_steps=probe,
               recheck_eps_rel=1e-6)
    res = {}
    with R.Governor(params, cfg) as g:
        for mode in ("graph", "direct", "graph_after_retune"):
            g.set_profiling(mode == "direct")
            if mode == "graph_after_retune" and kind == "spec":
                g.set_tuning(16, probe)
            out = []
            for t, (v_prev, r, x_t) in enumerate(cases):
                g.sample_scenarios(seed, t)
                out.append(g.step(x_t, r, v_prev))
            res[mode] = out
        g.set_profiling(False)
    assert res["graph"] == res["direct"] == res["graph_after_retune"]
    if kind != "ksection":
        for t, ((v_prev, r, x_t), (_, k, f)) in enumerate(zip(cases, res["graph"])):
            d = orc.sample_disturbances(seed, t, N, H, inputs.DIST_AMP)
            assert (k, f) == orc.bisect_joint(params, orc.cfg(H=H, N=N), x_t, v_prev, r, 12, d)
