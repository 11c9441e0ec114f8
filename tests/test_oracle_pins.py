"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Nothing here runs on a GPU.  Each test names the passage or the identity it
checks.  The paper (arXiv 2510.08288) prints no numeric example, so the pins
are library routines (numpy's Philox, scipy's expm / DOP853), closed forms,
brute force on tiny inputs and the identities the paper states (Alg. 1 is
Alg. 2 with d = 0 and N_sim = 1; grid search equals bisection on the dyadic
grid; more scenarios never raise kappa).
"""
import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.linalg import expm

from paper_2510_08288_gb300 import inputs


# ---------------------------------------------------------------- Philox ----
@pytest.mark.parametrize("key", [0, 5, 2**63 + 12345, 2**64 - 1])
def test_philox_matches_numpy(orc, key):
    """Philox4x64-10 (Salmon et al. SC'11) equals numpy.random.Philox, an
    independent implementation; numpy advances word 0 of the counter before
    each block, so its block n is ours at counter n + 1."""
    for start in (0, 7, 2**40):
        bg = np.random.Philox(key=key, counter=start)
        raw = bg.random_raw(12)
        kw = bg.state["state"]["key"]
        for blk in range(3):
            mine = orc.philox4x64_10([start + 1 + blk, 0, 0, 0], kw)
            np.testing.assert_array_equal(raw[4 * blk:4 * blk + 4], mine)


def test_philox_full_counter_matches_numpy(orc):
    """All four counter words enter the block (numpy counter set explicitly)."""
    ctr = np.array([3, 0xDEADBEEF, 17, 1], dtype=np.uint64)
    bg = np.random.Philox(key=np.array([11, 22], dtype=np.uint64),
                          counter=np.array([2, 0xDEADBEEF, 17, 1], dtype=np.uint64))
    raw = bg.random_raw(4)
    np.testing.assert_array_equal(raw, orc.philox4x64_10(ctr, [11, 22]))


def test_disturbance_range_and_moments(orc):
    """d_j^k i.i.d. uniform on [-a, a) per component (Sec. IV-A ranges)."""
    amp = inputs.DIST_AMP
    d = orc.sample_disturbances(3, 9, 512, 200, amp)
    for i, a in enumerate(amp):
        di = d[i]
        assert di.min() >= -a and di.max() < a
        assert abs(di.mean()) < 0.02 * a
        assert abs(di.var() / (a * a / 3.0) - 1.0) < 0.02
    # scenarios are independent of N: a prefix of a larger draw (nested sets)
    d_small = orc.sample_disturbances(3, 9, 100, 200, amp)
    np.testing.assert_array_equal(d_small, d[:, :, :100])
    # a different update index draws new scenarios (redrawn every RG step)
    d_next = orc.sample_disturbances(3, 10, 100, 200, amp)
    assert not np.any(d_next == d_small)


# ------------------------------------------------------------------- RK4 ----
def _linear_system():
    rng = np.random.default_rng(4)
    A = -np.diag([3.0, 1.0, 0.4]) + 0.5 * (rng.standard_normal((3, 3)) - rng.standard_normal((3, 3)).T)
    B = rng.standard_normal(3)
    return A, B


def test_rk4_one_step_taylor_closed_form(orc):
    """On x' = Ax + Bu one classical RK4 step is exactly the degree-4 Taylor
    polynomial of the flow: x+ = T4(hA) x + h (I + hA/2 + (hA)^2/6 + (hA)^3/24) B u."""
    A, B = _linear_system()
    x = np.array([0.3, -1.2, 2.0])
    u = 0.7
    for h in (0.01, 0.1, 0.37):
        M = h * A
        I3 = np.eye(3)
        T4 = I3 + M + M @ M / 2 + M @ M @ M / 6 + M @ M @ M @ M / 24
        S = I3 + M / 2 + M @ M / 6 + M @ M @ M / 24
        want = T4 @ x + h * S @ (B * u)
        got = orc.rk4_linear(A, B, u, x, h)
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-14)


def test_rk4_global_order_four_vs_expm(orc):
    """Global error against the matrix-exponential solution falls as h^4."""
    A, B = _linear_system()
    x0 = np.array([1.0, 0.5, -0.5])
    u, T = 0.3, 2.0
    eAT = expm(A * T)
    exact = eAT @ x0 + np.linalg.solve(A, (eAT - np.eye(3)) @ (B * u))
    errs = []
    for n in (20, 40, 80):
        h = T / n
        x = x0.copy()
        for _ in range(n):
            x = orc.rk4_linear(A, B, u, x, h)
        errs.append(np.linalg.norm(x - exact))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((slopes > 3.8) & (slopes < 4.3)), slopes


def test_fc3_rk4_order_four_vs_dop853(orc, params):
    """The FC3 RK4 step converges at order 4 against scipy's DOP853 run on the
    same vector field (catches a wrong stage weight or stage point)."""
    x0 = orc.equilibrium(params, 100.0)
    I_new, T = 250.0, 0.1
    ref = solve_ivp(lambda t, x: orc.rhs(params, x, I_new), (0.0, T), x0, method="DOP853",
                    rtol=1e-13, atol=1e-9).y[:, -1]
    errs = []
    for n in (40, 80, 160):
        x = x0.copy()
        for _ in range(n):
            x = orc.rk4_step(params, x, I_new, T / n)
        errs.append(np.max(np.abs(x - ref) / np.abs(ref)))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((slopes > 3.6) & (slopes < 4.4)), (errs, slopes)


# ------------------------------------------------------------------- FC3 ----
def test_fc3_output_scales_inversely_with_current(orc, params):
    """OER = O2 supplied / O2 consumed, and consumption is proportional to the
    stack current (Faraday): h(x, 2I) = h(x, I) / 2."""
    x = np.array([120000.0, 5000.0, 130000.0])
    for I in (50.0, 123.4, 300.0):
        assert orc.output(params, x, 2 * I) == pytest.approx(orc.output(params, x, I) / 2, rel=1e-15)


def test_fc3_current_enters_only_the_cathode_balance(orc, params):
    """Only the cathode mass balance consumes O2: d(dp_ca/dt)/dI is the
    constant -R_a T_st / V_ca * M_O2 n_cell / (4 F); the other rates do not
    depend on I except through the controller's feed-forward (omega row)."""
    P = dict(zip(inputs.FC3_PARAM_NAMES, params))
    x = np.array([118000.0, 4600.0, 129000.0])
    f1, f2 = orc.rhs(params, x, 100.0), orc.rhs(params, x, 180.0)
    slope = -P["R_a"] * P["T_st"] / P["V_ca"] * P["M_O2"] * P["n_cell"] / (4 * P["faraday"])
    assert (f2[0] - f1[0]) / 80.0 == pytest.approx(slope, rel=1e-9)
    assert f2[2] == f1[2]


def test_fc3_total_mass_balance(orc, params):
    """Sum of the two manifold balances: the orifice flow between them cancels,
    so V_ca dp_ca + V_sm dp_sm = R T (W_cp - W_ca - W_O2) and is unchanged by
    the orifice coefficient k_sm."""
    x = np.array([121000.0, 5200.0, 133000.0])
    P = dict(zip(inputs.FC3_PARAM_NAMES, params))
    a = orc.rhs(params, x, 150.0)
    b = orc.rhs(inputs.fc3_params(k_sm=2 * P["k_sm"]), x, 150.0)
    tot = lambda f: P["V_ca"] * f[0] + P["V_sm"] * f[2]
    assert tot(a) == pytest.approx(tot(b), rel=1e-9, abs=1e-9)
    assert a[1] == b[1]


@pytest.mark.parametrize("I", [50.0, 100.0, 175.0, 250.0, 300.0])
def test_equilibrium_residual_and_stability(orc, params, I):
    """x_eq(v) found by the 1-D flow reduction zeroes all three balances of the
    full right-hand side; the Jacobian there is Hurwitz and every eigenvalue
    times dt lies well inside RK4's stability region (the model's acceptance
    conditions; the closed loop is stable as Sec. II-A assumes)."""
    x = orc.equilibrium(params, I)
    f = orc.rhs(params, x, I)
    P = dict(zip(inputs.FC3_PARAM_NAMES, params))
    RT = P["R_a"] * P["T_st"]
    W = P["k_sm"] * (x[2] - x[0])
    assert abs(f[0]) < 1e-9 * RT / P["V_ca"] * W
    assert abs(f[2]) < 1e-9 * RT / P["V_sm"] * W
    assert abs(f[1]) < 1e-6 * abs(x[1])
    J = np.zeros((3, 3))
    for i in range(3):
        h = 1e-6 * abs(x[i])
        e = np.zeros(3)
        e[i] = h
        J[:, i] = (orc.rhs(params, x + e, I) - orc.rhs(params, x - e, I)) / (2 * h)
    lam = np.linalg.eigvals(J) * inputs.DT
    assert np.all(lam.real < 0)
    assert np.all(np.abs(lam) < 1.5)          # RK4 real-axis limit is about 2.785
    y = orc.output(params, x, I)
    assert 2.15 < y < 2.25


def test_zero_disturbance_equilibrium_stays_put(orc, params):
    """With d = 0 and x_t = x_eq(v) the RK4 trajectory stays on x_eq to roundoff."""
    I = 140.0
    x = orc.equilibrium(params, I)
    y = x.copy()
    for _ in range(2000):
        y = orc.rk4_step(params, y, I, inputs.DT)
    np.testing.assert_allclose(y, x, rtol=1e-9)


def test_current_step_violates_oer_without_governor(orc, params):
    """A step of the current from 100 A to 250 A drives OER below 1.9 (the
    transient the governor exists for, Sec. IV-A) and the loop settles back."""
    x = orc.equilibrium(params, 100.0)
    ys = []
    for _ in range(600):
        ys.append(orc.output(params, x, 250.0))
        x = orc.rk4_step(params, x, 250.0, inputs.DT)
    assert min(ys) < 1.9
    assert ys[-1] > 2.15


# -------------------------------------------------------------- searches ----
def _problem(orc, params, H=40, N=3, seed=7):
    x = orc.equilibrium(params, 100.0)
    d = orc.sample_disturbances(seed, 0, N, H, inputs.DIST_AMP)
    return x, d


def _dyadic_truth(orc, params, c, x, v_prev, r, n_kappa, d):
    grid = np.arange(2 ** (n_kappa - 1) + 1) / 2.0 ** (n_kappa - 1)
    adm, _, _, _ = orc.eval_candidates(params, c, x, v_prev, r, grid, d)
    feas = adm.astype(bool)
    return grid, feas


@pytest.mark.parametrize("r", [120.0, 180.0, 250.0, 300.0, 60.0, 100.0])
def test_bisection_equals_bruteforce_dyadic_grid(orc, params, r):
    """Alg. 1 on the joint predicate with N_kappa iterations returns the largest
    admissible point of {m 2^(1-N_kappa)} when admissibility is downward closed
    in kappa; Alg. 2 (min over scenarios, Sec. II-C) and Alg. 3 with
    M = 2^(N_kappa-1) + 1 (Eq. 5) return the same kappa."""
    n_kappa = 8
    x, d = _problem(orc, params)
    c = orc.cfg(H=40, N=3)
    grid, feas = _dyadic_truth(orc, params, c, x, 100.0, r, n_kappa, d)
    first_bad = np.argmin(feas) if not feas.all() else len(feas)
    assert not feas[first_bad:].any(), "predicate not monotone on this case"
    want = grid[first_bad - 1] if first_bad > 0 else 0.0
    kj, fj = orc.bisect_joint(params, c, x, 100.0, r, n_kappa, d)
    k2, _ = orc.alg2(params, c, x, 100.0, r, n_kappa, d)
    k3, f3 = orc.alg3(params, c, x, 100.0, r, 2 ** (n_kappa - 1) + 1, d)
    assert kj == want and k2 == want and k3 == want
    assert 0.0 <= kj <= 1.0
    if r == 100.0:
        assert kj == 1.0


def test_alg1_is_alg2_without_disturbance(orc, params):
    """Alg. 1 is Alg. 2 with d_t = 0 and N_sim = 1 (Sec. II-C)."""
    x = orc.equilibrium(params, 90.0)
    c = orc.cfg(H=300, N=1)
    zero = np.zeros((3, 300, 1))
    for r in (95.0, 110.0, 160.0, 280.0, 55.0):
        k1, f1 = orc.alg1(params, c, x, 90.0, r, 12)
        k2, f2 = orc.alg2(params, c, x, 90.0, r, 12, zero)
        assert k1 == k2 and f1 == f2


def test_more_scenarios_never_raise_kappa(orc, params):
    """Adding scenarios (nested draws) can only remove admissible candidates,
    so Alg. 3 and Alg. 2 return non-increasing kappa as N_sim grows."""
    x = orc.equilibrium(params, 100.0)
    prev3 = prev2 = 1.0
    for N in (1, 2, 4, 8, 16):
        d = orc.sample_disturbances(11, 3, N, 120, inputs.DIST_AMP)
        c = orc.cfg(H=120, N=N)
        k3, _ = orc.alg3(params, c, x, 100.0, 240.0, 65, d)
        k2, _ = orc.alg2(params, c, x, 100.0, 240.0, 10, d)
        assert k3 <= prev3 and k2 <= prev2
        prev3, prev2 = k3, k2


def test_early_exit_does_not_change_decisions(orc, params):
    """Stopping a rollout at its first violation (Sec. III-B/C) leaves every
    P entry and every candidate decision unchanged."""
    x, d = _problem(orc, params, H=80, N=6)
    kap = np.linspace(0.0, 1.0, 21)
    a1, s1, P1, st1 = orc.eval_candidates(params, orc.cfg(H=80, N=6, early_exit=1), x, 100.0, 250.0, kap, d, True)
    a0, s0, P0, st0 = orc.eval_candidates(params, orc.cfg(H=80, N=6, early_exit=0), x, 100.0, 250.0, kap, d, True)
    np.testing.assert_array_equal(a1, a0)
    np.testing.assert_array_equal(P1, P0)
    np.testing.assert_array_equal(s1[a1 == 1], s0[a0 == 1])
    assert st1 < st0


def test_hold_is_admissible_at_equilibrium(orc, params):
    """x_t = x_eq(v_prev), no disturbance: kappa = 0 keeps the loop at its
    equilibrium whose OER exceeds 1.9, so P's kappa = 0 row is all ones."""
    v_prev = 200.0
    x = orc.equilibrium(params, v_prev)
    zero = np.zeros((3, 200, 4))
    adm, ms, P, _ = orc.eval_candidates(params, orc.cfg(H=200, N=4), x, v_prev, 300.0, [0.0], zero, True)
    assert adm[0] == 1 and P.all()
    assert ms[0] == pytest.approx(orc.output(params, x, v_prev) - 1.9, rel=1e-9)


def test_steady_state_tightening(orc, params):
    """y_ss(v) must lie in the tightened set: with eps = 0 the bound is y_min,
    with eps = 1 it is y_c; OER_ss ~ 2.2 passes the first and fails y_c = 2.3."""
    I = 150.0
    y_ss = orc.output(params, orc.equilibrium(params, I), I)
    assert orc.ss_ok(params, orc.cfg(eps_ss=0.0), I)
    assert not orc.ss_ok(params, orc.cfg(eps_ss=1.0, y_c=y_ss + 1e-6), I)
    assert orc.ss_ok(params, orc.cfg(eps_ss=1.0, y_c=y_ss - 1e-6), I)
    assert orc.ss_ok(params, orc.cfg(ss_check=0, eps_ss=1.0, y_c=9.0), I)


def test_infeasible_everywhere_holds(orc, params):
    """Nothing admissible (y_min above every reachable OER): Alg. 1 and Alg. 3
    return kappa = 0 (hold v_prev) and flag it."""
    x = orc.equilibrium(params, 100.0)
    d = orc.sample_disturbances(1, 0, 2, 30, inputs.DIST_AMP)
    c = orc.cfg(H=30, N=2, y_min=5.0)
    assert orc.bisect_joint(params, c, x, 100.0, 200.0, 10, d) == (0.0, 1)
    assert orc.alg3(params, c, x, 100.0, 200.0, 9, d) == (0.0, 1)
    assert orc.ksection(params, c, x, 100.0, 200.0, 9, 3, d) == (0.0, 1)


def test_ksection_one_round_is_alg3_and_brackets_the_boundary(orc, params):
    """One k-section round is the grid of Alg. 3; after R rounds the result is
    admissible and the next point one cell up is not (monotone case)."""
    x, d = _problem(orc, params, H=60, N=4)
    c = orc.cfg(H=60, N=4)
    M = 9
    assert orc.ksection(params, c, x, 100.0, 250.0, M, 1, d) == orc.alg3(params, c, x, 100.0, 250.0, M, d)
    k, _ = orc.ksection(params, c, x, 100.0, 250.0, M, 3, d)
    width = (1.0 / (M - 1)) / (M + 1) ** 2
    a, _, _, _ = orc.eval_candidates(params, c, x, 100.0, 250.0, [k, k + width], d)
    assert a[0] == 1 and a[1] == 0


def test_threads_do_not_change_results(orc, params):
    """The threaded evaluation (Sec. III-B scheme) equals the sequential one."""
    x, d = _problem(orc, params, H=100, N=16)
    c = orc.cfg(H=100, N=16, early_exit=0)
    kap = np.linspace(0, 0.3, 13)
    r1 = orc.eval_candidates(params, c, x, 100.0, 250.0, kap, d, True, nthreads=1)
    r4 = orc.eval_candidates(params, c, x, 100.0, 250.0, kap, d, True, nthreads=4)
    for a, b in zip(r1[:3], r4[:3]):
        np.testing.assert_array_equal(a, b)


def test_governed_reference_is_eq2(orc):
    """v = v_prev + kappa (r - v_prev) evaluated as written (Eq. 2)."""
    rng = np.random.default_rng(0)
    for _ in range(100):
        vp, r, k = rng.uniform(50, 300), rng.uniform(50, 300), rng.uniform()
        assert orc.governed(vp, r, k) == vp + k * (r - vp)
    assert orc.governed(80.0, 200.0, 0.0) == 80.0
    assert orc.governed(80.0, 200.0, 1.0) == 200.0


def test_non_finite_state_is_a_violation(orc, params):
    """A non-finite state or output counts as a violation (slack -inf)."""
    c = orc.cfg(H=10, N=1)
    s, _ = orc.rollout(params, c, [np.nan, 3000.0, 120000.0], 100.0)
    assert s == -np.inf


# --------------------------------------------------- parametric uncertainty --
def test_param_multipliers_range_moments_and_mask(orc):
    """Per-scenario multipliers m_p^k uniform on [1 - rho, 1 + rho) for every
    uncertain parameter, exactly 1 for the rest; i.i.d. over k and p; redrawn
    with the update index; nested in N."""
    rho, mask = 0.1, inputs.FC3_UNCERTAIN_MASK
    m = orc.sample_param_multipliers(7, 3, 4096, rho, mask)
    unc = np.array([(mask >> p) & 1 for p in range(orc.nparam())], dtype=bool)
    assert unc.sum() == len(inputs.FC3_UNCERTAIN)
    np.testing.assert_array_equal(m[:, ~unc], 1.0)
    mu = m[:, unc]
    assert mu.min() >= 1.0 - rho and mu.max() < 1.0 + rho
    assert np.all(np.abs(mu.mean(axis=0) - 1.0) < 0.006)
    assert np.all(np.abs(mu.var(axis=0) / (rho * rho / 3.0) - 1.0) < 0.08)
    # distinct parameters of one scenario are not the same draw
    c = np.corrcoef(mu.T)
    assert np.max(np.abs(c - np.eye(c.shape[0]))) < 0.06
    np.testing.assert_array_equal(orc.sample_param_multipliers(7, 3, 100, rho, mask), m[:100])
    assert not np.any(orc.sample_param_multipliers(7, 4, 100, rho, mask)[:, unc] == m[:100, unc])
    np.testing.assert_array_equal(orc.sample_param_multipliers(7, 3, 64, 0.0, mask), 1.0)


def test_param_multiplier_words_from_philox(orc):
    """m_p^k comes from word p % 4 of the Philox block at counter
    (p / 4, k, update, 2): the stream-2 blocks, pinned to numpy's Philox
    above, mapped to 1 + rho (2u - 1) with u the top 53 bits over 2^53."""
    rho, seed, upd = 0.25, 99, 12
    m = orc.sample_param_multipliers(seed, upd, 5, rho, (1 << orc.nparam()) - 1)
    for k in range(5):
        for p in range(orc.nparam()):
            w = int(orc.philox4x64_10([p // 4, k, upd, 2], [seed, 0])[p % 4])
            u = (w >> 11) / 2.0**53
            assert m[k, p] == 1.0 + rho * (2.0 * u - 1.0)


def test_param_multipliers_scale_scenario_parameters(orc, params):
    """With multipliers loaded, scenario k's rollout is the nominal rollout of
    the model with parameters theta * m^k (only scenario k's row is used),
    and leaving the context restores the nominal model."""
    N, H = 6, 120
    c = orc.cfg(H=H, N=N, early_exit=0)
    x = orc.equilibrium(params, 120.0)
    d = orc.sample_disturbances(1, 0, N, H, inputs.DIST_AMP)
    m = orc.sample_param_multipliers(1, 0, N, 0.1, (1 << orc.nparam()) - 1)
    nominal = [orc.rollout(params, c, x, 180.0, d, k)[0] for k in range(N)]
    with orc.param_multipliers(m):
        scaled = [orc.rollout(params, c, x, 180.0, d, k)[0] for k in range(N)]
    direct = [orc.rollout(params * m[k], c, x, 180.0, d, k)[0] for k in range(N)]
    assert scaled == direct
    assert all(a != b for a, b in zip(scaled, nominal))
    assert [orc.rollout(params, c, x, 180.0, d, k)[0] for k in range(N)] == nominal
    # multipliers of one make no difference
    with orc.param_multipliers(np.ones_like(m)):
        assert [orc.rollout(params, c, x, 180.0, d, k)[0] for k in range(N)] == nominal


# ------------------------------------------------- adjoint's objective ----
def _slack_by_steps(orc, p, x_t, I, d, k, jstar, dt=0.01, y_min=1.9):
    """s_jstar^k by the real-valued primitives one step at a time: jstar RK4
    steps of scenario k, each followed by its disturbance, then h - y_min."""
    x = np.array(x_t, dtype=float)
    for j in range(jstar):
        x = orc.rk4_step(p, x, I, dt) + d[:, j, k]
    return orc.output(p, x, I) - y_min


def test_min_slack_argmin_is_the_brute_force_minimum(orc, params):
    """The adjoint's objective g = min_k min_j s_j^k over the full horizon
    (j = 0 included) and its first argmin in (k, then j) order, against every
    slack computed step by step from the real primitives."""
    H, N = 40, 4
    x = orc.equilibrium(params, 100.0) * np.array([1.03, 0.98, 1.01])
    d = orc.sample_disturbances(11, 0, N, H, inputs.DIST_AMP)
    for kappa in (0.0, 0.05, 0.3):
        I = orc.governed(100.0, 250.0, kappa)
        S = np.array([[_slack_by_steps(orc, params, x, I, d, k, j) for j in range(H + 1)] for k in range(N)])
        g, k, j = orc.min_slack_argmin(params, orc.cfg(H=H, N=N), x, I, d)
        assert g == pytest.approx(S.min(), rel=1e-13, abs=1e-13)
        assert (k, j) == tuple(int(i) for i in np.unravel_index(np.argmin(S), S.shape))


@pytest.mark.parametrize("with_multipliers", [False, True])
@pytest.mark.parametrize("k,jstar", [(0, 0), (1, 17), (2, 40)])
def test_slack_gradient_matches_central_differences(orc, params, k, jstar, with_multipliers):
    """The complex-step gradient of s_jstar^k (kappa, x_t, theta; Squire and
    Trapp 1998, a separate complex-valued copy of the model) against central
    differences of the real-valued primitives with relative steps 1e-6; its
    real part equals the real-valued slack.  With parameter multipliers the
    derivative is taken with respect to the nominal theta."""
    H, N, v_prev, r, kappa = 40, 3, 100.0, 250.0, 0.1
    x = orc.equilibrium(params, v_prev) * np.array([1.02, 0.99, 1.01])
    d = orc.sample_disturbances(7, 0, N, H, inputs.DIST_AMP)
    m = orc.sample_param_multipliers(3, 0, N, 0.1, (1 << orc.nparam()) - 1) if with_multipliers else None
    c = orc.cfg(H=H, N=N)

    def s_real(p, x_t, kap):
        pk = p * m[k] if m is not None else p
        return _slack_by_steps(orc, pk, x_t, orc.governed(v_prev, r, kap), d, k, jstar)

    with orc.param_multipliers(m):
        s, grad = orc.slack_grad(params, c, x, v_prev, r, kappa, d, k, jstar)
    assert s == pytest.approx(s_real(params, x, kappa), rel=1e-13, abs=1e-14)
    fd = [(s_real(params, x, kappa + 1e-6) - s_real(params, x, kappa - 1e-6)) / 2e-6]
    for i in range(3):
        h = 1e-6 * abs(x[i])
        e = np.zeros(3)
        e[i] = h
        fd.append((s_real(params, x + e, kappa) - s_real(params, x - e, kappa)) / (2 * h))
    for i in range(orc.nparam()):
        h = 1e-6 * abs(params[i]) if params[i] != 0 else 1e-6
        e = np.zeros(orc.nparam())
        e[i] = h
        fd.append((s_real(params + e, x, kappa) - s_real(params - e, x, kappa)) / (2 * h))
    fd = np.array(fd)
    scale = np.abs(grad) + np.abs(fd)
    assert np.all(np.abs(grad - fd) <= 1e-5 * scale + 1e-12), np.max(np.abs(grad - fd) / np.maximum(scale, 1e-300))
    if jstar > 0:
        assert np.count_nonzero(grad) == grad.size  # every parameter reaches a state after one step


# ----------------------------------------------------------- closed loop ----
def _numpy_block(ctr, key):
    """Philox4x64-10 block at counter ctr from numpy.random.Philox (which adds
    one to the 256-bit counter, with carries, before each block)."""
    c = [int(w) for w in ctr]
    v = (c[0] | (c[1] << 64) | (c[2] << 128) | (c[3] << 192)) - 1
    words = [(v >> (64 * i)) & (2**64 - 1) for i in range(4)]
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(words, dtype=np.uint64))
    return bg.random_raw(4)


def _sym(w, a):
    """a (2u - 1), u = (w >> 11) 2^-53 (the uniform mapping of the draws)."""
    return a * (2.0 * ((int(w) >> 11) * 2.0 ** -53) - 1.0)


def test_closed_loop_is_sample_search_govern_plant(orc, params):
    """Fig. 1's loop, two updates written out from its pieces: update t draws
    its scenarios from Philox counters (j, k, t0 + t, 0), runs Alg. 1 on the
    joint predicate from (x_t, v_{t-1}, r_t), applies Eq. 2, and the plant
    takes one RK4 step at v_t plus its own draw from counter (0, 0, t0 + t, 1).
    The draws are recomputed from numpy's Philox, so a wrong update index,
    stream, setpoint or order in the oracle's loop fails this test."""
    N, H, seed, t0 = 8, 120, 77, 5
    amp, pamp = np.array(inputs.DIST_AMP), np.array([30.0, 5.0, 20.0])
    c = orc.cfg(H=H, N=N)
    x0 = orc.equilibrium(params, 100.0) * np.array([1.0, 1.01, 0.995])
    r_seq = np.array([230.0, 120.0])
    v, kap, fl, xs = orc.closed_loop(params, c, x0, 100.0, r_seq, seed, t0, amp, pamp, search=0, n_kappa=12)
    x, vp = x0.copy(), 100.0
    for t in range(2):
        d = orc.sample_disturbances(seed, t0 + t, N, H, amp)
        for (j, k) in ((1, 0), (7, 5), (H - 1, N - 1)):
            w = _numpy_block([j, k, t0 + t, 0], [seed, 0])
            for i in range(3):
                assert d[i, j, k] == _sym(w[i], amp[i])
        k_t, f_t = orc.bisect_joint(params, c, x, vp, r_seq[t], 12, d)
        v_t = vp + k_t * (r_seq[t] - vp)
        wp = _numpy_block([0, 0, t0 + t, 1], [seed, 0])
        x = orc.rk4_step(params, x, v_t, 0.01) + np.array([_sym(wp[i], pamp[i]) for i in range(3)])
        assert (kap[t], fl[t], v[t]) == (k_t, f_t, v_t)
        np.testing.assert_array_equal(xs[t + 1], x)
        vp = v_t
    assert 0.0 < kap[0] < 1.0      # the first update governs (kappa neither 0 nor 1)
