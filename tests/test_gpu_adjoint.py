"""Discrete adjoint of the robust objective on the GPU, through the C ABI.

g(kappa) = min over scenarios and steps of the slack (Alg. 3's test is
g >= 0).  The GPU's reverse sweep of RK4 (with checkpointing) is compared with
the FP64 oracle's complex-step derivative at the same argmin, with central
finite differences of the GPU's own g, and through the autograd wrapper; the
Newton search it drives is judged against 20-step bisection.
"""
import numpy as np
import pytest

from paper_2510_08288_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_08288_gb300 import build as B
    B.build()
    from paper_2510_08288_gb300 import rrg
    return rrg


def _gov(R, params, N, H, **kw):
    base = dict(horizon=H, n_scenarios=N, max_candidates=16, precision=R.FP64)
    base.update(kw)
    return R.Governor(params, R.rrg_config_default(**base))


@pytest.mark.parametrize("checkpoint", [1, 7, 50, 1000])
def test_adjoint_fp64_matches_complex_step(R, orc, params, checkpoint):
    N, H = 48, 300
    x_t = orc.equilibrium(params, 100.0) * np.array([1.0, 1.02, 1.01])
    with _gov(R, params, N, H) as g:
        g.sample_scenarios(4, 2)
        d = orc.sample_disturbances(4, 2, N, H, inputs.DIST_AMP)
        for kappa in (0.05, 0.1, 0.3):
            gv, grad, ks, js = g.slack_gradient(x_t, 100.0, 250.0, kappa, checkpoint, R.FP64)
            c = orc.cfg(H=H, N=N, early_exit=0)
            go, ko, jo = orc.min_slack_argmin(params, c, x_t, orc.governed(100.0, 250.0, kappa), d)
            assert (ks, js) == (ko, jo)
            assert gv == pytest.approx(go, rel=1e-10, abs=1e-12)
            so, gro = orc.slack_grad(params, c, x_t, 100.0, 250.0, kappa, d, ko, jo)
            scale = np.maximum(np.abs(gro), 1e-12 * np.max(np.abs(gro)))
            np.testing.assert_allclose(grad, gro, rtol=1e-7, atol=0)
            assert np.all(np.abs(grad - gro) <= 1e-7 * scale + 1e-14)


@pytest.mark.parametrize("checkpoint", [1, 7, 50, 800])
def test_adjoint_late_argmin_matches_complex_step(R, orc, params, checkpoint):
    """kappa = 0 (hold) from the 100 A equilibrium: the minimum slack comes
    late in the horizon (step 489 of 800), so the reverse sweep spans many
    checkpoint segments (489 at checkpoint 1, a partial last one at 7 and
    50, one at 800), all recomputed in parallel before the adjoint sweep."""
    N, H = 32, 800
    x_t = orc.equilibrium(params, 100.0)
    with _gov(R, params, N, H) as g:
        g.sample_scenarios(9, 0)
        d = orc.sample_disturbances(9, 0, N, H, inputs.DIST_AMP)
        gv, grad, ks, js = g.slack_gradient(x_t, 100.0, 250.0, 0.0, checkpoint, R.FP64)
    c = orc.cfg(H=H, N=N, early_exit=0)
    go, ko, jo = orc.min_slack_argmin(params, c, x_t, orc.governed(100.0, 250.0, 0.0), d)
    assert (ks, js) == (ko, jo) and jo > 400
    assert gv == pytest.approx(go, rel=1e-10, abs=1e-12)
    _, gro = orc.slack_grad(params, c, x_t, 100.0, 250.0, 0.0, d, ko, jo)
    np.testing.assert_allclose(grad, gro, rtol=1e-7, atol=1e-14 * np.max(np.abs(gro)))


def test_adjoint_forward_pass_is_timed_as_a_rollout(R, orc, params):
    """With profiling on, a gradient's forward pass (all scenarios, full
    horizon) is one timed rollout launch of the seven the call makes on a
    binary64 handle (candidate set-up 2, binary64 scenario fill 2, forward,
    argmin, reverse); a binary32 gradient on a binary32 handle reads the
    stored binary32 draw and skips the fill."""
    N, H = 256, 300
    x_t = orc.equilibrium(params, 100.0)
    with _gov(R, params, N, H) as g:
        g.sample_scenarios(2, 0)
        g.reset_stats()
        g.set_profiling(True)
        for prec in (R.FP32, R.FP64):
            g.slack_gradient(x_t, 100.0, 250.0, 0.1, 50, prec)
        st = g.stats()
    assert st["launches"] == 12 and st["rollout_launches"] == 2
    assert st["timed_rollouts"] == 2 and st["rollout_ms"] > 0
    with _gov(R, params, N, H, precision=R.FP32_RECHECK) as g:
        g.sample_scenarios(2, 0)
        g.reset_stats()
        g.slack_gradient(x_t, 100.0, 250.0, 0.1, 50, R.FP32)
        assert g.stats()["launches"] == 4


def test_adjoint_fp32_close_to_fp64(R, orc, params):
    N, H = 64, 400
    x_t = orc.equilibrium(params, 120.0)
    with _gov(R, params, N, H) as g:
        g.sample_scenarios(1, 1)
        g64, gr64, k64, j64 = g.slack_gradient(x_t, 120.0, 260.0, 0.08, 50, R.FP64)
        g32, gr32, k32, j32 = g.slack_gradient(x_t, 120.0, 260.0, 0.08, 50, R.FP32)
    assert (k32, j32) == (k64, j64)
    assert abs(g32 - g64) < 2e-4
    big = np.abs(gr64) > 1e-6 * np.max(np.abs(gr64))
    np.testing.assert_allclose(gr32[big], gr64[big], rtol=2e-3)


def test_adjoint_kappa_matches_central_differences(R, orc, params):
    """dg/dkappa against central differences (h = 1e-6) of the GPU's own g,
    at kappas where the argmin does not switch inside [kappa - h, kappa + h]."""
    N, H = 40, 250
    x_t = orc.equilibrium(params, 100.0)
    h = 1e-6
    with _gov(R, params, N, H) as g:
        g.sample_scenarios(6, 0)
        for kappa in (0.04, 0.09, 0.2):
            g0, grad, ks, js = g.slack_gradient(x_t, 100.0, 250.0, kappa)
            gp, _, kp, jp = g.slack_gradient(x_t, 100.0, 250.0, kappa + h)
            gm, _, km, jm = g.slack_gradient(x_t, 100.0, 250.0, kappa - h)
            if (kp, jp) != (ks, js) or (km, jm) != (ks, js):
                continue
            assert grad[0] == pytest.approx((gp - gm) / (2 * h), rel=1e-5)


def test_adjoint_full_size_workload(R, orc, params):
    """4,096 scenarios x 1,000 steps, checkpoint every 50 steps (the adjoint
    workload), FP64: value, argmin and gradient equal the oracle's."""
    w = inputs.WORKLOADS["adjoint"]
    N, H, C = w["N"], w["H"], w["checkpoint"]
    x_t = orc.equilibrium(params, 100.0)
    with _gov(R, params, N, H) as g:
        g.sample_scenarios(3, 0)
        d = orc.sample_disturbances(3, 0, N, H, inputs.DIST_AMP)
        gv, grad, ks, js = g.slack_gradient(x_t, 100.0, 250.0, 0.1, C, R.FP64)
    c = orc.cfg(H=H, N=N, early_exit=0)
    go, ko, jo = orc.min_slack_argmin(params, c, x_t, orc.governed(100.0, 250.0, 0.1), d)
    assert (ks, js) == (ko, jo) and gv == pytest.approx(go, rel=1e-10)
    _, gro = orc.slack_grad(params, c, x_t, 100.0, 250.0, 0.1, d, ko, jo)
    np.testing.assert_allclose(grad, gro, rtol=1e-7, atol=1e-14 * np.max(np.abs(gro)))


def test_autograd_function(R, orc, params):
    import torch
    from paper_2510_08288_gb300 import autograd as A
    N, H = 32, 200
    x_t = orc.equilibrium(params, 100.0)
    with _gov(R, params, N, H) as g:
        g.sample_scenarios(2, 0)
        kap = torch.tensor(0.07, dtype=torch.float64, requires_grad=True)
        xt = torch.tensor(x_t, dtype=torch.float64, requires_grad=True)
        th = torch.tensor(params, dtype=torch.float64, requires_grad=True)
        out = A.min_slack(kap, xt, th, g, 100.0, 250.0)
        (2.0 * out).backward()
        gv, grad, _, _ = g.slack_gradient(x_t, 100.0, 250.0, 0.07)
    assert out.item() == gv
    assert kap.grad.item() == pytest.approx(2 * grad[0], rel=1e-15)
    np.testing.assert_allclose(xt.grad.numpy(), 2 * grad[1:4], rtol=1e-15)
    np.testing.assert_allclose(th.grad.numpy(), 2 * grad[4:], rtol=1e-15)


@pytest.mark.parametrize("case", [(100.0, 250.0), (150.0, 290.0), (220.0, 300.0), (80.0, 60.0)])
def test_newton_search_agrees_with_bisection(R, orc, params, case):
    """The adjoint-driven Newton search lands within one bracket of the
    20-iteration joint bisection (Alg. 1) and needs fewer gradient
    evaluations than bisection needs rollout rounds."""
    v_prev, r = case
    N, H = 64, 400
    x_t = orc.equilibrium(params, v_prev)
    tol = 2.0 ** -19
    with _gov(R, params, N, H, precision=R.FP32_RECHECK, recheck_eps_rel=1e-4) as g:
        g.sample_scenarios(8, 1)
        k_n, fl, it = g.newton_search(x_t, r, v_prev, tol=tol, max_iter=40)
    d = orc.sample_disturbances(8, 1, N, H, inputs.DIST_AMP)
    k_b, f_b = orc.bisect_joint(params, orc.cfg(H=H, N=N), x_t, v_prev, r, 20, d)
    assert fl == f_b
    assert abs(k_n - k_b) <= tol + 2.0 ** -19
    assert it <= 20


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_multi_kappa_gradients_equal_single_calls(R, orc, params, precision):
    """rrg_slack_gradients at m kappas gives each kappa's single-call result
    bit for bit (each kappa's forward lanes, argmin and reverse sweep are its
    own), with the steady-state outcome of each."""
    N, H = 96, 300
    prec = R.FP64 if precision == "fp64" else R.FP32
    x_t = orc.equilibrium(params, 100.0) * np.array([1.0, 1.02, 1.01])
    kappas = np.array([0.0, 0.05, 0.1, 0.3, 0.9])
    with _gov(R, params, N, H, precision=R.FP32_RECHECK) as g:
        g.sample_scenarios(4, 2)
        gm, grm, km, jm, ss = g.slack_gradients(x_t, 100.0, 250.0, kappas, 7, prec)
        for i, k in enumerate(kappas):
            g1, gr1, k1, j1 = g.slack_gradient(x_t, 100.0, 250.0, k, 7, prec)
            assert (gm[i], km[i], jm[i]) == (g1, k1, j1)
            np.testing.assert_array_equal(grm[i], gr1)
    assert np.all(ss == 1)
    if prec == R.FP64:
        d = orc.sample_disturbances(4, 2, N, H, inputs.DIST_AMP)
        c = orc.cfg(H=H, N=N, early_exit=0)
        for i in (1, 3):
            go, ko, jo = orc.min_slack_argmin(params, c, x_t, orc.governed(100.0, 250.0, kappas[i]), d)
            assert (km[i], jm[i]) == (ko, jo) and gm[i] == pytest.approx(go, rel=1e-10, abs=1e-12)


def test_newton_search_full_size_workload(R, orc, params):
    """4,096 scenarios x 1,000 steps, checkpoint 50, binary32 gradients: the
    search lands within one bracket of the oracle's 20-iteration joint
    bisection (own draw), with the bracket judged by the binary32 + binary64
    recheck evaluation at the benchmark's band."""
    w = inputs.WORKLOADS["adjoint"]
    N, H, C = w["N"], w["H"], w["checkpoint"]
    tol = 2.0 ** -19
    x_t = orc.equilibrium(params, 100.0)
    with _gov(R, params, N, H, precision=R.FP32_RECHECK, recheck_eps_rel=1e-6, max_candidates=32) as g:
        g.sample_scenarios(3, 0)
        k_n, fl, it = g.newton_search(x_t, 250.0, 100.0, tol=tol, max_iter=40, checkpoint=C, precision=R.FP32)
    d = orc.sample_disturbances(3, 0, N, H, inputs.DIST_AMP)
    k_b, f_b = orc.bisect_joint(params, orc.cfg(H=H, N=N), x_t, 100.0, 250.0, 20, d,
                                nthreads=min(16, __import__("os").cpu_count() or 1))
    assert fl == f_b
    assert abs(k_n - k_b) <= tol + 2.0 ** -19
    assert it <= 12


def test_gradient_graph_equals_direct_launches(R, orc, params):
    """rrg_slack_gradients replays its kernels as a captured graph keyed by
    (m, checkpoint, precision) and the adjoint buffers; with the library's
    rollout timing on it launches them directly.  Both give the same bits,
    across calls with new inputs and after the call's shape changes."""
    N, H = 512, 300
    cases = [(orc.equilibrium(params, 100.0), 100.0, 250.0, [0.1]),
             (orc.equilibrium(params, 150.0) * np.array([1.01, 0.99, 1.0]), 150.0, 90.0, [0.3, 0.6]),
             (orc.equilibrium(params, 100.0), 100.0, 250.0, [0.05, 0.1, 0.2])]
    res = {}
    with _gov(R, params, N, H, precision=R.FP32_RECHECK) as g:
        g.sample_scenarios(3, 1)
        for mode in ("graph", "direct", "graph_again"):
            g.set_profiling(mode == "direct")
            out = []
            for x_t, v_prev, r, kap in cases:
                for prec in (R.FP32, R.FP64):
                    out.append(g.slack_gradients(x_t, v_prev, r, kap, 50, prec))
            res[mode] = out
        g.set_profiling(False)
    for a, b, c in zip(res["graph"], res["direct"], res["graph_again"]):
        for u, v, w in zip(a, b, c):
            np.testing.assert_array_equal(u, v)
            np.testing.assert_array_equal(u, w)
