"""Two candidates per thread (rrg_set_pairing) against one per thread.

The TMA ring, which takes precedence over pairing on large launches, is off
in these tests (RRG_TMA_NEVER), so the paired kernel is the one compared.

A paired thread runs candidates A and B of the same scenario off one load of
each disturbance, with the same per-trajectory arithmetic as a single lane:
the admissible flags, the P entries, every search result and the min slack
of every admissible candidate are identical in every mode (without an early
exit, every min slack).  The rows of a launch are paired 2y, 2y + 1, so odd
candidate counts leave a row alone in the last pair; scenario counts that are
not a multiple of the block leave a ragged tail.  The oracle draws its own
disturbances (and parameter multipliers) for the decisions it is compared on.
"""
import os

import numpy as np
import pytest

from paper_2510_08288_gb300 import inputs

pytestmark = pytest.mark.gpu
NTH = max(1, min(16, os.cpu_count() or 1))
BAND_REL = 1e-6
MASK = inputs.FC3_UNCERTAIN_MASK


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
    c = dict(horizon=H, n_scenarios=N, max_candidates=32, n_bisect=12, search=R.SEARCH_SPEC_BISECT,
             precision=R.FP32_RECHECK, early_exit=R.EXIT_CANDIDATE, recheck_eps_rel=BAND_REL,
             param_unc_mask=MASK)
    c.update(kw)
    return R.rrg_config_default(**c)


def _gov(R, params, cfg):
    g = R.Governor(params, cfg)
    g.set_tma(R.TMA_NEVER)
    return g


def _same_slack(a, b):
    """Bit-identical, NaN (a candidate failing the steady-state check) included."""
    a, b = np.asarray(a), np.asarray(b)
    assert a.shape == b.shape
    np.testing.assert_array_equal(np.isnan(a), np.isnan(b))
    np.testing.assert_array_equal(a[~np.isnan(a)], b[~np.isnan(b)])


@pytest.mark.parametrize("N,H", [(8192, 200), (300, 65), (129, 33), (1, 17)])
@pytest.mark.parametrize("prec", ["fp32", "fp32_recheck"])
@pytest.mark.parametrize("unc", [0.0, 0.1])
@pytest.mark.parametrize("early", [0, 1, 2])
def test_pairs_equal_single_lanes(R, orc, params, N, H, prec, unc, early):
    p = R.FP32 if prec == "fp32" else R.FP32_RECHECK
    kappas = np.linspace(0.0, 1.0, 13)   # 13 rows: the last pair has one
    x_t = orc.equilibrium(params, 100.0) * np.array([1.0, 1.03, 1.0])
    res = {}
    with _gov(R, params, _cfg(R, N, H, precision=p, early_exit=early, param_unc_rel=unc)) as g:
        assert g.get_pairing() == R.PAIR_FILLED
        g.sample_scenarios(5, 2)
        for mode in (R.PAIR_NEVER, R.PAIR_ALWAYS, R.PAIR_FILLED):
            g.set_pairing(mode)
            assert g.get_pairing() == mode
            res[mode] = (g.eval_candidates(x_t, 100.0, 250.0, kappas, want_P=True),
                         g.eval_candidates(x_t, 100.0, 250.0, kappas))
    (a0, m0, P0), (b0, n0, _) = res[R.PAIR_NEVER]
    for mode in (R.PAIR_ALWAYS, R.PAIR_FILLED):
        (a1, m1, P1), (b1, n1, _) = res[mode]
        np.testing.assert_array_equal(a1, a0)
        np.testing.assert_array_equal(b1, b0)
        np.testing.assert_array_equal(P1, P0)
        if early == 0:
            _same_slack(m1, m0)
            _same_slack(n1, n0)
        else:
            _same_slack(m1[a0 == 1], m0[a0 == 1])
            _same_slack(n1[b0 == 1], n0[b0 == 1])
    assert 0 < int(a0.sum()) < len(kappas) or N == 1


@pytest.mark.parametrize("unc", [0.0, 0.1])
def test_paired_recheck_decides_like_the_oracle(R, orc, params, unc):
    """Binary32 pairs + binary64 recheck at the benchmark's band: the oracle's
    per-scenario decisions (P) and admissible flags, candidates around the
    boundary (many near-zero lanes)."""
    N, H, seed, upd = 1000, 120, 3, 4
    # the boundary: kappa ~ 0.1 for the nominal model, lower with uncertain parameters
    kappas = np.linspace(0.0, 0.06, 25) if unc else np.linspace(0.09, 0.115, 26)
    x_t = orc.equilibrium(params, 100.0)
    with _gov(R, params, _cfg(R, N, H, early_exit=R.EXIT_LANE, param_unc_rel=unc)) as g:
        g.set_pairing(R.PAIR_ALWAYS)
        g.sample_scenarios(seed, upd)
        adm, _, P = g.eval_candidates(x_t, 100.0, 250.0, kappas, want_P=True)
    d = orc.sample_disturbances(seed, upd, N, H, inputs.DIST_AMP)
    mult = orc.sample_param_multipliers(seed, upd, N, unc, MASK) if unc else None
    with orc.param_multipliers(mult):
        a_o, _, P_o, _ = orc.eval_candidates(params, orc.cfg(H=H, N=N, early_exit=0), x_t, 100.0, 250.0,
                                             kappas, d, want_P=True, nthreads=NTH)
    np.testing.assert_array_equal(adm, a_o)
    np.testing.assert_array_equal(P, P_o)
    assert 0 < int(a_o.sum()) < len(kappas)


SEARCHES = [("spec", dict(search=3, probe_steps=0)), ("spec_probe", dict(search=3, probe_steps=128)),
            ("ksection", dict(search=2, n_rounds=3)), ("bisect", dict(search=0))]


@pytest.mark.parametrize("name,kw", SEARCHES, ids=[s[0] for s in SEARCHES])
def test_searches_are_unchanged_by_pairing(R, orc, params, name, kw):
    """Every search gives the same (v_t, kappa, flags) in the three modes;
    the speculative bisection and the bisection give the oracle's joint
    bisection over all scenarios."""
    N, H, seed, upd = 2048, 600, 3, 7
    cases = [(100.0, 250.0, orc.equilibrium(params, 100.0)),
             (180.0, 90.0, orc.equilibrium(params, 180.0) * np.array([1.02, 0.99, 1.01])),
             (60.0, 280.0, orc.equilibrium(params, 60.0))]
    out = {}
    with _gov(R, params, _cfg(R, N, H, **kw)) as g:
        g.sample_scenarios(seed, upd)
        for mode in (R.PAIR_NEVER, R.PAIR_FILLED, R.PAIR_ALWAYS):
            g.set_pairing(mode)
            out[mode] = [g.step(x_t, r, v_prev) for v_prev, r, x_t in cases]
    assert out[R.PAIR_FILLED] == out[R.PAIR_NEVER] == out[R.PAIR_ALWAYS]
    if name in ("spec", "spec_probe", "bisect"):
        d = orc.sample_disturbances(seed, upd, N, H, inputs.DIST_AMP)
        for (v_prev, r, x_t), (_, k, f) in zip(cases, out[R.PAIR_ALWAYS]):
            k_o, f_o = orc.bisect_joint(params, orc.cfg(H=H, N=N), x_t, v_prev, r, 12, d, nthreads=NTH)
            assert (k, f) == (k_o, f_o), (v_prev, r)


@pytest.mark.parametrize("use_graph", [True, False])
def test_closed_loop_is_unchanged_by_pairing(R, orc, params, use_graph):
    """The closed loop (graph replays and direct launches) across a level
    change gives the same trajectory in every mode; setting the mode discards
    the cached graph."""
    N, H, T = 4096, 400, 6
    x0 = orc.equilibrium(params, 100.0)
    r_seq = np.array([250.0] * 3 + [120.0] * 3)
    runs = []
    with _gov(R, params, _cfg(R, N, H, max_candidates=16)) as g:
        for mode in (R.PAIR_NEVER, R.PAIR_ALWAYS, R.PAIR_NEVER, R.PAIR_FILLED):
            g.set_pairing(mode)
            runs.append(g.closed_loop(x0, 100.0, r_seq, 9, 0, inputs.DIST_AMP, use_graph=use_graph))
    for r in runs[1:]:
        for a, b in zip(r, runs[0]):
            np.testing.assert_array_equal(np.asarray(a), np.asarray(b))


def test_autotune_pairing_keeps_the_result(R, orc, params):
    N, H = 8192, 300
    x_t = orc.equilibrium(params, 100.0)
    with _gov(R, params, _cfg(R, N, H, max_candidates=16)) as g:
        g.sample_scenarios(1, 1)
        want = g.step(x_t, 250.0, 100.0)
        mode, ms = g.autotune_pairing(x_t, 250.0, 100.0, repeats=2)
        assert mode in (R.PAIR_NEVER, R.PAIR_FILLED, R.PAIR_ALWAYS)
        assert g.get_pairing() == mode
        assert len(ms) == 3 and all(t > 0.0 for t in ms)
        assert ms[mode] == min(ms)
        assert g.step(x_t, 250.0, 100.0) == want


def test_pairing_mode_is_validated(R, params):
    with _gov(R, params, _cfg(R, 64, 10)) as g:
        for bad in (-1, 3):
            with pytest.raises(R.RrgError):
                g.set_pairing(bad)
        assert g.get_pairing() == R.PAIR_FILLED


def test_paired_steps_are_counted(R, orc, params):
    """rrg_stats.lane_steps_paired: none without pairing, and with it a share
    of lane_steps (the steps a survivor runs alone are not paired)."""
    N, H = 4096, 300
    x_t = orc.equilibrium(params, 100.0)
    with _gov(R, params, _cfg(R, N, H, max_candidates=16, search=R.SEARCH_KSECTION, n_rounds=3)) as g:
        g.sample_scenarios(1, 1)
        for mode in (R.PAIR_NEVER, R.PAIR_ALWAYS):
            g.set_pairing(mode)
            g.reset_stats()
            g.step(x_t, 150.0, 100.0)
            st = g.stats()
            if mode == R.PAIR_NEVER:
                assert st["lane_steps_paired"] == 0
            else:
                assert 0 < st["lane_steps_paired"] <= st["lane_steps"]
