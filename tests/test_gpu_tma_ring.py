"""The binary32 ring through the Tensor Memory Accelerator (rrg_set_tma).

RRG_TMA_ALWAYS forces the TMA for every ring launch and RRG_TMA_NEVER the
per-lane copies, so each test runs both paths on the same launches.

Launches that leave most warp slots empty bring the stored disturbances into
a shared-memory ring.  With the TMA, one tensor copy per warp fills a
32-scenario x 16-step x 3-component box (zeros past the array); without it,
each lane issues its own 4-byte copies.  The arithmetic is the same, so the
two give identical flags, P entries and min slacks (every min slack without
an early exit, the admissible candidates' with one), and the oracle's
decisions.  Scenario counts that are not a multiple of the 32-lane box leave
a ragged last warp; horizons that are not a multiple of 16 end in a partial
chunk; probes that are not a multiple of 16 start the continuation mid-chunk.
"""
import os

import numpy as np
import pytest

from paper_2510_08288_gb300 import inputs

pytestmark = pytest.mark.gpu
NTH = max(1, min(16, os.cpu_count() or 1))
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
    c = dict(horizon=H, n_scenarios=N, max_candidates=16, n_bisect=12, search=R.SEARCH_SPEC_BISECT,
             precision=R.FP32_RECHECK, early_exit=R.EXIT_CANDIDATE, recheck_eps_rel=1e-6,
             param_unc_mask=MASK, probe_steps=0)
    c.update(kw)
    return R.rrg_config_default(**c)


def _same(a, b):
    a, b = np.asarray(a), np.asarray(b)
    np.testing.assert_array_equal(np.isnan(a), np.isnan(b))
    np.testing.assert_array_equal(a[~np.isnan(a)], b[~np.isnan(b)])


@pytest.mark.parametrize("N,H", [(1000, 203), (4096, 2000), (36, 65), (300, 16), (1028, 33)])
@pytest.mark.parametrize("prec", ["fp32", "fp32_recheck"])
@pytest.mark.parametrize("unc", [0.0, 0.1])
@pytest.mark.parametrize("early", [0, 1, 2])
def test_tma_ring_equals_async_ring(R, orc, params, N, H, prec, unc, early):
    p = R.FP32 if prec == "fp32" else R.FP32_RECHECK
    kappas = np.linspace(0.0, 1.0, 13)
    x_t = orc.equilibrium(params, 100.0) * np.array([1.0, 1.03, 1.0])
    res = {}
    with R.Governor(params, _cfg(R, N, H, precision=p, early_exit=early, param_unc_rel=unc)) as g:
        assert g.get_tma() == R.TMA_AUTO
        g.sample_scenarios(5, 2)
        for mode in (R.TMA_ALWAYS, R.TMA_NEVER):
            g.set_tma(mode)
            assert g.get_tma() == mode
            g.reset_stats()
            res[mode] = g.eval_candidates(x_t, 100.0, 250.0, kappas, want_P=True)
            assert g.stats()["wait_timeouts"] == 0
    (a1, m1, P1), (a0, m0, P0) = res[R.TMA_ALWAYS], res[R.TMA_NEVER]
    np.testing.assert_array_equal(a1, a0)
    np.testing.assert_array_equal(P1, P0)
    if early == 0:
        _same(m1, m0)
    else:
        _same(m1[a0 == 1], m0[a0 == 1])


@pytest.mark.parametrize("unc", [0.0, 0.1])
def test_tma_ring_decides_like_the_oracle(R, orc, params, unc):
    """At the benchmark's band, candidates around the boundary (many near-zero
    lanes, rechecked in binary64): the oracle's P and flags; the oracle draws
    its own disturbances and multipliers."""
    N, H, seed, upd = 1000, 203, 3, 4
    kappas = np.linspace(0.0, 0.06, 25) if unc else np.linspace(0.09, 0.115, 26)
    x_t = orc.equilibrium(params, 100.0)
    with R.Governor(params, _cfg(R, N, H, max_candidates=32, early_exit=R.EXIT_LANE, param_unc_rel=unc)) as g:
        g.set_tma(R.TMA_ALWAYS)
        g.sample_scenarios(seed, upd)
        adm, _, P = g.eval_candidates(x_t, 100.0, 250.0, kappas, want_P=True)
        assert g.stats()["wait_timeouts"] == 0
    d = orc.sample_disturbances(seed, upd, N, H, inputs.DIST_AMP)
    mult = orc.sample_param_multipliers(seed, upd, N, unc, MASK) if unc else None
    with orc.param_multipliers(mult):
        a_o, _, P_o, _ = orc.eval_candidates(params, orc.cfg(H=H, N=N, early_exit=0), x_t, 100.0, 250.0,
                                             kappas, d, want_P=True, nthreads=NTH)
    np.testing.assert_array_equal(adm, a_o)
    np.testing.assert_array_equal(P, P_o)
    assert 0 < int(a_o.sum()) < len(kappas)


@pytest.mark.parametrize("probe", [1, 20, 128])
def test_tma_ring_in_pipelined_searches(R, orc, params, probe):
    """Probe and continuation launches (the continuation starts at the probe's
    step, mid-chunk unless the probe is a multiple of 16): the same result
    with and without the TMA, and the oracle's joint bisection."""
    N, H, seed, upd = 1024, 500, 3, 7
    cases = [(100.0, 250.0, orc.equilibrium(params, 100.0)),
             (180.0, 90.0, orc.equilibrium(params, 180.0) * np.array([1.02, 0.99, 1.01]))]
    out = {}
    with R.Governor(params, _cfg(R, N, H, max_candidates=64, probe_steps=probe)) as g:
        g.sample_scenarios(seed, upd)
        for mode in (R.TMA_ALWAYS, R.TMA_NEVER, R.TMA_AUTO):
            g.set_tma(mode)
            g.reset_stats()
            out[mode] = [g.step(x_t, r, v_prev) for v_prev, r, x_t in cases]
            assert g.stats()["wait_timeouts"] == 0
    assert out[R.TMA_ALWAYS] == out[R.TMA_NEVER] == out[R.TMA_AUTO]
    d = orc.sample_disturbances(seed, upd, N, H, inputs.DIST_AMP)
    for (v_prev, r, x_t), (_, k, f) in zip(cases, out[R.TMA_ALWAYS]):
        assert (k, f) == orc.bisect_joint(params, orc.cfg(H=H, N=N), x_t, v_prev, r, 12, d, nthreads=NTH)


@pytest.mark.parametrize("use_graph", [True, False])
def test_tma_ring_closed_loop(R, orc, params, use_graph):
    """The closed loop alternates two scenario pairs (two tensor maps, the
    second made when the loop first runs): the same trajectory with and
    without the TMA, across a level change."""
    N, H = 1024, 300
    x0 = orc.equilibrium(params, 100.0)
    r_seq = np.array([250.0] * 3 + [120.0] * 3)
    runs = []
    with R.Governor(params, _cfg(R, N, H, max_candidates=64, probe_steps=32)) as g:
        for mode in (R.TMA_ALWAYS, R.TMA_NEVER, R.TMA_AUTO):
            g.set_tma(mode)
            g.reset_stats()
            runs.append(g.closed_loop(x0, 100.0, r_seq, 9, 0, inputs.DIST_AMP, use_graph=use_graph))
            assert g.stats()["wait_timeouts"] == 0
    for r in runs[1:]:
        for a, b in zip(r, runs[0]):
            np.testing.assert_array_equal(np.asarray(a), np.asarray(b))


def test_tma_availability(R, params):
    """No TMA ring where the tensor map cannot describe the array: a row
    stride that is not a multiple of 16 bytes, or no stored binary32 array."""
    with R.Governor(params, _cfg(R, 37, 20)) as g:
        assert g.get_tma() == R.TMA_NEVER
        for mode in (R.TMA_AUTO, R.TMA_ALWAYS):
            with pytest.raises(R.RrgError):
                g.set_tma(mode)
        g.set_tma(R.TMA_NEVER)
    with R.Governor(params, _cfg(R, 64, 20, precision=R.FP32, early_exit=R.EXIT_LANE,
                                 scenarios_in_register=1)) as g:
        assert g.get_tma() == R.TMA_NEVER
    with R.Governor(params, _cfg(R, 64, 20)) as g:
        assert g.get_tma() == R.TMA_AUTO
        for bad in (-1, 3):
            with pytest.raises(R.RrgError):
                g.set_tma(bad)


def test_tma_wait_timeout_is_reported_and_the_handle_recovers(R, orc, params):
    """Bounded waits (RRG_INJECT_TMA_NO_COPY: the ring issues no copies, so
    nothing ever arrives): every warp's wait runs out within its limit, the
    launch returns, rrg_stats.wait_timeouts counts the warps, and every lane
    that was running reports a violation, so no candidate is admissible and P
    is all zero.  With the switch off the same handle gives its normal
    results again."""
    N, H = 1000, 100
    kappas = np.linspace(0.0, 0.2, 7)
    x_t = orc.equilibrium(params, 100.0)
    with R.Governor(params, _cfg(R, N, H, early_exit=R.EXIT_LANE)) as g:
        g.set_tma(R.TMA_ALWAYS)
        g.sample_scenarios(1, 1)
        a0, m0, P0 = g.eval_candidates(x_t, 100.0, 250.0, kappas, want_P=True)
        assert a0.any()
        g.set_injection(R.INJECT_TMA_NO_COPY)
        g.reset_stats()
        a1, _, P1 = g.eval_candidates(x_t, 100.0, 250.0, kappas, want_P=True)
        st = g.stats()
        assert st["wait_timeouts"] > 0
        assert not a1.any() and not P1.any()
        g.set_injection(0)
        g.reset_stats()
        a2, m2, P2 = g.eval_candidates(x_t, 100.0, 250.0, kappas, want_P=True)
        assert g.stats()["wait_timeouts"] == 0
        with pytest.raises(R.RrgError):
            g.set_injection(2)
    np.testing.assert_array_equal(a2, a0)
    np.testing.assert_array_equal(P2, P0)
    _same(m2, m0)


def test_tma_auto_takes_large_launches_only(R, orc, params):
    """RRG_TMA_AUTO: launches of at least 24 warps per SM (8,192 scenarios x
    16 candidates: 27 per SM) take the TMA ring, ahead of pairing; small ones
    (1,024 x 16: 3.4 per SM) keep the per-lane copies; results equal."""
    x_t = orc.equilibrium(params, 100.0)
    kappas = np.linspace(0.0, 1.0, 16)
    res = {}
    for N, want_tma in ((8192, True), (1024, False)):
        with R.Governor(params, _cfg(R, N, 200, early_exit=R.EXIT_NONE, precision=R.FP32)) as g:
            g.sample_scenarios(2, 2)
            for mode in (R.TMA_AUTO, R.TMA_NEVER):
                g.set_tma(mode)
                g.reset_stats()
                res[(N, mode)] = g.eval_candidates(x_t, 100.0, 250.0, kappas)
                st = g.stats()
                used = st["lane_steps_tma"] > 0
                assert used == (want_tma and mode == R.TMA_AUTO), (N, mode)
                if used:
                    assert st["lane_steps_tma"] == st["lane_steps"]
                    assert st["lane_steps_paired"] == 0
            a0, m0, _ = res[(N, R.TMA_AUTO)]
            a1, m1, _ = res[(N, R.TMA_NEVER)]
            np.testing.assert_array_equal(a0, a1)
            _same(m0, m1)


# ------------------------------------------- two candidates per thread --
@pytest.mark.parametrize("N,H", [(1000, 203), (4096, 600), (36, 65)])
@pytest.mark.parametrize("prec", ["fp32", "fp32_recheck"])
@pytest.mark.parametrize("unc", [0.0, 0.1])
@pytest.mark.parametrize("early", [0, 1, 2])
def test_tma_pairs_equal_single_lanes(R, orc, params, N, H, prec, unc, early):
    """Two candidates per thread on the TMA ring (RRG_TMA_ALWAYS with
    RRG_PAIR_ALWAYS) against one per thread on the per-lane ring: identical
    flags, P and min slacks (every one without an early exit, the admissible
    candidates' with one); 13 rows leave the last pair with one candidate."""
    p = R.FP32 if prec == "fp32" else R.FP32_RECHECK
    kappas = np.linspace(0.0, 1.0, 13)
    x_t = orc.equilibrium(params, 100.0) * np.array([1.0, 1.03, 1.0])
    with R.Governor(params, _cfg(R, N, H, precision=p, early_exit=early, param_unc_rel=unc)) as g:
        g.sample_scenarios(5, 2)
        g.set_tma(R.TMA_NEVER)
        g.set_pairing(R.PAIR_NEVER)
        a0, m0, P0 = g.eval_candidates(x_t, 100.0, 250.0, kappas, want_P=True)
        g.set_tma(R.TMA_ALWAYS)
        g.set_pairing(R.PAIR_ALWAYS)
        g.reset_stats()
        a1, m1, P1 = g.eval_candidates(x_t, 100.0, 250.0, kappas, want_P=True)
        st = g.stats()
    assert st["wait_timeouts"] == 0
    assert st["lane_steps_paired"] > 0
    assert st["lane_steps_tma"] == st["lane_steps"] - st["lane_steps_fp64"]
    np.testing.assert_array_equal(a1, a0)
    np.testing.assert_array_equal(P1, P0)
    if early == 0:
        _same(m1, m0)
    else:
        _same(m1[a0 == 1], m0[a0 == 1])


@pytest.mark.parametrize("unc", [0.0, 0.1])
def test_tma_pairs_decide_like_the_oracle(R, orc, params, unc):
    N, H, seed, upd = 1000, 203, 3, 4
    kappas = np.linspace(0.0, 0.06, 25) if unc else np.linspace(0.09, 0.115, 26)
    x_t = orc.equilibrium(params, 100.0)
    with R.Governor(params, _cfg(R, N, H, max_candidates=32, early_exit=R.EXIT_LANE, param_unc_rel=unc)) as g:
        g.set_tma(R.TMA_ALWAYS)
        g.set_pairing(R.PAIR_ALWAYS)
        g.sample_scenarios(seed, upd)
        adm, _, P = g.eval_candidates(x_t, 100.0, 250.0, kappas, want_P=True)
        assert g.stats()["lane_steps_paired"] > 0
    d = orc.sample_disturbances(seed, upd, N, H, inputs.DIST_AMP)
    mult = orc.sample_param_multipliers(seed, upd, N, unc, MASK) if unc else None
    with orc.param_multipliers(mult):
        a_o, _, P_o, _ = orc.eval_candidates(params, orc.cfg(H=H, N=N, early_exit=0), x_t, 100.0, 250.0,
                                             kappas, d, want_P=True, nthreads=NTH)
    np.testing.assert_array_equal(adm, a_o)
    np.testing.assert_array_equal(P, P_o)


@pytest.mark.parametrize("probe", [0, 20])
def test_tma_pairs_in_searches_and_closed_loop(R, orc, params, probe):
    """Searches (pipelined rounds keep single lanes, the rounds after them
    pair) and the closed loop give the same results with pairs on the TMA
    ring as with single lanes on the per-lane ring, and the oracle's joint
    bisection."""
    N, H, seed, upd = 1024, 500, 3, 7
    cases = [(100.0, 250.0, orc.equilibrium(params, 100.0)),
             (180.0, 90.0, orc.equilibrium(params, 180.0) * np.array([1.02, 0.99, 1.01]))]
    r_seq = np.array([250.0] * 2 + [120.0] * 2)
    out, loops = {}, {}
    with R.Governor(params, _cfg(R, N, H, max_candidates=64, probe_steps=probe)) as g:
        for tma, pair in ((R.TMA_ALWAYS, R.PAIR_ALWAYS), (R.TMA_NEVER, R.PAIR_NEVER)):
            g.set_tma(tma)
            g.set_pairing(pair)
            g.sample_scenarios(seed, upd)
            out[tma] = [g.step(x_t, r, v_prev) for v_prev, r, x_t in cases]
            loops[tma] = g.closed_loop(orc.equilibrium(params, 100.0), 100.0, r_seq, 9, 0, inputs.DIST_AMP)
            assert g.stats()["wait_timeouts"] == 0
    assert out[R.TMA_ALWAYS] == out[R.TMA_NEVER]
    for a, c in zip(loops[R.TMA_ALWAYS], loops[R.TMA_NEVER]):
        np.testing.assert_array_equal(np.asarray(a), np.asarray(c))
    d = orc.sample_disturbances(seed, upd, N, H, inputs.DIST_AMP)
    for (v_prev, r, x_t), (_, k, f) in zip(cases, out[R.TMA_ALWAYS]):
        assert (k, f) == orc.bisect_joint(params, orc.cfg(H=H, N=N), x_t, v_prev, r, 12, d, nthreads=NTH)


def test_tma_pairs_wait_timeout(R, orc, params):
    """The injected timeout with pairs: counted, nothing admissible, and the
    handle recovers."""
    N, H = 1000, 100
    kappas = np.linspace(0.0, 0.2, 7)
    x_t = orc.equilibrium(params, 100.0)
    with R.Governor(params, _cfg(R, N, H, early_exit=R.EXIT_LANE)) as g:
        g.set_tma(R.TMA_ALWAYS)
        g.set_pairing(R.PAIR_ALWAYS)
        g.sample_scenarios(1, 1)
        a0, _, P0 = g.eval_candidates(x_t, 100.0, 250.0, kappas, want_P=True)
        g.set_injection(R.INJECT_TMA_NO_COPY)
        g.reset_stats()
        a1, _, P1 = g.eval_candidates(x_t, 100.0, 250.0, kappas, want_P=True)
        assert g.stats()["wait_timeouts"] > 0 and not a1.any() and not P1.any()
        g.set_injection(0)
        a2, _, P2 = g.eval_candidates(x_t, 100.0, 250.0, kappas, want_P=True)
    np.testing.assert_array_equal(a2, a0)
    np.testing.assert_array_equal(P2, P0)
