"""Batched instances (many independent RG problems in one persistent launch
per round) against the oracle, through the C ABI.

Instance s draws its scenarios with seed + s, so each instance's result must
equal the oracle's Alg. 3 or k-section on that instance's own draw; the
batch's binary32 rollouts with the binary64 recheck decide like binary64
whenever the band covers the binary32 error (same tolerances as the
single-problem tests: identical kappa, v_t and flags).
"""
import numpy as np
import pytest

from paper_2510_08288_gb300 import inputs

pytestmark = pytest.mark.gpu

BAND = 2e-4 / 1.9


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_08288_gb300 import build as B
    B.build()
    from paper_2510_08288_gb300 import rrg
    return rrg


def _problem(orc, params, S, seed, **kw):
    b = inputs.batched_instances(S, seed, **kw)
    x = np.array([orc.equilibrium(params, b["v_prev"][s]) * b["xfac"][s] for s in range(S)])
    return b, x


def _cfg(R, M, search, **kw):
    base = dict(max_candidates=M, n_rounds=3, search=search, precision=R.FP32_RECHECK,
                early_exit=R.EXIT_CANDIDATE, recheck_eps_rel=BAND)
    base.update(kw)
    return R.rrg_config_default(**base)


def _oracle(orc, params, kind, x, v_prev, r, d, N, H, M, rounds=3):
    c = orc.cfg(H=H, N=N)
    if kind == "grid":
        return orc.alg3(params, c, x, v_prev, r, M, d)
    return orc.ksection(params, c, x, v_prev, r, M, rounds, d)


@pytest.mark.parametrize("kind", ["ksection", "grid"])
@pytest.mark.parametrize("M", [2, 7, 32])
def test_batch_step_matches_oracle(R, orc, params, kind, M):
    S, seed, upd = 9, 7, 3
    b, x = _problem(orc, params, S, 5, N_lo=1, N_hi=300, H_lo=1, H_hi=250)
    search = R.SEARCH_KSECTION if kind == "ksection" else R.SEARCH_GRID
    with R.BatchGovernor(params, _cfg(R, M, search), b["N"], b["H"]) as g:
        v, k, f = g.step(x, b["r"], b["v_prev"], seed, upd)
    for s in range(S):
        N, H = int(b["N"][s]), int(b["H"][s])
        d = orc.sample_disturbances(seed + s, upd, N, H, inputs.DIST_AMP)
        ko, fo = _oracle(orc, params, kind, x[s], b["v_prev"][s], b["r"][s], d, N, H, M)
        assert (k[s], f[s]) == (ko, fo), s
        assert v[s] == orc.governed(b["v_prev"][s], b["r"][s], ko)


def test_batch_uneven_sizes_and_invalid_instance(R, orc, params):
    """Very uneven instances (1 .. 3,000 scenarios, horizons 1 .. 900), one
    with a non-finite state (holds with flag bit 1), one with r = v_prev."""
    N = np.array([1, 3000, 64, 129, 1, 700, 2], dtype=np.int32)
    H = np.array([900, 50, 1, 333, 2, 120, 600], dtype=np.int32)
    S = N.shape[0]
    v_prev = np.array([100.0, 150.0, 60.0, 220.0, 80.0, 120.0, 290.0])
    r = np.array([250.0, 160.0, 300.0, 100.0, 80.0, 200.0, 60.0])
    x = np.array([orc.equilibrium(params, v) for v in v_prev])
    x[2, 1] = np.nan
    with R.BatchGovernor(params, _cfg(R, 16, R.SEARCH_KSECTION), N, H) as g:
        v, k, f = g.step(x, r, v_prev, 11, 0)
    assert f[2] & 2 and k[2] == 0.0 and v[2] == v_prev[2]
    for s in range(S):
        if s == 2:
            continue
        d = orc.sample_disturbances(11 + s, 0, int(N[s]), int(H[s]), inputs.DIST_AMP)
        ko, fo = _oracle(orc, params, "ksection", x[s], v_prev[s], r[s], d, int(N[s]), int(H[s]), 16)
        assert (k[s], f[s]) == (ko, fo), s
    assert k[4] == 1.0


def test_all_rollout_variants_agree_and_autotune_picks_one(R, orc, params):
    S = 12
    b, x = _problem(orc, params, S, 9, N_lo=16, N_hi=2000, H_lo=50, H_hi=400)
    with R.BatchGovernor(params, _cfg(R, 16, R.SEARCH_KSECTION), b["N"], b["H"]) as g:
        outs = []
        for var in range(R.BATCH_VARIANTS):
            g.set_variant(var)
            assert g.get_variant()[0] == var
            outs.append(g.step(x, b["r"], b["v_prev"], 3, 1))
        best, ms = g.autotune(x, b["r"], b["v_prev"], 3, 1, repeats=1)
        assert 0 <= best < R.BATCH_VARIANTS and g.get_variant()[0] == best
        assert np.all(ms > 0) and ms[best] == ms.min()
        after = g.step(x, b["r"], b["v_prev"], 3, 1)
    for o in outs[1:] + [after]:
        for a, c in zip(outs[0], o):
            np.testing.assert_array_equal(a, c)


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_closed_loop_matches_oracle(R, orc, params, use_graph):
    """T closed-loop updates of every instance (plants included) equal the
    oracle's closed loop of each instance with seed + s; a continued loop
    (two calls) equals one call."""
    S, T, M, seed, t0 = 5, 4, 8, 21, 2
    b, x0 = _problem(orc, params, S, 13, N_lo=4, N_hi=200, H_lo=20, H_hi=160)
    r_seq = np.stack([inputs.staircase(T, 2, 2, seed=40 + s) for s in range(S)], axis=1)
    amp = inputs.DIST_AMP
    with R.BatchGovernor(params, _cfg(R, M, R.SEARCH_KSECTION), b["N"], b["H"]) as g:
        v, k, f, xs = g.closed_loop(x0, b["v_prev"], r_seq, seed, t0, amp, use_graph=use_graph)
    for s in range(S):
        c = orc.cfg(H=int(b["H"][s]), N=int(b["N"][s]))
        vo, ko, fo, xo = orc.closed_loop(params, c, x0[s], b["v_prev"][s], r_seq[:, s], seed + s, t0, amp, amp,
                                         search=2, M=M, rounds=3)
        np.testing.assert_array_equal(k[:, s], ko)
        np.testing.assert_array_equal(f[:, s], fo)
        np.testing.assert_array_equal(v[:, s], vo)
        np.testing.assert_allclose(xs[:, s], xo, rtol=1e-10)


def test_batch_closed_loop_continues(R, orc, params):
    import torch
    S, T, M, seed = 4, 4, 8, 5
    b, x0 = _problem(orc, params, S, 17, N_lo=4, N_hi=100, H_lo=20, H_hi=100)
    r_seq = np.stack([inputs.staircase(T, 2, 2, seed=60 + s) for s in range(S)], axis=1)
    amp = inputs.DIST_AMP
    cfg = _cfg(R, M, R.SEARCH_KSECTION)
    with R.BatchGovernor(params, cfg, b["N"], b["H"]) as g:
        one = g.closed_loop(x0, b["v_prev"], r_seq, seed, 0, amp)
    with R.BatchGovernor(params, cfg, b["N"], b["H"]) as g:
        dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
        dr = dev(r_seq.reshape(-1))
        ov = torch.zeros(T * S, dtype=torch.float64, device="cuda")
        ok = torch.zeros_like(ov)
        of = torch.zeros(T * S, dtype=torch.int32, device="cuda")
        ox = torch.zeros((T + 1) * S * 3, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        R.rrg_batch_closed_loop_dev(g.h, dev(x0.reshape(-1)), dev(b["v_prev"]), dr, 2, seed, 0, amp, True,
                                    ov, ok, of, ox)
        # an unrelated update in between (its draw may overwrite the pair
        # holding the loop's next update)
        g.step(x0, b["r"], b["v_prev"], 77, 3)
        R.rrg_batch_closed_loop_dev(g.h, None, None, dr, 2, seed, 0, amp, True, ov, ok, of, ox)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ok.cpu().numpy().reshape(T, S), one[1])
        np.testing.assert_array_equal(ox.cpu().numpy().reshape(T + 1, S, 3), one[3])


def test_batch_stats_count_steps(R, orc, params):
    S = 3
    b, x = _problem(orc, params, S, 23, N_lo=10, N_hi=50, H_lo=10, H_hi=40)
    with R.BatchGovernor(params, _cfg(R, 4, R.SEARCH_GRID, early_exit=R.EXIT_NONE), b["N"], b["H"]) as g:
        g.set_profiling(True)
        g.step(x, b["r"], b["v_prev"], 1, 0)
        st = g.stats()
    # no early exit: every candidate that passes the steady-state check runs N H steps
    assert st["lane_steps"] - st["lane_steps_fp64"] <= int(np.sum(4 * b["N"] * b["H"]))
    assert st["rollout_launches"] == 1 and st["timed_rollouts"] == 1 and st["rollout_ms"] > 0


def test_batch_recheck_runs_only_to_the_last_uncertain_step(R, orc, params):
    """As the single-problem test: disturbance-free instances whose hold
    candidate sits 1e-7 above y_min at j = 0 only; the grid's kappa = 0 is
    admissible, every lane of it is rechecked, and no binary64 step runs."""
    S, N, H = 3, 200, 300
    x = np.array([orc.equilibrium(params, 100.0) * np.array([1.0, 1.0, 0.999])] * S)
    y_min = orc.output(params, x[0], 100.0) - 1e-7
    cfg = _cfg(R, 4, R.SEARCH_GRID, y_min=y_min, ss_check=0, dist_amp=(0.0, 0.0, 0.0),
               recheck_eps_rel=1e-6, early_exit=R.EXIT_LANE)
    with R.BatchGovernor(params, cfg, [N] * S, [H] * S) as g:
        v, k, f = g.step(x, np.full(S, 150.0), np.full(S, 100.0), 0, 0)
        st = g.stats()
    for s in range(S):
        ko, fo = orc.alg3(params, orc.cfg(H=H, N=N, y_min=y_min, ss_check=0), x[s], 100.0, 150.0, 4,
                          np.zeros((3, H, N)))
        assert (k[s], f[s]) == (ko, fo) == (0.0, 0)
    assert st["rechecked"] == S * N and st["lane_steps_fp64"] == 0


def test_full_size_batch_update_matches_single_problems_and_oracle(R, orc, params):
    """The batched workload at full size (256 instances, N_s up to 8,192,
    H_s up to 4,000, k-section with 32 candidates x 3 rounds, seed 2, in the
    variant the autotuner picks): every instance's kappa equals the
    single-problem search on the same draw (seed + s), and the oracle's on
    the cheapest instances."""
    S, seed, upd, M = 256, 2, 0, 32
    b, x = _problem(orc, params, S, seed)
    cfg = _cfg(R, M, R.SEARCH_KSECTION, recheck_eps_rel=1e-6)
    with R.BatchGovernor(params, cfg, b["N"], b["H"]) as g:
        g.autotune(x, b["r"], b["v_prev"], seed, upd, repeats=1)
        v, k, f = g.step(x, b["r"], b["v_prev"], seed, upd)
    for s in range(S):
        N, H = int(b["N"][s]), int(b["H"][s])
        c1 = R.rrg_config_default(horizon=H, n_scenarios=N, max_candidates=M, n_rounds=3,
                                  search=R.SEARCH_KSECTION, precision=R.FP32_RECHECK,
                                  early_exit=R.EXIT_CANDIDATE, recheck_eps_rel=1e-6)
        with R.Governor(params, c1) as g1:
            g1.sample_scenarios(seed + s, upd)
            assert g1.step(x[s], b["r"][s], b["v_prev"][s]) == (v[s], k[s], f[s]), s
    cheapest = sorted(range(S), key=lambda s: int(b["N"][s]) * int(b["H"][s]))[:6]
    for s in cheapest:
        N, H = int(b["N"][s]), int(b["H"][s])
        d = orc.sample_disturbances(seed + s, upd, N, H, inputs.DIST_AMP)
        ko, fo = _oracle(orc, params, "ksection", x[s], b["v_prev"][s], b["r"][s], d, N, H, M)
        assert (k[s], f[s]) == (ko, fo), s


# ----------------------------------------------- speculative bisection ----
@pytest.mark.parametrize("width", [1, 2, 3, 8, 31, 64])
def test_batch_spec_bisect_is_alg1_for_every_width(R, orc, params, width):
    """RRG_SEARCH_SPEC_BISECT batches: every instance's kappa and flags equal
    the oracle's joint bisection (Alg. 1, N_kappa = 12) on the instance's own
    draw, whatever the tree width, with the binary32 + recheck rollouts at
    the benchmark's band."""
    S, seed, upd = 9, 7, 3
    b, x = _problem(orc, params, S, 5, N_lo=1, N_hi=300, H_lo=1, H_hi=250)
    cfg = _cfg(R, 64, R.SEARCH_SPEC_BISECT, n_bisect=12, recheck_eps_rel=1e-6)
    with R.BatchGovernor(params, cfg, b["N"], b["H"]) as g:
        g.set_width(width)
        assert g.get_width() == width
        v, k, f = g.step(x, b["r"], b["v_prev"], seed, upd)
        st = g.stats()
    for s in range(S):
        N, H = int(b["N"][s]), int(b["H"][s])
        d = orc.sample_disturbances(seed + s, upd, N, H, inputs.DIST_AMP)
        k_o, f_o = orc.bisect_joint(params, orc.cfg(H=H, N=N), x[s], b["v_prev"][s], b["r"][s], 12, d)
        assert (k[s], f[s]) == (k_o, f_o), s
        assert v[s] == b["v_prev"][s] + k_o * (b["r"][s] - b["v_prev"][s])
    # rounds: enough trees of this width for 12 iterations from kappa = 1
    d0 = max(dd for dd in range(1, 13) if 2 ** (dd - 1) <= width)
    d1 = max(dd for dd in range(1, 13) if 2 ** dd - 1 <= width)
    assert st["rounds"] == 1 + -(-(12 - min(d0, 12)) // d1)


def test_batch_width_autotune_keeps_every_result(R, orc, params):
    """The width autotuner times whole updates for each tree size and keeps
    the fastest; every instance's kappa is the same at every width."""
    S = 6
    b, x = _problem(orc, params, S, 9, N_lo=64, N_hi=512, H_lo=100, H_hi=400)
    cfg = _cfg(R, 32, R.SEARCH_SPEC_BISECT, n_bisect=12, recheck_eps_rel=1e-6)
    with R.BatchGovernor(params, cfg, b["N"], b["H"]) as g:
        _, k_ref, f_ref = g.step(x, b["r"], b["v_prev"], 4, 0)
        w, ws, ms = g.autotune_width(x, b["r"], b["v_prev"], 4, 0, repeats=1)
        assert w in ws and np.all(ms > 0) and list(ws) == sorted(ws) and ws[0] == 1 and ws[-1] == 32
        assert g.get_width() == w
        for width in (1, 7, 32):
            g.set_width(width)
            _, k, f = g.step(x, b["r"], b["v_prev"], 4, 0)
            np.testing.assert_array_equal(k, k_ref)
            np.testing.assert_array_equal(f, f_ref)
    with R.BatchGovernor(params, _cfg(R, 8, R.SEARCH_KSECTION), b["N"], b["H"]) as g:
        with pytest.raises(R.RrgError):
            g.set_width(4)


PAIR_VARIANT = 8   # warp tiles of two candidates per thread


@pytest.mark.parametrize("width", [1, 3, 7])
@pytest.mark.parametrize("kind", ["spec", "ksection"])
def test_batch_pair_tiles_match_single_tiles_and_oracle(R, orc, params, width, kind):
    """The paired warp-tile variant (candidate slots 2p and 2p + 1 in one
    thread; an odd round leaves the last pair with one) gives every
    instance's kappa and flags of the single warp tiles and of the oracle,
    for the speculative bisection at odd tree widths and for the k-section
    (odd grid 7)."""
    S, seed, upd = 9, 7, 3
    b, x = _problem(orc, params, S, 5, N_lo=1, N_hi=300, H_lo=1, H_hi=250)
    if kind == "spec":
        cfg = _cfg(R, 64, R.SEARCH_SPEC_BISECT, n_bisect=12, recheck_eps_rel=1e-6)
    else:
        cfg = _cfg(R, 7, R.SEARCH_KSECTION, recheck_eps_rel=1e-6)
    with R.BatchGovernor(params, cfg, b["N"], b["H"]) as g:
        if kind == "spec":
            g.set_width(width)
        out = {}
        for var in (7, PAIR_VARIANT):
            g.set_variant(var)
            out[var] = g.step(x, b["r"], b["v_prev"], seed, upd)
    for a, c in zip(out[7], out[PAIR_VARIANT]):
        np.testing.assert_array_equal(a, c)
    v, k, f = out[PAIR_VARIANT]
    for s in range(S):
        N, H = int(b["N"][s]), int(b["H"][s])
        d = orc.sample_disturbances(seed + s, upd, N, H, inputs.DIST_AMP)
        if kind == "spec":
            k_o, f_o = orc.bisect_joint(params, orc.cfg(H=H, N=N), x[s], b["v_prev"][s], b["r"][s], 12, d)
        else:
            k_o, f_o = _oracle(orc, params, "ksection", x[s], b["v_prev"][s], b["r"][s], d, N, H, 7)
        assert (k[s], f[s]) == (k_o, f_o), s


SPLIT_VARIANT = 9  # warp tiles of 16 scenarios, two lanes per trajectory


@pytest.mark.parametrize("early", ["none", "lane", "candidate"])
@pytest.mark.parametrize("kind", ["spec", "ksection"])
def test_batch_split_tiles_match_single_tiles_and_oracle(R, orc, params, early, kind):
    """Two lanes per trajectory (role 0 the linear flow derivatives, role 1
    the compressor speed's, swapped by shuffles): every instance's v_t, kappa
    and flags equal the one-lane warp tiles' and the oracle's, for scenario
    counts that leave a ragged 16-scenario tile and horizons shorter than the
    prefetch block; without early exit both count the same lane-steps."""
    S, seed, upd = 9, 7, 3
    b, x = _problem(orc, params, S, 5, N_lo=1, N_hi=300, H_lo=1, H_hi=250)
    ex = {"none": R.EXIT_NONE, "lane": R.EXIT_LANE, "candidate": R.EXIT_CANDIDATE}[early]
    if kind == "spec":
        cfg = _cfg(R, 64, R.SEARCH_SPEC_BISECT, n_bisect=12, recheck_eps_rel=1e-6, early_exit=ex)
    else:
        cfg = _cfg(R, 7, R.SEARCH_KSECTION, recheck_eps_rel=1e-6, early_exit=ex)
    out, steps = {}, {}
    with R.BatchGovernor(params, cfg, b["N"], b["H"]) as g:
        if kind == "spec":
            g.set_width(7)
        for var in (7, SPLIT_VARIANT):
            g.set_variant(var)
            assert g.get_variant()[0] == var
            g.reset_stats()
            out[var] = g.step(x, b["r"], b["v_prev"], seed, upd)
            st = g.stats()
            steps[var] = st["lane_steps"] - st["lane_steps_fp64"]
        assert g.get_variant()[1] == 16
    for a, c in zip(out[7], out[SPLIT_VARIANT]):
        np.testing.assert_array_equal(a, c)
    if early == "none":
        assert steps[7] == steps[SPLIT_VARIANT] > 0
    v, k, f = out[SPLIT_VARIANT]
    for s in range(S):
        N, H = int(b["N"][s]), int(b["H"][s])
        d = orc.sample_disturbances(seed + s, upd, N, H, inputs.DIST_AMP)
        if kind == "spec":
            k_o, f_o = orc.bisect_joint(params, orc.cfg(H=H, N=N), x[s], b["v_prev"][s], b["r"][s], 12, d)
        else:
            k_o, f_o = _oracle(orc, params, "ksection", x[s], b["v_prev"][s], b["r"][s], d, N, H, 7)
        assert (k[s], f[s]) == (k_o, f_o), s
