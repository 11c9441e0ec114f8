"""Alg. 1 rounds for evaluations the caller runs (rrg_bisect_init / plan /
decide): host logic of the library, no GPU.

The evaluations come from the FP64 oracle (orc.eval_candidates on the whole
scenario set, or the AND over contiguous shards of it), so the loop's kappa
must equal the oracle's own joint bisection (orc.bisect_joint) for every
round width; on arbitrary predicates, monotone or not, it must equal Alg. 1
run node by node.
"""
import numpy as np
import pytest

from paper_2510_08288_gb300 import inputs


@pytest.fixture(scope="module")
def R():
    from paper_2510_08288_gb300 import build as B
    B.build()
    from paper_2510_08288_gb300 import rrg
    return rrg


def _run(R, n_bisect, m_max, evaluate):
    s = R.rrg_bisect_init(n_bisect)
    rounds, evals = 0, 0
    while not s.done:
        kap = R.rrg_bisect_plan(s, m_max)
        assert 1 <= kap.size <= m_max
        R.rrg_bisect_decide(s, evaluate(kap))
        rounds += 1
        evals += kap.size
    assert R.rrg_bisect_plan(s, m_max).size == 0
    return s.kappa_opt, (0 if s.any else 1), rounds, evals


def _alg1(n_bisect, pred):
    """Alg. 1 node by node on a predicate (kappa = 1 first; an admissible
    kappa = 1 ends it)."""
    lo, hi, k, kopt, any_ = 0.0, 1.0, 1.0, 0.0, False
    for _ in range(n_bisect):
        if pred(k):
            kopt, any_ = k, True
            if k == 1.0:
                break
            lo = k
        else:
            hi = k
        k = (lo + hi) / 2.0
    return kopt, (0 if any_ else 1)


@pytest.mark.parametrize("case", [(100.0, 250.0), (150.0, 290.0), (220.0, 300.0), (80.0, 60.0)])
@pytest.mark.parametrize("m_max", [1, 2, 3, 7, 16, 64])
def test_rounds_give_the_oracles_joint_bisection(R, orc, params, case, m_max):
    v_prev, r = case
    N, H, nb = 16, 150, 12
    x_t = orc.equilibrium(params, v_prev)
    d = orc.sample_disturbances(4, 1, N, H, inputs.DIST_AMP)
    c = orc.cfg(H=H, N=N)
    ev = lambda kap: orc.eval_candidates(params, c, x_t, v_prev, r, kap, d)[0]
    k, f, rounds, _ = _run(R, nb, m_max, ev)
    k_o, f_o = orc.bisect_joint(params, c, x_t, v_prev, r, nb, d)
    assert (k, f) == (k_o, f_o)
    if m_max >= 7 and k_o not in (0.0, 1.0):
        assert rounds < nb


@pytest.mark.parametrize("m_max", [1, 8, 64])
def test_two_scenario_shards_combined_by_and(R, orc, params, m_max):
    """Shards [0, 9) and [9, 20) of one draw, each evaluated on its own, the
    flags combined by AND: the unsharded joint bisection's kappa."""
    N, H, nb = 20, 200, 14
    v_prev, r = 100.0, 250.0
    x_t = orc.equilibrium(params, v_prev)
    d = orc.sample_disturbances(6, 3, N, H, inputs.DIST_AMP)
    shards = [np.ascontiguousarray(d[:, :, :9]), np.ascontiguousarray(d[:, :, 9:])]

    def ev(kap):
        a = [orc.eval_candidates(params, orc.cfg(H=H, N=sd.shape[2]), x_t, v_prev, r, kap, sd)[0]
             for sd in shards]
        return np.minimum(a[0], a[1])
    k, f, _, _ = _run(R, nb, m_max, ev)
    assert (k, f) == orc.bisect_joint(params, orc.cfg(H=H, N=N), x_t, v_prev, r, nb, d)


@pytest.mark.parametrize("seed", range(40))
def test_any_predicate_gives_alg1(R, seed):
    """Random predicates, monotone or not, and random round widths: the
    rounds' walk is Alg. 1's path through the same outcomes."""
    rng = np.random.default_rng(seed)
    nb = int(rng.integers(1, 16))
    table = {}

    def pred(k):
        if k not in table:
            table[k] = bool(rng.random() < 0.5) if seed % 2 else bool(k <= 0.37 + 0.01 * seed)
        return table[k]
    m_max = int(rng.integers(1, 40))
    k, f, _, evals = _run(R, nb, m_max, lambda kap: np.array([pred(x) for x in kap], dtype=np.uint8))
    assert (k, f) == _alg1(nb, pred)


def test_round_sizes_and_errors(R):
    s = R.rrg_bisect_init(12)
    # a kappa = 1 root: its admissible branch ends the search, so 2^(d-1) nodes
    assert R.rrg_bisect_plan(s, 64).size == 64
    assert R.rrg_bisect_plan(s, 63).size == 32
    kap = R.rrg_bisect_plan(s, 4)
    np.testing.assert_array_equal(kap, [1.0, 0.5, 0.25, 0.75])
    with pytest.raises(R.RrgError):
        R.rrg_bisect_decide(s, np.ones(3, dtype=np.uint8))        # not a round size
    R.rrg_bisect_decide(s, np.array([0, 1, 0, 0], dtype=np.uint8))
    assert (s.iter, s.lo, s.hi, s.kappa, s.kappa_opt) == (3, 0.5, 0.75, 0.625, 0.5)
    # off the root: 2^d - 1 nodes, limited by the iterations left
    assert R.rrg_bisect_plan(s, 64).size == 63
    assert R.rrg_bisect_plan(s, 6).size == 3
    s.iter = 10
    assert R.rrg_bisect_plan(s, 64).size == 3
    for bad in (0, 63):
        with pytest.raises(R.RrgError):
            R.rrg_bisect_init(bad)
    done = R.rrg_bisect_init(1)
    R.rrg_bisect_decide(done, np.array([1], dtype=np.uint8))
    assert done.done and done.kappa_opt == 1.0
    with pytest.raises(R.RrgError):
        R.rrg_bisect_decide(done, np.array([1], dtype=np.uint8))
