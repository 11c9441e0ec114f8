"""Scenario sharding through the C ABI on one GPU.

Handles whose rrg_config.scenario_base are 0, n_1, n_1 + n_2, ... hold
consecutive shards of one scenario set: their draws are the unsharded
handle's columns (disturbances and parameter multipliers), and the
speculative bisection run by rounds around an AND of their admissible flags
(shard.sharded_search with rrg_bisect_plan / rrg_bisect_decide) gives the
unsharded handle's device-resident search and the oracle's joint bisection
over all scenarios (the oracle draws its own disturbances).  On one GPU the
shards are evaluated one after the other; across GPUs the AND is the
all-reduce of shard.allreduce_candidates.
"""
import os

import numpy as np
import pytest

from paper_2510_08288_gb300 import inputs
from paper_2510_08288_gb300 import shard

pytestmark = pytest.mark.gpu
NTH = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_08288_gb300 import build as B
    B.build()
    from paper_2510_08288_gb300 import rrg
    return rrg


def _cfg(R, N, H, base=0, **kw):
    c = dict(horizon=H, n_scenarios=N, max_candidates=64, n_bisect=12, search=R.SEARCH_SPEC_BISECT,
             precision=R.FP32_RECHECK, early_exit=R.EXIT_CANDIDATE, recheck_eps_rel=1e-6,
             scenario_base=base, probe_steps=0)
    c.update(kw)
    return R.rrg_config_default(**c)


def _shards(sizes):
    bases = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    return list(zip(sizes, bases))


@pytest.mark.parametrize("precision", ["fp32_recheck", "fp64"])
@pytest.mark.parametrize("sizes", [(1024, 1024), (700, 1348), (512, 512, 1024)])
def test_sharded_search_equals_unsharded_and_oracle(R, orc, params, precision, sizes):
    N, H, seed, upd = int(sum(sizes)), 600, 3, 7
    prec = R.FP32_RECHECK if precision == "fp32_recheck" else R.FP64
    cases = [(100.0, 250.0, orc.equilibrium(params, 100.0)),
             (180.0, 90.0, orc.equilibrium(params, 180.0) * np.array([1.02, 0.99, 1.01])),
             (60.0, 280.0, orc.equilibrium(params, 60.0))]
    hs = [R.Governor(params, _cfg(R, n, H, int(b), precision=prec)) for n, b in _shards(sizes)]
    try:
        with R.Governor(params, _cfg(R, N, H, precision=prec)) as g:
            g.sample_scenarios(seed, upd)
            for h in hs:
                h.sample_scenarios(seed, upd)
            d = orc.sample_disturbances(seed, upd, N, H, inputs.DIST_AMP)
            for v_prev, r, x_t in cases:
                _, k_u, f_u = g.step(x_t, r, v_prev)

                def evaluate(kap):
                    res = [h.eval_candidates(x_t, v_prev, r, kap) for h in hs]
                    a = np.min(np.stack([q[0] for q in res]), axis=0)
                    s = np.min(np.stack([q[1] for q in res]), axis=0)
                    return a, s
                k_s, f_s, rounds = shard.sharded_search(evaluate, 12, 64, combine=lambda a, s: (a, s))
                k_o, f_o = orc.bisect_joint(params, orc.cfg(H=H, N=N), x_t, v_prev, r, 12, d, nthreads=NTH)
                assert (k_s, f_s) == (k_u, f_u) == (k_o, f_o), (v_prev, r)
                assert rounds <= 3
    finally:
        for h in hs:
            h.close()


def test_shard_draws_are_the_unsharded_columns(R, params):
    """Disturbances (binary64 values regenerated from the binary32 draw) and
    parametric multipliers of a shard equal the unsharded handle's columns."""
    N, H, seed, upd = 96, 40, 11, 4
    kw = dict(param_unc_rel=0.1, param_unc_mask=inputs.FC3_UNCERTAIN_MASK)
    with R.Governor(params, _cfg(R, N, H, **kw)) as g:
        g.sample_scenarios(seed, upd)
        d_all, m_all = g.get_scenarios(), g.get_param_multipliers()
    for n, b in _shards((30, 66)):
        with R.Governor(params, _cfg(R, n, H, int(b), **kw)) as h:
            h.sample_scenarios(seed, upd)
            np.testing.assert_array_equal(h.get_scenarios(), d_all[:, :, b:b + n])
            np.testing.assert_array_equal(h.get_param_multipliers(), m_all[b:b + n])


def test_shard_with_in_register_scenarios(R, orc, params):
    """Disturbances drawn inside the trajectory loop use the global index too:
    the shard's P rows equal the unsharded handle's columns."""
    N, H, seed, upd = 256, 300, 5, 2
    kap = np.linspace(0.05, 0.15, 8)
    x_t = orc.equilibrium(params, 100.0)
    kw = dict(precision=R.FP32, early_exit=R.EXIT_LANE, scenarios_in_register=1)
    with R.Governor(params, _cfg(R, N, H, **kw)) as g:
        g.sample_scenarios(seed, upd)
        _, _, P = g.eval_candidates(x_t, 100.0, 250.0, kap, want_P=True)
    with R.Governor(params, _cfg(R, 156, H, 100, **kw)) as h:
        h.sample_scenarios(seed, upd)
        _, _, Ph = h.eval_candidates(x_t, 100.0, 250.0, kap, want_P=True)
    np.testing.assert_array_equal(Ph, P[:, 100:])


def test_scenario_base_is_validated(R, params):
    for bad in (-1, 2**62 + 1):
        with pytest.raises(R.RrgError):
            R.Governor(params, _cfg(R, 8, 10, bad))
    with pytest.raises(R.RrgError):
        R.BatchGovernor(params, _cfg(R, 8, 10, 5, search=R.SEARCH_KSECTION), np.array([8], dtype=np.int32),
                        np.array([10], dtype=np.int32))
