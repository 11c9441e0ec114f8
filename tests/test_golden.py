"""Regression fixtures in tests/golden (written by tests/golden/make_golden.py
from the FP64 oracle alone; the paper prints no worked example to store).

not gpu: the oracle still reproduces them.  gpu: the CUDA path, in the
benchmark's configurations, lands on the same kappas.
"""
import json
import os

import numpy as np
import pytest

from paper_2510_08288_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_oracle_reproduces_the_single_update_fixture(orc, params):
    g = _load("single_update.json")
    w = g["workload"]
    x_t = orc.equilibrium(params, w["v_prev"])
    np.testing.assert_allclose(x_t, g["x_t"], rtol=1e-13)
    d = orc.sample_disturbances(w["seed"], w["update"], w["N"], w["H"], inputs.DIST_AMP)
    k, f = orc.bisect_joint(params, orc.cfg(H=w["H"], N=w["N"]), x_t, w["v_prev"], w["r"], w["n_bisect"], d)
    assert (k, f) == (g["kappa"], g["flags"])
    # Alg. 3 on the dyadic grid of the same resolution lands on the same kappa
    assert (g["kappa_alg3_dyadic_grid"], g["flags_alg3"]) == (g["kappa"], g["flags"])
    assert g["v_t"] == w["v_prev"] + k * (w["r"] - w["v_prev"])


def test_oracle_reproduces_the_closed_loop_prefix(orc, params):
    """The first 3 of the fixture's 10 updates (the rest is checked on the GPU)."""
    g = _load("closed_loop_prefix.json")
    w = g["workload"]
    x0 = orc.equilibrium(params, w["v0"])
    v, k, f, xs = orc.closed_loop(params, orc.cfg(H=w["H"], N=w["N"]), x0, w["v0"], np.array(g["r"][:3]),
                                  w["seed"], w["t0"], inputs.DIST_AMP, inputs.DIST_AMP, search=0,
                                  n_kappa=w["n_bisect"], nthreads=os.cpu_count() or 1)
    np.testing.assert_array_equal(k, g["kappa"][:3])
    np.testing.assert_array_equal(f, g["flags"][:3])
    np.testing.assert_allclose(xs, np.array(g["x"][:4]), rtol=1e-13)


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_08288_gb300 import build as B
    B.build()
    from paper_2510_08288_gb300 import rrg
    return rrg


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32_recheck"])
def test_gpu_single_update_matches_the_fixture(R, params, prec):
    g = _load("single_update.json")
    w = g["workload"]
    cfg = R.rrg_config_default(horizon=w["H"], n_scenarios=w["N"], max_candidates=64, n_bisect=w["n_bisect"],
                               search=R.SEARCH_SPEC_BISECT, precision={"fp64": R.FP64, "fp32_recheck": R.FP32_RECHECK}[prec])
    with R.Governor(params, cfg) as gov:
        gov.sample_scenarios(w["seed"], w["update"])
        v_t, k, f = gov.step(np.array(g["x_t"]), w["r"], w["v_prev"])
    assert (k, f, v_t) == (g["kappa"], g["flags"], g["v_t"])


@pytest.mark.gpu
@pytest.mark.parametrize("use_graph", [False, True])
def test_gpu_closed_loop_matches_the_fixture(R, params, use_graph):
    """The benchmark's closed loop (FP32 rollouts + FP64 recheck, speculative
    bisection with the tuned shape) over the fixture's 10 updates."""
    g = _load("closed_loop_prefix.json")
    w = g["workload"]
    cfg = R.rrg_config_default(horizon=w["H"], n_scenarios=w["N"], max_candidates=64, n_bisect=w["n_bisect"],
                               search=R.SEARCH_SPEC_BISECT, precision=R.FP32_RECHECK,
                               early_exit=R.EXIT_CANDIDATE, recheck_eps_rel=1e-6)
    with R.Governor(params, cfg) as gov:
        gov.set_tuning(64, 32)
        x0 = np.array(g["x"][0])
        v, k, f, xs = gov.closed_loop(x0, w["v0"], np.array(g["r"]), w["seed"], w["t0"], inputs.DIST_AMP,
                                      use_graph=use_graph)
    np.testing.assert_array_equal(k, g["kappa"])
    np.testing.assert_array_equal(f, g["flags"])
    np.testing.assert_array_equal(v, g["v"])
    np.testing.assert_allclose(xs, np.array(g["x"]), rtol=1e-10)
