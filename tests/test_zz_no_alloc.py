"""rrg_eval_candidates_static: the allocation-free candidate evaluation.

Some callers cannot allocate device memory while they run, for example a
fixed-rate control task or a host program that owns all device memory through
its own pool, so they cannot create a handle.  This entry point serves them
from one fixed device array inside the library.  These tests call it through
the C ABI on caller-owned device buffers and check that two calls in a row
give the same decisions and slacks as rrg_eval_candidates on a handle, and
that sizes beyond the array's limits are refused with a clear error.

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test; it also passes on its own.
"""
import numpy as np
import pytest

from paper_2510_08288_gb300 import inputs

pytestmark = pytest.mark.gpu

SLACK_RTOL = 1e-9     # the binary64 tolerance of the parity tests


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_08288_gb300 import build as B
    B.build()
    from paper_2510_08288_gb300 import rrg as R
    return torch, R


@pytest.mark.parametrize("precision", ["fp64", "fp32_recheck"])
def test_static_matches_handle_on_two_calls(env, precision):
    torch, R = env
    p = inputs.fc3_params()
    N, H = 96, 300
    prec = R.FP64 if precision == "fp64" else R.FP32_RECHECK
    cfg = R.rrg_config_default(horizon=H, n_scenarios=N, max_candidates=16, precision=prec,
                               early_exit=R.EXIT_CANDIDATE, recheck_eps_rel=1e-4)
    dev = torch.device("cuda")
    with R.Governor(p, cfg) as g:
        g.sample_scenarios(3, 0)
        d = g.get_scenarios()
        x100, _ = g.equilibrium(100.0)
        x150, _ = g.equilibrium(150.0)
        calls = [(x100, 100.0, 250.0, np.linspace(0.05, 0.15, 11)),
                 (x150, 150.0, 60.0, np.array([0.0, 0.5, 1.0]))]
        d64 = torch.tensor(d, dtype=torch.float64, device=dev)
        d32 = d64.float()
        torch.cuda.synchronize()
        for x, vp, r, kap in calls:
            want_adm, want_ms, _ = g.eval_candidates(x, vp, r, kap)
            m = len(kap)
            dx = torch.tensor(x, dtype=torch.float64, device=dev)
            dk = torch.tensor(kap, dtype=torch.float64, device=dev)
            dadm = torch.full((m,), 7, dtype=torch.uint8, device=dev)
            dms = torch.full((m,), -1.0, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            R.rrg_eval_candidates_static(p, cfg, None, d64, d32, dx, vp, r, dk, m, dadm, dms)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(dadm.cpu().numpy(), want_adm)
            np.testing.assert_allclose(dms.cpu().numpy(), want_ms, rtol=SLACK_RTOL, atol=1e-12)


def test_static_rejects_sizes_beyond_its_scratch(env):
    torch, R = env
    p = inputs.fc3_params()
    dev = torch.device("cuda")
    cfg = R.rrg_config_default(horizon=10, n_scenarios=4096, max_candidates=128, precision=R.FP64)
    d64 = torch.zeros(3 * 10 * 4096, dtype=torch.float64, device=dev)
    dx = torch.tensor([1.1e5, 3e3, 1.2e5], dtype=torch.float64, device=dev)
    dk = torch.zeros(128, dtype=torch.float64, device=dev)
    dadm = torch.zeros(128, dtype=torch.uint8, device=dev)
    with pytest.raises(R.RrgError) as e:          # more candidates than the scratch holds
        R.rrg_eval_candidates_static(p, cfg, None, d64, None, dx, 100.0, 200.0, dk, 65, dadm)
    assert e.value.code == R.RRG_EINVAL and "1..64" in str(e.value)
    with pytest.raises(R.RrgError) as e:          # 64 x 4096 trajectories > 131072
        R.rrg_eval_candidates_static(p, cfg, None, d64, None, dx, 100.0, 200.0, dk, 64, dadm)
    assert e.value.code == R.RRG_EINVAL and "scratch limit" in str(e.value)
