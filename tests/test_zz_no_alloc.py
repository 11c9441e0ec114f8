"""rrg_eval_candidates_static: the allocation-free candidate evaluation.

Some callers cannot allocate device memory while they run, for example a
fixed-rate control task or a host program that owns all device memory through
its own pool, so they cannot create a handle.  This entry point serves them
from one fixed device array inside the library.  These tests call it through
the C ABI on caller-owned device buffers and check, on two calls in a row,
that it gives the same decisions and slacks as rrg_eval_candidates on a handle
and as the FP64 oracle on the same scenarios; that it works on a side stream,
without the optional outputs and at exactly its stated limits; and that sizes
beyond those limits are refused with a clear error.

The scenarios come from the oracle's own sampler; the handle and the static
call both receive them as explicit arrays (the binary32 copy is the
round-to-nearest of each binary64 value on both).

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test; it also passes on its own.
"""
import numpy as np
import pytest

from paper_2510_08288_gb300 import inputs

pytestmark = pytest.mark.gpu

SLACK_RTOL = 1e-9     # the binary64 tolerance of the parity tests
SLACK32_TOL = 2e-4    # binary32 slack band of the parity tests (OER units)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_08288_gb300 import build as B
    B.build()
    from paper_2510_08288_gb300 import rrg as R
    return torch, R


def _static(torch, R, p, cfg, stream, d, x, vp, r, kap, want_ms=True, with64=True):
    """One static call on fresh device buffers; returns (adm, min_slack or None)."""
    dev = torch.device("cuda")
    m = len(kap)
    d64 = torch.tensor(d, dtype=torch.float64, device=dev)
    d32 = d64.float()
    dx = torch.tensor(x, dtype=torch.float64, device=dev)
    dk = torch.tensor(kap, dtype=torch.float64, device=dev)
    dadm = torch.full((m,), 7, dtype=torch.uint8, device=dev)
    dms = torch.full((m,), -1.0, dtype=torch.float64, device=dev) if want_ms else None
    torch.cuda.synchronize()
    R.rrg_eval_candidates_static(p, cfg, stream, d64 if with64 else None, d32, dx, vp, r, dk, m, dadm, dms)
    if stream is not None:
        stream.synchronize()
    torch.cuda.synchronize()
    return dadm.cpu().numpy(), (dms.cpu().numpy() if want_ms else None)


def _oracle(orc, p, N, H, x, vp, r, kap, d, **kw):
    c = orc.cfg(H=H, N=N, early_exit=0, **kw)
    a, ms, _, _ = orc.eval_candidates(p, c, x, vp, r, kap, d)
    return a, ms


@pytest.mark.parametrize("precision", ["fp64", "fp32_recheck", "fp32"])
def test_static_matches_handle_and_oracle_on_two_calls(env, orc, precision):
    torch, R = env
    p = inputs.fc3_params()
    N, H = 96, 300
    prec = {"fp64": R.FP64, "fp32_recheck": R.FP32_RECHECK, "fp32": R.FP32}[precision]
    cfg = R.rrg_config_default(horizon=H, n_scenarios=N, max_candidates=16, precision=prec,
                               early_exit=R.EXIT_CANDIDATE, recheck_eps_rel=SLACK32_TOL / 1.9)
    d = orc.sample_disturbances(3, 0, N, H, inputs.DIST_AMP)
    x100, x150 = orc.equilibrium(p, 100.0), orc.equilibrium(p, 150.0)
    calls = [(x100, 100.0, 250.0, np.linspace(0.05, 0.15, 11)),
             (x150, 150.0, 60.0, np.array([0.0, 0.5, 1.0]))]
    with R.Governor(p, cfg) as g:
        g.set_scenarios(d)
        for x, vp, r, kap in calls:
            want_adm, want_ms, _ = g.eval_candidates(x, vp, r, kap)
            adm, ms = _static(torch, R, p, cfg, None, d, x, vp, r, kap, with64=precision != "fp32")
            # the same kernels on the same scenarios as the handle (the min
            # slack of an inadmissible candidate depends on when its early
            # exits land, so only the admissible ones are compared)
            np.testing.assert_array_equal(adm, want_adm)
            sel = want_adm == 1
            np.testing.assert_allclose(ms[sel], want_ms[sel], rtol=SLACK_RTOL, atol=1e-12)
            # and the FP64 oracle on its own draw of the scenarios
            a_o, ms_o = _oracle(orc, p, N, H, x, vp, r, kap, d)
            ok = a_o == 1
            if precision == "fp32":
                # plain binary32: decisions differ only inside the slack band
                differ = adm != a_o
                assert np.all(np.abs(ms_o[differ]) < SLACK32_TOL)
                np.testing.assert_allclose(ms[ok], ms_o[ok], rtol=0, atol=SLACK32_TOL)
            else:
                np.testing.assert_array_equal(adm, a_o)
                if precision == "fp64":
                    np.testing.assert_allclose(ms[ok], ms_o[ok], rtol=SLACK_RTOL, atol=1e-12)
                else:
                    np.testing.assert_allclose(ms[ok], ms_o[ok], rtol=0, atol=SLACK32_TOL)


def test_static_on_a_side_stream_without_min_slack(env, orc):
    """A non-default stream and d_min_slack = NULL: the flags equal the
    handle's and the oracle's, on two calls in a row."""
    torch, R = env
    p = inputs.fc3_params()
    N, H = 64, 200
    cfg = R.rrg_config_default(horizon=H, n_scenarios=N, max_candidates=8, precision=R.FP32_RECHECK,
                               early_exit=R.EXIT_LANE, recheck_eps_rel=SLACK32_TOL / 1.9)
    d = orc.sample_disturbances(8, 2, N, H, inputs.DIST_AMP)
    x = orc.equilibrium(p, 120.0)
    s = torch.cuda.Stream()
    with R.Governor(p, cfg) as g:
        g.set_scenarios(d)
        for kap in (np.linspace(0.0, 0.2, 8), np.array([0.03, 0.9])):
            want, _, _ = g.eval_candidates(x, 120.0, 280.0, kap)
            adm, _ = _static(torch, R, p, cfg, s, d, x, 120.0, 280.0, kap, want_ms=False)
            np.testing.assert_array_equal(adm, want)
            a_o, _ = _oracle(orc, p, N, H, x, 120.0, 280.0, kap, d)
            np.testing.assert_array_equal(adm, a_o)


def test_static_at_its_limits(env, orc):
    """Exactly at the limits (m = 64 candidates, m * N = 131,072
    trajectories), with a recheck band so wide that nearly every trajectory
    lands on the recheck list and fills that part of the scratch: the same
    flags and slacks as the handle, on a side stream, twice in a row."""
    torch, R = env
    p = inputs.fc3_params()
    N, H, m = 2048, 40, 64
    assert m * N == 131072
    cfg = R.rrg_config_default(horizon=H, n_scenarios=N, max_candidates=m, precision=R.FP32_RECHECK,
                               early_exit=R.EXIT_NONE, recheck_eps_rel=0.5)
    d = orc.sample_disturbances(11, 4, N, H, inputs.DIST_AMP)
    x = orc.equilibrium(p, 100.0)
    kap = np.linspace(0.0, 0.12, m)
    s = torch.cuda.Stream()
    with R.Governor(p, cfg) as g:
        g.set_scenarios(d)
        want_adm, want_ms, _ = g.eval_candidates(x, 100.0, 250.0, kap)
        st = g.stats()
        assert st["rechecked"] > N * m // 2      # the wide band lists most trajectories
        sel = want_adm == 1
        for _ in range(2):
            adm, ms = _static(torch, R, p, cfg, s, d, x, 100.0, 250.0, kap)
            np.testing.assert_array_equal(adm, want_adm)
            np.testing.assert_allclose(ms[sel], want_ms[sel], rtol=SLACK_RTOL, atol=1e-12)
    assert 0 < int(want_adm.sum()) < m
    # sampled candidates against the oracle (every trajectory of each)
    for i in (0, m // 2, m - 1):
        a_o, ms_o = _oracle(orc, p, N, H, x, 100.0, 250.0, kap[i:i + 1], d)
        assert adm[i] == a_o[0]
        if a_o[0]:
            assert ms[i] == pytest.approx(ms_o[0], rel=SLACK_RTOL, abs=1e-12)


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
    with pytest.raises(R.RrgError) as e:          # binary32 rollouts need the binary32 copy
        cfg32 = R.rrg_config_default(horizon=10, n_scenarios=64, max_candidates=8, precision=R.FP32)
        R.rrg_eval_candidates_static(p, cfg32, None, d64, None, dx, 100.0, 200.0, dk, 8, dadm)
    assert e.value.code == R.RRG_EINVAL
