"""The C ABI library loads and exports every entry point include/rrg.h declares
(no compute calls: these tests run without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rrg.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rrg_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_08288_gb300 import build as B
    return ctypes.CDLL(B.build())


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("rrg_create", "rrg_sample_scenarios", "rrg_eval_candidates", "rrg_step", "rrg_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2510_08288_gb300 import rrg as R
    for n in _declared():
        assert hasattr(R, n), n


def _c_layout(struct, fields, tmp_path):
    """sizeof and offsetof of a struct of include/rrg.h, as the C compiler
    lays it out (gcc, the host ABI the binding runs on)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    inc = os.path.join(ROOT, "include")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rrg.h"', 'int main(void) {',
             '  printf("%%zu\\n", sizeof(%s));' % struct]
    lines += ['  printf("%%zu\\n", offsetof(%s, %s));' % (struct, f) for f in fields]
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return int(out[0]), [int(x) for x in out[1:]]


@pytest.mark.parametrize("name", ["RrgConfig", "RrgStats"])
def test_struct_layout_matches_c_compiler(name, tmp_path):
    """The ctypes mirrors have the C compiler's size and field offsets."""
    from paper_2510_08288_gb300 import rrg as R
    cls = getattr(R, name)
    struct = {"RrgConfig": "rrg_config", "RrgStats": "rrg_stats"}[name]
    fields = [f[0] for f in cls._fields_]
    size, offs = _c_layout(struct, fields, tmp_path)
    assert ctypes.sizeof(cls) == size
    assert [getattr(cls, f).offset for f in fields] == offs


def test_config_defaults_and_create_validation_without_gpu():
    """Defaults are the paper's fuel-cell values; an invalid configuration is
    rejected before any device work, so this runs on a CPU-only host."""
    from paper_2510_08288_gb300 import inputs
    from paper_2510_08288_gb300 import rrg as R
    c = R.rrg_config_default()
    assert c.dt == 0.01 and c.y_min == 1.9 and list(c.dist_amp) == [50.0, 10.0, 50.0]
    bad = R.rrg_config_default(horizon=0)
    with pytest.raises(R.RrgError) as e:
        R.rrg_create(inputs.fc3_params(), bad)
    assert e.value.code == R.RRG_EINVAL and "horizon" in str(e.value)
    with pytest.raises(R.RrgError):
        R.rrg_create(inputs.fc3_params()[:5], c)
    with pytest.raises(R.RrgError):
        R.rrg_create(inputs.fc3_params(), R.rrg_config_default(search=R.SEARCH_GRID, max_candidates=1))
    # parametric uncertainty: rho in [0, 1), mask within the parameter vector
    assert c.param_unc_rel == 0.0 and c.param_unc_mask == inputs.FC3_UNCERTAIN_MASK
    for kw in (dict(param_unc_rel=1.0), dict(param_unc_rel=-0.1), dict(param_unc_rel=float("nan")),
               dict(param_unc_rel=0.1, param_unc_mask=1 << 27)):
        with pytest.raises(R.RrgError) as e:
            R.rrg_create(inputs.fc3_params(), R.rrg_config_default(**kw))
        assert e.value.code == R.RRG_EINVAL and "param_unc" in str(e.value)


def test_static_entry_rejects_parametric_uncertainty_without_gpu():
    """The allocation-free entry point has no multiplier storage: it refuses
    param_unc_rel != 0 before touching the device."""
    from paper_2510_08288_gb300 import inputs
    from paper_2510_08288_gb300 import rrg as R
    p = np.ascontiguousarray(inputs.fc3_params())
    cfg = R.rrg_config_default(param_unc_rel=0.1)
    rc = R.lib.rrg_eval_candidates_static(p.ctypes.data_as(ctypes.c_void_p), 27, ctypes.byref(cfg), None,
                                          None, None, None, 100.0, 200.0, None, 1, None, None)
    assert rc == R.RRG_ENOTIMPL and "parametric" in R.rrg_last_error(None)


def test_oracle_and_library_share_no_code():
    """The CUDA sources never include oracle files and the oracle never
    includes the library's headers."""
    csrc = os.path.join(ROOT, "paper_2510_08288_gb300", "csrc")
    for f in os.listdir(csrc):
        assert "oracle" not in open(os.path.join(csrc, f)).read().lower()
    osrc = open(os.path.join(ROOT, "oracle", "rrg_oracle.c")).read()
    assert "#include \"" not in osrc and "rrg.h" not in osrc
    for f in ("rrg.py", "build.py", "inputs.py"):
        assert "import oracle" not in open(os.path.join(ROOT, "paper_2510_08288_gb300", f)).read()
        assert "from oracle" not in open(os.path.join(ROOT, "paper_2510_08288_gb300", f)).read()


def test_batch_create_validation_without_gpu():
    """The batched entry point rejects bad shapes and unsupported options
    before any device work."""
    from paper_2510_08288_gb300 import inputs
    from paper_2510_08288_gb300 import rrg as R
    p = inputs.fc3_params()
    ok = R.rrg_config_default(search=R.SEARCH_KSECTION, precision=R.FP32_RECHECK)
    cases = [
        (ok, [10, 0], [5, 5], R.RRG_EINVAL),
        (ok, [10], [0], R.RRG_EINVAL),
        (ok, [], [], R.RRG_EINVAL),
        (ok, [1] * 1025, [1] * 1025, R.RRG_EINVAL),
        (R.rrg_config_default(search=R.SEARCH_BISECT, precision=R.FP32_RECHECK), [4], [4], R.RRG_ENOTIMPL),
        (R.rrg_config_default(search=R.SEARCH_GRID, precision=R.FP64), [4], [4], R.RRG_ENOTIMPL),
        (R.rrg_config_default(search=R.SEARCH_GRID, precision=R.FP32_RECHECK, param_unc_rel=0.1), [4], [4],
         R.RRG_ENOTIMPL),
        (R.rrg_config_default(search=R.SEARCH_GRID, precision=R.FP32_RECHECK, max_candidates=1024), [2 ** 21], [4],
         R.RRG_EINVAL),
    ]
    for cfg, ns, hz, code in cases:
        with pytest.raises(R.RrgError) as e:
            R.rrg_batch_create(p, cfg, ns, hz)
        assert e.value.code == code, (ns, hz, str(e.value))


def test_step_latency_rejects_a_null_handle():
    """The latency probe validates its arguments before touching a device."""
    from paper_2510_08288_gb300 import rrg as R
    c = ctypes.c_double(0.0)
    assert R.lib.rrg_step_latency(None, 100.0, 10, ctypes.byref(c)) == R.RRG_EINVAL


def test_handle_entry_points_reject_a_null_handle():
    """Every handle entry point returns RRG_EINVAL for a null handle before it
    touches a device (the adjoint, the Newton search, profiling, statistics)."""
    from paper_2510_08288_gb300 import rrg as R
    x = (ctypes.c_double * 3)(1.0, 2.0, 3.0)
    g = ctypes.c_double(0.0)
    grad = (ctypes.c_double * 31)()
    k, j = ctypes.c_int64(0), ctypes.c_int64(0)
    assert R.lib.rrg_slack_gradient(None, x, 100.0, 250.0, 0.1, 50, R.FP32, ctypes.byref(g), grad,
                                    ctypes.byref(k), ctypes.byref(j)) == R.RRG_EINVAL
    kap = ctypes.c_double(0.0)
    fl, it = ctypes.c_int32(0), ctypes.c_int32(0)
    assert R.lib.rrg_newton_search(None, x, 250.0, 100.0, 1e-6, 10, 50, R.FP32, ctypes.byref(kap),
                                   ctypes.byref(fl), ctypes.byref(it)) == R.RRG_EINVAL
    assert R.lib.rrg_set_profiling(None, 1) == R.RRG_EINVAL
    st = R.RrgStats()
    assert R.lib.rrg_get_stats(None, ctypes.byref(st)) == R.RRG_EINVAL
