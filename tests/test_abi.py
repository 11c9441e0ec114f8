"""The C ABI library loads and exports every entry point include/rrg.h declares
(no compute calls: these tests run without a GPU)."""
import ctypes
import os
import re

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


def test_config_struct_layout_matches_header():
    """The ctypes mirror has the size of the C struct (checked via offsets)."""
    from paper_2510_08288_gb300 import rrg as R
    assert ctypes.sizeof(R.RrgConfig) == 8 + 9 * 4 + 4 + 4 * 8 + 3 * 8 + 8
    assert R.RrgConfig.y_min.offset == 48


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
