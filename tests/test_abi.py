"""The C-ABI library loads and exports every entry point include/bps.h declares
(no compute: runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "bps.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bps_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1306_1821_gb300 import bps
    from paper_1306_1821_gb300 import build as b
    if not os.path.exists(bps.LIB_PATH):
        b.build()
    return bps.load()


def test_header_declares_the_path():
    names = declared()
    for n in ["bps_create", "bps_set_data", "bps_set_state", "bps_get_state", "bps_hmc_step",
              "bps_sample_power", "bps_sample_bias_norm", "bps_jump", "bps_gibbs_iterate",
              "bps_last_error", "bps_destroy"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1306_1821_gb300 import bps
    for n in declared():
        assert hasattr(lib, n), n
        assert n in bps.declared_symbols(), f"binding lacks {n}"


def test_version_without_gpu(lib):
    assert lib.bps_version().decode().startswith("bps")
