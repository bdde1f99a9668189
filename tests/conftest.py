import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_addoption(parser):
    parser.addoption("--pcr-debug-build", action="store_true", default=False,
                     help="run the tests against libpcr_debug.so (device bounds checks and counters) "
                          "instead of libpcr.so")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size cases (tens of seconds or more)")
    if config.getoption("--pcr-debug-build"):
        from paper_2104_07526_gb300 import build, pcr
        build.build()
        build.build(debug=True)
        pcr._lib = pcr.load_library(pcr.DEBUG_LIB_PATH)


def read_golden(name: str):
    """Non-comment, non-empty lines of a golden fixture, split on ';'."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([c.strip() for c in line.split(";")])
    return rows


@pytest.fixture(scope="session")
def oracle():
    from oracle import pyoracle
    pyoracle.lib()
    return pyoracle
