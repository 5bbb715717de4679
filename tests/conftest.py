import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library, built in-tree for sm_103a (GPU tests only)."""
    from paper_0910_0329_gb300 import build_lib, dpm

    build_lib.build()
    return dpm.lib()


@pytest.fixture(scope="session")
def tables_ctx(gpu_lib):
    """A context with tables for the three materials and the default parameters."""
    from paper_0910_0329_gb300 import dpm
    from paper_0910_0329_gb300 import workloads as W

    d = dpm.Dpm(0, W.MATERIALS, W.DEFAULT_PARAMS)
    yield d
    d.close()
