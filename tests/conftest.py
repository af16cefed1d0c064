import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: larger CPU cases")


@pytest.fixture(scope="session")
def small_geom():
    """4 pores x 32 nodes + 256-node wall |x/4|^8 + |y|^8 = 1 (384 nodes)."""
    import stokes_inputs as si
    return si.pipe10_geometry(0, n_outer=256, n_pores=4, n_per_pore=32)


@pytest.fixture(scope="session")
def pipe10_geom():
    import stokes_inputs as si
    return si.cached_geometry("pipe10", 0)
