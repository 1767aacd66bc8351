import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def small_sphere_oracle():
    from oracle.oracle import OracleMesh
    from paper_2009_00706_gb300 import inputs as I
    w = I.small_sphere()
    m = OracleMesh(w.lo, w.hi, w.base_level, w.regions, w.triangles(), w.lmax)
    return w, m
