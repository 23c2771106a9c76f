import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def grid():
    import oracle
    from paper_2212_10733_gb300 import synth
    vpar, vperp, vol = synth.grid_arrays()
    return oracle.Grid(vpar=vpar, vperp=vperp, vol_uniform=vol)
