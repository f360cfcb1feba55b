import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than ~30 s on CPU")


@pytest.fixture(scope="session")
def libncs():
    """The built CUDA library (built in-tree on first use)."""
    from paper_1906_04209_gb300 import build, ncs
    if not os.path.exists(ncs.LIB_PATH):
        build.build()
    return ncs.load()


_PRE = {}


@pytest.fixture(scope="session")
def small_pre():
    """Small oracle precomputes, keyed by mode: eps = 0.1, K = 10 (M = 3)."""
    from oracle import operator as O

    def get(mode, K=10, eps=0.1, npan=6, nord=10, ntheta=24, tau=1e-11):
        key = (mode, K, eps, npan, nord, ntheta, tau)
        if key not in _PRE:
            _PRE[key] = O.make_precompute(eps, mode, K, npan=npan, nord=nord, ntheta=ntheta, tau=tau)
        return _PRE[key]
    return get
