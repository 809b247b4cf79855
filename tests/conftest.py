"""Shared pytest configuration: the ``gpu`` marker, the import path and the brute-force ray fan of
the 64 x 64 heterogeneous TTI pin (shared by the oracle tests that compare with it)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line('markers', 'gpu: needs a CUDA GPU (GB300, sm_103a) and the built library')
    config.addinivalue_line('markers', 'slow: longer CPU test (still part of the CPU suite)')


@pytest.fixture(scope='session')
def tti64_shooter():
    """The Lagrangian ray shooter's arrivals on the 64 x 64 x 64 TTI medium (2048 rays)."""
    import synthmedia
    from oracle import shooter as SH
    p = synthmedia.tti_heterogeneous(n=64, n_theta=64, length=2560.0, steps=400, freqs=(10.0,))
    fan = SH.shoot(p, n_rays=2048)
    cnt, first, arr = SH.arrivals(p, fan)
    return p, fan, cnt, first, arr
