import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def obs_small():
    from paper_2507_22128_gb300 import synth
    return synth.plain_small(seed=0)


@pytest.fixture(scope="session")
def obs_wstack():
    """Reduced medium recipe: 256x256 at 1", 16 w-planes, 24 antennas x 40
    times x 2 channels (w-stacked parity case)."""
    from paper_2507_22128_gb300 import synth
    return synth.medium(seed=11, n_times=40, n=256, n_wplanes=16, n_ant=24, n_chan=2)


@pytest.fixture(scope="session")
def obs_large():
    """Reduced large recipe: 256x256 at 0.5", 32 w-planes, 128 antennas on a
    10 km spiral x 6 times x 1 channel (P = 4 parity case)."""
    from paper_2507_22128_gb300 import synth
    return synth.large(seed=3, n_times=6, n=256, n_chan=1)
