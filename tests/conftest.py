import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    # launch-variant cache of the autotuner: keep tests independent of any cache a
    # benchmark run may have written for this user
    import tempfile
    os.environ.setdefault("SPH_AUTOTUNE_CACHE",
                          os.path.join(tempfile.mkdtemp(prefix="sph_tune_"), "autotune.json"))
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")
