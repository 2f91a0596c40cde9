import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: large sizes; still part of the default run")


@pytest.fixture(scope="session")
def sr():
    """The product library (CUDA path through the C-ABI). Fails loudly if the
    extension is missing: there is no fallback."""
    import paper_2004_05371_gb300 as sr_mod
    sr_mod.load()
    return sr_mod
