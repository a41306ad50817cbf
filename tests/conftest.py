import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
for p in (ROOT, os.path.join(ROOT, "tests")):
    if p not in sys.path:
        sys.path.insert(0, p)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def spinodal64():
    """64^3 Cahn-Hilliard mask, 1000 steps, porosity 0.70, mask seed 0."""
    from paper_2604_13929_gb300 import inputs
    return inputs.spinodal_mask(64, 0.70, 1000, seed=0, device="cpu")


@pytest.fixture(scope="session")
def spinodal32_90():
    """32^3 Cahn-Hilliard mask, 400 steps, porosity 0.90 (small, for the oracle)."""
    from paper_2604_13929_gb300 import inputs
    return inputs.spinodal_mask(32, 0.90, 400, seed=1, device="cpu")
