import os
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libamr")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    return oracle.load()


@pytest.fixture(scope="session")
def tiny():
    from paper_1210_8014_gb300 import inputs
    tree, cams = inputs.tiny_workload()
    return tree, cams[0]


@pytest.fixture(scope="session")
def zoom_tree():
    """The 193M-leaf level-22 zoom tree, generated once per test session."""
    from paper_1210_8014_gb300 import inputs
    return inputs.zoom_tree()
