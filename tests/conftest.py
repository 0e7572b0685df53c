import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session", autouse=True)
def _built_host_libs():
    """The oracle and the fixture mesher are plain C; compile them if needed."""
    import oracle
    from paper_2605_26137_b300 import build as pkg_build
    oracle.build()
    pkg_build.build_synth()
    yield
