import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU and the compiled CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session", autouse=True)
def _input_cache(tmp_path_factory):
    # keep generated meshes inside the test session unless a cache is set
    if not os.environ.get("DEC_INPUT_CACHE"):
        os.environ["DEC_INPUT_CACHE"] = str(
            tmp_path_factory.mktemp("dec_inputs"))
    yield
