import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session", autouse=True)
def _blas_threads():
    # numpy and scipy each bundle an OpenBLAS; two full-size thread pools
    # thrash on the small matrices of the oracle.
    try:
        from threadpoolctl import threadpool_limits
        with threadpool_limits(limits=min(4, os.cpu_count() or 1)):
            yield
    except ImportError:
        yield
