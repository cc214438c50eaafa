import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a); run with -m gpu")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.load()
    return oracle


FULL_SIZE_MODULE = "test_gpu_full_size.py"


def pytest_collection_finish(session):
    # the full-size parity tests need minutes of single-threaded oracle work: start it in
    # spawned worker processes as soon as the run is known to include them
    if session.config.option.collectonly:
        return
    if any(item.nodeid.split("::")[0].endswith(FULL_SIZE_MODULE) for item in session.items):
        from tests import oracle_pool

        oracle_pool.start()


def pytest_sessionfinish(session, exitstatus):
    import sys as _sys

    mod = _sys.modules.get("tests.oracle_pool")
    if mod is not None:
        mod.stop()
