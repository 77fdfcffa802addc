import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libinolf.so")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session", autouse=True)
def _host_builds():
    """Compile the host-only pieces the CPU tests need (g++/gcc, seconds)."""
    import oracle
    from paper_2303_04086_gb300 import synth
    synth.build()
    oracle.build()


@pytest.fixture(scope="session", autouse=True)
def _device_flag_checks():
    """Every asynchronous render / backward call made through the Python
    binding in the tests waits for its kernels and fails on a device-side
    failure flag (a traversal overflow, a bounded wait that ran out)."""
    from paper_2303_04086_gb300 import inolf
    inolf.check_device_flags(True)
    yield
    inolf.check_device_flags(False)


@pytest.fixture(scope="session")
def tiny():
    from paper_2303_04086_gb300 import synth
    return synth.tiny_scene(seed=0)


@pytest.fixture(scope="session")
def tiny_oracle(tiny):
    import oracle
    return oracle.Oracle(tiny)


@pytest.fixture(scope="session")
def tiny_cam():
    from paper_2303_04086_gb300 import synth
    return synth.camera((0.0, 0.0, 3.0))
