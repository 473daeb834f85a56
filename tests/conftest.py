import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the native library")


@pytest.fixture(scope="session")
def datadir(tmp_path_factory):
    # tmpfs when there is one: its files can be mapped for the GPU (GFS_XFER_MAPPED)
    if os.path.isdir("/dev/shm") and os.access("/dev/shm", os.W_OK):
        import shutil
        import tempfile
        d = tempfile.mkdtemp(prefix="gfs_tests_", dir="/dev/shm")
        yield d
        shutil.rmtree(d, ignore_errors=True)
    else:
        yield str(tmp_path_factory.mktemp("gfs_data"))


def pytest_runtest_setup(item):
    if item.get_closest_marker("gpu") is not None:
        import torch
        if not torch.cuda.is_available():
            pytest.fail("GPU test run without a CUDA device (deselect with -m 'not gpu')")
