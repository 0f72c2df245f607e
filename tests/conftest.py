import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def M():
    import paper_1506_05393_gb300 as M
    M.lib()
    return M


@pytest.fixture(scope="session")
def ctx(M):
    """One library context on cuda:0 for the whole GPU session."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected but no CUDA device is visible")
    torch.cuda.init()
    c = M.mrf_ctx_create(0, 0)
    yield c
    M.mrf_ctx_destroy(c)


class DevView:
    """__cuda_array_interface__ view of a raw device pointer (no copy)."""

    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"shape": (int(nbytes),), "typestr": "|u1", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def device_bytes(ptr, nbytes):
    """A uint8 CUDA tensor aliasing library-owned device memory."""
    import torch
    return torch.as_tensor(DevView(ptr, nbytes), device="cuda")
