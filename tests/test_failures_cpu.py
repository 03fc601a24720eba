"""Failure reporting on the host, without a GPU: an injected device-allocation failure comes
back as BD_ERR_NOMEM (the code a real out-of-memory error gives), not as a generic CUDA error,
and the injection fires once."""

import numpy as np
import pytest

import paper_1501_02237_gb300 as bd
from paper_1501_02237_gb300._lib import BD_ERR_CUDA, BD_ERR_NOMEM

SMALL = np.array([[0, 0], [1, 0], [0, 1], [1, 1], [2, 1]])


@pytest.fixture(autouse=True)
def _disarm():
    yield
    bd.inject_alloc_failure(-1)


def test_injected_allocation_failure_is_nomem():
    bd.inject_alloc_failure(0)
    with pytest.raises(bd.BinodegError) as e:
        bd.Plan(SMALL)  # a new plan allocates its device buffers first
    assert e.value.code == BD_ERR_NOMEM
    assert "out of memory" in str(e.value)


def test_injection_fires_once_and_disarms():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present: the GPU test covers the recovery")
    bd.inject_alloc_failure(0)
    with pytest.raises(bd.BinodegError) as e:
        bd.Plan(SMALL)
    assert e.value.code == BD_ERR_NOMEM
    # consumed: the next allocation is a real one, which fails without a device as a CUDA error
    with pytest.raises(bd.BinodegError) as e:
        bd.Plan(SMALL)
    assert e.value.code == BD_ERR_CUDA
    # disarmed explicitly: never fires
    bd.inject_alloc_failure(5)
    bd.inject_alloc_failure(-1)
    with pytest.raises(bd.BinodegError) as e:
        bd.Plan(SMALL)
    assert e.value.code == BD_ERR_CUDA
