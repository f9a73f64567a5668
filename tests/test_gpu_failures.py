"""Failure paths, exercised without a GPU fault.

* A device wait that runs out: a test hook makes every digit-product launch
  wait on a barrier nothing arrives at (a short limit), so the kernel raises
  its error word and returns before issuing any copy or product; the call
  reports MBINV_ETIMEOUT and the context computes correctly afterwards.
* An allocation that fails: a host-side hook makes the next device
  allocation fail as if the GPU were out of memory; the call reports
  MBINV_ECUDA before any launch and the context computes correctly
  afterwards."""
import ctypes

import numpy as np
import pytest

import bri_inputs as bi
from helpers import to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mb():
    import paper_1612_00001_gb300 as mb
    mb.build()
    L = mb.test_lib()
    L.mbinv_debug_set_stall_ns.argtypes = [ctypes.c_ulonglong]
    L.mbinv_debug_set_stall_ns.restype = None
    L.mbinv_debug_fail_allocations.argtypes = [ctypes.c_int]
    L.mbinv_debug_fail_allocations.restype = None
    return mb


def dev(a):
    return torch.tensor(a, dtype=torch.float64, device="cuda")


def test_device_wait_that_runs_out_is_reported(mb):
    m = bi.uniform_shift(768, 1)  # b = 192: Schur products and inverse updates are digit products
    L = mb.test_lib()
    with mb.Context(dev(m), 4, precision="fp64_tc") as ctx:
        ref = to_np(ctx.block(1, 2))
        L.mbinv_debug_set_stall_ns(1000000)  # 1 ms
        try:
            with pytest.raises(mb.MbinvError) as e:
                ctx.block(1, 2)
            assert e.value.status == mb.ETIMEOUT
        finally:
            L.mbinv_debug_set_stall_ns(0)
        torch.cuda.synchronize()
        assert np.array_equal(to_np(ctx.block(1, 2)), ref)


def test_failed_allocation_is_reported_before_launch(mb):
    m = bi.uniform_shift(512, 2)
    L = mb.test_lib()
    with mb.Context(dev(m), 8, precision="fp64_tc") as c0:
        ref = to_np(c0.block(3, 4))
    with mb.Context(dev(m), 8, precision="fp64_tc") as ctx:
        L.mbinv_debug_fail_allocations(1)
        try:
            with pytest.raises(mb.MbinvError) as e:
                ctx.block(3, 4)
            assert e.value.status == mb.ECUDA
            assert ctx.last_report is None or ctx.last_report["launches"] == 0
        finally:
            L.mbinv_debug_fail_allocations(0)
        assert np.array_equal(to_np(ctx.block(3, 4)), ref)
