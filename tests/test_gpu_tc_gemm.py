"""The tcgen05 tensor-core product alone, against a plain FP64 product of the
same operands (through a test hook of libmbinv, not the public header)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hook():
    import paper_1612_00001_gb300 as mb
    mb.build()
    f = mb.test_lib().mbinv_debug_tc_gemm
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int] * 6 + [ctypes.c_void_p]
    return f


def run(hook, m, n, k, S, count, mode=0, seed=0):
    g = torch.Generator(device="cpu").manual_seed(seed)
    A = torch.randn(count, m, k, generator=g).cuda()
    B = torch.randn(count, k, n, generator=g).cuda()
    C = torch.zeros(count, m, n, device="cuda")
    rc = hook(A.data_ptr(), B.data_ptr(), C.data_ptr(), m, n, k, S, count, mode,
              torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    ref = torch.bmm(A.double(), B.double())
    return C.double(), ref


# BF16 keeps 8 significant bits per slice: 1 slice ~ 2^-8 relative per
# operand, 2 slices ~ 2^-16, 3 slices ~ 2^-24 (plus FP32 accumulation).
TOL = {1: 2e-2, 2: 1e-4, 3: 2e-6}


@pytest.mark.parametrize("S", [1, 2, 3])
def test_single_tile(hook, S):
    C, ref = run(hook, 128, 128, 64, S, 1)
    err = float((C - ref).norm() / ref.norm())
    assert err < TOL[S], err


@pytest.mark.parametrize("m,n,k,count", [(512, 512, 512, 3), (200, 136, 100, 2), (384, 256, 960, 1)])
def test_grouped_ragged(hook, m, n, k, count):
    for S in (1, 3):
        C, ref = run(hook, m, n, k, S, count, seed=m + k)
        err = float((C - ref).norm() / ref.norm())
        assert err < TOL[S], (S, err)


def test_transposed_slice_epilogue(hook):
    C, ref = run(hook, 256, 384, 192, 3, 2, mode=1)
    err = float((C - ref).norm() / ref.norm())
    assert err < TOL[3], err
