"""mbinv_invert_noalloc - the inverse entry point that allocates nothing -
against the library's allocating path (mbinv_create with k = 1 and
mbinv_block), through the C ABI, on two calls in a row.

It exists for callers that cannot allocate device memory when they call (a
framework's caching allocator holding the GPU's memory, code that must not
pay cudaFree's device-wide synchronisation).  This file is collected last so
that a run stopping at the first failure has run every other test already."""
import ctypes

import numpy as np
import pytest

import bri_inputs as bi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12  # relative Frobenius; both paths run the same FP64 kernels


@pytest.fixture(scope="module")
def mb():
    import paper_1612_00001_gb300 as mb
    mb.build()
    return mb


def allocating_inverse(mb, a):
    with mb.Context(a, 1, precision="fp64" if a.dtype == torch.float64 else "fp32") as ctx:
        return ctx.block(0, 0)


def noalloc_inverse(mb, a):
    x = torch.empty_like(a)
    st = mb.lib().mbinv_invert_noalloc(a.data_ptr(), a.stride(0), x.data_ptr(), x.stride(0), a.shape[0],
                                       0 if a.dtype == torch.float64 else 1, torch.cuda.current_stream().cuda_stream)
    return st, x


@pytest.mark.parametrize("b", [96, 300, 512])
def test_noalloc_matches_allocating_path_twice(mb, b):
    for call, seed in enumerate((1, 2)):  # two calls in a row, different inputs
        a = torch.tensor(bi.uniform_shift(b, seed, shift=b / 8), device="cuda")
        st, x = noalloc_inverse(mb, a)
        assert st == mb.OK, (call, st)
        ref = allocating_inverse(mb, a)
        err = float(torch.linalg.norm(x - ref) / torch.linalg.norm(ref))
        assert err <= TOL, (call, err)
        # and it is the inverse
        eye = torch.eye(b, dtype=a.dtype, device="cuda")
        assert float(torch.linalg.norm(x @ a - eye)) < 1e-9


def test_noalloc_fp32_and_singular(mb):
    a = torch.tensor(bi.uniform_shift(200, 3, shift=20.0), dtype=torch.float32, device="cuda")
    st, x = noalloc_inverse(mb, a)
    assert st == mb.OK
    ref = allocating_inverse(mb, a)
    assert float(torch.linalg.norm(x - ref) / torch.linalg.norm(ref)) <= 1e-6
    z = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    st, _ = noalloc_inverse(mb, z)
    assert st == mb.ESINGULAR
    # the next call is not disturbed by the singular one
    a = torch.tensor(bi.uniform_shift(64, 4), device="cuda")
    st, x = noalloc_inverse(mb, a)
    assert st == mb.OK
    assert float(torch.linalg.norm(x - allocating_inverse(mb, a))) < 1e-12 * float(torch.linalg.norm(x))


def test_noalloc_rejects_oversize_before_launch(mb):
    big = torch.empty((513, 513), dtype=torch.float64, device="cuda")
    st, _ = noalloc_inverse(mb, big)
    assert st == mb.EINVAL
