"""The library's planner (host code, no GPU): its distinct frames per block
agree with the oracle's memoized recursion (Sec. 3.1 frames, memoized on
identity), its leaves are the order-2 frames, and its inverse and product work
per block are the pinned G(k), I(k) of the memoized DAG with distinct pivots
inverted once (Sec. 5, 7)."""
import ctypes

import pytest

import bri_inputs as bi
import oracle


@pytest.fixture(scope="module")
def plan():
    import paper_1612_00001_gb300 as mb
    mb.build()
    f = mb.lib().mbinv_debug_plan
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    f.restype = ctypes.c_int

    def run(k, i, j, pad_last=False):
        out = (ctypes.c_double * 6)()
        assert f(k, i, j, int(pad_last), out) == 0, (k, i, j)
        return dict(zip(("frames", "leaves", "inversions", "slots", "gemm_b3", "inv_b3"), out))
    return run


@pytest.mark.parametrize("k", [2, 3, 4, 5, 6, 7, 8])
def test_frames_match_oracle(plan, k):
    m = bi.uniform_shift(k, 4)
    for (i, j) in [(0, 0), (k - 1, 0), (0, k - 1), (k // 2, k - 1), (k - 1, k - 1)]:
        _, st, stats = oracle.bri_block(m, k, i, j, memo=True)
        assert st == oracle.OK
        p = plan(k, i, j)
        assert p["frames"] == stats["frames"], (k, i, j)
        # one order-2 frame per kept (row, column) pair around the pivot block
        assert p["leaves"] == (k - 1) ** 2
        # distinct pivots inverted once: never more inverses than the oracle's
        # one per reduction, and two b^3 of inverse work per inverse
        assert p["inversions"] <= stats["inversions"]
        assert p["inv_b3"] == 2 * p["inversions"]


def test_padded_requests_match_oracle(plan):
    k = 5
    m = bi.uniform_shift(k, 3)
    for (i, j) in [(4, 1), (2, 4), (4, 4), (1, 2)]:
        _, st, stats = oracle.bri_block(m, k, i, j, memo=True, pad_last=True)
        assert st == oracle.OK
        assert plan(k, i, j, pad_last=True)["frames"] == stats["frames"], (i, j)


def test_k8_and_k16_counts(plan):
    for (i, j) in [(0, 0), (3, 6), (7, 7)]:
        p = plan(8, i, j)
        assert (p["frames"], p["inversions"], p["gemm_b3"], p["inv_b3"], p["slots"]) == (270, 148, 996, 296, 292)
    assert plan(16, 0, 15)["frames"] == 3502


def test_invalid_arguments():
    import paper_1612_00001_gb300 as mb
    f = mb.lib().mbinv_debug_plan
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    out = (ctypes.c_double * 6)()
    assert f(8, 8, 0, 0, out) == -1
    assert f(8, 0, -1, 0, out) == -1
    assert f(0, 0, 0, 0, out) == -1
    assert f(8, 0, 0, 0, None) == -1
