"""The library's schedules run on scalars (b = 1) on the host, against the
oracle.  With b = 1 every step of the recursion is one IEEE operation, so a
schedule that reads the right values in the right order reproduces the
oracle's memoized recursion (O2) bit for bit: the level-by-level schedule of
merged runs, and the depth-first bounded schedule whatever its slot budget
(values evicted to "host memory" and brought back, blocks of M loaded on
demand).  No GPU: the hook builds the plan and interprets it."""
import ctypes

import numpy as np
import pytest

import bri_inputs as bi
import oracle


@pytest.fixture(scope="module")
def run():
    import paper_1612_00001_gb300 as mb
    mb.build()
    f = mb.test_lib().mbinv_debug_run_schedule_scalar
    dp = ctypes.POINTER(ctypes.c_double)
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                  ctypes.c_int, dp, dp, dp]
    f.restype = ctypes.c_int

    def go(m, k, reqs, mode, slots=0, host_m=False):
        m = np.ascontiguousarray(m, dtype=np.float64)
        flat = (ctypes.c_int * (2 * len(reqs)))(*[x for ij in reqs for x in ij])
        outs = np.zeros(len(reqs))
        stats = np.zeros(7)
        rc = f(k, len(reqs), flat, mode, slots, int(host_m), m.ctypes.data_as(dp), outs.ctypes.data_as(dp),
               stats.ctypes.data_as(dp))
        return rc, outs, dict(zip(("steps", "slots", "spill", "loads", "spills", "inversions", "gemm_b3"), stats))
    return go


def oracle_scalars(m, k, reqs):
    out = []
    for i, j in reqs:
        v, st, _ = oracle.bri_block(m, k, i, j, memo=True)
        assert st == oracle.OK
        out.append(v[0, 0])
    return np.array(out)


@pytest.mark.parametrize("k", [3, 5, 8])
def test_level_schedule_of_merged_runs_equals_oracle(run, k):
    m = bi.uniform_shift(k, 11)
    reqs = [(i, j) for i in range(k) for j in range(k)]
    rc, outs, st = run(m, k, reqs, 0)
    assert rc == 0
    assert np.array_equal(outs, oracle_scalars(m, k, reqs))


@pytest.mark.parametrize("k,slots,host_m", [(6, 8, True), (6, 8, False), (8, 12, True), (8, 40, True),
                                            (10, 16, True)])
def test_bounded_schedule_equals_oracle_in_few_slots(run, k, slots, host_m):
    m = bi.uniform_shift(k, 12)
    reqs = [(0, k - 1), (k - 1, 0), (2, 2)]
    rc, outs, st = run(m, k, reqs, 1, slots, host_m)
    assert rc == 0, rc
    assert np.array_equal(outs, oracle_scalars(m, k, reqs))
    assert st["slots"] <= slots
    # work is the level schedule's: the same values, each computed once
    rc0, outs0, st0 = run(m, k, reqs, 0)
    assert (st["inversions"], st["gemm_b3"]) == (st0["inversions"], st0["gemm_b3"])
    assert np.array_equal(outs, outs0)
    if host_m:
        assert st["loads"] >= k * k  # every block of M read from the host at least once


def test_bounded_schedule_spills_only_when_short_of_slots(run):
    k = 8
    m = bi.uniform_shift(k, 13)
    reqs = [(3, 5)]
    rc, _, roomy = run(m, k, reqs, 1, 4096, False)
    assert rc == 0 and roomy["spills"] == 0 and roomy["loads"] == 0
    rc, outs, tight = run(m, k, reqs, 1, 10, False)
    assert rc == 0 and tight["spills"] > 0 and tight["loads"] >= tight["spills"]
    assert tight["slots"] <= 10 < roomy["slots"]
    assert np.array_equal(outs, oracle_scalars(m, k, reqs))


def test_bounded_schedule_refuses_too_few_slots(run):
    m = bi.uniform_shift(6, 1)
    rc, _, _ = run(m, 6, [(0, 5)], 1, 3, True)
    assert rc == -2
