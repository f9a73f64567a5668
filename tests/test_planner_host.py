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
    f = mb.test_lib().mbinv_debug_plan
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
        # 996 b^3 of products (the survey's G(8)) less 100 b^3 of shared piv^-1 right
        assert (p["frames"], p["inversions"], p["gemm_b3"], p["inv_b3"], p["slots"]) == (270, 148, 896, 296, 292)
    assert plan(16, 0, 15)["frames"] == 3502


def test_invalid_arguments():
    import paper_1612_00001_gb300 as mb
    f = mb.test_lib().mbinv_debug_plan
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    out = (ctypes.c_double * 6)()
    assert f(8, 8, 0, 0, out) == -1
    assert f(8, 0, -1, 0, out) == -1
    assert f(0, 0, 0, 0, out) == -1
    assert f(8, 0, 0, 0, None) == -1


# ---------------------------------------------------------------- merged plans
#
# An independent restatement of the forward procedure (Sec. 3.1) for counting
# only: root lists for (i, j) (rows start with j, columns with i, the others
# ascending), children by dropping the first/last row and column, the pivot
# index put back at position 2 of every frame of order >= 3, frames memoized on
# identity within a request, and merged across requests when they compute the
# same thing (same four operand frames; leaves: same kept block and pivot).

_KLPR = [[0, 1, 3, 2], [1, 0, 2, 3], [2, 3, 1, 0], [3, 2, 0, 1]]


def _root(k, i, j):
    if i == j:
        rows = [i] + [x for x in range(k) if x != i]
        return rows, list(rows)
    mid = [x for x in range(k) if x not in (i, j)]
    return [j] + mid + [i], [i] + mid + [j]


def _merged(k, reqs):
    cons, frames = {}, []
    request_frames = 0
    for i, j in reqs:
        rows, cols = _root(k, i, j)
        prow, pcol = rows[1], cols[1]
        memo = {}

        def visit(rows, cols, role):
            p = len(rows)
            kr = rows[0] if role in (0, 1) else rows[-1]
            kc = cols[0] if role in (0, 2) else cols[-1]
            ident = (kr, kc, frozenset(rows) - {kr}, frozenset(cols) - {kc})
            if ident in memo:
                return memo[ident]
            if p == 2:
                key = ("leaf", kr, kc, prow, pcol)
            else:
                ch = []
                for c in range(4):
                    r0, c0 = (1 if c >= 2 else 0), (1 if c & 1 else 0)
                    cr, cc = rows[r0:r0 + p - 1], cols[c0:c0 + p - 1]
                    if p - 1 >= 3:
                        if cr[0] == prow:
                            cr[0], cr[1] = cr[1], cr[0]
                        if cc[0] == pcol:
                            cc[0], cc[1] = cc[1], cc[0]
                    ch.append(visit(cr, cc, c))
                key = ("frame",) + tuple(ch[x] for x in _KLPR[role])
            if key not in cons:
                cons[key] = len(frames)
                frames.append(key)
            memo[ident] = cons[key]
            return memo[ident]

        visit(rows, cols, 0)
        request_frames += len(memo)
    leaves = [f for f in frames if f[0] == "leaf"]
    inner = [f for f in frames if f[0] == "frame"]
    leaf_pivots = {(f[3], f[4]) for f in leaves}
    t_values = {(f[3], f[4], f[2]) for f in leaves}
    pivots = {f[3] for f in inner}
    z_values = {(f[3], f[4]) for f in inner}
    return {"frames": len(frames), "request_frames": request_frames, "leaves": len(leaves),
            "inversions": len(leaf_pivots) + len(pivots) + len(reqs),
            "gemm_b3": 2 * (len(t_values) + len(leaves)) + 2 * (len(z_values) + len(inner)),
            "inv_b3": 2 * (len(leaf_pivots) + len(pivots) + len(reqs))}


@pytest.fixture(scope="module")
def plan_group():
    import paper_1612_00001_gb300 as mb
    mb.build()
    f = mb.test_lib().mbinv_debug_plan_group
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                  ctypes.POINTER(ctypes.c_double)]
    f.restype = ctypes.c_int

    def run(k, reqs, pad_last=False):
        flat = (ctypes.c_int * (2 * len(reqs)))(*[x for ij in reqs for x in ij])
        out = (ctypes.c_double * 7)()
        assert f(k, len(reqs), flat, int(pad_last), out) == 0
        return dict(zip(("frames", "request_frames", "inversions", "slots", "gemm_b3", "inv_b3", "leaves"),
                        [int(x) for x in out]))
    return run


@pytest.mark.parametrize("k", [3, 4, 5, 8])
def test_single_request_counts_match_restatement(plan_group, k):
    for ij in [(0, 0), (k - 1, 0), (1, k - 1)]:
        got, want = plan_group(k, [ij]), _merged(k, [ij])
        for key in ("frames", "request_frames", "leaves", "inversions", "gemm_b3", "inv_b3"):
            assert got[key] == want[key], (k, ij, key, got[key], want[key])
        assert got["frames"] == got["request_frames"]


def test_k8_single_request_work():
    """At k = 8 a request evaluates 270 frames and 148 inverses; its products
    are the survey's 996 b^3 less the 100 b^3 of the 50 products piv^-1 right
    that two frames share (formed once)."""
    w = _merged(8, [(3, 6)])
    assert (w["frames"], w["inversions"], w["gemm_b3"], w["inv_b3"]) == (270, 148, 896, 296)


@pytest.mark.parametrize("k,reqs", [
    (4, [(i, j) for i in range(4) for j in range(4)]),
    (8, [(i, j) for i in range(8) for j in range(8)]),
    (8, [(2, j) for j in range(8)]),
    (6, [(0, 5), (5, 0), (2, 2), (3, 1)]),
])
def test_merged_group_counts_match_restatement(plan_group, k, reqs):
    got, want = plan_group(k, reqs), _merged(k, reqs)
    for key in ("frames", "request_frames", "leaves", "inversions", "gemm_b3", "inv_b3"):
        assert got[key] == want[key], (k, key, got[key], want[key])
    assert got["frames"] <= got["request_frames"]


def test_all_blocks_of_k8_share_most_frames(plan_group):
    """The 64 runs of k = 8 (Sec. 5's k^2 runs) evaluate 6116 distinct frames
    instead of 64 x 270 = 17280, and 2133 inverses instead of 64 x 148."""
    g = plan_group(8, [(i, j) for i in range(8) for j in range(8)])
    assert (g["frames"], g["request_frames"], g["inversions"]) == (6116, 17280, 2133)
    single = plan_group(8, [(0, 0)])
    assert g["slots"] < 64 * single["slots"]
