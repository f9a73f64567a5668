"""The pins catch plausible mistakes: each test here plants one mistake in a
copy of the oracle's C source (on the CPU), builds it, and checks that the
pins that pass on the real oracle - brute force against LAPACK for k = 2..4
(which holds the k = 2 closed form) and the worked 4x4 example of Sec. 4
assembled from its printed frames - fail on it.  Dropping the exchange that
keeps M_22 at (2,2) is invisible to brute force (any elimination order gives
the inverse in exact arithmetic); the printed frames catch it."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import bri_inputs as bi

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "bri_oracle.c")

MUTATIONS = {
    # wrong role formula: B reduces as if it were A's pivot layout
    "role_B_swapped": ("case 1: return schur_reduce(R, bb, ldb, a, lda, c, ldc, d, ldd, out);",
                       "case 1: return schur_reduce(R, bb, ldb, d, ldd, c, ldc, a, lda, out);"),
    # wrong sign of the Schur update
    "sign": ("out[r * b + c] = kept[r * ldk + c] - out[r * b + c];",
             "out[r * b + c] = kept[r * ldk + c] + out[r * b + c];"),
    # the exchange that keeps M_22 at (2,2) dropped
    "no_exchange": ("if (cr[0] == R->piv_row) { int t = cr[0]; cr[0] = cr[1]; cr[1] = t; }",
                    "if (0) { int t = cr[0]; cr[0] = cr[1]; cr[1] = t; }"),
    # transposed operand in the plain product
    "transposed_B": ("c[q] = c[q] + a * brow[q];", "c[q] = c[q] + a * B[q * ldb + t];"),
    # the final column interchanges of Gauss-Jordan dropped
    "no_unswap": ("if (p != j)\n            for (int64_t r = 0; r < n; ++r) {",
                  "if (0)\n            for (int64_t r = 0; r < n; ++r) {"),
    # rows and columns of the permutation for (i, j) exchanged
    "root_transposed": ("rows[0] = j; cols[0] = i;\n    for (int x = 0; x < k; ++x)",
                        "rows[0] = i; cols[0] = j;\n    for (int x = 0; x < k; ++x)"),
    # one term of the elimination dropped (no update of the pivot column)
    "dropped_term": ("xi[j] = 0.0;\n            for (int64_t c = 0; c < n; ++c) xi[c] = xi[c] - f * xj[c];",
                     "xi[j] = 0.0;\n            for (int64_t c = 0; c < n; ++c) if (c != j) xi[c] = xi[c] - f * xj[c];"),
}


def _bind(L):
    dp = ctypes.POINTER(ctypes.c_double)
    i64 = ctypes.c_int64
    L.orc_bri_block.argtypes = [dp, i64, i64, i64, i64, i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                ctypes.POINTER(ctypes.c_int64)]
    L.orc_bri_block.restype = ctypes.c_int
    L.orc_gj_inverse.argtypes = [i64, dp, i64, dp, i64]
    L.orc_gj_inverse.restype = ctypes.c_int
    L.orc_matmul.argtypes = [i64, i64, i64, dp, i64, dp, i64, dp, i64]
    L.orc_matmul.restype = None
    return L


def build_mutant(tmp, name):
    text = open(SRC).read()
    old, new = {**MUTATIONS, **FLOOR_MUTATIONS}[name]
    assert old in text, f"mutation site of {name} not found"
    src = os.path.join(tmp, f"{name}.c")
    open(src, "w").write(text.replace(old, new, 1))
    so = os.path.join(tmp, f"{name}.so")
    subprocess.run(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", src, "-o", so, "-lm"],
                   check=True)
    return _bind(ctypes.CDLL(so))


def _worked_example_ok(L):
    """Sec. 4: N_11 assembled from the printed frames (tests/golden/frames_k4.txt)
    with the library's own primitives equals its recursion bit for bit, and the
    recursion visits the 14 distinct frames of k = 4."""
    dp = ctypes.POINTER(ctypes.c_double)
    b = 2
    m = np.ascontiguousarray(bi.uniform_shift(4 * b, 21))
    blk = {(r, c): np.ascontiguousarray(m[r * b:(r + 1) * b, c * b:(c + 1) * b]) for r in range(4) for c in range(4)}

    def inv(a):
        a = np.ascontiguousarray(a)
        x = np.empty_like(a)
        L.orc_gj_inverse(b, a.ctypes.data_as(dp), b, x.ctypes.data_as(dp), b)
        return x

    def mm(a, c):
        a, c = np.ascontiguousarray(a), np.ascontiguousarray(c)
        o = np.empty((b, b))
        L.orc_matmul(b, b, b, a.ctypes.data_as(dp), b, c.ctypes.data_as(dp), b, o.ctypes.data_as(dp), b)
        return o

    def schur(kept, left, piv, right):
        return kept - mm(left, mm(inv(piv), right))

    frames = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "frames_k4.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, r, c = (x.strip() for x in line.split("|"))
        frames[name] = ([int(x) - 1 for x in r.split()], [int(x) - 1 for x in c.split()])
    P = (1, 1)

    def leaf(rows, cols):
        (x,) = [q for q in rows if q != P[0]]
        (y,) = [q for q in cols if q != P[1]]
        return schur(blk[x, y], blk[x, P[1]], blk[P], blk[P[0], y])

    lv = {}
    for nm in "ABCD":
        r, c = frames["M>" + nm]
        v = {"A": leaf(r[:2], c[:2]), "B": leaf(r[:2], c[1:]), "C": leaf(r[1:], c[:2]), "D": leaf(r[1:], c[1:])}
        lv[nm] = {"A": schur(v["A"], v["B"], v["D"], v["C"]), "B": schur(v["B"], v["A"], v["C"], v["D"]),
                  "C": schur(v["C"], v["D"], v["B"], v["A"]), "D": schur(v["D"], v["C"], v["A"], v["B"])}[nm]
    n11 = inv(schur(lv["A"], lv["B"], lv["D"], lv["C"]))
    out = np.empty((b, b))
    stats = (ctypes.c_int64 * 4)()
    st = L.orc_bri_block(m.ctypes.data_as(dp), 4 * b, 4, b, 0, 0, 1, 0, 0, out.ctypes.data_as(dp), stats)
    return st == 0 and np.array_equal(out, n11) and stats[2] == 14


def pins_pass(L):
    """The brute-force pin (all blocks, k = 2..4, which contains the k = 2
    closed form) and the worked example of Sec. 4."""
    if not _worked_example_ok(L):
        return False
    dp = ctypes.POINTER(ctypes.c_double)
    for k, b, seed in [(2, 3, 5), (3, 3, 1), (4, 2, 7)]:
        m = np.ascontiguousarray(bi.uniform_shift(k * b, seed, shift=k * b / 4))
        inv = np.linalg.inv(m)
        for i in range(k):
            for j in range(k):
                out = np.empty((b, b))
                stats = (ctypes.c_int64 * 4)()
                st = L.orc_bri_block(m.ctypes.data_as(dp), k * b, k, b, i, j, 1, 0, 0, out.ctypes.data_as(dp), stats)
                ref = inv[i * b:(i + 1) * b, j * b:(j + 1) * b]
                if st != 0 or not np.all(np.isfinite(out)):
                    return False
                if np.linalg.norm(out - ref) > 1e-12 * np.linalg.norm(ref):
                    return False
    return True


# Mistakes in the re-associated evaluation that the sensitivity floor rests on
# (the parity rule's 10 x floor): the scalar pin of the floor must fail.
FLOOR_MUTATIONS = {
    # the re-associated order silently evaluated like the plain one
    "reassoc_ignored": ("if (!R->reassoc) {", "if (1) {"),
}


def floor_pins_pass(L):
    """k = 2, b = 1: the floor written out in IEEE double (see
    tests/test_oracle.py) against the mutant's two evaluation orders."""
    dp = ctypes.POINTER(ctypes.c_double)
    nonzero = 0
    for t in range(40):
        v = bi.uniform_pm1(77, t, 4)
        b_, c, d = float(v[1]) + 2.0, float(v[2]) + 2.0, float(v[3]) + 4.0
        a = b_ * c / d + 1e-3 * float(v[0])
        dinv = 1.0 / d
        n1 = 1.0 / (a - b_ * (dinv * c))
        n2 = 1.0 / (a - (b_ * dinv) * c)
        m = np.ascontiguousarray(np.array([[a, b_], [c, d]]))
        got = []
        for reassoc in (0, 1):
            out = np.empty((1, 1))
            stats = (ctypes.c_int64 * 4)()
            if L.orc_bri_block(m.ctypes.data_as(dp), 2, 2, 1, 0, 0, 1, reassoc, 0, out.ctypes.data_as(dp), stats):
                return False
            got.append(out[0, 0])
        if got[0] != n1 or got[1] != n2:
            return False
        nonzero += n1 != n2
    return nonzero >= 10


@pytest.fixture(scope="module")
def tmpdir_():
    d = tempfile.mkdtemp(prefix="oracle_mut_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


def test_unmutated_copy_passes(tmpdir_):
    text = open(SRC).read()
    src = os.path.join(tmpdir_, "clean.c")
    open(src, "w").write(text)
    so = os.path.join(tmpdir_, "clean.so")
    subprocess.run(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", src, "-o", so, "-lm"],
                   check=True)
    L = _bind(ctypes.CDLL(so))
    assert pins_pass(L)
    assert floor_pins_pass(L)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmpdir_, name):
    assert not pins_pass(build_mutant(tmpdir_, name)), f"mutation {name} survived the pins"


@pytest.mark.parametrize("name", sorted(FLOOR_MUTATIONS))
def test_planted_floor_mistake_is_caught(tmpdir_, name):
    assert not floor_pins_pass(build_mutant(tmpdir_, name)), f"mutation {name} survived the floor pin"
