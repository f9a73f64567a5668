"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every test here runs on the CPU only.  The oracle is checked against values
that do not come from itself: the closed-form 2x2 block inverse (Eq. invSchur),
the frames printed in the worked 4x4 example (Sec. 4), Theorem 1's operation
count, block-diagonal and block-triangular matrices with known inverses, the
augmented matrix of Eq. inverse_M_augmented, brute force by LAPACK on tiny
inputs, and exact invariances (power-of-two scaling).
"""
import itertools
import os

import numpy as np
import pytest

import bri_inputs as bi
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def blocks(m, b):
    k = m.shape[0] // b
    return {(r, c): m[r * b:(r + 1) * b, c * b:(c + 1) * b] for r in range(k) for c in range(k)}


# ----------------------------------------------------------- Gauss-Jordan

@pytest.mark.parametrize("n", [1, 2, 5, 16, 33])
def test_gj_matches_lapack(n):
    m = bi.uniform_shift(n, 11, shift=0.5)  # weak shift: pivoting matters
    x, st = oracle.gj_inverse(m)
    assert st == oracle.OK
    ref = np.linalg.inv(m)
    cond = np.linalg.cond(m)
    assert oracle.rel_fro(x, ref) <= 50 * n * cond * np.finfo(float).eps


def test_gj_needs_row_interchange():
    # zero in the leading position: only row interchanges make it solvable
    m = np.array([[0.0, 2.0, 1.0], [1.0, 1.0, 0.0], [3.0, 0.0, 1.0]])
    x, st = oracle.gj_inverse(m)
    assert st == oracle.OK
    assert np.allclose(x @ m, np.eye(3), atol=1e-15)


def test_gj_permutation_matrix_exact():
    p = np.eye(7)[[3, 0, 6, 1, 5, 2, 4]]
    x, st = oracle.gj_inverse(p)
    assert st == oracle.OK
    assert np.array_equal(x, p.T)


def test_gj_singular_detected():
    m = bi.uniform_shift(6, 3)
    m[4] = 2.0 * m[1] - m[0]
    _, st = oracle.gj_inverse(m)
    assert st == oracle.SINGULAR
    _, st = oracle.gj_inverse(np.zeros((3, 3)))
    assert st == oracle.SINGULAR
    m = bi.uniform_shift(4, 1)
    m[2, 2] = np.nan
    _, st = oracle.gj_inverse(m)
    assert st == oracle.SINGULAR


def test_matmul_is_plain_product():
    a = bi.uniform_pm1(1, 1, 12).reshape(3, 4)
    b = bi.uniform_pm1(1, 2, 20).reshape(4, 5)
    c = oracle.matmul(a, b)
    # sum in increasing inner index, no fused multiply-add
    ref = np.zeros((3, 5))
    for t in range(4):
        ref = ref + a[:, t:t + 1] * b[t:t + 1, :]
    assert np.array_equal(c, ref)


# ----------------------------------------------------- k = 2: Eq. invSchur

@pytest.mark.parametrize("b", [1, 3, 8])
def test_k2_against_schur_block_inverse(b):
    """Eq. invSchur: E = (M/D)^-1, F = -(M/D)^-1 B D^-1,
    G = -D^-1 C (M/D)^-1, H = D^-1 + D^-1 C (M/D)^-1 B D^-1."""
    m = bi.uniform_shift(2 * b, 5)
    bl = blocks(m, b)
    A, B, C, D = bl[0, 0], bl[0, 1], bl[1, 0], bl[1, 1]
    Di = np.linalg.inv(D)
    S = np.linalg.inv(A - B @ Di @ C)
    ref = {(0, 0): S, (0, 1): -S @ B @ Di, (1, 0): -Di @ C @ S, (1, 1): Di + Di @ C @ S @ B @ Di}
    for (i, j), r in ref.items():
        n_ij, st, stats = oracle.bri_block(m, 2, i, j, memo=False)
        assert st == oracle.OK
        assert stats["schur_ops"] == 1
        assert oracle.rel_fro(n_ij, r) <= 1e-14, (i, j)


# ------------------------------------------------ Theorem 1 operation count

def test_theorem1_schur_op_count():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "schur_op_counts.txt")) if not l.startswith("#")]
    for k, count in ((int(a), int(c)) for a, c in rows):
        m = bi.uniform_shift(k, 2)  # b = 1
        _, st, stats = oracle.bri_block(m, k, 0, 0, memo=False)
        assert st == oracle.OK
        assert stats["schur_ops"] == count == sum(4 ** d for d in range(k - 1))
        assert stats["inversions"] == count + 1  # one per reduction + the final one


def test_memo_frame_counts():
    """Distinct frame identities per block: one shared value per identity."""
    expect = {2: 1, 3: 5, 4: 14, 5: 37, 6: 82, 7: 157, 8: 270}
    for k, cnt in expect.items():
        m = bi.uniform_shift(k, 4)
        for (i, j) in [(0, 0), (k - 1, 0), (0, k - 1), (k // 2, k - 1)]:
            _, st, stats = oracle.bri_block(m, k, i, j, memo=True)
            assert st == oracle.OK
            assert stats["frames"] == cnt, (k, i, j)


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_o1_equals_o2_bitwise(k):
    m = bi.uniform_shift(2 * k, 9)
    for i, j in [(0, 0), (1, k - 1), (k - 1, 0), (k - 1, k - 1)]:
        a, st1, _ = oracle.bri_block(m, k, i, j, memo=False)
        b, st2, _ = oracle.bri_block(m, k, i, j, memo=True)
        assert st1 == st2 == oracle.OK
        assert np.array_equal(a, b)


# ------------------------------------------------- worked example, Sec. 4

def _golden_frames():
    out = {}
    for line in open(os.path.join(GOLDEN, "frames_k4.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, r, c = (s.strip() for s in line.split("|"))
        out[name] = ([int(x) - 1 for x in r.split()], [int(x) - 1 for x in c.split()])
    return out


def _schur(kept, left, piv, right):
    """kept - left (piv^-1 right) with the oracle's own primitives."""
    pinv, st = oracle.gj_inverse(piv)
    assert st == oracle.OK
    return kept - oracle.matmul(left, oracle.matmul(pinv, right))


def test_worked_example_4x4_bitwise():
    """N_11 of a 4x4 block matrix assembled by hand from the printed frames
    (Eq. frames4x4Matrix), the leaf rule of Eqs. FA2-FD2 (Schur complement of
    M_22 in every 2x2 frame), the level-2 reductions of Eqs. Schur_Phi_2_A-D
    and Eq. blockmatrix4x4 equals the oracle's result bit for bit."""
    b = 3
    m = bi.uniform_shift(4 * b, 21)
    bl = blocks(m, b)
    fr = _golden_frames()
    P = (1, 1)  # M_22, 0-based

    # the printed splits of M>B agree with Step 1 applied to the printed M>B
    r, c = fr["M>B"]
    assert fr["M>B>A"] == (r[:2], c[:2]) and fr["M>B>B"] == (r[:2], c[1:])
    assert fr["M>B>C"] == (r[1:], c[:2]) and fr["M>B>D"] == (r[1:], c[1:])

    def leaf(rows, cols):
        # Schur complement of M_22 in a 2x2 frame: the entry opposite M_22
        # minus (its row, M_22's column) M_22^-1 (M_22's row, its column)
        (x,) = [q for q in rows if q != P[0]]
        (y,) = [q for q in cols if q != P[1]]
        return _schur(bl[x, y], bl[x, P[1]], bl[P], bl[P[0], y])

    def split(rows, cols):
        return {"A": (rows[:2], cols[:2]), "B": (rows[:2], cols[1:]),
                "C": (rows[1:], cols[:2]), "D": (rows[1:], cols[1:])}

    level = {}
    for name in "ABCD":
        v = {ch: leaf(*rc) for ch, rc in split(*fr["M>" + name]).items()}
        if name == "A":    # Eq. Schur_Phi_2_A: (./D)
            level[name] = _schur(v["A"], v["B"], v["D"], v["C"])
        elif name == "B":  # Eq. Schur_Phi_2_B: (./C)
            level[name] = _schur(v["B"], v["A"], v["C"], v["D"])
        elif name == "C":  # Eq. Schur_Phi_2_C: (./B)
            level[name] = _schur(v["C"], v["D"], v["B"], v["A"])
        else:              # Eq. Schur_Phi_2_D: (./A)
            level[name] = _schur(v["D"], v["C"], v["A"], v["B"])
    root = _schur(level["A"], level["B"], level["D"], level["C"])  # Eq. blockmatrix4x4
    n11, st = oracle.gj_inverse(root)
    assert st == oracle.OK

    got, st, _ = oracle.bri_block(m, 4, 0, 0, memo=False)
    assert st == oracle.OK
    assert np.array_equal(got, n11)
    assert oracle.rel_fro(got, np.linalg.inv(m)[:b, :b]) < 1e-14


def test_leaf_formulas_of_frame_B():
    """Eqs. FA2-FD2: the four leaf values of M>B, as frames of the oracle."""
    b = 2
    m = bi.uniform_shift(4 * b, 8)
    bl = blocks(m, b)
    fr = _golden_frames()
    expect = {
        "A": _schur(bl[0, 2], bl[0, 1], bl[1, 1], bl[1, 2]),  # M13 - M12 M22^-1 M23
        "B": _schur(bl[0, 3], bl[0, 1], bl[1, 1], bl[1, 3]),  # M14 - M12 M22^-1 M24
        "C": _schur(bl[2, 2], bl[2, 1], bl[1, 1], bl[1, 2]),  # M33 - M32 M22^-1 M23
        "D": _schur(bl[2, 3], bl[2, 1], bl[1, 1], bl[1, 3]),  # M34 - M32 M22^-1 M24
    }
    for role in "ABCD":
        rows, cols = fr["M>B>" + role]
        v, st, _ = oracle.bri_frame(m, b, rows, cols, role, 1, 1)
        assert st == oracle.OK
        assert np.array_equal(v, expect[role]), role


# ------------------------------------------------------------- brute force

@pytest.mark.parametrize("k,b", [(2, 3), (3, 3), (4, 3), (5, 2), (6, 2)])
def test_all_blocks_against_dense_inverse(k, b):
    m = bi.uniform_shift(k * b, 31 + k)
    ref = np.linalg.inv(m)
    dense, st = oracle.dense_inverse(m)
    assert st == oracle.OK
    assert oracle.rel_fro(dense, ref) < 1e-14
    for i, j in itertools.product(range(k), range(k)):
        n_ij, st, _ = oracle.bri_block(m, k, i, j)
        assert st == oracle.OK
        blk = ref[i * b:(i + 1) * b, j * b:(j + 1) * b]
        assert oracle.rel_fro(n_ij, blk) < 1e-12, (i, j)


def test_root_lists_reading():
    """The permutation that puts block (i, j) of the inverse at the top-left:
    rows start with j, columns with i, and inv(M[rows][:, cols]) has N_ij in
    its top-left corner."""
    k, b = 5, 2
    m = bi.uniform_shift(k * b, 3)
    ref = np.linalg.inv(m)
    for i, j in itertools.product(range(k), range(k)):
        rows, cols = oracle.root_lists(k, i, j)
        assert rows[0] == j and cols[0] == i and sorted(rows) == sorted(cols) == list(range(k))
        ri = np.concatenate([np.arange(r * b, (r + 1) * b) for r in rows])
        ci = np.concatenate([np.arange(c * b, (c + 1) * b) for c in cols])
        pinv = np.linalg.inv(m[np.ix_(ri, ci)])
        assert np.allclose(pinv[:b, :b], ref[i * b:(i + 1) * b, j * b:(j + 1) * b], rtol=0, atol=1e-15)


# ------------------------------------------------------- structured inputs

def test_block_diagonal():
    k, b = 4, 3
    m = bi.block_diagonal(k, b, 6)
    for i in range(k):
        n_ii, st, _ = oracle.bri_block(m, k, i, i)
        assert st == oracle.OK
        assert oracle.rel_fro(n_ii, np.linalg.inv(m[i * b:(i + 1) * b, i * b:(i + 1) * b])) < 1e-15
    # an off-diagonal block of the inverse is zero: no recursion can invert to it
    _, st, _ = oracle.bri_block(m, k, 0, 1)
    assert st == oracle.SINGULAR


def test_block_upper_triangular():
    k, b = 4, 3
    m = bi.block_upper_triangular(k, b, 7)
    ref = np.linalg.inv(m)
    for i, j in [(0, 0), (2, 2), (0, 3), (1, 2)]:
        n_ij, st, _ = oracle.bri_block(m, k, i, j)
        assert st == oracle.OK
        assert oracle.rel_fro(n_ij, ref[i * b:(i + 1) * b, j * b:(j + 1) * b]) < 1e-14, (i, j)
    for i in range(k):
        d = np.linalg.inv(m[i * b:(i + 1) * b, i * b:(i + 1) * b])
        n_ii, _, _ = oracle.bri_block(m, k, i, i)
        assert oracle.rel_fro(n_ii, d) < 1e-14
    _, st, _ = oracle.bri_block(m, k, 3, 0)  # strictly lower: the block is zero
    assert st == oracle.SINGULAR


def test_power_of_two_scaling_is_exact():
    k, b = 4, 4
    m = bi.uniform_shift(k * b, 12)
    for s in (-3, 5):
        for i, j in [(0, 0), (2, 1)]:
            a, _, _ = oracle.bri_block(m, k, i, j)
            c, _, _ = oracle.bri_block(m * 2.0 ** s, k, i, j)
            assert np.array_equal(c, a * 2.0 ** (-s))


def test_symmetric_input_gives_transposed_blocks():
    k, b = 4, 4
    m = bi.spd(k * b, 1e2, 2)
    for i, j in [(0, 1), (1, 3), (2, 0)]:
        a, _, _ = oracle.bri_block(m, k, i, j)
        c, _, _ = oracle.bri_block(m, k, j, i)
        assert oracle.rel_fro(a, c.T) < 1e-12


# ------------------------------------------------------------ augmentation

def test_augmented_matrix():
    """Eq. inverse_M_augmented: Gamma^-1 = diag(M^-1, I)."""
    n, k = 10, 4
    m = bi.uniform_shift(n, 13)
    ref = np.linalg.inv(m)
    g, b, l = oracle.augment(m, k)
    assert (b, l) == (3, 2)
    ginv = np.linalg.inv(g)
    assert np.allclose(ginv[:n, :n], ref, atol=1e-15) and np.allclose(ginv[n:, n:], np.eye(l))
    cpl = bi.pad_columns(n, l, 1)
    for i, j in itertools.product(range(k), range(k)):
        gi, _, _ = oracle.augment(m, k, i, j, coupling=cpl)
        n_ij, st, _ = oracle.bri_block(gi, k, i, j, pad_last=True)
        assert st == oracle.OK, (i, j)
        r0, r1 = i * b, min((i + 1) * b, n)
        c0, c1 = j * b, min((j + 1) * b, n)
        assert oracle.rel_fro(n_ij[:r1 - r0, :c1 - c0], ref[r0:r1, c0:c1]) < 1e-13, (i, j)
    # with the plain border, blocks that touch the padding are singular
    _, st, _ = oracle.bri_block(g, k, 0, 3)
    assert st == oracle.SINGULAR
    _, st, _ = oracle.bri_block(g, k, 3, 0)
    assert st == oracle.SINGULAR


@pytest.mark.parametrize("n,k", [(22, 5), (31, 6), (61, 8)])
def test_augmented_matrix_larger_k(n, k):
    """For k >= 5 the padded block must be the pivot index of requests that do
    not touch it: elsewhere some inverted frame keeps padded rows, which are
    zero, and the recursion stops on a singular pivot."""
    m = bi.uniform_shift(n, 3)
    ref = np.linalg.inv(m)
    b = -(-n // k)
    l = k * b - n
    cpl = bi.pad_columns(n, l, 0)
    for i, j in itertools.product(range(k), range(k)):
        g, _, _ = oracle.augment(m, k, i, j, coupling=cpl)
        n_ij, st, _ = oracle.bri_block(g, k, i, j, pad_last=True)
        assert st == oracle.OK, (i, j)
        r0, r1 = i * b, min((i + 1) * b, n)
        c0, c1 = j * b, min((j + 1) * b, n)
        # the parity rule against truth: the fixed bar plus 10 x the recursion's
        # own rounding sensitivity, which grows with k (1e-10 at k = 8)
        bound = 1e-11 + 10 * oracle.sensitivity_floor(g, k, i, j, pad_last=True)
        assert oracle.rel_fro(n_ij[:r1 - r0, :c1 - c0], ref[r0:r1, c0:c1]) < bound, (i, j)
    g, _, _ = oracle.augment(m, k)
    _, st, _ = oracle.bri_block(g, k, 0, 1, pad_last=False)
    assert st == oracle.SINGULAR
    rows, cols = oracle.root_lists(k, 0, 1, pad_last=True)
    assert rows == [1, k - 1] + list(range(2, k - 1)) + [0] and cols == [0, k - 1] + list(range(2, k - 1)) + [1]


# -------------------------------------------- residual, refinement, adjoint

def test_residual_and_refinement_are_second_order():
    k, b = 4, 4
    n = k * b
    m = bi.uniform_shift(n, 14)
    inv = np.linalg.inv(m)
    i, j = 1, 3
    xr, yc = inv[i * b:(i + 1) * b, :], inv[:, j * b:(j + 1) * b]
    assert np.abs(oracle.block_row_residual(m, xr, i, b)).max() < 1e-14
    for eps in (1e-4, 1e-6):
        dx = eps * bi.uniform_pm1(1, 1, b * n).reshape(b, n)
        dy = eps * bi.uniform_pm1(1, 2, n * b).reshape(n, b)
        fixed = oracle.refine_block(m, xr + dx, yc + dy, i, j, b)
        exact = inv[i * b:(i + 1) * b, j * b:(j + 1) * b]
        # the corrected block differs from N_ij by exactly -dX M dY
        assert np.allclose(fixed - exact, -(dx @ m @ dy), atol=1e-15 + 1e-9 * eps * eps)


def test_adjoint_against_central_differences():
    k, b = 4, 2
    n = k * b
    m = bi.spd(n, 1e1, 3)
    g = bi.gaussian_matrix(b, b, 5)
    i, j = 2, 1
    an = oracle.adjoint(np.linalg.inv(m), g, i, j, b)
    fd = np.zeros_like(m)
    h = 1e-6
    for r in range(n):
        for c in range(n):
            e = np.zeros_like(m)
            e[r, c] = h
            lp = np.sum(g * np.linalg.inv(m + e)[i * b:(i + 1) * b, j * b:(j + 1) * b])
            lm = np.sum(g * np.linalg.inv(m - e)[i * b:(i + 1) * b, j * b:(j + 1) * b])
            fd[r, c] = (lp - lm) / (2 * h)
    assert oracle.rel_fro(an, fd) < 1e-7


def test_sensitivity_floor_small_for_dominant_matrix():
    m = bi.uniform_shift(64, 1)
    f = oracle.sensitivity_floor(m, 4, 0, 0)
    assert 0.0 < f < 1e-14


def _scalar_floor(a, b_, c, d):
    """The floor of the k = 2, b = 1 case written out in IEEE double (Python
    floats, one rounding per operation, no fused multiply-add): the root is
    the leaf a - b d^-1 c (Eq. invSchur, E = (A - B D^-1 C)^-1), evaluated as
    b * (d^-1 * c) and as (b * d^-1) * c; N_00 is the inverse of each."""
    dinv = 1.0 / d
    n1 = 1.0 / (a - b_ * (dinv * c))
    n2 = 1.0 / (a - (b_ * dinv) * c)
    return abs(n2 - n1) / abs(n1), n1


def test_sensitivity_floor_pinned_on_scalars():
    """k = 2 with b = 1: every step of both evaluation orders is a single
    IEEE operation, so the floor is fixed by the arithmetic itself.  It must
    equal the written-out relative difference exactly, be nonzero where the
    two orders round differently, and be exactly zero where every operation
    is exact."""
    found_nonzero = 0
    for t in range(40):
        v = bi.uniform_pm1(77, t, 4)
        b_, c, d = float(v[1]) + 2.0, float(v[2]) + 2.0, float(v[3]) + 4.0
        # a close to b c / d: the difference cancels, so a rounding of the
        # product shows in N_00
        a = b_ * c / d + 1e-3 * float(v[0])
        m = np.array([[a, b_], [c, d]])
        want, n00 = _scalar_floor(a, b_, c, d)
        got, st, _ = oracle.bri_block(m, 2, 0, 0)
        assert st == oracle.OK and got[0, 0] == n00
        assert oracle.sensitivity_floor(m, 2, 0, 0) == want
        found_nonzero += want > 0.0
    # the re-association really rounds differently on generic inputs
    assert found_nonzero >= 10
    # small integers and a power-of-two pivot: every product and difference
    # is exact in both orders, so the floor is exactly zero
    m = np.array([[7.0, 3.0], [5.0, 4.0]])
    assert oracle.sensitivity_floor(m, 2, 0, 0) == 0.0


def test_sensitivity_floor_zero_when_products_are_exact():
    """k = 4, b = 2, block upper triangular with power-of-two diagonal blocks
    and small integers above: every pivot inverse and every Schur product is
    exact in either order, so the two evaluations agree bit for bit (floor
    exactly zero) and equal the dense inverse; strictly lower requests are
    structurally singular (Sec. 1: the inverted submatrices must be
    nonsingular)."""
    b, k = 2, 4
    m = np.zeros((k * b, k * b))
    for t in range(k):
        m[t * b:(t + 1) * b, t * b:(t + 1) * b] = np.diag([2.0 ** (t + 1), 2.0 ** t])
    ints = [1.0, -2.0, 3.0, 1.0, -1.0, 2.0]
    q = 0
    for r in range(k):
        for c in range(r + 1, k):
            m[r * b, c * b + 1] = ints[q % 6]
            m[r * b + 1, c * b] = ints[(q + 1) % 6]
            q += 1
    inv = np.linalg.inv(m)
    for i, j in [(0, 0), (0, 2), (1, 2), (1, 3), (3, 3)]:
        n_ij, st, _ = oracle.bri_block(m, k, i, j)
        assert st == oracle.OK
        assert np.allclose(n_ij, inv[i * b:(i + 1) * b, j * b:(j + 1) * b], rtol=0, atol=1e-15), (i, j)
        assert oracle.sensitivity_floor(m, k, i, j) == 0.0, (i, j)
    # a generic perturbation of the same matrix makes it nonzero
    m2 = m + 1e-3 * bi.uniform_pm1(5, 0, (k * b) ** 2).reshape(k * b, k * b)
    assert oracle.sensitivity_floor(m2, k, 1, 2) > 0.0
