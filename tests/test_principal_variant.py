"""The principal-Schur-complement variant (the reformulation around M/A that
Sec. 8 names as future work), on the CPU: the oracle's restatement pinned
against LAPACK, closed forms and IEEE arithmetic, and the library's schedule
of it interpreted on scalars (b = 1) against the oracle bit for bit."""
import ctypes

import numpy as np
import pytest

import bri_inputs as bi
import oracle


@pytest.mark.parametrize("k", [2, 3, 5, 6])
def test_variant_oracle_matches_dense_inverse(k):
    b = 4
    m = bi.uniform_shift(k * b, 40 + k)
    inv = np.linalg.inv(m)
    for i in range(k):
        for j in range(k):
            got, st = oracle.principal_block(m, k, i, j)
            assert st == oracle.OK
            assert oracle.rel_fro(got, inv[i * b:(i + 1) * b, j * b:(j + 1) * b]) < 1e-13, (k, i, j)


def test_variant_on_scalars_is_the_written_out_formula():
    """k = 2, b = 1: N_01 = -(b/a) / (d - c (b/a)) with 1/x inverses, each
    step one IEEE operation."""
    for t in range(20):
        v = bi.uniform_pm1(91, t, 4)
        a, b_, c, d = float(v[0]) + 3.0, float(v[1]), float(v[2]), float(v[3]) + 3.0
        m = np.array([[a, b_], [c, d]])
        z = (1.0 / a) * b_
        want = -(z * (1.0 / (d - c * z)))
        got, st = oracle.principal_block(m, 2, 0, 1)
        assert st == oracle.OK and got[0, 0] == want
        got, st = oracle.principal_block(m, 2, 1, 1)
        assert got[0, 0] == 1.0 / (d - c * ((1.0 / a) * b_))


def test_variant_block_diagonal_closed_form():
    """Block-diagonal M: N_ii = M_ii^-1 and every off-diagonal block is zero -
    where the paper's recursion meets singular non-principal pivots (Sec. 1:
    the inverted submatrices must be nonsingular)."""
    k, b = 4, 8
    m = bi.block_diagonal(k, b, 3)
    for i in range(k):
        got, st = oracle.principal_block(m, k, i, i)
        assert st == oracle.OK
        assert oracle.rel_fro(got, np.linalg.inv(m[i * b:(i + 1) * b, i * b:(i + 1) * b])) < 1e-14
    got, st = oracle.principal_block(m, k, 0, 3)
    assert st == oracle.OK and np.all(got == 0.0)
    _, st, _ = oracle.bri_block(m, k, 0, 3)
    assert st == oracle.SINGULAR


def test_variant_is_stable_where_the_recursion_is_not():
    """Haar U diag(sigma) V^T with cond 1e4, k = 6, b = 16: the paper's order
    loses most digits (its own sensitivity floor is far above the rounding
    level), the principal variant stays near cond x unit roundoff."""
    k, b = 6, 16
    m = bi.haar_svd(k * b, 1e4, 2)
    inv = np.linalg.inv(m)
    i, j = 1, 4
    ref = inv[i * b:(i + 1) * b, j * b:(j + 1) * b]
    paper, st, _ = oracle.bri_block(m, k, i, j)
    assert st == oracle.OK
    var, st = oracle.principal_block(m, k, i, j)
    assert st == oracle.OK
    e_paper, e_var = oracle.rel_fro(paper, ref), oracle.rel_fro(var, ref)
    assert e_var < 1e-10 and e_var < e_paper / 100, (e_paper, e_var)


@pytest.fixture(scope="module")
def interp():
    import paper_1612_00001_gb300 as mb
    mb.build()
    f = mb.test_lib().mbinv_debug_run_schedule_scalar
    dp = ctypes.POINTER(ctypes.c_double)
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                  ctypes.c_int, dp, dp, dp]
    f.restype = ctypes.c_int

    def go(m, k, i, j):
        m = np.ascontiguousarray(m, dtype=np.float64)
        flat = (ctypes.c_int * 2)(i, j)
        outs = np.zeros(1)
        stats = np.zeros(7)
        rc = f(k, 1, flat, 2, 0, 0, m.ctypes.data_as(dp), outs.ctypes.data_as(dp), stats.ctypes.data_as(dp))
        return rc, outs[0], stats
    return go


@pytest.mark.parametrize("k", [2, 3, 6, 9])
def test_variant_schedule_on_scalars_equals_oracle(interp, k):
    m = bi.uniform_shift(k, 17)
    for i, j in [(0, 0), (0, k - 1), (k - 1, 1), (k // 2, k // 2)]:
        rc, got, stats = interp(m, k, i, j)
        assert rc == 0
        want, st = oracle.principal_block(m, k, i, j)
        assert st == oracle.OK and got == want[0, 0], (k, i, j)
