"""The digit-split FP64 product on the tensor cores, alone (through a test
hook of libmbinv, not the public header).

Two kinds of check:
* bit for bit against the same scheme written out with Python integers
  (row exponents, 56-bit fixed point, balanced base-128 digits, the 36 digit
  pairs with p + q <= 7, one rounding of the exact integer sum, one rounding
  of the Schur update), which pins the kernel's arithmetic exactly;
* against an FP64 product, within the scheme's error bound
  |err_ij| <= K 2^-53 max|a_i.| max|b_.j| (dropped pairs and the rounding of
  the fixed-point entries) plus FP64 rounding of the result.
"""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KCHUNK = 512  # K of one exact accumulation


@pytest.fixture(scope="module")
def hook():
    import paper_1612_00001_gb300 as mb
    mb.build()
    f = mb.test_lib().mbinv_debug_oz_gemm
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int] * 4 + [ctypes.c_double] * 2 + [ctypes.c_void_p]
    return f


def run(hook, A, B, Cin, alpha, beta):
    """A (count, m, k), B (count, k, n), Cin (count, m, n) or None; numpy FP64."""
    count, m, k = A.shape
    n = B.shape[2]
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    dCin = torch.from_numpy(np.ascontiguousarray(Cin)).cuda() if Cin is not None else None
    dC = torch.full((count, m, n), float("nan"), dtype=torch.float64, device="cuda")
    rc = hook(dA.data_ptr(), dB.data_ptr(), dCin.data_ptr() if dCin is not None else None, dC.data_ptr(),
              m, n, k, count, alpha, beta, torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    return dC.cpu().numpy()


# ------------------------------------------------------------------ the scheme with Python integers
def row_exponents(M):
    """E_r with 2^E_r > max |M[r, :]| (the frexp exponent of the maximum)."""
    mx = np.max(np.abs(M), axis=1)
    return np.array([math.frexp(float(v))[1] if v != 0 else 0 for v in mx], dtype=np.int64)


def digits(M, E):
    """Balanced base-128 digits (8, rows, K) of round(M 2^(55 - E)), ties away from zero."""
    mant, ex = np.frexp(M)
    Mi = (np.abs(mant) * 2.0 ** 53).astype(np.int64)  # |M| = Mi 2^(ex - 53), exact
    sh = ex.astype(np.int64) + 2 - E[:, None]
    X = np.zeros(M.shape, dtype=np.int64)
    pos = sh >= 0
    X[pos] = Mi[pos] << sh[pos]
    neg = (~pos) & (sh >= -54)
    r = -sh[neg]
    X[neg] = (Mi[neg] + (np.int64(1) << (r - 1))) >> r
    X = np.where(M < 0, -X, X)
    d = np.zeros((8,) + M.shape, dtype=np.int64)
    for p in range(7, 0, -1):
        rr = X & 127
        rr = np.where(rr >= 64, rr - 128, rr)
        d[p] = rr
        X = (X - rr) >> 7
    d[0] = X
    assert np.all(np.abs(d) <= 64)
    return d


def scheme(A, B, Cin, alpha, beta):
    """out = beta Cin + alpha A B for one problem, as the kernel computes it."""
    m, k = A.shape
    n = B.shape[1]
    EA, EB = row_exponents(A), row_exponents(B.T)
    dA, dB = digits(A, EA), digits(np.ascontiguousarray(B.T), EB)
    out = np.zeros((m, n)) if Cin is None else Cin.copy()
    for c, k0 in enumerate(range(0, k, KCHUNK)):
        sl = slice(k0, min(k, k0 + KCHUNK))
        G = np.zeros((8, m, n), dtype=np.int64)
        for p in range(8):
            for q in range(8 - p):
                G[p + q] += dA[p][:, sl] @ dB[q][:, sl].T
        assert np.all(np.abs(G) <= 2 ** 24)
        b_ = beta if c == 0 else 1.0
        for i in range(m):
            for j in range(n):
                S = sum(int(G[g, i, j]) * 128 ** (7 - g) for g in range(8))
                v = math.ldexp(float(S), int(EA[i] + EB[j] - 61))  # float(S): one rounding, ties to even
                y = alpha * v
                if Cin is None and c == 0:
                    out[i, j] = y
                elif b_ == 1.0:
                    out[i, j] = out[i, j] + y
                else:
                    out[i, j] = math.fma(b_, out[i, j], y) if hasattr(math, "fma") else b_ * out[i, j] + y
    return out


def operands(count, m, n, k, seed, spread=20):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((count, m, k)) * np.exp2(rng.integers(-spread, spread + 1, (count, m, 1)))
    B = rng.standard_normal((count, k, n)) * np.exp2(rng.integers(-spread, spread + 1, (count, 1, n)))
    C = rng.standard_normal((count, m, n))
    return A, B, C


@pytest.mark.parametrize("m,n,k,count", [(128, 64, 64, 1), (200, 100, 300, 2), (130, 70, 600, 1)])
def test_bitwise_against_integer_scheme(hook, m, n, k, count):
    A, B, C = operands(count, m, n, k, seed=m + n + k)
    for alpha, beta, cin in [(-1.0, 1.0, C), (1.0, 0.0, None)]:
        got = run(hook, A, B, cin, alpha, beta)
        for g in range(count):
            want = scheme(A[g], B[g], None if cin is None else cin[g], alpha, beta)
            assert np.array_equal(got[g], want), (alpha, g, np.max(np.abs(got[g] - want)))


def test_bitwise_with_group_sums_past_2_22(hook):
    """Entries whose six leading balanced digits are all 63 make the group
    sums of K = 512 exceed 2^22 (group 5: 6 pairs x 512 x 63^2 > 2^23), where
    the epilogue's FP32-add shortcut would not be exact: the warps holding
    such rows must take the conversions.  Rows 0-15 and 64-79 of A hold the
    value, the others random entries (warps see both), and the result is still
    the integer scheme bit for bit."""
    x = 63.0 * sum(128.0 ** (7 - p) for p in range(6)) * 2.0 ** -55  # digits 63 x 6, 0, 0 (row exponent 0)
    E = row_exponents(np.array([[x]]))
    d = digits(np.array([[x]]), E)
    assert [int(v) for v in d[:, 0, 0]] == [63] * 6 + [0, 0]
    rng = np.random.default_rng(12)
    m, n, k = 128, 64, 512
    A = rng.standard_normal((1, m, k))
    A[0, 0:16, :] = x
    A[0, 64:80, :] = x
    B = np.full((1, k, n), x)
    B[0, :, 40:] = rng.standard_normal((k, n - 40))
    C = rng.standard_normal((1, m, n))
    G5 = 6 * k * 63 * 63
    assert G5 > 2 ** 22
    got = run(hook, A, B, C, -1.0, 1.0)
    want = scheme(A[0], B[0], C[0], -1.0, 1.0)
    assert np.array_equal(got[0], want), np.max(np.abs(got[0] - want))


def bound(A, B, ref, k):
    amax = np.max(np.abs(A), axis=2, keepdims=True)
    bmax = np.max(np.abs(B), axis=1, keepdims=True)
    return k * 2.0 ** -53 * amax * bmax + 4 * 2.0 ** -53 * np.abs(ref)


@pytest.mark.parametrize("m,n,k,count,spread", [(512, 512, 512, 3, 0), (1000, 700, 1200, 1, 10),
                                                (64, 64, 16, 4, 30)])
def test_fp64_accuracy(hook, m, n, k, count, spread):
    A, B, C = operands(count, m, n, k, seed=7 + k, spread=spread)
    got = run(hook, A, B, C, -1.0, 1.0)
    tA, tB, tC = (torch.from_numpy(x).cuda() for x in (A, B, C))
    ref = (tC - torch.bmm(tA, tB)).cpu().numpy()
    err = np.abs(got - ref)
    assert np.all(err <= bound(A, B, ref, k)), float(np.max(err / bound(A, B, ref, k)))


def test_non_finite_rows_and_zero_operands(hook):
    A, B, C = operands(1, 128, 128, 128, seed=3, spread=0)
    A[0, 5, 17] = np.nan
    B[0, 9, 40] = np.inf  # column 40 of B
    got = run(hook, A, B, C, -1.0, 1.0)
    ref = C[0] - A[0] @ B[0]
    assert np.all(np.isnan(got[0, 5, :]))
    assert np.all(np.isnan(got[0, :, 40]))
    mask = np.ones((128, 128), bool)
    mask[5, :] = False
    mask[:, 40] = False
    assert np.allclose(got[0][mask], ref[mask], rtol=1e-13, atol=1e-12)
    Z = np.zeros_like(A)
    got = run(hook, Z, np.zeros_like(B), C, -1.0, 1.0)
    assert np.array_equal(got, C)
