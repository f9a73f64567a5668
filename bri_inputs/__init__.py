"""Seeded synthetic inputs for Block Recursive Inversion (BRI).

This module is shared by the CPU oracle's tests, the GPU parity tests and the
benchmark.  It holds no arithmetic of the inversion method itself: it only
draws matrices whose shapes and value distributions follow the workloads the
method is exercised on, plus the structured matrices whose inverses have
closed forms (block-diagonal, block-triangular).

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: draw number ``t`` of stream ``(seed, stream)`` is
``mix(base + (t + 1) * GOLDEN)`` with ``base = mix(seed ^ mix(stream))``, so
every element can be produced independently and on any machine bit-exactly.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream identifiers, so that different quantities drawn with the same seed
# never share random numbers.
STREAM_UNIFORM = 1
STREAM_GAUSS_U = 2
STREAM_GAUSS_V = 3
STREAM_GAUSS_Q = 4
STREAM_HOUSE = 5
STREAM_PAD = 6
STREAM_BATCH = 7
STREAM_W = 8
STREAM_STRUCT = 9


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws ``offset .. offset+count-1`` of the SplitMix64 stream (uint64)."""
    base = _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ _mix(np.uint64(stream)))
    t = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(base + t * GOLDEN)


def uniform01(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of each draw times 2^-53."""
    u = splitmix64(seed, stream, count, offset)
    return (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_pm1(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [-1, 1)."""
    return 2.0 * uniform01(seed, stream, count, offset) - 1.0


def gaussian(seed: int, stream: int, count: int) -> np.ndarray:
    """Standard normal draws by the Box-Muller transform of pairs of uniforms."""
    pairs = (count + 1) // 2
    u = uniform01(seed, stream, 2 * pairs)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * pairs)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


# ---------------------------------------------------------------- workloads

def uniform_shift(n: int, seed: int, shift: float | None = None) -> np.ndarray:
    """Entries i.i.d. uniform[-1, 1) plus ``shift * I`` (default ``n``):
    strictly diagonally dominant, the first two workloads' first family."""
    a = uniform_pm1(seed, STREAM_UNIFORM, n * n).reshape(n, n)
    a[np.diag_indices(n)] += float(n if shift is None else shift)
    return a


def haar_orthogonal(n: int, seed: int, stream: int) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a Gaussian matrix with the
    signs of R's diagonal moved into Q (Mezzadri, Notices AMS 54, 2007)."""
    g = gaussian(seed, stream, n * n).reshape(n, n)
    q, r = np.linalg.qr(g)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d[None, :]


def log_spaced(n: int, kappa: float) -> np.ndarray:
    """sigma_t = 10^(-log10(kappa) * t / (n - 1)), t = 0..n-1: from 1 down
    to 1/kappa, so the condition number is exactly kappa."""
    if n == 1:
        return np.ones(1)
    t = np.arange(n, dtype=np.float64)
    return 10.0 ** (-np.log10(kappa) * t / (n - 1))


def haar_svd(n: int, kappa: float, seed: int) -> np.ndarray:
    """M = U diag(sigma) V^T with Haar U, V and log-spaced sigma (cond = kappa)."""
    u = haar_orthogonal(n, seed, STREAM_GAUSS_U)
    v = haar_orthogonal(n, seed, STREAM_GAUSS_V)
    s = log_spaced(n, kappa)
    return (u * s[None, :]) @ v.T


def householder_product_apply(x: np.ndarray, vs: np.ndarray, side: str) -> np.ndarray:
    """Applies H_1 H_2 ... H_r (H = I - 2 v v^T / v^T v) to x from the left
    (``side='left'``) or its transpose from the right."""
    y = x.copy()
    if side == "left":
        for v in vs[::-1]:
            y -= (2.0 / (v @ v)) * np.outer(v, v @ y)
    else:
        for v in vs[::-1]:
            y -= (2.0 / (v @ v)) * np.outer(y @ v, v)
    return y


def householder_svd(n: int, kappa: float, seed: int, reflectors: int = 64) -> np.ndarray:
    """M = U diag(sigma) V^T where U and V are each a product of ``reflectors``
    Householder reflections with Gaussian vectors (small n only on the host)."""
    vu = gaussian(seed, STREAM_HOUSE, reflectors * n).reshape(reflectors, n)
    vv = gaussian(seed + 0x5151, STREAM_HOUSE, reflectors * n).reshape(reflectors, n)
    s = log_spaced(n, kappa)
    m = np.diag(s)
    m = householder_product_apply(m, vu, "left")
    m = householder_product_apply(m, vv, "right")
    return m


def spd(n: int, kappa: float, seed: int) -> np.ndarray:
    """Symmetric positive definite M = Q diag(mu) Q^T, Q Haar, eigenvalues
    mu_t log-spaced in [1, kappa] so that cond(M) = kappa."""
    q = haar_orthogonal(n, seed, STREAM_GAUSS_Q)
    mu = 1.0 / log_spaced(n, kappa)
    m = (q * mu[None, :]) @ q.T
    return 0.5 * (m + m.T)


def gaussian_matrix(rows: int, cols: int, seed: int, stream: int = STREAM_W) -> np.ndarray:
    return gaussian(seed, stream, rows * cols).reshape(rows, cols)


# ---------------------------------------------------- structured test inputs

def block_diagonal(k: int, b: int, seed: int) -> np.ndarray:
    """k x k block-diagonal matrix with diagonally dominant diagonal blocks."""
    n = k * b
    m = np.zeros((n, n))
    for t in range(k):
        blk = uniform_pm1(seed, STREAM_STRUCT, b * b, offset=t * b * b).reshape(b, b)
        blk[np.diag_indices(b)] += b
        m[t * b:(t + 1) * b, t * b:(t + 1) * b] = blk
    return m


def block_upper_triangular(k: int, b: int, seed: int) -> np.ndarray:
    """Dense blocks on and above the block diagonal, zero below it."""
    n = k * b
    m = uniform_shift(n, seed)
    for r in range(k):
        for c in range(r):
            m[r * b:(r + 1) * b, c * b:(c + 1) * b] = 0.0
    return m


def pad_columns(n: int, l: int, seed: int) -> np.ndarray:
    """The n x l uniform[-1, 1) coupling block used when a matrix whose order
    is not a multiple of k is bordered up to a multiple (see the padding
    reading in the library's documentation)."""
    return uniform_pm1(seed, STREAM_PAD, n * l).reshape(n, l)


def ragged_batch(count: int, seed: int, nmin: int = 256, nmax: int = 4096,
                 kmin: int = 2, kmax: int = 8, round_to: int = 64):
    """Problem list of the batched uneven workload: n uniform in [nmin, nmax]
    rounded to a multiple of ``round_to``, k uniform in {kmin..kmax}, one block
    (i, j) drawn uniformly.  Returns a list of dicts (n, k, i, j, seed)."""
    u = uniform01(seed, STREAM_BATCH, 4 * count).reshape(count, 4)
    out = []
    for t in range(count):
        n = nmin + int(u[t, 0] * (nmax - nmin + 1))
        n = max(round_to, int(round(n / round_to)) * round_to)
        n = min(max(n, nmin), nmax)
        k = kmin + int(u[t, 1] * (kmax - kmin + 1))
        i = int(u[t, 2] * k)
        j = int(u[t, 3] * k)
        out.append(dict(n=n, k=k, i=i, j=j, seed=seed * 100003 + t))
    return out
