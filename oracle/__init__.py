"""CPU oracle for Block Recursive Inversion (arXiv:1612.00001).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``.  The library never imports it and
it imports nothing from the library.

The arithmetic of the paper's recursion lives in ``bri_oracle.c`` (plain C,
FP64, no fused multiply-add); this module loads it with ctypes and adds the
plain definitions the tests compare against:

* ``bri_block``          N_ij by the recursion, literal (memo=False, O1) or
                         memoized on frame identity (memo=True, O2).
* ``dense_inverse``      M^-1 by Gauss-Jordan with partial pivoting (O3).
* ``augment``            the bordered matrix of Sec. 3 (Eq. M_augmented) and
                         the coupled variant used for requests that touch the
                         padded block.
* ``block_row_residual`` E_i^T - X_i M, the defining property of block row i
                         of the inverse.
* ``refine_block``       N_ij <- X_i E_j + (E_i^T - X_i M) Y_j.
* ``adjoint``            dL/dM = -(M^-T)[:, rows i] G (M^-T)[cols j, :].
* ``principal_block``    N_ij by the principal-Schur-complement variant.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, SINGULAR = 0, 1, 2, 3
ROLE = {"A": 0, "B": 1, "C": 2, "D": 3}


def build(force: bool = False) -> str:
    """Compiles bri_oracle.c with gcc (OpenMP, no FP contraction)."""
    src = os.path.join(_HERE, "bri_oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", src, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            i64, dp, ip = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
            L.orc_matmul.argtypes = [i64, i64, i64, dp, i64, dp, i64, dp, i64]
            L.orc_matmul.restype = None
            L.orc_gj_inverse.argtypes = [i64, dp, i64, dp, i64]
            L.orc_gj_inverse.restype = ctypes.c_int
            L.orc_bri_frame.argtypes = [dp, i64, i64, ip, ip, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                        ctypes.POINTER(ctypes.c_int64)]
            L.orc_bri_frame.restype = ctypes.c_int
            L.orc_bri_block.argtypes = [dp, i64, i64, i64, i64, i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                        ctypes.POINTER(ctypes.c_int64)]
            L.orc_bri_block.restype = ctypes.c_int
            L.orc_root_lists.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ip]
            L.orc_root_lists.restype = None
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_set_num_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(t: int) -> None:
    lib().orc_set_num_threads(int(t))


# --------------------------------------------------------------- primitives

def matmul(a, b) -> np.ndarray:
    """Plain triple-loop product (sum in increasing inner index, no FMA)."""
    a, b = _f64(a), _f64(b)
    m, kk = a.shape
    kk2, n = b.shape
    assert kk == kk2
    c = np.empty((m, n))
    lib().orc_matmul(m, n, kk, _dp(a), kk, _dp(b), n, _dp(c), n)
    return c


def gj_inverse(a):
    """(X, status): Gauss-Jordan inverse with partial pivoting (first max)."""
    a = _f64(a)
    n = a.shape[0]
    x = np.empty_like(a)
    st = lib().orc_gj_inverse(n, _dp(a), n, _dp(x), n)
    return x, st


def dense_inverse(m):
    """O3: the whole inverse by Gauss-Jordan with partial pivoting."""
    return gj_inverse(m)


def root_lists(k: int, i: int, j: int, pad_last: bool = False):
    r = (ctypes.c_int * k)()
    c = (ctypes.c_int * k)()
    lib().orc_root_lists(k, i, j, int(pad_last), r, c)
    return list(r), list(c)


def bri_frame(m, b: int, rows, cols, role, piv_row: int, piv_col: int, memo=False, reassoc=False):
    """Value of one frame (ordered block-row and block-column lists, role
    'A'..'D').  Returns (value, status, stats)."""
    m = _f64(m)
    p = len(rows)
    r = (ctypes.c_int * p)(*rows)
    c = (ctypes.c_int * p)(*cols)
    out = np.empty((b, b))
    stats = (ctypes.c_int64 * 4)()
    role = ROLE[role] if isinstance(role, str) else int(role)
    st = lib().orc_bri_frame(_dp(m), m.shape[1], b, r, c, p, role, piv_row, piv_col, int(memo), int(reassoc),
                             _dp(out), stats)
    return out, st, dict(schur_ops=stats[0], inversions=stats[1], frames=stats[2], memo_hits=stats[3])


def bri_block(m, k: int, i: int, j: int, memo: bool = True, reassoc: bool = False, pad_last: bool = False):
    """N_ij by the paper's recursion.  m must be (k*b) x (k*b); pad_last
    marks a matrix bordered by augment() (see root_lists).  Returns
    (N_ij, status, stats)."""
    m = _f64(m)
    n = m.shape[0]
    assert n % k == 0, "use augment() first when k does not divide n"
    b = n // k
    out = np.empty((b, b))
    stats = (ctypes.c_int64 * 4)()
    st = lib().orc_bri_block(_dp(m), n, k, b, i, j, int(memo), int(reassoc), int(pad_last), _dp(out), stats)
    return out, st, dict(schur_ops=stats[0], inversions=stats[1], frames=stats[2], memo_hits=stats[3])


# ------------------------------------------------------------ augmentation

def augment(m, k: int, i: int | None = None, j: int | None = None, coupling=None):
    """Borders M (n x n) up to order k*b, b = ceil(n/k), l = k*b - n.

    Plain reading (Eq. M_augmented): Gamma = [[M, 0], [0, I_l]], so that
    Gamma^-1 = diag(M^-1, I_l) (Eq. inverse_M_augmented).  Every off-diagonal
    block of Gamma^-1 that touches the padded rows or columns is then
    singular and cannot come out of the recursion, so for a request (i, k-1)
    with i != k-1 the border is [[M, B'], [0, I]] (inverse [[M^-1, -M^-1 B'],
    [0, I]]), and for (k-1, j) it is [[M, 0], [C', I]] (inverse
    [[M^-1, 0], [-C' M^-1, I]]); the top-left n x n block of the inverse is
    M^-1 either way.  ``coupling`` is B' (n x l) or C'^T (n x l).  Requests
    that do not touch the last block keep the plain border and must be run
    with pad_last=True (the padded block becomes the pivot index; with it
    anywhere else, frames that keep the padded rows are singular).
    Returns (Gamma, b, l)."""
    m = _f64(m)
    n = m.shape[0]
    b = -(-n // k)
    l = k * b - n
    g = np.zeros((k * b, k * b))
    g[:n, :n] = m
    g[n:, n:] = np.eye(l)
    if l and i is not None and j is not None and i != j:
        if coupling is None:
            raise ValueError("coupling block required for a request touching the padded block")
        cpl = _f64(coupling)
        if j == k - 1:
            g[:n, n:] = cpl
        elif i == k - 1:
            g[n:, :n] = cpl.T
    return g, b, l


# ------------------------------------------------------- plain definitions

def block_row_residual(m, x_row, i: int, b: int) -> np.ndarray:
    """E_i^T - X_i M for X_i (b x n): zero exactly when X_i is block row i of M^-1."""
    m = _f64(m)
    r = -(_f64(x_row) @ m)
    r[:, i * b:(i + 1) * b] += np.eye(b)
    return r


def refine_block(m, x_row, y_col, i: int, j: int, b: int) -> np.ndarray:
    """One two-sided correction N_ij <- X_i E_j + (E_i^T - X_i M) Y_j.  With
    dX = X_i - (M^-1)_{i,:} and dY = Y_j - (M^-1)_{:,j} the corrected block
    differs from N_ij by -dX M dY."""
    x_row, y_col = _f64(x_row), _f64(y_col)
    r = block_row_residual(m, x_row, i, b)
    return x_row[:, j * b:(j + 1) * b] + r @ y_col


def adjoint(minv, g, i: int, j: int, b: int) -> np.ndarray:
    """dL/dM for L = sum(G * (M^-1)_ij): -(M^-1)^T[:, rows of block i] G
    (M^-1)^T[cols of block j, :], i.e. -(X_i)^T G (Y_j)^T."""
    minv = _f64(minv)
    x_row = minv[i * b:(i + 1) * b, :]
    y_col = minv[:, j * b:(j + 1) * b]
    return -(x_row.T @ _f64(g) @ y_col.T)


def principal_block(m, k: int, i: int, j: int):
    """N_ij by the principal-Schur-complement variant (the reformulation
    around M/A, Eq. SchurofA, that Sec. 8 names as future work): the blocks
    other than i and j are eliminated in ascending order,
        S[r][q] <- S[r][q] - S[r][c] (S[c][c]^-1 S[c][q]),
    each pivot S[c][c] a principal Schur complement; then N_ii = S_ii^-1, or
    N_ij = -(S_ii^-1 S_ij) (S_jj - S_ji S_ii^-1 S_ij)^-1 for i != j.  Products
    and inverses are the oracle's own (plain loops, Gauss-Jordan).  Returns
    (N_ij, status)."""
    m = _f64(m)
    n = m.shape[0]
    assert n % k == 0
    b = n // k
    S = {(r, q): m[r * b:(r + 1) * b, q * b:(q + 1) * b].copy() for r in range(k) for q in range(k)}
    order = [x for x in range(k) if x not in (i, j)]
    alive = order + ([i] if i == j else [i, j])
    for t, c in enumerate(order):
        p, st = gj_inverse(S[c, c])
        if st:
            return None, st
        rest = alive[t + 1:]
        z = {q: matmul(p, S[c, q]) for q in rest}
        for r in rest:
            for q in rest:
                S[r, q] = S[r, q] - matmul(S[r, c], z[q])
    pi, st = gj_inverse(S[i, i])
    if st:
        return None, st
    if i == j:
        return pi, OK
    z = matmul(pi, S[i, j])
    t_ = S[j, j] - matmul(S[j, i], z)
    ti, st = gj_inverse(t_)
    if st:
        return None, st
    return -matmul(z, ti), OK


def rel_fro(a, ref) -> float:
    a, ref = np.asarray(a, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    d = np.linalg.norm(ref)
    return float(np.linalg.norm(a - ref) / (d if d > 0 else 1.0))


def sensitivity_floor(m, k: int, i: int, j: int, pad_last: bool = False) -> float:
    """|O2 - O2'|_F / |O2|_F where O2' evaluates every Schur product as
    (left * pivot^-1) * right instead of left * (pivot^-1 * right): the
    method's own sensitivity to the order of rounding."""
    a, st, _ = bri_block(m, k, i, j, memo=True, reassoc=False, pad_last=pad_last)
    b_, st2, _ = bri_block(m, k, i, j, memo=True, reassoc=True, pad_last=pad_last)
    if st or st2:
        return float("nan")
    return rel_fro(b_, a)
