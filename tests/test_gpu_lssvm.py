"""The LS-SVM application without storing M (Sec. 5 and Sec. 7, Eq. A):
A_gamma = [[0, 1^T], [1, K + I/gamma]] with the RBF kernel of Gaussian points,
produced block by block on the GPU by the library's producer and never
stored; only the blocks near the diagonal are requested (what the
cross-validation of LS-SVMs reads).

Inputs: n = 2047 points of dimension 8 drawn N(0, 1) (the paper draws randn
points; it prints neither n, dim, sigma nor gamma: sigma = 2, gamma = 10
here), so A_gamma has order 2048 = 8 x 256."""
import ctypes

import numpy as np
import pytest

import bri_inputs as bi
import oracle
from helpers import oracle_block, parity_tol, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NPTS, DIM, SIGMA, GAMMA, K = 2047, 8, 2.0, 10.0, 8


@pytest.fixture(scope="module")
def mb():
    import paper_1612_00001_gb300 as mb
    mb.build()
    return mb


def a_gamma(x, sigma, gamma):
    """Eq. A written out (numpy, FP64)."""
    d2 = ((x[:, None, :] - x[None, :, :]) ** 2).sum(-1)
    kg = np.exp(-d2 / (2.0 * sigma * sigma)) + np.eye(x.shape[0]) / gamma
    n = x.shape[0]
    a = np.zeros((n + 1, n + 1))
    a[0, 1:] = 1.0
    a[1:, 0] = 1.0
    a[1:, 1:] = kg
    return a


@pytest.fixture(scope="module")
def points():
    return bi.gaussian_matrix(NPTS, DIM, 31)


def produced_matrix(mb, x):
    """The producer called directly for the whole matrix (test only)."""
    L = mb.lib()
    p = mb.Rbf(x.data_ptr(), NPTS, DIM, SIGMA, GAMMA)
    a = torch.empty((NPTS + 1, NPTS + 1), dtype=torch.float64, device="cuda")
    rc = L.mbinv_rbf_block(0, 0, NPTS + 1, NPTS + 1, a.data_ptr(), NPTS + 1, 0,
                           torch.cuda.current_stream().cuda_stream, ctypes.cast(ctypes.pointer(p), ctypes.c_void_p))
    assert rc == 0
    torch.cuda.synchronize()
    return to_np(a)


def test_producer_matches_eq_a(mb, points):
    x = torch.tensor(points, device="cuda")
    got = produced_matrix(mb, x)
    ref = a_gamma(points, SIGMA, GAMMA)
    assert got[0, 0] == 0.0 and np.all(got[0, 1:] == 1.0) and np.all(got[1:, 0] == 1.0)
    assert np.abs(got - ref).max() <= 4e-16 * np.abs(ref).max()


@pytest.mark.parametrize("prec", ["fp64_tc", "fp64"])
def test_near_diagonal_blocks_without_storing_the_matrix(mb, points, prec):
    """Blocks (i, i) and (i, i +- 1) of A_gamma^-1 from the produced matrix,
    under a cap of half of A_gamma's own bytes (the device never holds
    A_gamma, nor half of it beside the workspace), against the oracle run on the
    same entries, at the FP64 bar max(1e-11, 10 x floor)."""
    x = torch.tensor(points, device="cuda")
    a = produced_matrix(mb, x)
    m = NPTS + 1
    cap = m * m * 8 // 2
    ctx = mb.Context.from_rbf(x, K, SIGMA, GAMMA, precision=prec, cap=cap)
    ij = [(i, i) for i in range(K)] + [(i, i + 1) for i in range(K - 1)] + [(i + 1, i) for i in range(K - 1)]
    outs = [to_np(o) for o in ctx.blocks(ij)]
    rep = ctx.last_report
    assert rep["peak_device_bytes"] <= cap
    assert rep["frames"] < rep["request_frames"]
    for (i, j), got in zip(ij, outs):
        tol, floor = parity_tol(a, K, i, j, 1e-11)
        err = oracle.rel_fro(got, oracle_block(a, K, i, j))
        assert err <= tol, (prec, i, j, err, tol)
    # symmetric matrix: N_ji and N_ij^T are two runs of the recursion, equal
    # within its sensitivity
    tol, floor = parity_tol(a, K, 2, 1, 1e-11)
    assert oracle.rel_fro(outs[K + 1].T, outs[2 * K]) <= (tol if prec == "fp64" else 2 ** 7 * tol)
    ctx.close()
