"""Mixed path (tcgen05 BF16-slice Schur products, FP64 pivot inverses, FP32
frame values) and its refinement, against the CPU oracle through the C ABI.

Bounds: the FP32-grade sweep (3 slices) 1e-4 (the plain-FP32 tolerance) at
k = 4; the refined block 1e-10 (relative Frobenius error against the dense
inverse, the refined target)."""
import numpy as np
import pytest

import bri_inputs as bi
import oracle
from helpers import oracle_block, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mb():
    import paper_1612_00001_gb300 as mb
    mb.build()
    return mb


def test_mixed_sweep_small_config(mb):
    m = bi.uniform_shift(256, 0)
    M = torch.tensor(m, dtype=torch.float32, device="cuda")
    ctx = mb.Context(M, 4, precision="mixed", slices=3)
    ref32 = m.astype(np.float32).astype(np.float64)
    for i, j in [(0, 0), (1, 3), (3, 2)]:
        got = to_np(ctx.block(i, j))
        err = oracle.rel_fro(got, oracle_block(ref32, 4, i, j))
        assert err < 1e-4, (i, j, err)


@pytest.mark.parametrize("slices,tol", [(2, 5e-3), (1, 1.0)])
def test_mixed_fewer_slices_runs(mb, slices, tol):
    m = bi.uniform_shift(256, 0)
    M = torch.tensor(m, dtype=torch.float32, device="cuda")
    got = to_np(mb.Context(M, 4, precision="mixed", slices=slices).block(0, 0))
    err = oracle.rel_fro(got, np.linalg.inv(m)[:64, :64])
    assert np.isfinite(got).all() and err < tol, err


def test_mixed_ragged_block(mb):
    """b = 100 and b = 200: tiles with zero-padded edges."""
    for n, k in [(300, 3), (600, 3)]:
        m = bi.uniform_shift(n, 4, shift=n / 4)
        M = torch.tensor(m, dtype=torch.float32, device="cuda")
        ctx = mb.Context(M, k, precision="mixed")
        ref32 = m.astype(np.float32).astype(np.float64)
        for i, j in [(0, 0), (2, 1)]:
            got = to_np(ctx.block(i, j))
            err = oracle.rel_fro(got, oracle_block(ref32, k, i, j))
            assert err < 1e-4, (n, i, j, err)


def test_mixed_fp64_input(mb):
    m = bi.uniform_shift(256, 5)
    ctx = mb.Context(torch.tensor(m, device="cuda"), 4, precision="mixed")
    got = to_np(ctx.block(2, 1))
    assert oracle.rel_fro(got, oracle_block(m, 4, 2, 1)) < 1e-4


def test_mixed_refined_reaches_fp64_accuracy(mb):
    m = bi.uniform_shift(256, 0)
    ctx = mb.Context(torch.tensor(m, device="cuda"), 4, precision="mixed", refine=1)
    inv = np.linalg.inv(m)
    for i, j in [(0, 0), (0, 1), (3, 2)]:
        got = to_np(ctx.block(i, j))
        err = oracle.rel_fro(got, inv[i * 64:(i + 1) * 64, j * 64:(j + 1) * 64])
        assert err < 1e-10, (i, j, err)
        assert ctx.last_report["rel_residual"] < 1e-3


def _mixed_k8(mb, i, j):
    m = bi.uniform_shift(512, 2)
    M = torch.tensor(m, dtype=torch.float32, device="cuda")
    got = to_np(mb.Context(M, 8, precision="mixed").block(i, j))
    ref32 = m.astype(np.float32).astype(np.float64)
    floor = oracle.sensitivity_floor(ref32, 8, i, j)
    return got, oracle.rel_fro(got, oracle_block(ref32, 8, i, j)), floor


def test_mixed_k8_block00_meets_the_fp32_bar(mb):
    """n = 512, k = 8 (b = 64): 270 frames, grouped launches of up to 100
    products.  Block (0,0) meets the parity rule max(1e-4, 10 x floor)."""
    got, err, floor = _mixed_k8(mb, 0, 0)
    assert err <= max(1e-4, 10.0 * floor), (err, floor)


@pytest.mark.parametrize("i,j", [(5, 2), (7, 0)])
def test_mixed_k8_offdiagonal_misses_the_fp32_bar(mb, i, j):
    """The same matrix, off-diagonal blocks: the parity rule is NOT met and the
    test states so.  FP32 frame values carry unit roundoff 2^-24 and the k = 8
    recursion amplifies rounding by floor / 2^-53 (the oracle's own
    sensitivity at FP64), so the expected error is near 2^29 x floor, far
    above 10 x floor.  Asserted: the error is above the bar, and within
    10 x the floor scaled to FP32 unit roundoff (a wrong result still fails).
    One refinement step does not rescue such a sweep (its error squared
    stays far above 1e-10)."""
    got, err, floor = _mixed_k8(mb, i, j)
    bar = max(1e-4, 10.0 * floor)
    assert np.isfinite(got).all()
    assert err > bar, ("the FP32-valued sweep met the FP32 bar", err, bar)
    assert err <= 10.0 * 2.0 ** 29 * floor, (err, floor)


def test_mixed_refined_many_blocks_share_rows_and_columns(mb):
    """Refining all 16 blocks at once computes each needed block row and
    column once; every block still reaches the refined accuracy and equals
    the block refined alone."""
    m = bi.uniform_shift(256, 3)
    M = torch.tensor(m, device="cuda")
    ctx = mb.Context(M, 4, precision="mixed", refine=1)
    ij = [(i, j) for i in range(4) for j in range(4)]
    outs = ctx.blocks(ij)
    inv = np.linalg.inv(m)
    for (i, j), o in zip(ij, outs):
        got = to_np(o)
        assert oracle.rel_fro(got, inv[i * 64:(i + 1) * 64, j * 64:(j + 1) * 64]) < 1e-10, (i, j)
    alone = to_np(mb.Context(M, 4, precision="mixed", refine=1).block(2, 1))
    assert oracle.rel_fro(alone, to_np(outs[9])) < 1e-13
