"""The unrefined sweep at the bench's block size: n = 4096, k = 8 (b = 512),
uniform[-1,1) + n I, on both FP64-valued paths, sampled blocks against the
oracle (the memoized recursion in plain FP64) element by element at the FP64
bar max(1e-11, 10 x floor).  This reaches the b = 512 tile and K paths of the
digit products (one K chunk of 512) and of the FP64 tile products, and the
64-column panels of the pivot inverses, in the same grouped launches the
bench uses (all sampled blocks' runs executed together)."""
import numpy as np
import pytest

import bri_inputs as bi
import oracle
from helpers import oracle_block, parity_tol, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-11
N, K = 4096, 8
BLOCKS = [(0, 0), (2, 5)]


@pytest.fixture(scope="module")
def mb():
    import paper_1612_00001_gb300 as mb
    mb.build()
    return mb


@pytest.fixture(scope="module")
def matrix_and_refs():
    m = bi.uniform_shift(N, 0)
    refs = {}
    for i, j in BLOCKS:
        tol, floor = parity_tol(m, K, i, j, TOL_FP64)
        refs[i, j] = (oracle_block(m, K, i, j), tol, floor)
    return m, refs


@pytest.mark.parametrize("prec", ["fp64_tc", "fp64"])
def test_unrefined_b512_against_oracle(mb, matrix_and_refs, prec):
    m, refs = matrix_and_refs
    with mb.Context(torch.tensor(m, device="cuda"), K, precision=prec, refine=0) as ctx:
        outs = [to_np(x) for x in ctx.blocks(BLOCKS, width=len(BLOCKS))]
        assert 0 < ctx.last_report["frames"] <= 270 * len(BLOCKS)
    for (i, j), got in zip(BLOCKS, outs):
        ref, tol, floor = refs[i, j]
        assert np.isfinite(got).all()
        err = oracle.rel_fro(got, ref)
        assert err <= tol, (prec, i, j, err, tol, floor)
