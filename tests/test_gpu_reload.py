"""mbinv_reload: a context re-reads M after the caller changed its contents
(the next matrix of a stream of one shape), keeping its plans, workspace and
captured launch graphs.  The blocks after a reload must be bit for bit those
of a fresh context on the new matrix, and the new matrix's blocks must match
the oracle at the FP64 bar max(1e-11, 10 x floor) (where k divides n)."""
import numpy as np
import pytest

import bri_inputs as bi
from helpers import oracle_block, parity_tol, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mb():
    import paper_1612_00001_gb300 as mb
    mb.build()
    return mb


REQ = [(0, 1), (2, 2), (3, 0)]


def blocks_of(ctx):
    return [to_np(o) for o in ctx.blocks(REQ)]


@pytest.mark.parametrize("where,n,prec,dt", [("host", 512, "fp64_tc", "f64"), ("host", 512, "fp64", "f64"),
                                             ("device", 512, "fp64_tc", "f64"),
                                             ("device_padded", 510, "fp64_tc", "f64"),
                                             ("device", 512, "fp64_tc", "f32")])
def test_reload_equals_a_fresh_context(mb, where, n, prec, dt):
    """dt = f32: an FP32 M on an FP64-valued path is converted on the device
    (staged, then widened) at creation and again at every reload."""
    k = 4
    tdt = torch.float64 if dt == "f64" else torch.float32
    m1, m2 = bi.uniform_shift(n, 1), bi.uniform_shift(n, 2)
    if dt == "f32":
        m2 = m2.astype(np.float32).astype(np.float64)  # the values the context sees
    if where == "host":
        buf = torch.tensor(m1, dtype=tdt).pin_memory()
    else:
        buf = torch.tensor(m1, dtype=tdt, device="cuda")
    ctx = mb.Context(buf, k, precision=prec, out_dtype=torch.float64)
    first = blocks_of(ctx)
    ctx.reload(torch.tensor(m2, dtype=tdt))
    torch.cuda.synchronize()
    got = blocks_of(ctx)
    fresh_buf = torch.tensor(m2, dtype=tdt, device="cuda" if where != "host" else "cpu")
    with mb.Context(fresh_buf, k, precision=prec, out_dtype=torch.float64) as fresh:
        want = blocks_of(fresh)
    for (i, j), a, b_, f in zip(REQ, got, want, first):
        assert np.array_equal(a, b_), (where, i, j)
        assert not np.array_equal(a, f), (where, i, j)
        if n % k:
            continue  # the bordered matrix's parity is pinned by the padding tests
        tol, floor = parity_tol(m2, k, i, j, 1e-11)
        ref = oracle_block(m2, k, i, j)
        err = np.linalg.norm(a - ref) / np.linalg.norm(ref)
        assert err <= tol, (where, i, j, err, tol)
    ctx.close()


def test_reload_of_a_produced_matrix_is_refused_on_the_python_side_only(mb):
    """A context that produces M has nothing to re-read: the binding refuses
    new contents, the C call itself returns MBINV_OK."""
    x = torch.randn(255, 4, dtype=torch.float64, device="cuda")
    ctx = mb.Context.from_rbf(x, 4, 2.0, 10.0)
    with pytest.raises(ValueError):
        ctx.reload(torch.zeros(256, 256, dtype=torch.float64))
    ctx.reload()
    ctx.close()
