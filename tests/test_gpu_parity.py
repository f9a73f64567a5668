"""GPU path against the CPU oracle, through the C ABI (libmbinv.so).

Every comparison is element by element on the same seeded inputs; the bound
is max(fixed tolerance, 10 x the oracle's own sensitivity floor), written in
each test.  The fixed tolerances: 1e-11 (FP64), 1e-4 (FP32)."""
import itertools

import numpy as np
import pytest

import bri_inputs as bi
import oracle
from helpers import oracle_block, parity_tol, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-11
TOL_FP32 = 1e-4


@pytest.fixture(scope="module")
def mb():
    import paper_1612_00001_gb300 as mb
    mb.build()
    return mb


def dev(a, dtype=torch.float64):
    return torch.tensor(a, dtype=dtype, device="cuda")


@pytest.mark.parametrize("i,j", [(0, 0), (1, 3), (3, 0), (2, 2)])
def test_fp64_small_config_blocks(mb, i, j):
    """n=256, k=4 (b=64), uniform[-1,1] + n I."""
    m = bi.uniform_shift(256, 0)
    ctx = mb.Context(dev(m), 4, precision="fp64")
    got = to_np(ctx.block(i, j))
    ref = oracle_block(m, 4, i, j)
    tol, floor = parity_tol(m, 4, i, j, TOL_FP64)
    err = oracle.rel_fro(got, ref)
    assert err <= tol, (err, tol, floor)
    rep = ctx.last_report
    assert rep["frames"] == 14 and rep["inversions"] == 4  # P, 2 distinct pivots, root


def test_fp64_all_blocks_against_dense_inverse(mb):
    m = bi.uniform_shift(256, 1)
    ctx = mb.Context(dev(m), 4)
    full = to_np(ctx.all_blocks())
    dense, st = oracle.dense_inverse(m)
    assert st == oracle.OK
    for i, j in itertools.product(range(4), range(4)):
        s = np.s_[i * 64:(i + 1) * 64, j * 64:(j + 1) * 64]
        assert oracle.rel_fro(full[s], dense[s]) < 1e-12, (i, j)


@pytest.mark.parametrize("n,k", [(300, 3), (600, 3), (400, 2), (520, 5)])
def test_fp64_ragged_tiles_and_blocked_inverse(mb, n, k):
    """b = 100, 200, 200, 104: tiles with ragged edges; b > 128 takes the
    blocked elimination with a ragged last panel."""
    m = bi.uniform_shift(n, 3, shift=n / 8)
    ctx = mb.Context(dev(m), k)
    for i, j in [(0, 0), (k - 1, 0), (1, k - 1)]:
        got = to_np(ctx.block(i, j))
        ref = oracle_block(m, k, i, j)
        tol, floor = parity_tol(m, k, i, j, TOL_FP64)
        assert oracle.rel_fro(got, ref) <= tol, (i, j, oracle.rel_fro(got, ref), tol)


def test_fp64_single_block_inverse_k1(mb):
    m = bi.uniform_shift(333, 5, shift=10.0)
    ctx = mb.Context(dev(m), 1)
    got = to_np(ctx.block(0, 0))
    ref, st = oracle.gj_inverse(m)
    assert oracle.rel_fro(got, ref) < 1e-13


def test_fp64_host_buffers(mb):
    m = bi.uniform_shift(128, 7)
    ctx = mb.Context(torch.tensor(m), 4)  # host M, host out
    got = ctx.block(2, 1, on_host=True)
    assert got.device.type == "cpu"
    ref = oracle_block(m, 4, 2, 1)
    assert oracle.rel_fro(to_np(got), ref) < 1e-12


def test_fp64_padding_border(mb):
    """n = 250, k = 4 (b = 63, l = 2) and n = 250, k = 6 (b = 42, l = 2):
    Eq. M_augmented, coupling border for requests that touch the padded
    block, padded block as pivot index for the others."""
    for n, k, seed in [(250, 4, 17), (250, 6, 5)]:
        _padding_case(mb, n, k, seed)


def _padding_case(mb, n, k, seed):
    m = bi.uniform_shift(n, 8)
    ctx = mb.Context(dev(m), k, pad_seed=seed)
    inv = np.linalg.inv(m)
    b = -(-n // k)
    cpl = bi.pad_columns(n, k * b - n, seed)
    for i, j in itertools.product(range(k), range(k)):
        got = to_np(ctx.block(i, j))
        g, _, _ = oracle.augment(m, k, i, j, coupling=cpl)
        ref = oracle_block(g, k, i, j, pad_last=True)
        r1, c1 = min(b, n - i * b), min(b, n - j * b)
        assert got.shape == (r1, c1)
        tol, _ = parity_tol(g, k, i, j, TOL_FP64, pad_last=True)
        assert oracle.rel_fro(got, ref[:r1, :c1]) <= tol, (i, j)
        assert oracle.rel_fro(got, inv[i * b:i * b + r1, j * b:j * b + c1]) < 1e-11


def test_fp64_singular_pivot_reported(mb):
    m = bi.block_diagonal(4, 16, 3)
    ctx = mb.Context(dev(m), 4)
    with pytest.raises(mb.MbinvError) as e:
        ctx.block(0, 1)
    assert e.value.status == mb.ESINGULAR
    # the context stays usable
    got = to_np(ctx.block(2, 2))
    assert oracle.rel_fro(got, np.linalg.inv(m[32:48, 32:48])) < 1e-14


def test_fp64_nan_input_is_singular(mb):
    m = bi.uniform_shift(64, 2)
    m[5, 7] = np.nan
    ctx = mb.Context(dev(m), 4)
    with pytest.raises(mb.MbinvError) as e:
        ctx.block(0, 0)
    assert e.value.status == mb.ESINGULAR


def test_power_of_two_scaling_bitwise(mb):
    m = bi.uniform_shift(384, 4)
    a = to_np(mb.Context(dev(m), 4).block(1, 2))
    c = to_np(mb.Context(dev(m * 8.0), 4).block(1, 2))
    assert np.array_equal(c * 8.0, a)


def test_fp32_small_config(mb):
    m = bi.uniform_shift(256, 0)
    m32 = m.astype(np.float32)
    ctx = mb.Context(dev(m32, torch.float32), 4, precision="fp32")
    for i, j in [(0, 0), (3, 1)]:
        got = to_np(ctx.block(i, j))
        ref = oracle_block(m32.astype(np.float64), 4, i, j)
        err = oracle.rel_fro(got, ref)
        assert err <= TOL_FP32, err


def test_fp64_block_row_and_col(mb):
    m = bi.uniform_shift(192, 9)
    ctx = mb.Context(dev(m), 3)
    row = to_np(ctx.block_row(1))
    col = to_np(ctx.block_col(2))
    inv = np.linalg.inv(m)
    assert oracle.rel_fro(row, inv[64:128, :]) < 1e-12
    assert oracle.rel_fro(col, inv[:, 128:192]) < 1e-12
    # block row times M is block row of I
    r = oracle.block_row_residual(m, row, 1, 64)
    assert np.abs(r).max() < 1e-12


def test_backward_against_reference_and_central_differences(mb):
    n, k, b, i, j = 64, 4, 16, 2, 1
    m = bi.spd(n, 1e1, 3)
    g = bi.gaussian_matrix(b, b, 5)
    ref = oracle.adjoint(np.linalg.inv(m), g, i, j, b)
    M = dev(m).requires_grad_(True)
    out = mb.block(M, k, i, j)
    (out * dev(g)).sum().backward()
    got = to_np(M.grad)
    assert oracle.rel_fro(got, ref) < 1e-12
    # directional central differences through the GPU forward path
    rng = np.random.default_rng(0)
    for _ in range(3):
        v = rng.standard_normal((n, n))
        h = 1e-5
        lp = float((to_np(mb.Context(dev(m + h * v), k).block(i, j)) * g).sum())
        lm = float((to_np(mb.Context(dev(m - h * v), k).block(i, j)) * g).sum())
        fd = (lp - lm) / (2 * h)
        an = float((got * v).sum())
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_batched_problems(mb):
    probs = bi.ragged_batch(6, 3, nmin=64, nmax=320, kmin=2, kmax=5)
    tensors, refs = [], []
    for p in probs:
        m = bi.uniform_shift(p["n"], p["seed"])
        tensors.append((dev(m), p["k"], p["i"], p["j"]))
        g, b, l = oracle.augment(m, p["k"], p["i"], p["j"], coupling=bi.pad_columns(p["n"], (-p["n"]) % p["k"], 0))
        ref = oracle_block(g, p["k"], p["i"], p["j"], pad_last=l > 0)
        refs.append(ref)
    outs, statuses, rep, st = mb.batched_blocks(tensors)
    assert st == mb.OK and all(s == mb.OK for s in statuses)
    for o, r in zip(outs, refs):
        o = to_np(o)
        assert oracle.rel_fro(o, r[:o.shape[0], :o.shape[1]]) < 1e-10


def test_cap_too_small_is_refused_before_launch(mb):
    m = bi.uniform_shift(512, 1)
    ctx = mb.Context(dev(m), 8, cap=1 << 16)
    with pytest.raises(mb.MbinvError) as e:
        ctx.block(0, 0)
    assert e.value.status == mb.ENOMEM_CAP


def test_cap_respected_by_chunked_schedule(mb):
    """n = 2048, k = 8 (b = 256): under a cap below the unconstrained peak the
    planner chunks the Schur temporaries and the inverse batches; same result."""
    m = bi.uniform_shift(2048, 1)
    full = mb.Context(dev(m), 8)
    a = to_np(full.block(3, 4))
    need = full.last_report["peak_device_bytes"]
    cap = int(need * 0.85)
    small = mb.Context(dev(m), 8, cap=cap)
    c = to_np(small.block(3, 4))
    assert small.last_report["peak_device_bytes"] <= cap
    assert oracle.rel_fro(c, a) < 1e-13


def test_requests_run_together_match_one_at_a_time(mb):
    """mbinv_blocks runs several independent requests level by level in the
    same grouped launches; each block is bit for bit the one-at-a-time block."""
    m = bi.uniform_shift(512, 6)
    ctx = mb.Context(dev(m), 8)
    ij = [(0, 0), (3, 5), (7, 1), (2, 2), (6, 7)]
    together = [to_np(x) for x in ctx.blocks(ij)]
    for (i, j), t in zip(ij, together):
        one = to_np(mb.Context(dev(m), 8).block(i, j))
        assert np.array_equal(t, one), (i, j)
        assert oracle.rel_fro(t, oracle_block(m, 8, i, j)) <= parity_tol(m, 8, i, j, TOL_FP64)[0]


def test_requests_together_with_padding_and_host_outputs(mb):
    n, k = 250, 4
    m = bi.uniform_shift(n, 8)
    ctx = mb.Context(dev(m), k, pad_seed=3)
    ij = [(0, 1), (1, 3), (3, 0), (3, 3), (2, 2)]
    outs = [torch.empty((ctx.extent(i), ctx.extent(j)), dtype=torch.float64) for i, j in ij]  # host
    ctx.blocks(ij, outs=outs)
    inv = np.linalg.inv(m)
    b = ctx.b
    for (i, j), o in zip(ij, outs):
        ref = inv[i * b:i * b + ctx.extent(i), j * b:j * b + ctx.extent(j)]
        assert oracle.rel_fro(o.numpy(), ref) < 1e-11, (i, j)


def test_mixed_requests_together(mb):
    m = bi.uniform_shift(256, 0)
    M = torch.tensor(m, dtype=torch.float32, device="cuda")
    ctx = mb.Context(M, 4, precision="mixed")
    ij = [(0, 0), (1, 3), (3, 2)]
    together = [to_np(x) for x in ctx.blocks(ij)]
    for (i, j), t in zip(ij, together):
        one = to_np(mb.Context(M, 4, precision="mixed").block(i, j))
        assert np.array_equal(t, one), (i, j)


def test_k16_blocks_and_cap(mb):
    """k = 16 (3502 distinct frames per block), b = 32, against the oracle; then
    under a cap well below the unconstrained workspace."""
    n, k = 512, 16
    m = bi.uniform_shift(n, 12)
    ctx = mb.Context(dev(m), k)
    for i, j in [(0, 0), (15, 3), (7, 9)]:
        got = to_np(ctx.block(i, j))
        assert ctx.last_report["frames"] == 3502
        tol, floor = parity_tol(m, k, i, j, TOL_FP64)
        assert oracle.rel_fro(got, oracle_block(m, k, i, j)) <= tol, (i, j)
    need = ctx.last_report["peak_device_bytes"]
    small = mb.Context(dev(m), k, cap=int(need * 0.6))
    got = to_np(small.block(15, 3))
    assert small.last_report["peak_device_bytes"] <= int(need * 0.6)
    assert oracle.rel_fro(got, to_np(ctx.block(15, 3))) < 1e-12
