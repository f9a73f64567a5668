"""The panel-cluster autotuner: it times batched inverses of synthetic
matrices for each cluster bias, keeps the fastest, writes its choice to a
cache file that a context reads back, and changes no result bit (the
cluster size moves rows between CTAs; every row is eliminated by the same
operations)."""
import numpy as np
import pytest

import bri_inputs as bi
from helpers import to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mb():
    import paper_1612_00001_gb300 as mb
    mb.build()
    return mb


def test_autotune_writes_cache_and_keeps_results(mb, tmp_path):
    m = bi.uniform_shift(2048, 8)
    M = torch.tensor(m, device="cuda")
    with mb.Context(M, 4, precision="fp64_tc") as c0:  # b = 512, leaf pivot batch of 1
        before = to_np(c0.block(1, 2))
    path = tmp_path / "tune.txt"
    bias, secs = mb.autotune(512, 1, "fp64_tc", str(path))
    assert -2 <= bias <= 2 and secs > 0
    fields = path.read_text().split()
    assert [int(x) for x in fields[:4]] == [512, 1, 3, bias]
    bias2, _ = mb.autotune(512, 8, "fp64_tc", str(path))
    assert len(path.read_text().splitlines()) == 2
    with mb.Context(M, 4, precision="fp64_tc", tune_cache_path=str(path)) as c1:
        after = to_np(c1.block(1, 2))
    assert np.array_equal(before, after)


def test_forced_cluster_biases_change_no_bit(mb, tmp_path):
    """Biases -2 and +2 written to a cache file: one- and two-CTA clusters,
    and (past the heuristic's 8) the non-portable 16-CTA clusters the tuner
    may pick for small batches.  Every bias gives the same bits; the cache's
    last word restores bias 0 for the rest of the process."""
    m = bi.uniform_shift(2048, 9)
    M = torch.tensor(m, device="cuda")
    keys = [1, 2, 4, 8, 16]

    def run(bias):
        path = tmp_path / f"bias{bias}.txt"
        path.write_text("".join(f"512 {c} 3 {bias} 1.0\n" for c in keys))
        with mb.Context(M, 4, precision="fp64_tc", tune_cache_path=str(path)) as c:
            return [to_np(c.block(i, j)) for i, j in [(1, 2), (3, 3)]]

    try:
        base = run(0)
        for bias in (2, -2):
            got = run(bias)
            for a, b_ in zip(got, base):
                assert np.array_equal(a, b_), bias
    finally:
        run(0)
