"""A prepared build (mphf_build_prepare / _enqueue / _finish): its device
work has no allocation and no host synchronisation, so it can be captured
once in a CUDA graph and replayed on new keys.  Every replay must store the
words of mphf_build_ex on the same keys; a code longer than reserved, and a
failing build, are reported by finish() and leave the handle unusable."""
import numpy as np
import pytest

from paper_2212_09562_b300 import mphf as M
from paper_2212_09562_b300 import workloads as W
from test_gpu_parity import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2212_09562_b300 import build
    build.build()
    M.lib()
    return t


def same(a, b):
    x, y = a.host_arrays(), b.host_arrays()
    for k in ("values", "node_off", "cum_keys", "bit_pos", "gr", "ef"):
        assert np.array_equal(x[k], y[k]), k
    assert a.info.gr_bits == b.info.gr_bits and a.info.n_nodes == b.info.n_nodes
    for k in ("leaf", "lower1", "lower2", "upper"):
        assert a.stats()[k] == b.stats()[k], k


CASES = [  # (leaf, bucket, leaf method, tree, key bytes, n)
    (8, 100, M.PLAIN, M.TREE_RECSPLIT, 8, 20_000),
    (12, 1000, M.ROTATION, M.TREE_RECSPLIT, 16, 60_000),
    (16, 2000, M.ROTATION, M.TREE_RECSPLIT, 8, 50_000),
    (24, 2000, M.SHOCKHASH, M.TREE_FANOUT2, 8, 40_000),
    (5, 7, M.ROTATION, M.TREE_RECSPLIT, 8, 3),
]


@pytest.mark.parametrize("leaf,bucket,bij,tree,kb,n", CASES)
def test_prepared_build_equals_the_plain_build(torch, leaf, bucket, bij, tree, kb, n):
    keys = W.random_keys(n, kb, 8100 + n)
    dk = to_dev(torch, keys)
    h = M.MPHF.prepare(n, leaf, bucket, bij, key_bytes=kb, tree=tree)
    with pytest.raises(M.MPHFError):
        h.query(dk)  # not usable before finish
    h.enqueue(dk)
    h.finish()
    one = M.MPHF.build(dk, leaf, bucket, bij, tree=tree)
    same(h, one)
    assert np.array_equal(h.query(dk).cpu().numpy(), one.query(dk).cpu().numpy())
    assert h.verify(dk) == 0
    assert h.serialize() == one.serialize()


def test_graph_replays_build_new_keys(torch):
    """Captured once, the graph rebuilds from whatever keys sit in its input
    buffer: three key sets, each equal to its plain build."""
    n, leaf, bucket = 120_000, 12, 1000
    buf = torch.empty(n, dtype=torch.int64, device="cuda")
    h = M.MPHF.prepare(n, leaf, bucket, True)
    s = torch.cuda.Stream()
    buf.copy_(torch.from_numpy(W.distinct_u64(n, 8200).view(np.int64)))
    torch.cuda.synchronize()
    h.enqueue(buf, stream=s)  # an eager run first: lazy module loading happens outside capture
    h.finish(stream=s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        h.enqueue(buf, stream=s)
    for seed in (8201, 8202, 8203):
        keys = W.distinct_u64(n, seed)
        buf.copy_(torch.from_numpy(keys.view(np.int64)))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        h.finish(stream=s)
        dk = to_dev(torch, keys)
        same(h, M.MPHF.build(dk, leaf, bucket, True))
        assert h.verify(dk) == 0


def test_code_longer_than_reserved_is_refused(torch):
    n = 10_000
    dk = to_dev(torch, W.distinct_u64(n, 8300))
    h = M.MPHF.prepare(n, 8, 100, True, gr_capacity_bits=4096)  # the code needs about 18,000 bits
    h.enqueue(dk)
    with pytest.raises(M.MPHFError) as e:
        h.finish()
    assert e.value.code == M.ECAPACITY
    with pytest.raises(M.MPHFError):
        h.query(dk)


def test_failing_build_and_recovery(torch):
    n = 5_000
    keys = W.distinct_u64(n, 8400)
    bad = keys.copy()
    bad[7] = bad[4000]
    h = M.MPHF.prepare(n, 8, 100, True)
    h.enqueue(to_dev(torch, bad))
    with pytest.raises(M.MPHFError) as e:
        h.finish()
    assert e.value.code == M.EDUPLICATE
    dk = to_dev(torch, keys)
    h.enqueue(dk)  # the same handle builds again
    h.finish()
    same(h, M.MPHF.build(dk, 8, 100, True))


def test_enqueue_after_a_plain_build_of_smaller_buckets(torch):
    """A plain build of small buckets between two enqueues must not leave the
    search kernel's shared-memory limit below what the prepared build
    launches with (room for the largest bucket a build accepts)."""
    n = 20_000
    dk = to_dev(torch, W.distinct_u64(n, 8450))
    h = M.MPHF.prepare(n, 8, 100, True)
    h.enqueue(dk)
    h.finish()
    small = M.MPHF.build(to_dev(torch, W.distinct_u64(500, 8451)), 8, 10, True)
    assert small.info.n == 500
    h.enqueue(dk)
    h.finish()
    same(h, M.MPHF.build(dk, 8, 100, True))
