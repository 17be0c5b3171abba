"""Prepared builds searched together (mphf_batch_prepare / _enqueue /
_finish): the buckets of every member go through one persistent search
launch, enqueued without allocation or host synchronisation, so the whole
batch can be captured once in a CUDA graph and replayed on new keys.  Every
member must store the words of its plain build (mphf_build_ex) and of
mphf_build_batch; a failing member fails alone."""
import ctypes

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


# (n, leaf, bucket, leaf method, tree, key bytes): mixed leaf sizes, methods,
# trees and key sizes, a one-key build and uneven sizes
MEMBERS = [
    (20_000, 8, 100, M.PLAIN, M.TREE_RECSPLIT, 8),
    (60_000, 12, 1000, M.ROTATION, M.TREE_RECSPLIT, 16),
    (30_000, 16, 2000, M.ROTATION, M.TREE_RECSPLIT, 8),
    (40_000, 24, 2000, M.SHOCKHASH, M.TREE_FANOUT2, 8),
    (1, 8, 100, M.ROTATION, M.TREE_RECSPLIT, 8),
    (3_333, 5, 7, M.ROTATION, M.TREE_RECSPLIT, 8),
]


def prepare_all(members):
    return [M.MPHF.prepare(n, l, b, bij, key_bytes=kb, tree=t) for n, l, b, bij, t, kb in members]


def test_batch_equals_plain_builds_and_the_oracle(torch, orc):
    keys = [W.random_keys(n, kb, 8500 + i) for i, (n, _, _, _, _, kb) in enumerate(MEMBERS)]
    dk = [to_dev(torch, k) for k in keys]
    hs = prepare_all(MEMBERS)
    batch = M.PreparedBatch(hs)
    batch.enqueue(dk)
    assert batch.finish() == [M.OK] * len(MEMBERS)
    for h, d, k, (n, l, b, bij, t, kb) in zip(hs, dk, keys, MEMBERS):
        one = M.MPHF.build(d, l, b, bij, tree=t)
        same(h, one)
        assert h.verify(d) == 0
        assert h.serialize() == one.serialize()
    # each group of members with one bucket size, leaf method and tree also
    # through mphf_build_batch
    groups = {}
    for i, (n, l, b, bij, t, kb) in enumerate(MEMBERS):
        groups.setdefault((b, bij, t), []).append(i)
    for (b, bij, t), idx in groups.items():
        built = M.build_batch([dk[i] for i in idx], [MEMBERS[i][1] for i in idx], bucket_size=b,
                              rotation=bij, tree=t, tuned=False)
        for i, one in zip(idx, built):
            same(hs[i], one)
    # and one member straight against the oracle
    o = orc.build_mphf(keys[0], 8, 100, M.PLAIN, threads=8)
    assert np.array_equal(hs[0].host_arrays()["values"], o.values)
    assert np.array_equal(hs[0].host_arrays()["gr"], o.gr)


def test_captured_batch_replays_on_new_keys(torch):
    """One graph holds the whole batch; three key sets in its input buffers,
    every member equal to its plain build each time."""
    members = [(50_000, 16, 2000, M.ROTATION, M.TREE_RECSPLIT, 8),
               (20_000, 8, 100, M.ROTATION, M.TREE_RECSPLIT, 8),
               (70_000, 12, 1000, M.ROTATION, M.TREE_RECSPLIT, 8)]
    bufs = [torch.empty(n, dtype=torch.int64, device="cuda") for n, *_ in members]
    hs = prepare_all(members)
    batch = M.PreparedBatch(hs)
    s = torch.cuda.Stream()
    for i, b in enumerate(bufs):
        b.copy_(torch.from_numpy(W.distinct_u64(b.shape[0], 8600 + i).view(np.int64)))
    torch.cuda.synchronize()
    batch.enqueue(bufs, stream=s)  # eager first: lazy module loading happens outside capture
    batch.finish(stream=s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        batch.enqueue(bufs, stream=s)
    for rep in range(3):
        keys = [W.distinct_u64(b.shape[0], 8700 + 10 * rep + i) for i, b in enumerate(bufs)]
        for b, k in zip(bufs, keys):
            b.copy_(torch.from_numpy(k.view(np.int64)))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert batch.finish(stream=s) == [M.OK] * len(members)
        for h, k, (n, l, bk, bij, t, kb) in zip(hs, keys, members):
            d = to_dev(torch, k)
            same(h, M.MPHF.build(d, l, bk, bij, tree=t))
            assert h.verify(d) == 0


def test_failing_member_fails_alone_and_the_batch_recovers(torch):
    members = [(4_000, 12, 200, M.ROTATION, M.TREE_RECSPLIT, 8)] * 4
    keys = [W.distinct_u64(4_000, 8800 + i) for i in range(4)]
    bad = keys[2].copy()
    bad[7] = bad[3000]
    hs = prepare_all(members)
    batch = M.PreparedBatch(hs)
    batch.enqueue([to_dev(torch, k) for k in keys[:2] + [bad] + keys[3:]])
    with pytest.raises(M.MPHFError) as e:
        batch.finish()
    assert e.value.code == M.EDUPLICATE
    with pytest.raises(M.MPHFError):
        hs[2].query(to_dev(torch, bad))  # the failed member is unusable
    for i in (0, 1, 3):
        d = to_dev(torch, keys[i])
        same(hs[i], M.MPHF.build(d, 12, 200, True))
    dk = [to_dev(torch, k) for k in keys]
    batch.enqueue(dk)  # the same batch builds again
    assert batch.finish() == [M.OK] * 4
    for h, d in zip(hs, dk):
        same(h, M.MPHF.build(d, 12, 200, True))


def test_batch_arguments_are_checked(torch):
    L = M.lib()
    a = M.MPHF.prepare(1000, 8, 100)
    b = M.MPHF.prepare(2000, 8, 100)
    plain = M.MPHF.build(to_dev(torch, W.distinct_u64(1000, 8900)), 8, 100)
    out = ctypes.c_void_p()

    def prep(handles, threads=0):
        arr = (ctypes.c_void_p * len(handles))(*[h._h.value for h in handles])
        return L.mphf_batch_prepare(arr, len(handles), threads, 0, None, ctypes.byref(out))

    assert prep([a, a]) == M.EINVAL          # a handle twice
    assert prep([a, plain]) == M.EINVAL      # not a prepared build
    assert prep([a, b], threads=100) == M.EINVAL
    assert out.value is None
    batch = M.PreparedBatch([a, b])
    with pytest.raises(ValueError):
        batch.enqueue([to_dev(torch, W.distinct_u64(1000, 1))])  # one key set short
    with pytest.raises(ValueError):
        batch.enqueue([to_dev(torch, W.distinct_u64(1000, 1)),
                       to_dev(torch, W.distinct_u64(1999, 2))])  # wrong size
    ptrs = (ctypes.c_void_p * 2)(None, None)
    assert L.mphf_batch_enqueue(batch._b, ptrs, None) == M.EINVAL
    batch.close()
