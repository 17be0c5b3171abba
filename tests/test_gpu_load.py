"""Loading serialised functions on the device.

A function built on the GPU, serialised and loaded again has the same node
values, offsets and packed words, answers every query the same way, and
serialises to the same bytes.  A blob written from the oracle's arrays
loads into a function whose arrays and queries equal the oracle's: the
library's decoder reads the oracle's encoding (Section 2.2,
"Representation") word for word.
"""
import numpy as np
import pytest

from paper_2212_09562_b300 import mphf as M
from paper_2212_09562_b300 import workloads as W
from helpers import oracle_blob
from test_gpu_parity import to_dev

pytestmark = pytest.mark.gpu

ARRAYS = ("values", "node_off", "cum_keys", "bit_pos", "gr", "ef")
CASES = [  # (leaf, bucket, leaf method, tree, key bytes, n)
    (8, 100, M.PLAIN, M.TREE_RECSPLIT, 8, 5000),
    (12, 1000, M.ROTATION, M.TREE_RECSPLIT, 16, 20000),
    (16, 300, M.ROTATION, M.TREE_RECSPLIT, 8, 3000),
    (24, 2000, M.SHOCKHASH, M.TREE_FANOUT2, 8, 20000),
    (12, 300, M.SHOCKHASH, M.TREE_RECSPLIT, 8, 9000),
    (10, 500, M.PLAIN, M.TREE_FANOUT2, 16, 8000),
    (5, 1, M.ROTATION, M.TREE_RECSPLIT, 8, 50),
    (8, 100, M.ROTATION, M.TREE_RECSPLIT, 8, 1),
]


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2212_09562_b300 import build
    build.build()
    M.lib()
    return t


@pytest.mark.parametrize("leaf,bucket,bij,tree,kb,n", CASES)
def test_serialise_then_load_gives_the_same_function(torch, leaf, bucket, bij, tree, kb, n):
    keys = W.random_keys(n, kb, 13 * n + leaf)
    dkeys = to_dev(torch, keys)
    g = M.MPHF.build(dkeys, leaf, bucket, bij, tree=tree)
    blob = g.serialize()
    h = M.MPHF.load(bytes(bytearray(blob)))  # a fresh copy of the bytes
    a, b = g.host_arrays(), h.host_arrays()
    for k in ARRAYS:
        assert np.array_equal(a[k], b[k]), k
    for f in ("n", "nb", "n_nodes", "gr_bits", "gr_words", "ef_words", "max_bucket", "tree_shape",
              "leaf_size", "bucket_size", "key_bytes", "leaf_bijection"):
        assert getattr(g.info, f) == getattr(h.info, f), f
    assert h.serialize() == blob
    assert np.array_equal(h.query(dkeys).cpu().numpy(), g.query(dkeys).cpu().numpy())
    assert h.verify(dkeys) == 0 and h.verify_static(dkeys) == 0
    other = to_dev(torch, W.random_keys(20000, kb, 99 + leaf))
    assert np.array_equal(h.query(other).cpu().numpy(), g.query(other).cpu().numpy())
    st = h.stats()
    assert all(st[k] == (0, 0) for k in ("leaf", "lower1", "lower2", "upper"))


@pytest.mark.parametrize("leaf,bucket,bij,tree,kb,n", CASES)
def test_oracle_blobs_load_and_query_like_the_oracle(torch, orc, leaf, bucket, bij, tree, kb, n):
    keys = W.random_keys(n, kb, 29 * n + leaf)
    o = orc.build_mphf(keys, leaf, bucket, bij, threads=4, tree=tree)
    h = M.MPHF.load(oracle_blob(o, leaf, bucket, kb, bij, tree))
    a = h.host_arrays()
    for k, want in zip(ARRAYS, (o.values, o.node_off, o.cum_keys, o.bit_pos, o.gr, o.ef)):
        assert np.array_equal(a[k], want), k
    dkeys = to_dev(torch, keys)
    assert np.array_equal(h.query(dkeys).cpu().numpy().view(np.uint64), o.query(keys))
    assert h.verify(dkeys) == 0
    other = W.random_keys(20000, kb, 199 + leaf)
    assert np.array_equal(h.query(to_dev(torch, other)).cpu().numpy().view(np.uint64), o.query(other))


def test_empty_function_loads(torch, orc):
    g = M.MPHF.build(torch.empty(0, dtype=torch.int64, device="cuda"), 8, 100)
    h = M.MPHF.load(g.serialize())
    assert h.info.n == 0 and h.info.nb == 0 and h.info.n_nodes == 0
    assert np.array_equal(h.host_arrays()["ef"], g.host_arrays()["ef"])
    assert h.serialize() == g.serialize()


def test_damaged_blob_is_refused_before_the_device(torch):
    keys = W.random_keys(3000, 8, 5)
    g = M.MPHF.build(to_dev(torch, keys), 8, 100)
    blob = bytearray(g.serialize())
    blob[-1] ^= 0x80  # top bit of the last Elias-Fano high word: one more one
    before = M.kernel_launches()
    with pytest.raises(M.MPHFError) as e:
        M.MPHF.load(bytes(blob))
    assert e.value.code == M.EINVAL
    assert M.kernel_launches() == before


def test_serialised_fixture_loads_and_is_what_the_gpu_writes(torch):
    """The golden serialised function (written from the oracle alone)
    queries to its stored values on the device, and the GPU build of the
    same keys serialises to exactly its bytes."""
    from helpers import read_serialised_fixture
    p, blob, keys, values = read_serialised_fixture()
    dkeys = to_dev(torch, keys)
    h = M.MPHF.load(blob)
    assert np.array_equal(h.query(dkeys).cpu().numpy().view(np.uint64), values)
    g = M.MPHF.build(dkeys, p["leaf"], p["bucket"], p["bijection"], tree=p["tree"])
    assert g.serialize() == blob
