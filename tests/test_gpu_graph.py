"""The query path inside a CUDA graph.

mphf_query is one kernel launch with no allocation and no host
synchronisation, so a serving loop can capture it once and replay it for
every batch of keys.  The replayed graph must give the values of eager
queries, batch after batch.
"""
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


@pytest.mark.parametrize("bij,tree,leaf,bucket", [(M.ROTATION, M.TREE_RECSPLIT, 12, 1000),
                                                  (M.SHOCKHASH, M.TREE_FANOUT2, 24, 2000)])
def test_captured_query_replays_like_eager_queries(torch, bij, tree, leaf, bucket):
    n, batch = 50_000, 8192
    keys = W.random_keys(n, 8, 4100 + leaf)
    dkeys = to_dev(torch, keys)
    g = M.MPHF.build(dkeys, leaf, bucket, bij, tree=tree)
    buf = torch.empty(batch, dtype=torch.int64, device="cuda")
    out = torch.empty(batch, dtype=torch.int64, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # warm-up outside the capture
        buf.copy_(dkeys[:batch])
        g.query(buf, out=out)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        g.query(buf, out=out)
    launches = M.kernel_launches()
    rng = np.random.default_rng(7)
    for step in range(6):
        # in-set keys in a random order, and for odd steps half of them replaced by other keys
        pick = dkeys[torch.from_numpy(rng.choice(n, batch, replace=False)).cuda()]
        if step % 2:
            pick[: batch // 2] = to_dev(torch, W.random_keys(batch // 2, 8, 5000 + step))
        buf.copy_(pick)
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, g.query(pick))
    assert M.kernel_launches() == launches + 6  # the eager checks; replays launch through the graph
    assert g.verify(dkeys) == 0
