"""One function built in bucket-range shards (Section 5.2) on the device.

Ranks are emulated one after another on one GPU with the library's own
steps (route, shard build, pack, join); the joined function must equal the
single-GPU build of all keys word for word and query like it.  A real
multi-GPU run (one process per GPU, NCCL) runs when two or more GPUs are
present."""
import ctypes
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from paper_2212_09562_b300 import mphf as M
from paper_2212_09562_b300 import shard as S
from paper_2212_09562_b300 import workloads as W
from test_gpu_parity import to_dev

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2212_09562_b300 import build
    build.build()
    M.lib()
    return t


def emulate(torch, keys, world, leaf, bucket, bij, tree=M.TREE_RECSPLIT):
    """Every emulated rank routes its slice; each owner builds from what the
    others sent it; the packs are joined on the device."""
    ops = S.LibraryOps()
    n = len(keys)
    cuts = [n * r // world for r in range(world + 1)]
    inbox = [[] for _ in range(world)]
    for r in range(world):
        dk = to_dev(torch, keys[cuts[r]:cuts[r + 1]])
        routed, counts = ops.route(dk, n, bucket, world)
        off = 0
        for dst, c in enumerate(counts):
            inbox[dst].append(routed[off:off + c])
            off += c
        assert off == cuts[r + 1] - cuts[r]
    shards, packs = [], []
    for r in range(world):
        mine = torch.cat(inbox[r]) if inbox[r] else to_dev(torch, keys[:0])
        sh = ops.build_shard(mine.contiguous(), n, leaf, bucket, bij, tree, r, world)
        shards.append(sh)
        packs.append(ops.pack(sh))
    return ops.concat(packs), shards


CASES = [  # (world, leaf, bucket, leaf method, tree, key bytes, n)
    (2, 8, 100, M.ROTATION, M.TREE_RECSPLIT, 8, 50_000),
    (3, 12, 1000, M.ROTATION, M.TREE_RECSPLIT, 16, 60_000),
    (4, 16, 2000, M.ROTATION, M.TREE_RECSPLIT, 8, 30_000),
    (5, 8, 100, M.PLAIN, M.TREE_RECSPLIT, 8, 7_000),
    (3, 24, 2000, M.SHOCKHASH, M.TREE_FANOUT2, 8, 40_000),
    (8, 6, 50, M.ROTATION, M.TREE_RECSPLIT, 8, 300),   # 6 buckets: two ranks own none
    (2, 8, 100, M.ROTATION, M.TREE_RECSPLIT, 8, 1),
]


@pytest.mark.parametrize("world,leaf,bucket,bij,tree,kb,n", CASES)
def test_sharded_build_equals_the_single_build(torch, world, leaf, bucket, bij, tree, kb, n):
    keys = W.random_keys(n, kb, 6100 + n + world)
    dkeys = to_dev(torch, keys)
    full, shards = emulate(torch, keys, world, leaf, bucket, bij, tree)
    one = M.MPHF.build(dkeys, leaf, bucket, bij, tree=tree)
    a, b = full.host_arrays(), one.host_arrays()
    for k in ("values", "node_off", "cum_keys", "bit_pos", "gr", "ef"):
        assert np.array_equal(a[k], b[k]), k
    assert full.info.gr_bits == one.info.gr_bits and full.info.n_nodes == one.info.n_nodes
    st_full, st_one = full.stats(), one.stats()
    for k in ("leaf", "lower1", "lower2", "upper"):
        assert st_full[k] == st_one[k], k
    q = full.query(dkeys).cpu().numpy()
    assert np.array_equal(q, one.query(dkeys).cpu().numpy())
    assert full.verify(dkeys) == 0
    assert full.serialize() == one.serialize()


def test_shard_refuses_keys_of_other_ranks_and_queries(torch):
    keys = W.distinct_u64(20_000, 6200)
    dkeys = to_dev(torch, keys)
    ops = S.LibraryOps()
    with pytest.raises(M.MPHFError) as e:  # all keys, but rank 0 of 2 owns only half the buckets
        ops.build_shard(dkeys, len(keys), 8, 100, True, M.TREE_RECSPLIT, 0, 2)
    assert e.value.code == M.EINVAL
    routed, counts = ops.route(dkeys, len(keys), 100, 2)
    sh = ops.build_shard(routed[:counts[0]].contiguous(), len(keys), 8, 100, True, M.TREE_RECSPLIT, 0, 2)
    with pytest.raises(M.MPHFError):
        sh.query(dkeys)
    with pytest.raises(M.MPHFError):
        sh.serialize()
    # a join needs every rank's pack, in order
    sh1 = ops.build_shard(routed[counts[0]:].contiguous(), len(keys), 8, 100, True, M.TREE_RECSPLIT, 1, 2)
    p0, p1 = ops.pack(sh), ops.pack(sh1)
    for bad in ([p1, p0], [p0], [p0, p0]):
        with pytest.raises(M.MPHFError) as e:
            ops.concat(bad)
        assert e.value.code == M.EINVAL
    with pytest.raises(M.MPHFError) as e:  # a pack cut short
        ops.concat([p0, p1[: p1.numel() - 1]])
    assert e.value.code == M.EINVAL
    assert ops.concat([p0, p1]).verify(dkeys) == 0


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r'''
import os, sys
import numpy as np, torch, torch.distributed as dist
sys.path.insert(0, os.environ["ROOT"])
from paper_2212_09562_b300 import mphf as M, shard as S, workloads as W
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
torch.cuda.set_device(rank)
dist.init_process_group("nccl", device_id=torch.device("cuda", rank))
n = 200_000
keys = W.distinct_u64(n, 6300)
mine = keys[n * rank // world: n * (rank + 1) // world]
full, _ = S.build_sharded(torch.from_numpy(mine.view(np.int64)).cuda(), 12, 1000, True)
dk = torch.from_numpy(keys.view(np.int64)).cuda()
one = M.MPHF.build(dk, 12, 1000, True)
ok = full.serialize() == one.serialize() and full.verify(dk) == 0
dist.barrier()
dist.destroy_process_group()
sys.exit(0 if ok else 1)
'''


def test_sharded_build_on_every_gpu(torch, tmp_path):
    world = torch.cuda.device_count()
    if world < 2:
        pytest.skip("one GPU: the multi-process NCCL run needs two or more")
    script = tmp_path / "worker.py"
    script.write_text(WORKER)
    env = dict(os.environ, ROOT=ROOT, NCCL_NVLS_ENABLE="0")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={world}",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", str(script)]
    subprocess.run(cmd, env=env, check=True, timeout=600)
