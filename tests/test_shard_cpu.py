"""The sharded build's orchestration on CPU ranks (gloo, world size 2 and 3).

paper_2212_09562_b300.shard.build_sharded runs unchanged; its device steps
are replaced by the oracle: keys routed to the owner of their bucket (the
driver's partition rule), the owner's bucket range built by the oracle
(Section 5.2's consecutive range), packs joined by the reference joining of
shard_ref.  Every rank must end with the whole function of the union of all
ranks' keys, word for word the oracle's single build; the exchange must
deliver each key to exactly one rank, the owner of its bucket."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleOps:
    """build_sharded's device steps done by the CPU oracle on CPU tensors."""

    def __init__(self, orc, shard, leaf, bucket, rotation):
        self.O, self.S = orc, shard
        self.leaf, self.bucket, self.rotation = leaf, bucket, rotation
        self.received = None

    def _np(self, t):
        return t.numpy().view(np.uint64) if t.dim() == 1 else t.numpy()

    def route(self, keys, n_total, bucket_size, world):
        import torch
        from shard_ref import bucket_of_keys
        k = self._np(keys)
        nb = (n_total + bucket_size - 1) // bucket_size
        owner = self.S.bucket_owner(bucket_of_keys(self.O, k, nb), nb, world)
        order = np.argsort(owner, kind="stable")
        counts = np.bincount(owner, minlength=world)
        return torch.from_numpy(np.ascontiguousarray(k[order]).view(np.int64) if k.ndim == 1
                                else np.ascontiguousarray(k[order])), [int(c) for c in counts]

    def build_shard(self, keys, n_total, leaf, bucket, rotation, tree, rank, world):
        k = self._np(keys)
        self.received = k.copy()
        nb = (n_total + bucket - 1) // bucket
        lo, hi = self.S.bucket_range(rank, world, nb)
        return self.O.build_range(k, n_total, leaf, bucket, rotation, lo, hi, threads=2, tree=tree)

    def pack(self, o):
        import torch
        head = np.array([o.n, o.nb, o.n_nodes, o.gr_bits, len(o.gr)], np.uint64)
        words = np.concatenate([head, o.cum_keys, o.node_off, o.bit_pos, o.values, o.gr])
        return torch.from_numpy(words.view(np.int64).copy())

    def concat(self, packs):
        from shard_ref import concat_ranges
        parts = []
        for p in packs:
            w = p.numpy().view(np.uint64)
            n, nb, nn, bits, gw = (int(x) for x in w[:5])
            q = w[5:]
            parts.append({"n": n, "cum_keys": q[:nb + 1], "node_off": q[nb + 1:2 * nb + 2],
                          "bit_pos": q[2 * nb + 2:3 * nb + 3], "n_nodes": nn,
                          "values": q[3 * nb + 3:3 * nb + 3 + nn],
                          "gr": q[3 * nb + 3 + nn:3 * nb + 3 + nn + gw], "gr_bits": bits})
        return concat_ranges(parts)


def _rank_main(rank, world, port, out_dir, case):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_2212_09562_b300 import shard as S
    from paper_2212_09562_b300 import workloads as W
    leaf, bucket, rotation, kb, n = case
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # every rank starts from its own, uneven slice of the key set
    allkeys = W.random_keys(n, kb, 5100 + n)
    cuts = [0] + [n * (r + 1) * (r + 2) // (world * (world + 1)) for r in range(world)]
    mine = allkeys[cuts[rank]:cuts[rank + 1]]
    t = torch.from_numpy(np.ascontiguousarray(mine).view(np.int64) if kb == 8 else np.ascontiguousarray(mine))
    ops = OracleOps(O, S, leaf, bucket, rotation)
    full, _ = S.build_sharded(t, leaf, bucket, rotation, ops=ops)
    whole = O.build_mphf(allkeys, leaf, bucket, rotation, threads=2)
    ok = all(np.array_equal(full[k], getattr(whole, k))
             for k in ("cum_keys", "node_off", "bit_pos", "values", "gr")) and full["gr_bits"] == whole.gr_bits
    np.save(os.path.join(out_dir, f"ok{rank}.npy"), np.array([ok]))
    got = ops.received.view(np.uint8).reshape(len(ops.received), -1)
    np.save(os.path.join(out_dir, f"recv{rank}.npy"), got)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,case", [
    (2, (8, 100, True, 8, 20_000)),
    (3, (12, 300, True, 16, 9_000)),
    (2, (5, 7, False, 8, 90)),       # 13 buckets, some ranks' slices hold few keys
])
def test_sharded_build_equals_the_single_build(tmp_path, world, case):
    from oracle import oracle as O
    from paper_2212_09562_b300 import workloads as W
    from paper_2212_09562_b300 import shard as S
    from shard_ref import bucket_of_keys
    O.build()
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path), case), nprocs=world, join=True)
    assert all(bool(np.load(tmp_path / f"ok{r}.npy")[0]) for r in range(world))
    # the exchange gave every key to exactly the owner of its bucket
    leaf, bucket, rotation, kb, n = case
    allkeys = W.random_keys(n, kb, 5100 + n)
    nb = (n + bucket - 1) // bucket
    owner = S.bucket_owner(bucket_of_keys(O, allkeys, nb), nb, world)
    rows = allkeys.view(np.uint8).reshape(n, -1)
    for r in range(world):
        got = np.load(tmp_path / f"recv{r}.npy")
        want = rows[owner == r]
        assert sorted(map(bytes, got)) == sorted(map(bytes, want))


def test_partition_rule():
    from paper_2212_09562_b300 import shard as S
    for nb in (1, 2, 7, 1000, 5000):
        for world in (1, 2, 3, 8, 13):
            ranges = [S.bucket_range(r, world, nb) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == nb
            assert all(ranges[r][1] == ranges[r + 1][0] for r in range(world - 1))
            for b in range(nb):
                r = S.bucket_owner(b, nb, world)
                assert ranges[r][0] <= b < ranges[r][1]
