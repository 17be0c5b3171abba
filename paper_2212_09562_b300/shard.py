"""One function built across the GPUs of a torch.distributed group.

Section 5.2 of the paper builds the buckets in consecutive ranges, one range
per worker, and concatenates the workers' local Golomb-Rice sequences and
bucket offsets.  Here a worker is a rank with its own GPU:

1. every rank groups its own keys by the rank that owns their bucket
   (rank r owns buckets [floor(r nb / world), floor((r + 1) nb / world)),
   nb = ceil(n_total / bucket_size): a range of fingerprint hi words);
2. one all-to-all moves every key to its owner;
3. every rank builds its buckets (the same kernels as a whole build);
4. one all-gather gives every rank the packed shards of all ranks;
5. every rank joins them into the whole function, word for word the one a
   single GPU builds from all keys.

The collectives are torch.distributed calls on the group (NCCL for CUDA
tensors, gloo for CPU ones); the device work is the C ABI of libmphf
(mphf_shard_route, mphf_build_shard, mphf_shard_pack, mphf_shard_concat).
``ops`` can replace the device steps, which is how the orchestration is
tested on CPU ranks.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import mphf as M


def bucket_range(rank: int, world: int, nb: int) -> tuple[int, int]:
    """Buckets [lo, hi) of rank `rank` out of `world` (Section 5.2: consecutive ranges)."""
    return nb * rank // world, nb * (rank + 1) // world


def bucket_owner(b, nb: int, world: int):
    """The rank whose range holds bucket b (works elementwise on integer arrays)."""
    return ((b + 1) * world - 1) // nb


class LibraryOps:
    """The device steps through libmphf on the current CUDA device."""

    def route(self, keys, n_total: int, bucket_size: int, world: int):
        n, kb = M.key_layout(keys)
        out = keys.new_empty(keys.shape)
        counts = np.zeros(world, np.uint64)
        M._check(M.lib().mphf_shard_route(keys.data_ptr() if n else None, n, kb, n_total, bucket_size,
                                          world, out.data_ptr() if n else None, counts.ctypes.data,
                                          M._stream(None)), "mphf_shard_route")
        return out, [int(c) for c in counts]

    def build_shard(self, keys, n_total: int, leaf_size: int, bucket_size: int, rotation, tree: int,
                    rank: int, world: int):
        n, kb = M.key_layout(keys)
        p = M.default_params()
        p.leaf_size, p.bucket_size, p.key_bytes = leaf_size, bucket_size, kb
        p.leaf_bijection, p.tree_shape = M.bijection(rotation), tree
        h = ctypes.c_void_p()
        M._check(M.lib().mphf_build_shard(keys.data_ptr() if n else None, n, n_total, ctypes.byref(p),
                                          rank, world, M._stream(None), ctypes.byref(h)),
                 "mphf_build_shard")
        return M.MPHF(h.value)

    def pack(self, shard):
        torch = M._torch()
        size = ctypes.c_size_t()
        M._check(M.lib().mphf_shard_pack(shard._h, None, ctypes.byref(size), M._stream(None)),
                 "mphf_shard_pack")
        buf = torch.empty(size.value // 8, dtype=torch.int64, device="cuda")
        M._check(M.lib().mphf_shard_pack(shard._h, buf.data_ptr(), ctypes.byref(size),
                                         M._stream(None)), "mphf_shard_pack")
        return buf

    def concat(self, packs):
        count = len(packs)
        ptrs = (ctypes.c_void_p * count)(*[p.data_ptr() for p in packs])
        lens = (ctypes.c_size_t * count)(*[p.numel() * 8 for p in packs])
        h = ctypes.c_void_p()
        M._check(M.lib().mphf_shard_concat(ptrs, lens, count, None, M._stream(None), ctypes.byref(h)),
                 "mphf_shard_concat")
        return M.MPHF(h.value)


def _words(keys):
    """The keys as a flat int64 tensor (one or two words per key) and words per key."""
    torch = __import__("torch")
    if keys.dim() == 1:
        return keys.view(torch.int64), 1
    return keys.contiguous().view(torch.int64).reshape(-1), 2


def build_sharded(keys, leaf_size: int = 16, bucket_size: int = 2000, rotation=True,
                  tree: int = M.TREE_RECSPLIT, group=None, ops=None):
    """Builds one function over the union of every rank's `keys` (a tensor of
    this rank's keys: (n,) 64-bit or (n, 16) bytes / (n, 2) 64-bit) and returns
    it on every rank, with this rank's shard: (function, shard).  Collective:
    every rank of the group must call it."""
    import torch
    import torch.distributed as dist
    ops = ops or LibraryOps()
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    dev = keys.device
    n_local = int(keys.shape[0])
    t = torch.tensor([n_local], dtype=torch.int64, device=dev)
    dist.all_reduce(t, group=group)
    n_total = int(t.item())

    # 1-2: keys to the rank that owns their bucket (one all-to-all)
    routed, send = ops.route(keys, n_total, bucket_size, world)
    send_t = torch.tensor(send, dtype=torch.int64, device=dev)
    recv_t = torch.empty(world, dtype=torch.int64, device=dev)
    dist.all_to_all_single(recv_t, send_t, group=group)
    recv = [int(x) for x in recv_t.tolist()]
    flat, wpk = _words(routed)
    mine = torch.empty(sum(recv) * wpk, dtype=torch.int64, device=dev)
    dist.all_to_all_single(mine, flat, [c * wpk for c in recv], [c * wpk for c in send], group=group)
    if keys.dim() == 2:
        mine = mine.view(-1, 2) if keys.dtype != torch.uint8 else mine.view(torch.uint8).view(-1, 16)

    # 3: this rank's buckets
    shard = ops.build_shard(mine, n_total, leaf_size, bucket_size, rotation, tree, rank, world)

    # 4: every rank's pack on every rank (one all-gather, padded to the largest)
    pk = ops.pack(shard)
    size = torch.tensor([pk.numel()], dtype=torch.int64, device=dev)
    sizes = [torch.empty_like(size) for _ in range(world)]
    dist.all_gather(sizes, size, group=group)
    sizes = [int(s.item()) for s in sizes]
    cap = max(sizes)
    padded = torch.zeros(cap, dtype=torch.int64, device=dev)
    padded[: pk.numel()] = pk
    gathered = [torch.empty(cap, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(gathered, padded, group=group)

    # 5: the whole function
    full = ops.concat([g[:s] for g, s in zip(gathered, sizes)])
    return full, shard
