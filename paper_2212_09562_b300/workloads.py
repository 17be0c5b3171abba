"""Seeded synthetic workloads (keys and request streams) for tests and benchmarks.

This module only draws random inputs: it holds none of the hashing or search
arithmetic, so both the CUDA path and the CPU oracle can be fed from it.

The paper builds on synthetic keys only (Section 6, experimental setup:
random 128-bit integers used directly, or random strings).  The workloads:

* ``plain_l8``   n = 100,000 distinct uniform 64-bit keys, l = 8, b = 100, no rotation fitting
* ``rot_l12``    n = 1,000,000 distinct uniform 16-byte keys, l = 12, b = 1000, rotation fitting
* ``rot_l16``    n = 10,000,000 distinct uniform 64-bit keys, l = 16, b = 2000, rotation fitting
* ``shock_l16``  the keys and shape of ``rot_l16`` (another seed) with ShockHash leaves
  (Appendix C)
* ``shockf2_l24`` n = 10,000,000 distinct uniform 64-bit keys, l = 24, b = 2000, ShockHash
  leaves under a fanout-2 tree (the configuration of Appendix C)
* ``batch``      4,096 builds, n_i = floor(10^U(3,6)), l_i uniform in {8, 12, 16}, b = 2000
* ``serve``      Poisson request stream, mean 200/s, n ~ floor(10^U(4,7)) 16-byte keys, l = 16
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED_BASE = 12345


@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    leaf: int
    bucket: int
    key_bytes: int
    rotation: int  # leaf method: 0 / False plain, 1 / True rotation fitting, 2 ShockHash
    seed: int
    tree: int = 0  # 0 lower aggregation levels, 1 fanout 2 everywhere


WORKLOADS = {
    "plain_l8": Workload("plain_l8", 100_000, 8, 100, 8, False, SEED_BASE + 1),
    "rot_l12": Workload("rot_l12", 1_000_000, 12, 1000, 16, True, SEED_BASE + 2),
    "rot_l16": Workload("rot_l16", 10_000_000, 16, 2000, 8, True, SEED_BASE + 3),
    "shock_l16": Workload("shock_l16", 10_000_000, 16, 2000, 8, 2, SEED_BASE + 4),
    "shockf2_l24": Workload("shockf2_l24", 10_000_000, 24, 2000, 8, 2, SEED_BASE + 5, 1),
}


def distinct_u64(n: int, seed: int) -> np.ndarray:
    """n distinct uniform 64-bit keys in draw order (duplicates redrawn)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    keys = rng.integers(0, np.iinfo(np.uint64).max, size=n, dtype=np.uint64, endpoint=True)
    while True:
        _, first = np.unique(keys, return_index=True)
        if len(first) == n:
            return keys
        dup = np.ones(n, bool)
        dup[first] = False
        keys[dup] = rng.integers(0, np.iinfo(np.uint64).max, size=int(dup.sum()), dtype=np.uint64,
                                 endpoint=True)


def distinct_bytes16(n: int, seed: int) -> np.ndarray:
    """n distinct keys of 16 uniform bytes, shape (n, 16) uint8 (duplicates redrawn)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    keys = rng.integers(0, 256, size=(n, 16), dtype=np.uint8)
    while True:
        view = keys.view(np.dtype((np.void, 16))).reshape(n)
        _, first = np.unique(view, return_index=True)
        if len(first) == n:
            return keys
        dup = np.ones(n, bool)
        dup[first] = False
        keys[dup] = rng.integers(0, 256, size=(int(dup.sum()), 16), dtype=np.uint8)


def keys_for(w: Workload, n: int | None = None) -> np.ndarray:
    n = w.n if n is None else n
    return distinct_u64(n, w.seed) if w.key_bytes == 8 else distinct_bytes16(n, w.seed)


def random_keys(n: int, key_bytes: int, seed: int) -> np.ndarray:
    return distinct_u64(n, seed) if key_bytes == 8 else distinct_bytes16(n, seed)


def sample_buckets(nb: int, count: int, seed: int) -> np.ndarray:
    """A seeded sample of distinct bucket indices (sorted)."""
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    return np.sort(rng.choice(nb, size=min(count, nb), replace=False)).astype(np.uint64)


@dataclass(frozen=True)
class BatchInstance:
    n: int
    leaf: int
    seed: int


def batch_instances(count: int = 4096, seed: int = SEED_BASE + 4, lo_exp: float = 3.0,
                    hi_exp: float = 6.0, leaves=(8, 12, 16)) -> list[BatchInstance]:
    """Independent builds with log-uniform key counts and a leaf size drawn per build."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.floor(10.0 ** rng.uniform(lo_exp, hi_exp, size=count)).astype(np.int64)
    ls = rng.choice(np.asarray(leaves), size=count)
    return [BatchInstance(int(n), int(l), seed * 1000 + i) for i, (n, l) in enumerate(zip(ns, ls))]


def poisson_arrivals(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson request stream."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


def serve_sizes(count: int, seed: int, lo_exp: float = 4.0, hi_exp: float = 7.0) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    return np.floor(10.0 ** rng.uniform(lo_exp, hi_exp, size=count)).astype(np.int64)
