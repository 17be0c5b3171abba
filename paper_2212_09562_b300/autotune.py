"""Launch-shape autotuner for the search kernel.

For one leaf size and leaf method it builds a representative key set once per
candidate launch shape (threads per block, resident blocks per SM), times the
search kernel with the library's own CUDA events, checks that every candidate
produced the same function, and keeps the fastest.  Results are cached per
device name in a JSON file (``MPHF_TUNE_CACHE``, default
``~/.cache/mphf_tune.json``); ``tuned(leaf, rotation)`` returns the cached
shape or the library default.

    python -m paper_2212_09562_b300.autotune 8 12 16
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

from . import mphf as M
from . import workloads as W

CANDIDATES = [(128, 0), (256, 0), (512, 0), (256, 2), (512, 1)]
DEFAULT = (0, 0)  # library default (512 or 256 threads by tree and leaf size, as many blocks as fit)


def cache_path() -> str:
    return os.environ.get("MPHF_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "mphf_tune.json")


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _device_name() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _key(leaf: int, rotation, tree: int = M.TREE_RECSPLIT) -> str:
    """Cache key: device name, leaf size, leaf method and (fanout-2 only) tree shape."""
    k = f"{_device_name()}|l={leaf}|rot={M.bijection(rotation)}"
    return k if tree == M.TREE_RECSPLIT else f"{k}|tree={int(tree)}"


def tuned(leaf: int, rotation: bool = True, tree: int = M.TREE_RECSPLIT) -> tuple[int, int]:
    """(threads_per_block, blocks_per_sm) from the cache, else the library default."""
    entry = _load().get(_key(leaf, rotation, tree))
    return (int(entry["threads"]), int(entry["blocks_per_sm"])) if entry else DEFAULT


def tune(leaf: int, rotation: bool = True, n: int | None = None, bucket: int = 2000,
         candidates=CANDIDATES, save: bool = True, tree: int = M.TREE_RECSPLIT) -> dict:
    """Times every candidate shape on one build of n keys; returns the result record."""
    import torch
    if n is None:  # 1500 buckets of 2000 keys: five waves at the default shape, so the tail
        n = 3_000_000  # of the last wave does not decide (at 300 buckets it did)
    keys = torch.from_numpy(W.distinct_u64(n, 4711 + leaf).view(np.int64)).cuda()
    M.MPHF.build(keys[: min(n, 20_000)], leaf, bucket, rotation, tree=tree).close()  # warm-up
    times, ref = {}, None
    for threads, blocks in candidates:
        g = M.MPHF.build(keys, leaf, bucket, rotation, threads_per_block=threads,
                         blocks_per_sm=blocks, tree=tree)
        values = g.host_arrays()["values"]
        if ref is None:
            ref = values
        elif not np.array_equal(values, ref):
            raise RuntimeError(f"launch shape {(threads, blocks)} changed the result")
        times[(threads, blocks)] = g.stats()["ms"]["search"]
        g.close()
    best = min(times, key=times.get)
    rec = {"threads": best[0], "blocks_per_sm": best[1], "search_ms": times[best], "n": n,
           "bucket": bucket,
           "candidates": {f"{t}x{b}": ms for (t, b), ms in sorted(times.items())}}
    if save:
        data = _load()
        data[_key(leaf, rotation, tree)] = rec
        os.makedirs(os.path.dirname(cache_path()), exist_ok=True)
        tmp = cache_path() + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path())
    return rec


if __name__ == "__main__":
    for arg in sys.argv[1:] or ["16"]:
        print(arg, json.dumps(tune(int(arg))), flush=True)
