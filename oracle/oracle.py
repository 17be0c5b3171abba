"""ctypes wrapper around the plain CPU RecSplit oracle (``recsplit_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
CPU-baseline / reference legs of ``bench.py`` are the only callers.  The
product path never imports this module.

``build()`` compiles the C file with gcc into ``liboracle.so`` next to it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "recsplit_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

OK = 0
EINVAL = -1
ENOMEM = -2
EDUPLICATE = -4
ESEARCH_LIMIT = -5
EBUCKET = -7

MAX_BUCKET = 4096
DEFAULT_MAX_VALUE = (1 << 40) - 1

# leaf bijection methods (the ``rotation`` argument below takes a bool or one of these)
PLAIN = 0
ROTATION = 1
SHOCKHASH = 2
SH_SEED_BITS = 40          # a ShockHash leaf word: seed in bits 0..39, retrieval vector above
SH_RETRIEVAL_LEVEL = 63    # salt level of the retrieval rows
# tree shapes: RecSplit's two lower aggregation levels, or fanout 2 everywhere (Appendix C)
TREE_RECSPLIT = 0
TREE_FANOUT2 = 1
_FANOUT2_FLAG = 0x100      # carried on the leaf size argument of the C functions
STAT_KINDS = ("leaf", "lower1", "lower2", "upper")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, pthreads) if the library is missing or stale."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-fPIC", "-shared", "-pthread",
             SRC, "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB)
            u64, u32, p = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
            L.orc_mix64.restype = u64
            L.orc_mix64.argtypes = [u64]
            L.orc_fingerprint.argtypes = [p, u64, u32, p, p]
            L.orc_bucket_of.restype = u64
            L.orc_bucket_of.argtypes = [u64, u64]
            L.orc_fanouts.argtypes = [u32, p, p]
            L.orc_parts.restype = u32
            L.orc_parts.argtypes = [u32, u32, p]
            L.orc_count_nodes.restype = u64
            L.orc_count_nodes.argtypes = [u32, u32]
            L.orc_salt.restype = u64
            L.orc_salt.argtypes = [u32]
            L.orc_rotation_success_bound.restype = ctypes.c_double
            L.orc_rotation_success_bound.argtypes = [u32]
            L.orc_rotation_bound_given_a.restype = ctypes.c_double
            L.orc_rotation_bound_given_a.argtypes = [u32, u32]
            L.orc_plain_success.restype = ctypes.c_double
            L.orc_plain_success.argtypes = [u32]
            L.orc_split_success.restype = ctypes.c_double
            L.orc_split_success.argtypes = [u32, u32]
            L.orc_kiely_tau.restype = u32
            L.orc_kiely_tau.argtypes = [ctypes.c_double]
            L.orc_tau_table.argtypes = [u32, ctypes.c_int, u32, p]
            L.orc_build.restype = ctypes.c_int
            L.orc_build.argtypes = [p, u64, u32, u32, u32, ctypes.c_int, u64, ctypes.c_int,
                                    ctypes.POINTER(p)]
            L.orc_build_sample.restype = ctypes.c_int
            L.orc_build_range.restype = ctypes.c_int
            L.orc_build_range.argtypes = [p, u64, u32, u64, u32, u32, ctypes.c_int, u64, ctypes.c_int,
                                          u64, u64, p]
            L.orc_build_sample.argtypes = [p, u64, u32, u32, u32, ctypes.c_int, u64, ctypes.c_int,
                                           p, u64, p, p, p]
            L.orc_free.argtypes = [p]
            L.orc_query.argtypes = [p, p, u64, p]
            L.orc_sizes.argtypes = [p, p]
            L.orc_copy_out.argtypes = [p, p, p, p, p, p, p, p]
            L.orc_node_search.restype = ctypes.c_int
            L.orc_node_search.argtypes = [u32, ctypes.c_int, p, p, u32, u32, u64, p, p]
            L.orc_shockhash_orient_prob.restype = ctypes.c_double
            L.orc_shockhash_orient_prob.argtypes = [u32]
            L.orc_retrieval_solvable_prob.restype = ctypes.c_double
            L.orc_retrieval_solvable_prob.argtypes = [u32]
            L.orc_leaf_plain_early_exit.restype = u64
            L.orc_leaf_plain_early_exit.argtypes = [p, u32, p]
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _leaf(leaf: int, tree: int) -> int:
    if tree not in (TREE_RECSPLIT, TREE_FANOUT2):
        raise ValueError(f"unknown tree shape {tree!r}")
    return leaf | (_FANOUT2_FLAG if tree == TREE_FANOUT2 else 0)


def bij(rotation) -> int:
    """Leaf method code from a bool (rotation fitting on/off) or PLAIN/ROTATION/SHOCKHASH."""
    v = int(rotation)
    if v not in (PLAIN, ROTATION, SHOCKHASH):
        raise ValueError(f"unknown leaf method {rotation!r}")
    return v


def _key_bytes(keys: np.ndarray) -> tuple[np.ndarray, int]:
    """Keys as a contiguous byte view: (n,) uint64 -> 8 bytes, (n, 16) uint8 -> 16 bytes."""
    keys = np.ascontiguousarray(keys)
    if keys.dtype == np.uint64 and keys.ndim == 1:
        return keys, 8
    if keys.dtype == np.uint8 and keys.ndim == 2 and keys.shape[1] == 16:
        return keys, 16
    raise ValueError("keys must be (n,) uint64 or (n, 16) uint8")


def mix64(z: int) -> int:
    return int(lib().orc_mix64(z))


def fingerprint(keys: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    k, kb = _key_bytes(keys)
    n = k.shape[0]
    hi = np.empty(n, np.uint64)
    lo = np.empty(n, np.uint64)
    lib().orc_fingerprint(_ptr(k), n, kb, _ptr(hi), _ptr(lo))
    return hi, lo


def bucket_of(hi: int, nb: int) -> int:
    return int(lib().orc_bucket_of(hi, nb))


def fanouts(leaf: int, tree: int = TREE_RECSPLIT) -> tuple[int, int]:
    f1 = ctypes.c_uint32()
    f2 = ctypes.c_uint32()
    lib().orc_fanouts(_leaf(leaf, tree), ctypes.addressof(f1), ctypes.addressof(f2))
    return f1.value, f2.value


def parts(leaf: int, m: int, tree: int = TREE_RECSPLIT) -> list[int]:
    out = np.zeros(16, np.uint32)
    k = lib().orc_parts(_leaf(leaf, tree), m, _ptr(out))
    return [int(v) for v in out[:k]]


def count_nodes(leaf: int, m: int, tree: int = TREE_RECSPLIT) -> int:
    return int(lib().orc_count_nodes(_leaf(leaf, tree), m))


def salt(level: int) -> int:
    return int(lib().orc_salt(level))


def rotation_success_bound(m: int) -> float:
    return float(lib().orc_rotation_success_bound(m))


def rotation_bound_given_a(m: int, a: int) -> float:
    return float(lib().orc_rotation_bound_given_a(m, a))


def plain_success(m: int) -> float:
    return float(lib().orc_plain_success(m))


def split_success(leaf: int, m: int, tree: int = TREE_RECSPLIT) -> float:
    return float(lib().orc_split_success(_leaf(leaf, tree), m))


def kiely_tau(p: float) -> int:
    return int(lib().orc_kiely_tau(p))


def shockhash_orient_prob(m: int) -> float:
    return float(lib().orc_shockhash_orient_prob(m))


def retrieval_solvable_prob(m: int) -> float:
    return float(lib().orc_retrieval_solvable_prob(m))


def tau_table(leaf: int, rotation, max_m: int = MAX_BUCKET, tree: int = TREE_RECSPLIT) -> np.ndarray:
    out = np.zeros(max_m + 1, np.uint8)
    lib().orc_tau_table(_leaf(leaf, tree), bij(rotation), max_m, _ptr(out))
    return out


class OracleMPHF:
    """A function built by the oracle; arrays are copied out into numpy."""

    def __init__(self, handle: int, keys_bytes: int):
        self._h = handle
        self.key_bytes = keys_bytes
        L = lib()
        sz = np.zeros(8, np.uint64)
        L.orc_sizes(handle, _ptr(sz))
        self.n, self.nb, self.n_nodes, self.gr_bits, gr_words, ef_words, lc, lp = (int(v) for v in sz)
        self.ef_L = (lc, lp)
        nb = self.nb
        self.cum_keys = np.zeros(nb + 1, np.uint64)
        self.node_off = np.zeros(nb + 1, np.uint64)
        self.values = np.zeros(max(self.n_nodes, 1), np.uint64)[: self.n_nodes]
        self.bit_pos = np.zeros(nb + 1, np.uint64)
        self.gr = np.zeros(max(gr_words, 1), np.uint64)[:gr_words]
        self.ef = np.zeros(max(ef_words, 1), np.uint64)[:ef_words]
        st = np.zeros(8, np.uint64)
        L.orc_copy_out(handle, _ptr(self.cum_keys), _ptr(self.node_off), _ptr(self.values),
                       _ptr(self.bit_pos), _ptr(self.gr), _ptr(self.ef), _ptr(st))
        self.stats = {k: (int(st[2 * i]), int(st[2 * i + 1])) for i, k in enumerate(STAT_KINDS)}

    def query(self, keys: np.ndarray) -> np.ndarray:
        k, kb = _key_bytes(keys)
        assert kb == self.key_bytes
        out = np.empty(k.shape[0], np.uint64)
        lib().orc_query(self._h, _ptr(k), k.shape[0], _ptr(out))
        return out

    def close(self):
        if self._h:
            lib().orc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle build failed with code {code}")
        self.code = code


def build_mphf(keys: np.ndarray, leaf: int, bucket: int, rotation=True,
               max_value: int = DEFAULT_MAX_VALUE, threads: int = 1,
               tree: int = TREE_RECSPLIT) -> OracleMPHF:
    k, kb = _key_bytes(keys)
    h = ctypes.c_void_p()
    rc = lib().orc_build(_ptr(k), k.shape[0], kb, _leaf(leaf, tree), bucket, bij(rotation), max_value,
                         threads, ctypes.byref(h))
    if rc != OK:
        raise OracleError(rc)
    return OracleMPHF(h.value, kb)


def build_range(keys: np.ndarray, n_total: int, leaf: int, bucket: int, rotation, b_lo: int,
                b_hi: int, max_value: int = DEFAULT_MAX_VALUE, threads: int = 1,
                tree: int = TREE_RECSPLIT) -> OracleMPHF:
    """Buckets [b_lo, b_hi) of the function over n_total keys, from the keys of
    exactly those buckets (Section 5.2's consecutive bucket range).  Its
    cum_keys, node_off and bit_pos are local to the range (start at 0); gr is
    the range's own Golomb-Rice sequence.  Not queryable."""
    k, kb = _key_bytes(keys)
    h = ctypes.c_void_p()
    rc = lib().orc_build_range(_ptr(k), k.shape[0], kb, n_total, _leaf(leaf, tree), bucket,
                               bij(rotation), max_value, threads, b_lo, b_hi, ctypes.byref(h))
    if rc != OK:
        raise OracleError(rc)
    return OracleMPHF(h.value, kb)


def build_sample(keys: np.ndarray, leaf: int, bucket: int, rotation, buckets: np.ndarray,
                 max_value: int = DEFAULT_MAX_VALUE, threads: int = 1, tree: int = TREE_RECSPLIT):
    """Values of the listed buckets only: (values concatenated in list order,
    node count per listed bucket, stats dict)."""
    k, kb = _key_bytes(keys)
    buckets = np.ascontiguousarray(buckets, dtype=np.uint64)
    counts = np.zeros(len(buckets), np.uint64)
    cap = MAX_BUCKET * len(buckets)  # a bucket has fewer stored nodes than keys
    vals = np.zeros(max(cap, 1), np.uint64)
    st = np.zeros(8, np.uint64)
    rc = lib().orc_build_sample(_ptr(k), k.shape[0], kb, _leaf(leaf, tree), bucket, bij(rotation),
                                max_value, threads, _ptr(buckets), len(buckets), _ptr(vals),
                                _ptr(counts), _ptr(st))
    if rc != OK:
        raise OracleError(rc)
    total = int(counts.sum())
    stats = {kname: (int(st[2 * i]), int(st[2 * i + 1])) for i, kname in enumerate(STAT_KINDS)}
    return vals[:total].copy(), counts, stats


def node_search(leaf: int, rotation, lo: np.ndarray, hi: np.ndarray | None = None,
                depth: int = 0, max_value: int = DEFAULT_MAX_VALUE, tree: int = TREE_RECSPLIT):
    """Search one node's value directly: returns (rc, value, trials, evals)."""
    lo = np.ascontiguousarray(lo, dtype=np.uint64)
    hi = np.zeros_like(lo) if hi is None else np.ascontiguousarray(hi, dtype=np.uint64)
    x = np.zeros(1, np.uint64)
    st = np.zeros(2, np.uint64)
    rc = lib().orc_node_search(_leaf(leaf, tree), bij(rotation), _ptr(lo), _ptr(hi), len(lo), depth,
                               max_value, _ptr(x), _ptr(st))
    return rc, int(x[0]), int(st[0]), int(st[1])


def leaf_plain_early_exit(lo: np.ndarray) -> tuple[int, int]:
    lo = np.ascontiguousarray(lo, dtype=np.uint64)
    e = np.zeros(1, np.uint64)
    s = lib().orc_leaf_plain_early_exit(_ptr(lo), len(lo), _ptr(e))
    return int(s), int(e[0])
