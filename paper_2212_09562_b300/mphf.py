"""Python binding of libmphf (the C ABI in include/mphf.h).

Argument marshalling only: every step of a build or query runs in the CUDA
library.  PyTorch provides device memory and the current stream.  There is
no fallback: if the library is missing or cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# MPHF_LIBRARY selects another build of the same library (e.g. a tuning variant).
LIB_PATH = os.environ.get("MPHF_LIBRARY") or os.path.join(HERE, "libmphf.so")

OK = 0
EINVAL = -1
ENOMEM = -2
ECUDA = -3
EDUPLICATE = -4
ESEARCH_LIMIT = -5
EBUSY = -6
EBUCKET = -7
ENOTIMPL = -8
ETIMEOUT = -9
ECAPACITY = -10
MAX_BUCKET = 4096
VERIFY_STATIC_MAX_KEYS = 1 << 20
DEFAULT_MAX_VALUE = (1 << 40) - 1
LEAF_LOCKSTEP, LEAF_EARLY, LEAF_TABLE = 0, 1, 2
# leaf bijection methods; every ``rotation`` argument takes a bool or one of these
PLAIN, ROTATION, SHOCKHASH = 0, 1, 2
# tree shapes: RecSplit's lower aggregation levels, or fanout 2 everywhere (Appendix C)
TREE_RECSPLIT, TREE_FANOUT2 = 0, 1
SH_SEED_BITS = 40  # a ShockHash leaf's value: seed below bit 40, retrieval vector above


def bijection(rotation) -> int:
    """MPHF_BIJECTION_* code from a bool (rotation fitting on/off) or PLAIN/ROTATION/SHOCKHASH."""
    v = int(rotation)
    if v not in (PLAIN, ROTATION, SHOCKHASH):
        raise ValueError(f"unknown leaf method {rotation!r}")
    return v

_lock = threading.Lock()
_lib = None


class MPHFError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        msg = lib().mphf_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")
        self.code = code


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ctypes.c_void_p), ("free", ctypes.c_void_p), ("ctx", ctypes.c_void_p)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class TorchAllocator:
    """mphf_allocator hooks backed by torch's caching allocator, so that the
    library's device arrays count in torch's memory statistics and limits.
    ``live`` is the number of blocks handed out and not yet returned.  Keep
    the object alive while any function built with it exists (each MPHF
    holds a reference)."""

    def __init__(self):
        torch = _torch()
        self.live = 0

        def alloc(nbytes, stream, ctx):
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
            except Exception:  # out of memory: the library sees NULL
                return None
            self.live += 1
            return p

        def free(ptr, stream, ctx):
            torch.cuda.caching_allocator_delete(int(ptr))
            self.live -= 1

        self._alloc, self._free = _ALLOC_FN(alloc), _FREE_FN(free)
        self.struct = Allocator(ctypes.cast(self._alloc, ctypes.c_void_p),
                                ctypes.cast(self._free, ctypes.c_void_p), None)


class BuildParams(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_uint32), ("bucket_size", ctypes.c_uint32),
                ("key_bytes", ctypes.c_uint32), ("leaf_bijection", ctypes.c_uint32),
                ("max_value", ctypes.c_uint64), ("allocator", ctypes.c_void_p),
                ("threads_per_block", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32),
                ("leaf_method", ctypes.c_uint32), ("tree_shape", ctypes.c_uint32),
                ("seeds_per_thread", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("nb", ctypes.c_uint64), ("leaf_size", ctypes.c_uint32),
                ("bucket_size", ctypes.c_uint32), ("key_bytes", ctypes.c_uint32),
                ("leaf_bijection", ctypes.c_uint32), ("n_nodes", ctypes.c_uint64),
                ("gr_bits", ctypes.c_uint64), ("gr_words", ctypes.c_uint64),
                ("ef_words", ctypes.c_uint64), ("ef_low_bits", ctypes.c_uint32 * 2),
                ("ef_seq_words", ctypes.c_uint64 * 4), ("max_bucket", ctypes.c_uint32),
                ("tree_shape", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    _fields_ = [("trials", ctypes.c_uint64 * 4), ("evals", ctypes.c_uint64 * 4),
                ("ms_plan", ctypes.c_float), ("ms_search", ctypes.c_float),
                ("ms_pack", ctypes.c_float), ("ms_total", ctypes.c_float)]


class ServerCfg(ctypes.Structure):
    _fields_ = [("max_requests", ctypes.c_uint32), ("reserved_sms", ctypes.c_uint32),
                ("hbm_reserve_bytes", ctypes.c_uint64), ("idle_ms", ctypes.c_uint32),
                ("threads", ctypes.c_uint32)]


class RequestTimes(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_double), ("admitted", ctypes.c_double),
                ("finished", ctypes.c_double)]


class BuildDesc(ctypes.Structure):
    _fields_ = [("d_keys", ctypes.c_void_p), ("n", ctypes.c_uint64), ("leaf_size", ctypes.c_uint32),
                ("bucket_size", ctypes.c_uint32), ("key_bytes", ctypes.c_uint32),
                ("leaf_bijection", ctypes.c_uint32), ("max_value", ctypes.c_uint64),
                ("tree_shape", ctypes.c_uint32), ("seeds_per_thread", ctypes.c_uint32)]


# Every entry point of include/mphf.h: name -> (restype, argtypes)
_P, _U32, _U64, _I = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
SIGNATURES = {
    "mphf_default_params": (None, [_P]),
    "mphf_build": (_I, [_P, _U64, _U32, _U32, _P, _P]),
    "mphf_build_ex": (_I, [_P, _U64, _P, _P, _P]),
    "mphf_build_host": (_I, [_P, _U64, _P, _P, _P]),
    "mphf_query": (_I, [_P, _P, _U64, _P, _P]),
    "mphf_verify": (_I, [_P, _P, _U64, _P, _P]),
    "mphf_verify_static": (_I, [_P, _P, _U64, _P, _P]),
    "mphf_get_info": (_I, [_P, _P]),
    "mphf_get_values": (_I, [_P, _P, _P, _P, _P]),
    "mphf_get_bits": (_I, [_P, _P, _P, _P, _P]),
    "mphf_get_stats": (_I, [_P, _P]),
    "mphf_tau_table": (_I, [_U32, _U32, _U32, _U32, _P]),
    "mphf_serialize": (_I, [_P, _P, _P, _P]),
    "mphf_load_info": (_I, [_P, ctypes.c_size_t, _P]),
    "mphf_load": (_I, [_P, ctypes.c_size_t, _P, _P, _P]),
    "mphf_free": (_I, [_P]),
    "mphf_strerror": (ctypes.c_char_p, [_I]),
    "mphf_build_batch": (_I, [_P, _U32, _P, _P, _P]),
    "mphf_kernel_launches": (_U64, []),
    "mphf_server_create": (_I, [_P, _P]),
    "mphf_server_submit": (_I, [_P, _P, _P]),
    "mphf_server_poll": (_I, [_P, _U64, _U32, _P, _P, _P]),
    "mphf_server_destroy": (_I, [_P]),
    "mphf_build_prepare": (_I, [_U64, _P, _U64, _P]),
    "mphf_build_enqueue": (_I, [_P, _P, _P]),
    "mphf_build_finish": (_I, [_P, _P]),
    "mphf_batch_prepare": (_I, [_P, _U32, _U32, _U32, _P, _P]),
    "mphf_batch_enqueue": (_I, [_P, _P, _P]),
    "mphf_batch_finish": (_I, [_P, _P, _P]),
    "mphf_batch_free": (_I, [_P]),
    "mphf_shard_route": (_I, [_P, _U64, _U32, _U64, _U32, _U32, _P, _P, _P]),
    "mphf_build_shard": (_I, [_P, _U64, _U64, _P, _U32, _U32, _P, _P]),
    "mphf_shard_pack": (_I, [_P, _P, _P, _P]),
    "mphf_shard_concat": (_I, [_P, _P, _U32, _P, _P, _P]),
}


def lib() -> ctypes.CDLL:
    """Loads libmphf.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_2212_09562_b300.build`")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != OK:
        raise MPHFError(rc, what)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required")
    return torch


def _stream(stream) -> int:
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


class _DevArray:
    """Exposes a library-owned device array to torch (no copy)."""

    def __init__(self, ptr: int, count: int, typestr: str = "<u8"):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": typestr,
                                         "data": (ptr, False), "version": 3, "strides": None}


def _device_view(ptr: int, count: int):
    torch = _torch()
    if count == 0 or not ptr:
        return torch.zeros(0, dtype=torch.int64, device="cuda")
    return torch.as_tensor(_DevArray(ptr, count, "<i8"), device="cuda")


def key_layout(keys) -> tuple[int, int]:
    """(n, key_bytes) of a device key tensor: (n,) 64-bit, or (n, 16) bytes / (n, 2) 64-bit."""
    torch = _torch()
    if not keys.is_cuda or not keys.is_contiguous():
        raise ValueError("keys must be a contiguous CUDA tensor")
    if keys.numel() and keys.data_ptr() % 8:
        raise ValueError("keys must be 8-byte aligned")
    if keys.dim() == 1 and keys.element_size() == 8:
        return keys.shape[0], 8
    if keys.dim() == 2 and keys.dtype == torch.uint8 and keys.shape[1] == 16:
        return keys.shape[0], 16
    if keys.dim() == 2 and keys.element_size() == 8 and keys.shape[1] == 2:
        return keys.shape[0], 16
    raise ValueError("keys must be (n,) 64-bit or (n, 16) uint8 / (n, 2) 64-bit")


def host_key_bytes(keys: np.ndarray) -> int:
    """Key size of a host key array: (n,) of a 64-bit type, or (n, 16) uint8 / (n, 2) 64-bit."""
    if keys.ndim == 1 and keys.itemsize == 8:
        return 8
    if keys.ndim == 2 and keys.dtype == np.uint8 and keys.shape[1] == 16:
        return 16
    if keys.ndim == 2 and keys.itemsize == 8 and keys.shape[1] == 2:
        return 16
    raise ValueError("host keys must be (n,) 64-bit or (n, 16) uint8 / (n, 2) 64-bit")


def default_params() -> BuildParams:
    p = BuildParams()
    lib().mphf_default_params(ctypes.byref(p))
    return p


class MPHF:
    """A function built on the device by libmphf."""

    def __init__(self, handle: int, allocator: "TorchAllocator | None" = None):
        self._h = ctypes.c_void_p(handle)
        self._allocator = allocator  # frees of this function's arrays go through it
        info = Info()
        _check(lib().mphf_get_info(self._h, ctypes.byref(info)), "mphf_get_info")
        self.info = info

    # --- construction -------------------------------------------------------
    @classmethod
    def build(cls, keys, leaf_size: int = 16, bucket_size: int = 2000, rotation=True,
              max_value: int = DEFAULT_MAX_VALUE, threads_per_block: int = 0,
              blocks_per_sm: int = 0, stream=None, tuned: bool = False,
              leaf_method: int | None = None, tree: int = TREE_RECSPLIT,
              allocator: "TorchAllocator | None" = None, seeds_per_thread: int = 0) -> "MPHF":
        """rotation: True/False or PLAIN, ROTATION, SHOCKHASH (the leaf method);
        tree: TREE_RECSPLIT or TREE_FANOUT2;
        tuned=True takes the launch shape and seeds per thread from the
        autotuner's cache (the library default where nothing is cached);
        leaf_method: LEAF_LOCKSTEP (default), LEAF_EARLY or LEAF_TABLE;
        allocator: device memory hooks (default: the library's cudaMallocAsync)."""
        n, kb = key_layout(keys)
        if tuned and not threads_per_block and not blocks_per_sm and not seeds_per_thread:
            from .autotune import tuned as cached_shape
            threads_per_block, blocks_per_sm, seeds_per_thread = cached_shape(leaf_size, rotation, tree)
        p = default_params()
        p.leaf_size, p.bucket_size, p.key_bytes = leaf_size, bucket_size, kb
        p.leaf_bijection = bijection(rotation)
        p.tree_shape = tree
        p.max_value = max_value
        p.threads_per_block, p.blocks_per_sm = threads_per_block, blocks_per_sm
        p.seeds_per_thread = seeds_per_thread
        if leaf_method is not None:
            p.leaf_method = leaf_method
        if allocator is not None:
            p.allocator = ctypes.cast(ctypes.pointer(allocator.struct), ctypes.c_void_p)
        h = ctypes.c_void_p()
        rc = lib().mphf_build_ex(keys.data_ptr() if n else None, n, ctypes.byref(p),
                                 _stream(stream), ctypes.byref(h))
        _check(rc, "mphf_build_ex")
        return cls(h.value, allocator)

    @classmethod
    def prepare(cls, n: int, leaf_size: int = 16, bucket_size: int = 2000, rotation=True,
                key_bytes: int = 8, tree: int = TREE_RECSPLIT, max_value: int = DEFAULT_MAX_VALUE,
                seeds_per_thread: int = 0, gr_capacity_bits: int = 0) -> "MPHF":
        """A build of exactly n keys whose device work can be captured in a CUDA
        graph: enqueue(keys) issues it, finish() makes the function usable."""
        _torch()
        p = default_params()
        p.leaf_size, p.bucket_size, p.key_bytes = leaf_size, bucket_size, key_bytes
        p.leaf_bijection, p.tree_shape = bijection(rotation), tree
        p.max_value, p.seeds_per_thread = max_value, seeds_per_thread
        h = ctypes.c_void_p()
        _check(lib().mphf_build_prepare(n, ctypes.byref(p), gr_capacity_bits, ctypes.byref(h)),
               "mphf_build_prepare")
        obj = cls.__new__(cls)
        obj._h, obj._allocator, obj.info = h, None, Info()
        _check(lib().mphf_get_info(h, ctypes.byref(obj.info)), "mphf_get_info")
        return obj

    def enqueue(self, keys, stream=None):
        """Issues the prepared build of `keys` (n keys, the prepared key size) on
        the stream; capturable."""
        n, kb = key_layout(keys)
        if n != self.info.n or kb != self.info.key_bytes:
            raise ValueError("keys must be the prepared number and size")
        _check(lib().mphf_build_enqueue(self._h, keys.data_ptr(), _stream(stream)), "mphf_build_enqueue")

    def finish(self, stream=None):
        """Waits for the enqueued build and makes the function usable (raises its error)."""
        _check(lib().mphf_build_finish(self._h, _stream(stream)), "mphf_build_finish")
        _check(lib().mphf_get_info(self._h, ctypes.byref(self.info)), "mphf_get_info")

    @classmethod
    def build_host(cls, keys: np.ndarray, leaf_size: int = 16, bucket_size: int = 2000,
                   rotation=True, max_value: int = DEFAULT_MAX_VALUE,
                   stream=None, tree: int = TREE_RECSPLIT) -> "MPHF":
        """Build from keys in host memory (copied to the device inside the call)."""
        keys = np.ascontiguousarray(keys)
        kb = host_key_bytes(keys)
        p = default_params()
        p.leaf_size, p.bucket_size, p.key_bytes = leaf_size, bucket_size, kb
        p.leaf_bijection = bijection(rotation)
        p.tree_shape = tree
        p.max_value = max_value
        h = ctypes.c_void_p()
        rc = lib().mphf_build_host(keys.ctypes.data if len(keys) else None, len(keys),
                                   ctypes.byref(p), _stream(stream), ctypes.byref(h))
        _check(rc, "mphf_build_host")
        return cls(h.value)

    @classmethod
    def load(cls, blob: bytes, stream=None, allocator: "TorchAllocator | None" = None) -> "MPHF":
        """Rebuild a function on the current device from serialize()'s bytes
        (checked on the host first; a corrupt blob raises MPHFError EINVAL)."""
        _torch()
        h = ctypes.c_void_p()
        a = ctypes.byref(allocator.struct) if allocator is not None else None
        _check(lib().mphf_load(blob, len(blob), a, _stream(stream), ctypes.byref(h)), "mphf_load")
        return cls(h.value, allocator)

    # --- evaluation ---------------------------------------------------------
    def _count(self, keys) -> int:
        """Number of keys in a device tensor laid out like the built function's keys."""
        n, kb = key_layout(keys)
        if n and kb != self.info.key_bytes:
            raise ValueError("key size differs from the built function's")
        return n

    def query(self, keys, out=None, stream=None):
        torch = _torch()
        n = self._count(keys)
        if out is None:
            out = torch.empty(n, dtype=torch.int64, device=keys.device)
        elif (not out.is_cuda or out.device != keys.device or not out.is_contiguous()
              or out.element_size() != 8 or out.numel() < n or (n and out.data_ptr() % 8)):
            raise ValueError("out must be a contiguous 64-bit tensor of at least n elements "
                             "on the keys' device")
        _check(lib().mphf_query(self._h, keys.data_ptr() if n else None, n,
                                out.data_ptr() if n else None, _stream(stream)), "mphf_query")
        return out

    def verify(self, keys, stream=None) -> int:
        """Number of keys whose value is out of range or repeated (0 = bijection)."""
        n = self._count(keys)
        bad = ctypes.c_uint64()
        _check(lib().mphf_verify(self._h, keys.data_ptr() if n else None, n, ctypes.byref(bad),
                                 _stream(stream)), "mphf_verify")
        return int(bad.value)

    def verify_static(self, keys, stream=None) -> int:
        """Like verify(), without allocating device memory: a fixed scratch area
        reserved by the library serves every call (at most VERIFY_STATIC_MAX_KEYS
        keys; calls must not overlap on the device)."""
        n = self._count(keys)
        bad = ctypes.c_uint64()
        _check(lib().mphf_verify_static(self._h, keys.data_ptr() if n else None, n,
                                        ctypes.byref(bad), _stream(stream)), "mphf_verify_static")
        return int(bad.value)

    # --- contents -----------------------------------------------------------
    def device_arrays(self) -> dict:
        """Zero-copy torch views (int64) of the library-owned arrays."""
        ptrs = [ctypes.c_void_p() for _ in range(4)]
        _check(lib().mphf_get_values(self._h, *[ctypes.byref(p) for p in ptrs]), "mphf_get_values")
        gr, ef = ctypes.c_void_p(), ctypes.c_void_p()
        bits, words = ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().mphf_get_bits(self._h, ctypes.byref(gr), ctypes.byref(bits), ctypes.byref(ef),
                                   ctypes.byref(words)), "mphf_get_bits")
        nb = self.info.nb
        return {
            "values": _device_view(ptrs[0].value, self.info.n_nodes),
            "node_off": _device_view(ptrs[1].value, nb + 1),
            "cum_keys": _device_view(ptrs[2].value, nb + 1),
            "bit_pos": _device_view(ptrs[3].value, nb + 1),
            "gr": _device_view(gr.value, self.info.gr_words),
            "ef": _device_view(ef.value, words.value),
        }

    def host_arrays(self) -> dict:
        """The same arrays copied to host numpy uint64."""
        out = {}
        for k, v in self.device_arrays().items():
            out[k] = v.cpu().numpy().view(np.uint64).copy()
        return out

    def stats(self) -> dict:
        s = Stats()
        _check(lib().mphf_get_stats(self._h, ctypes.byref(s)), "mphf_get_stats")
        kinds = ("leaf", "lower1", "lower2", "upper")
        d = {k: (int(s.trials[i]), int(s.evals[i])) for i, k in enumerate(kinds)}
        d["ms"] = {"plan": s.ms_plan, "search": s.ms_search, "pack": s.ms_pack, "total": s.ms_total}
        return d

    def serialize(self, stream=None) -> bytes:
        n = ctypes.c_size_t()
        _check(lib().mphf_serialize(self._h, None, ctypes.byref(n), _stream(stream)), "mphf_serialize")
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().mphf_serialize(self._h, buf, ctypes.byref(n), _stream(stream)), "mphf_serialize")
        return buf.raw[: n.value]

    def close(self):
        if self._h and self._h.value:
            lib().mphf_free(self._h)
            self._h = ctypes.c_void_p()
        self._allocator = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def load_info(blob: bytes) -> Info:
    """Sizes of a serialised function, after the same host-side checks as
    MPHF.load (no device needed)."""
    info = Info()
    _check(lib().mphf_load_info(blob, len(blob), ctypes.byref(info)), "mphf_load_info")
    return info


def kernel_launches() -> int:
    """Kernels the library has launched in this process so far."""
    return int(lib().mphf_kernel_launches())


def tau_table(leaf_size: int, rotation, max_m: int = MAX_BUCKET,
              tree: int = TREE_RECSPLIT) -> np.ndarray:
    out = np.zeros(max_m + 1, np.uint8)
    _check(lib().mphf_tau_table(leaf_size, bijection(rotation), tree, max_m, out.ctypes.data),
           "mphf_tau_table")
    return out


def build_batch(keys_list, leaf_sizes, bucket_size: int = 2000, rotation=True,
                max_value: int = 0, stream=None, tree: int = TREE_RECSPLIT,
                tuned: bool = True) -> list[MPHF]:
    """Many independent builds in one call (see mphf_build_batch).  tuned:
    each build's seeds per thread from the autotuner's cache for its leaf size
    (the library default where nothing is cached)."""
    count = len(keys_list)
    if len(leaf_sizes) != count:
        raise ValueError("one leaf size per key set")
    spt = {}
    if tuned:
        from .autotune import tuned as cached_shape
        spt = {l: cached_shape(l, rotation, tree)[2] for l in set(leaf_sizes)}
    descs = (BuildDesc * max(count, 1))()
    for i, (k, l) in enumerate(zip(keys_list, leaf_sizes)):
        n, kb = key_layout(k)
        descs[i] = BuildDesc(k.data_ptr() if n else None, n, l, bucket_size, kb,
                             bijection(rotation), max_value, tree, spt.get(l, 0))
    outs = (ctypes.c_void_p * max(count, 1))()
    sts = (ctypes.c_int * max(count, 1))()
    rc = lib().mphf_build_batch(descs, count, _stream(stream), outs, sts)
    if rc != OK:
        for i in range(count):
            if outs[i]:
                lib().mphf_free(ctypes.c_void_p(outs[i]))
        _check(rc, "mphf_build_batch")
    return [MPHF(outs[i]) for i in range(count)]


class PreparedBatch:
    """Prepared builds (MPHF.prepare) searched by one persistent launch
    (mphf_batch_*): enqueue(keys_list) issues all of them without allocation
    or host synchronisation (capturable in a CUDA graph), finish() makes every
    member usable.  The members stay owned by the caller and must outlive the
    batch."""

    def __init__(self, members, threads: int = 0, blocks_per_sm: int = 0):
        _torch()
        self.members = list(members)
        count = len(self.members)
        hs = (ctypes.c_void_p * max(count, 1))(*[m._h.value for m in self.members])
        b = ctypes.c_void_p()
        _check(lib().mphf_batch_prepare(hs, count, threads, blocks_per_sm, None, ctypes.byref(b)),
               "mphf_batch_prepare")
        self._b = b
        self._ptrs = (ctypes.c_void_p * max(count, 1))()

    def enqueue(self, keys_list, stream=None):
        """Issues every member's build from keys_list[i] (its prepared n and key size)."""
        if len(keys_list) != len(self.members):
            raise ValueError("one key set per member")
        for i, (m, k) in enumerate(zip(self.members, keys_list)):
            n, kb = key_layout(k)
            if n != m.info.n or kb != m.info.key_bytes:
                raise ValueError(f"keys of member {i} must be its prepared number and size")
            self._ptrs[i] = k.data_ptr()
        _check(lib().mphf_batch_enqueue(self._b, self._ptrs, _stream(stream)), "mphf_batch_enqueue")

    def finish(self, stream=None) -> list[int]:
        """Waits and finishes every member; returns their codes (raises if any failed)."""
        count = len(self.members)
        sts = (ctypes.c_int * max(count, 1))()
        rc = lib().mphf_batch_finish(self._b, _stream(stream), sts)
        for m in self.members:
            _check(lib().mphf_get_info(m._h, ctypes.byref(m.info)), "mphf_get_info")
        _check(rc, "mphf_batch_finish")
        return [sts[i] for i in range(count)]

    def close(self):
        if getattr(self, "_b", None):
            lib().mphf_batch_free(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Build server with continuous batching (mphf_server_*): requests join one
    serving search on the device and complete one by one."""

    def __init__(self, max_requests: int = 64, reserved_sms: int = 4, hbm_reserve_bytes: int = 0,
                 idle_ms: int = 0, threads: int = 0):
        _torch()
        cfg = ServerCfg(max_requests, reserved_sms, hbm_reserve_bytes, idle_ms, threads)
        h = ctypes.c_void_p()
        _check(lib().mphf_server_create(ctypes.byref(cfg), ctypes.byref(h)), "mphf_server_create")
        self._h = h
        self._keep = {}  # ticket -> key tensor, alive until the request is polled

    def submit(self, keys, leaf_size: int = 16, bucket_size: int = 2000, rotation=True,
               max_value: int = 0, tree: int = TREE_RECSPLIT, seeds_per_thread: int = 0) -> int:
        n, kb = key_layout(keys)
        d = BuildDesc(keys.data_ptr() if n else None, n, leaf_size, bucket_size, kb,
                      bijection(rotation), max_value, tree, seeds_per_thread)
        t = ctypes.c_uint64()
        _check(lib().mphf_server_submit(self._h, ctypes.byref(d), ctypes.byref(t)),
               "mphf_server_submit")
        self._keep[t.value] = keys
        return t.value

    def poll(self, ticket: int, timeout_ms: int = 0):
        """None if not finished; else (status, MPHF or None, (submitted, admitted, finished))."""
        out, st, tm = ctypes.c_void_p(), ctypes.c_int(), RequestTimes()
        rc = lib().mphf_server_poll(self._h, ticket, timeout_ms, ctypes.byref(out),
                                    ctypes.byref(st), ctypes.byref(tm))
        if rc == ETIMEOUT:
            return None
        _check(rc, "mphf_server_poll")
        self._keep.pop(ticket, None)
        built = MPHF(out.value) if out.value else None
        return st.value, built, (tm.submitted, tm.admitted, tm.finished)

    def close(self):
        if self._h and self._h.value:
            lib().mphf_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
