"""Device memory through caller-supplied allocator hooks (mphf_allocator).

A build, a host-key build, a load and a verification take every device
array from the hooks and return every one of them; the function equals the
one built with the library's own allocator.  Failing the k-th allocation,
for every k a successful call makes, gives MPHF_ENOMEM with nothing left
allocated and no function returned.
"""
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


class CountingAllocator:
    """torch's caching allocator behind the hooks, counting calls; the
    allocation numbered fail_at (from 0) returns NULL."""

    def __init__(self, torch, fail_at=None):
        self.calls, self.live, self.fail_at = 0, 0, fail_at

        def alloc(nbytes, stream, ctx):
            k = self.calls
            self.calls += 1
            if k == self.fail_at:
                return None
            self.live += 1
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))

        def free(ptr, stream, ctx):
            torch.cuda.caching_allocator_delete(int(ptr))
            self.live -= 1

        self._a, self._f = M._ALLOC_FN(alloc), M._FREE_FN(free)
        self.struct = M.Allocator(ctypes.cast(self._a, ctypes.c_void_p),
                                  ctypes.cast(self._f, ctypes.c_void_p), None)

    def params(self, leaf, bucket, bij, tree, kb):
        p = M.default_params()
        p.leaf_size, p.bucket_size, p.key_bytes = leaf, bucket, kb
        p.leaf_bijection, p.tree_shape = bij, tree
        p.allocator = ctypes.cast(ctypes.pointer(self.struct), ctypes.c_void_p)
        return p


def _stream(torch):
    return torch.cuda.current_stream().cuda_stream


def test_torch_allocator_build_and_load(torch):
    keys = W.random_keys(20000, 8, 61)
    dkeys = to_dev(torch, keys)
    ref = M.MPHF.build(dkeys, 12, 500, M.ROTATION)
    a = M.TorchAllocator()
    before = torch.cuda.memory_allocated()
    g = M.MPHF.build(dkeys, 12, 500, M.ROTATION, allocator=a)
    assert a.live == 7  # values, node_off, cum_keys, bit_pos, gr, ef, directories
    assert torch.cuda.memory_allocated() > before
    for k, v in ref.host_arrays().items():
        assert np.array_equal(g.host_arrays()[k], v), k
    assert g.verify(dkeys) == 0 and a.live == 7  # verification scratch returned
    h = M.MPHF.load(g.serialize(), allocator=a)
    assert a.live == 14
    assert np.array_equal(h.query(dkeys).cpu().numpy(), ref.query(dkeys).cpu().numpy())
    g.close()
    h.close()
    assert a.live == 0


@pytest.mark.parametrize("leaf,bucket,bij,tree,kb,n", [
    (12, 500, M.ROTATION, M.TREE_RECSPLIT, 8, 20000),
    (8, 100, M.ROTATION, M.TREE_RECSPLIT, 16, 5000),   # 16-byte keys
    (24, 2000, M.SHOCKHASH, M.TREE_FANOUT2, 8, 10000),
    (8, 5, M.PLAIN, M.TREE_RECSPLIT, 8, 60000),        # more than 8192 buckets: other sort path
])
def test_every_allocation_failure_is_clean(torch, leaf, bucket, bij, tree, kb, n):
    keys = W.random_keys(n, kb, 71 + n)
    dkeys = to_dev(torch, keys)
    ok = CountingAllocator(torch)
    p = ok.params(leaf, bucket, bij, tree, kb)
    h = ctypes.c_void_p()
    assert M.lib().mphf_build_ex(dkeys.data_ptr(), n, ctypes.byref(p), _stream(torch),
                                 ctypes.byref(h)) == M.OK
    total = ok.calls
    ref = M.MPHF(h.value, ok)
    assert total > 10
    for k in range(total):
        a = CountingAllocator(torch, fail_at=k)
        q = a.params(leaf, bucket, bij, tree, kb)
        out = ctypes.c_void_p(7)
        rc = M.lib().mphf_build_ex(dkeys.data_ptr(), n, ctypes.byref(q), _stream(torch),
                                   ctypes.byref(out))
        assert rc == M.ENOMEM and out.value is None and a.live == 0, k
    # host keys: the key buffer is one more allocation
    host = CountingAllocator(torch)
    hp = host.params(leaf, bucket, bij, tree, kb)
    assert M.lib().mphf_build_host(np.ascontiguousarray(keys).ctypes.data, n, ctypes.byref(hp),
                                   _stream(torch), ctypes.byref(h)) == M.OK
    assert host.calls == total + 1
    built = M.MPHF(h.value, host)
    for k in ref.host_arrays():
        assert np.array_equal(built.host_arrays()[k], ref.host_arrays()[k]), k
    for k in (0, total // 2, total):
        a = CountingAllocator(torch, fail_at=k)
        q = a.params(leaf, bucket, bij, tree, kb)
        out = ctypes.c_void_p(7)
        rc = M.lib().mphf_build_host(np.ascontiguousarray(keys).ctypes.data, n, ctypes.byref(q),
                                     _stream(torch), ctypes.byref(out))
        assert rc == M.ENOMEM and out.value is None and a.live == 0, k
    # load, and verification through the function's own hooks
    blob = ref.serialize()
    for k in range(9):  # a load makes 8 allocations
        a = CountingAllocator(torch, fail_at=k)
        out = ctypes.c_void_p(7)
        rc = M.lib().mphf_load(blob, len(blob), ctypes.byref(a.struct), _stream(torch),
                               ctypes.byref(out))
        if k < 8:
            assert rc == M.ENOMEM and out.value is None and a.live == 0, k
        else:
            assert rc == M.OK and a.live == 7
            loaded = M.MPHF(out.value, a)
            for j in range(3):  # a verification makes 3 allocations
                a.fail_at = a.calls + j
                bad = ctypes.c_uint64(5)
                assert M.lib().mphf_verify(loaded._h, dkeys.data_ptr(), n, ctypes.byref(bad),
                                           _stream(torch)) == M.ENOMEM
                assert a.live == 7
            assert loaded.verify(dkeys) == 0
            loaded.close()
            assert a.live == 0
    built.close()
    ref.close()
    assert host.live == 0 and ok.live == 0
