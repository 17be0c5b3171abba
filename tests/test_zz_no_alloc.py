"""The bijection check that allocates no device memory (mphf_verify_static).

Callers whose device memory is owned by another allocator, or who sit on a
path where an allocation may stall the device, use this entry point instead of
mphf_verify.  It must report exactly what mphf_verify reports, call after
call, although every call reuses the same fixed scratch area.  This file is
collected last so that a failure here stops a run only after every other
test has run.
"""
import ctypes

import numpy as np
import pytest

from paper_2212_09562_b300 import mphf as M
from paper_2212_09562_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2212_09562_b300 import build
    build.build()
    M.lib()
    return t


def _stream(torch):
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(fn, h, dkeys, n, torch):
    bad = ctypes.c_uint64()
    rc = fn(h._h, ctypes.c_void_p(dkeys.data_ptr()), n, ctypes.byref(bad), _stream(torch))
    return rc, bad.value


@pytest.mark.parametrize("n,leaf,bucket,kb", [(200_000, 12, 1000, 8), (M.VERIFY_STATIC_MAX_KEYS, 8, 100, 16)])
def test_static_verify_matches_verify_on_two_calls(torch, n, leaf, bucket, kb):
    keys = W.random_keys(n, kb, 606 + kb)
    dkeys = torch.from_numpy(keys.view(np.int64) if kb == 8 else keys).cuda()
    h = M.MPHF.build(dkeys, leaf, bucket, True)
    L = M.lib()
    for _ in range(2):
        rc_a, bad_a = _check(L.mphf_verify, h, dkeys, n, torch)
        rc_b, bad_b = _check(L.mphf_verify_static, h, dkeys, n, torch)
        assert rc_a == M.OK and rc_b == M.OK
        assert bad_a == bad_b == 0
    # keys outside the built set collide: both checks count the same bad keys
    other = W.random_keys(n // 2, kb, 707 + kb)
    mixed = np.concatenate([keys[: n - n // 2], other])
    dmixed = torch.from_numpy(mixed.view(np.int64) if kb == 8 else mixed).cuda()
    for _ in range(2):
        rc_a, bad_a = _check(L.mphf_verify, h, dmixed, n, torch)
        rc_b, bad_b = _check(L.mphf_verify_static, h, dmixed, n, torch)
        assert rc_a == M.OK and rc_b == M.OK
        assert bad_a == bad_b and bad_a > 0


def test_static_verify_rejects_more_keys_than_its_scratch(torch):
    n = M.VERIFY_STATIC_MAX_KEYS + 1
    keys = W.distinct_u64(n, 808)
    dkeys = torch.from_numpy(keys.view(np.int64)).cuda()
    h = M.MPHF.build(dkeys, 8, 100, True)
    rc, bad = _check(M.lib().mphf_verify_static, h, dkeys, n, torch)
    assert rc == M.EINVAL and bad == 0
    assert h.verify(dkeys) == 0


def test_static_verify_makes_no_allocator_call(torch):
    """With h built through counting allocator hooks, mphf_verify takes its
    scratch from those hooks on every call, while mphf_verify_static asks for
    nothing: its scratch is the library's fixed device array."""
    from test_gpu_allocator import CountingAllocator
    n = 300_000
    keys = W.distinct_u64(n, 909)
    dkeys = torch.from_numpy(keys.view(np.int64)).cuda()
    A = CountingAllocator(torch)
    p = A.params(12, 1000, M.ROTATION, M.TREE_RECSPLIT, 8)
    hh = ctypes.c_void_p()
    L = M.lib()
    assert L.mphf_build_ex(ctypes.c_void_p(dkeys.data_ptr()), n, ctypes.byref(p), _stream(torch),
                           ctypes.byref(hh)) == M.OK
    h = M.MPHF(hh.value)
    try:
        before = A.calls
        rc_a, bad_a = _check(L.mphf_verify, h, dkeys, n, torch)
        assert rc_a == M.OK and bad_a == 0 and A.calls > before
        torch.cuda.synchronize()
        mem0 = torch.cuda.memory_allocated()
        for _ in range(2):
            before = A.calls
            rc_b, bad_b = _check(L.mphf_verify_static, h, dkeys, n, torch)
            assert rc_b == M.OK and bad_b == 0
            assert A.calls == before
        assert torch.cuda.memory_allocated() == mem0
    finally:
        h.close()
    assert A.live == 0
