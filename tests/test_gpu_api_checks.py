"""Host-side argument checks of the query entry points on a real function.

Each rejected call returns MPHF_EINVAL (or raises ValueError in the binding)
before any kernel is launched: the kernel-launch counter does not move and
the stream has nothing to run.  Pointers handed to the library here are
either valid or rejected on the host by construction; none reaches a kernel.
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


@pytest.fixture(scope="module")
def built(torch):
    keys = W.random_keys(3000, 8, 4242)
    dkeys = torch.from_numpy(keys.view(np.int64)).cuda()
    return M.MPHF.build(dkeys, 8, 100, M.ROTATION), dkeys


def test_misaligned_pointers_are_rejected_on_the_host(torch, built):
    g, dkeys = built
    n = dkeys.numel()
    out = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    before = M.kernel_launches()
    L = M.lib()
    # a key pointer 4 bytes into the tensor, an output pointer 4 bytes in
    assert L.mphf_query(g._h, dkeys.data_ptr() + 4, n - 1, out.data_ptr(), stream) == M.EINVAL
    assert L.mphf_query(g._h, dkeys.data_ptr(), n, out.data_ptr() + 4, stream) == M.EINVAL
    bad = ctypes.c_uint64(99)
    assert L.mphf_verify(g._h, dkeys.data_ptr() + 4, n - 1, ctypes.byref(bad), stream) == M.EINVAL
    assert bad.value == 0
    assert L.mphf_verify_static(g._h, dkeys.data_ptr() + 4, n - 1, ctypes.byref(bad),
                                stream) == M.EINVAL
    assert L.mphf_query(g._h, None, n, out.data_ptr(), stream) == M.EINVAL
    assert L.mphf_query(g._h, dkeys.data_ptr(), n, None, stream) == M.EINVAL
    assert M.kernel_launches() == before
    # the aligned call still works and gives the bijection
    assert L.mphf_query(g._h, dkeys.data_ptr(), n, out.data_ptr(), stream) == M.OK
    v = out[:n].cpu().numpy()
    assert np.array_equal(np.sort(v), np.arange(n))


def test_binding_checks_the_output_tensor(torch, built):
    g, dkeys = built
    n = dkeys.numel()
    before = M.kernel_launches()
    for out in (torch.empty(n - 1, dtype=torch.int64, device="cuda"),     # too short
                torch.empty(n, dtype=torch.int32, device="cuda"),         # 4-byte elements
                torch.empty(2 * n, dtype=torch.int64, device="cuda")[::2],  # not contiguous
                torch.empty(n, dtype=torch.int64)):                       # host memory
        with pytest.raises(ValueError):
            g.query(dkeys, out=out)
    assert M.kernel_launches() == before
    out = torch.full((n + 5,), -1, dtype=torch.int64, device="cuda")
    g.query(dkeys, out=out)
    torch.cuda.synchronize()
    assert np.array_equal(np.sort(out[:n].cpu().numpy()), np.arange(n))
    assert (out[n:] == -1).all()  # nothing written past n


def test_empty_function_rejects_queries(torch):
    g = M.MPHF.build(torch.empty(0, dtype=torch.int64, device="cuda"), 8, 100)
    assert g.info.n == 0
    keys = torch.arange(4, dtype=torch.int64, device="cuda")
    out = torch.empty(4, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert M.lib().mphf_query(g._h, keys.data_ptr(), 4, out.data_ptr(), stream) == M.EINVAL
    assert M.lib().mphf_query(g._h, keys.data_ptr(), 0, out.data_ptr(), stream) == M.OK


def test_keys_of_the_other_width_are_rejected(torch, built):
    """A function over 8-byte keys refuses 16-byte keys and the reverse: the C
    ABI takes no key length, so the binding checks it before any launch."""
    g8, dkeys8 = built
    keys16 = W.random_keys(500, 16, 4243)
    d16 = torch.from_numpy(np.ascontiguousarray(keys16)).cuda()
    g16 = M.MPHF.build(d16, 8, 100, M.ROTATION)
    before = M.kernel_launches()
    for g, wrong in ((g8, d16), (g16, dkeys8)):
        for call in (g.query, g.verify, g.verify_static):
            with pytest.raises(ValueError):
                call(wrong)
    assert M.kernel_launches() == before
    assert g16.verify(d16) == 0 and g8.verify_static(dkeys8) == 0
