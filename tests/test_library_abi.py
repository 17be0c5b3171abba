"""The C-ABI library loads without a GPU, exports every entry point that
include/mphf.h declares, and its host-side tables equal the oracle's.

The Golomb-Rice parameter per node size (Section 2.2, "Representation") is
computed independently by the library and by the oracle; parity of the
packed bits needs the two tables to be equal.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2212_09562_b300 import build as B
from paper_2212_09562_b300 import mphf as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return M.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mphf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mphf_[a-z_]+)\s*\(", text)))


def test_header_declares_the_binding_surface():
    names = declared_functions()
    assert set(names) == set(M.SIGNATURES), set(names) ^ set(M.SIGNATURES)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_error_strings(lib):
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8, -9):
        assert lib.mphf_strerror(code)
    assert lib.mphf_strerror(-4).decode().startswith("duplicate")


def test_default_params(lib):
    p = M.default_params()
    assert (p.leaf_size, p.bucket_size, p.key_bytes, p.leaf_bijection) == (16, 2000, 8, 1)
    assert p.max_value == M.DEFAULT_MAX_VALUE


def test_invalid_arguments_are_rejected_without_a_device(lib):
    h = ctypes.c_void_p()
    p = M.default_params()
    for field, value in [("leaf_size", 1), ("leaf_size", 25), ("bucket_size", 0),
                         ("bucket_size", 3001), ("key_bytes", 4), ("threads_per_block", 100),
                         ("leaf_bijection", 3), ("leaf_method", 3), ("tree_shape", 2)]:
        q = M.default_params()
        setattr(q, field, value)
        assert lib.mphf_build_ex(None, 0, ctypes.byref(q), None, ctypes.byref(h)) == M.EINVAL
    assert lib.mphf_build_ex(None, 5, ctypes.byref(p), None, ctypes.byref(h)) == M.EINVAL
    assert lib.mphf_query(None, None, 0, None, None) == M.EINVAL
    assert lib.mphf_tau_table(1, 1, 0, 10, None) == M.EINVAL
    out = np.zeros(11, np.uint8)
    assert lib.mphf_tau_table(8, 3, 0, 10, out.ctypes.data) == M.EINVAL
    assert lib.mphf_tau_table(8, 1, 2, 10, out.ctypes.data) == M.EINVAL


def test_host_builds_check_their_parameters_before_copying_keys(lib):
    """mphf_build_host rejects bad parameters and oversized n before it
    allocates device memory or reads the host keys."""
    h = ctypes.c_void_p(1)
    keys = np.zeros(4, np.uint64)
    p = M.default_params()
    assert lib.mphf_build_host(keys.ctypes.data, 1 << 32, ctypes.byref(p), None,
                               ctypes.byref(h)) == M.EINVAL
    assert h.value is None  # *out is cleared on every failure
    for field, value in [("leaf_size", 1), ("bucket_size", 0), ("key_bytes", 12),
                         ("leaf_bijection", 7), ("tree_shape", 5)]:
        q = M.default_params()
        setattr(q, field, value)
        assert lib.mphf_build_host(keys.ctypes.data, 4, ctypes.byref(q), None,
                                   ctypes.byref(h)) == M.EINVAL
    assert lib.mphf_build_host(None, 4, ctypes.byref(p), None, ctypes.byref(h)) == M.EINVAL
    assert lib.mphf_build_host(keys.ctypes.data, 4, None, None, ctypes.byref(h)) == M.EINVAL


def test_handle_calls_reject_null_handles_and_misaligned_keys(lib):
    bad = ctypes.c_uint64(7)
    n_len = ctypes.c_size_t(0)
    assert lib.mphf_verify(None, None, 0, ctypes.byref(bad), None) == M.EINVAL
    assert lib.mphf_verify_static(None, None, 0, ctypes.byref(bad), None) == M.EINVAL
    assert lib.mphf_serialize(None, None, ctypes.byref(n_len), None) == M.EINVAL
    assert lib.mphf_get_info(None, None) == M.EINVAL
    assert lib.mphf_get_stats(None, None) == M.EINVAL
    assert lib.mphf_free(None) == M.EINVAL
    assert lib.mphf_server_poll(None, 1, 0, None, None, None) == M.EINVAL
    assert lib.mphf_server_destroy(None) == M.EINVAL
    assert lib.mphf_build_batch(None, 0, None, None, None) == M.OK  # an empty batch
    assert lib.mphf_build_batch(None, 2, None, None, None) == M.EINVAL
    # prepared batches: checked before any device call
    out = ctypes.c_void_p(1)
    assert lib.mphf_batch_prepare(None, 1, 0, 0, None, ctypes.byref(out)) == M.EINVAL
    assert out.value is None
    fake = (ctypes.c_void_p * 1)(8)
    assert lib.mphf_batch_prepare(fake, 0, 0, 0, None, ctypes.byref(out)) == M.EINVAL
    assert lib.mphf_batch_prepare(fake, 1, 100, 0, None, ctypes.byref(out)) == M.EINVAL
    assert lib.mphf_batch_prepare(fake, 1, 0, 0, None, None) == M.EINVAL
    assert lib.mphf_batch_enqueue(None, None, None) == M.EINVAL
    assert lib.mphf_batch_finish(None, None, None) == M.EINVAL
    assert lib.mphf_batch_free(None) == M.EINVAL
    # keys must be 8-byte aligned: checked on the host, before any device work
    h = ctypes.c_void_p()
    assert lib.mphf_build_ex(12, 5, ctypes.byref(M.default_params()), None,
                             ctypes.byref(h)) == M.EINVAL
    assert lib.mphf_query(None, 12, 5, 16, None) == M.EINVAL


def test_binding_rejects_key_arrays_of_the_wrong_shape():
    assert M.host_key_bytes(np.zeros(3, np.uint64)) == 8
    assert M.host_key_bytes(np.zeros(3, np.int64)) == 8
    assert M.host_key_bytes(np.zeros((3, 16), np.uint8)) == 16
    assert M.host_key_bytes(np.zeros((3, 2), np.uint64)) == 16
    for bad in (np.zeros(3, np.uint32), np.zeros((3, 8), np.uint8), np.zeros((3, 3), np.uint64),
                np.zeros((2, 2, 2), np.uint64)):
        with pytest.raises(ValueError):
            M.host_key_bytes(bad)
    with pytest.raises(ValueError):
        M.MPHF.build_host(np.zeros(3, np.uint32), 8, 100)
    with pytest.raises(ValueError):
        M.build_batch([], [8])


@pytest.mark.parametrize("leaf", list(range(2, 25)))
@pytest.mark.parametrize("rotation", [M.PLAIN, M.ROTATION, M.SHOCKHASH])
@pytest.mark.parametrize("tree", [M.TREE_RECSPLIT, M.TREE_FANOUT2])
def test_tau_tables_equal_the_oracle(lib, orc, leaf, rotation, tree):
    assert np.array_equal(M.tau_table(leaf, rotation, tree=tree),
                          orc.tau_table(leaf, rotation, tree=tree))
