"""Batched builds: many independent functions through one persistent search
launch must equal the same builds made one by one, and the oracle.

A failing member (duplicate keys, bad parameters) fails alone; the others
are unaffected.
"""
import os

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


def dev(torch, keys):
    return torch.from_numpy(keys.view(np.int64) if keys.ndim == 1 else np.ascontiguousarray(keys)).cuda()


def same(a, b):
    ha, hb = a.host_arrays(), b.host_arrays()
    for k in ha:
        assert np.array_equal(ha[k], hb[k]), k
    sa, sb = a.stats(), b.stats()
    for k in ("leaf", "lower1", "lower2", "upper"):
        assert sa[k] == sb[k], k


def test_batch_equals_one_by_one_and_oracle(torch, orc):
    specs = [(0, 8, 8), (1, 12, 16), (100, 8, 8), (5000, 8, 16), (20000, 12, 8), (3000, 16, 8),
             (777, 5, 8), (40000, 8, 8), (2500, 16, 16), (12345, 12, 16), (2, 16, 8), (999, 20, 8)]
    keys = [W.random_keys(n, kb, 900 + i) for i, (n, l, kb) in enumerate(specs)]
    dkeys = [dev(torch, k) for k in keys]
    leaves = [l for _, l, _ in specs]
    bucket = 100
    batch = M.build_batch(dkeys, leaves, bucket_size=bucket)
    for i, (k, dk, l) in enumerate(zip(keys, dkeys, leaves)):
        one = M.MPHF.build(dk, l, bucket, True)
        same(batch[i], one)
        if len(k):
            assert batch[i].verify(dk) == 0
        if i % 3 == 0 and len(k) <= 20000:
            o = orc.build_mphf(k, l, bucket, True, threads=8)
            assert np.array_equal(batch[i].host_arrays()["values"], o.values)
            assert np.array_equal(batch[i].host_arrays()["gr"], o.gr)


def test_failing_member_does_not_disturb_the_others(torch):
    good = [W.distinct_u64(4000 + 100 * i, 950 + i) for i in range(4)]
    bad = W.distinct_u64(3000, 960)
    bad[7] = bad[2000]
    keys = good[:2] + [bad] + good[2:]
    dkeys = [dev(torch, k) for k in keys]
    descs = (M.BuildDesc * 6)()
    for i, dk in enumerate(dkeys):
        descs[i] = M.BuildDesc(dk.data_ptr(), dk.shape[0], 12, 200, 8, 1, 0, 0, 0)
    descs[5] = M.BuildDesc(dkeys[0].data_ptr(), dkeys[0].shape[0], 1, 200, 8, 1, 0, 0, 0)  # bad leaf size
    import ctypes
    outs = (ctypes.c_void_p * 6)()
    sts = (ctypes.c_int * 6)()
    stream = torch.cuda.current_stream().cuda_stream
    rc = M.lib().mphf_build_batch(descs, 6, stream, outs, sts)
    assert rc == M.EDUPLICATE
    assert list(sts) == [M.OK, M.OK, M.EDUPLICATE, M.OK, M.OK, M.EINVAL]
    assert not outs[2] and not outs[5]
    for i in (0, 1, 3, 4):
        built = M.MPHF(outs[i])
        same(built, M.MPHF.build(dkeys[i], 12, 200, True))


def test_batch_workload_sample(torch, orc):
    """64 builds of the batch workload (log-uniform sizes, leaf size drawn per
    build), sizes capped for test time; every member equals its plain build and
    a quarter are checked against the oracle."""
    inst = W.batch_instances(count=64, lo_exp=3.0, hi_exp=4.3)
    keys = [W.distinct_u64(x.n, x.seed) for x in inst]
    dkeys = [dev(torch, k) for k in keys]
    batch = M.build_batch(dkeys, [x.leaf for x in inst], bucket_size=2000)
    for i, (x, k, dk) in enumerate(zip(inst, keys, dkeys)):
        assert batch[i].verify(dk) == 0
        if i % 4 == 0:
            same(batch[i], M.MPHF.build(dk, x.leaf, 2000, True))
            if x.leaf < 16:
                o = orc.build_mphf(k, x.leaf, 2000, True, threads=8)
                assert np.array_equal(batch[i].host_arrays()["values"], o.values)


def test_batch_leaf16_members_match_the_oracle(torch, orc):
    """Members with l = 16 (the dominant cost of the batch workload) built in
    one batch with smaller ones, each equal to its oracle build word for word."""
    specs = [(20_000, 16), (1_500, 8), (30_000, 16), (7_000, 12), (3_000, 16)]
    keys = [W.distinct_u64(n, 1700 + i) for i, (n, _) in enumerate(specs)]
    dkeys = [dev(torch, k) for k in keys]
    batch = M.build_batch(dkeys, [l for _, l in specs], bucket_size=2000)
    for (n, l), k, dk, g in zip(specs, keys, dkeys, batch):
        o = orc.build_mphf(k, l, 2000, True, threads=os.cpu_count() or 4)
        a = g.host_arrays()
        for name, ref in (("values", o.values), ("node_off", o.node_off), ("cum_keys", o.cum_keys),
                          ("bit_pos", o.bit_pos), ("gr", o.gr), ("ef", o.ef)):
            assert np.array_equal(a[name], ref), (n, l, name)
        assert g.verify(dk) == 0
