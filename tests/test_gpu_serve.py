"""Serving with continuous batching: every served result equals the plain
build of the same request, alone or in a mix; admission follows arrival order
under a memory budget; timeouts and bad requests are reported, not hung on."""
import threading
import time

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


def requests(torch, count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(10 ** rng.uniform(3, 4.6))
        leaf = int(rng.choice([8, 12, 16]))
        kb = int(rng.choice([8, 16]))
        keys = W.random_keys(n, kb, seed * 100 + i)
        out.append((dev(torch, keys), leaf))
    return out


def poll_all(srv, tickets, timeout_s=300):
    res, t_end = {}, time.time() + timeout_s
    while len(res) < len(tickets) and time.time() < t_end:
        for t in tickets:
            if t not in res:
                r = srv.poll(t, 20)
                if r is not None:
                    res[t] = r
    assert len(res) == len(tickets), "requests did not finish"
    return res


def test_served_results_equal_plain_builds(torch):
    reqs = requests(torch, 16, 31)
    srv = M.Server(max_requests=8)
    tickets = []

    def arrive():  # staggered arrivals while earlier requests are on the device
        for dk, leaf in reqs:
            tickets.append(srv.submit(dk, leaf, 1000))
            time.sleep(0.003)

    th = threading.Thread(target=arrive)
    th.start()
    th.join()
    res = poll_all(srv, tickets)
    for t, (dk, leaf) in zip(tickets, reqs):
        st, built, (ts, ta, tf) = res[t]
        assert st == M.OK and built is not None
        assert ts <= ta <= tf
        same(built, M.MPHF.build(dk, leaf, 1000, True))
        assert built.verify(dk) == 0
    srv.close()


def test_alone_equals_in_mix(torch):
    reqs = requests(torch, 8, 32)
    probe_keys, probe_leaf = reqs[3]
    alone = M.Server(max_requests=1)
    t = alone.submit(probe_keys, probe_leaf, 500)
    st, a, _ = poll_all(alone, [t])[t]
    alone.close()
    mix = M.Server(max_requests=64)
    tickets = [mix.submit(dk, leaf, 500) for dk, leaf in reqs]
    res = poll_all(mix, tickets)
    st2, b, _ = res[tickets[3]]
    assert st == st2 == M.OK
    same(a, b)
    mix.close()


def test_fifo_admission_under_a_memory_budget(torch):
    free, _ = torch.cuda.mem_get_info()
    reqs = requests(torch, 6, 33)
    # reserve almost all free memory: only one request is admitted at a time
    srv = M.Server(max_requests=64, hbm_reserve_bytes=max(free - (64 << 20), 1))
    tickets = [srv.submit(dk, leaf, 500) for dk, leaf in reqs]
    res = poll_all(srv, tickets)
    admitted = [res[t][2][1] for t in tickets]
    assert admitted == sorted(admitted)
    assert all(res[t][0] == M.OK for t in tickets)
    srv.close()


def test_timeout_and_bad_requests(torch):
    keys = dev(torch, W.distinct_u64(300_000, 34))
    srv = M.Server(max_requests=4)
    t_big = srv.submit(keys, 16, 2000)
    assert srv.poll(t_big, 0) is None  # still running: reported, not waited on
    t_bad = srv.submit(keys, 1, 2000)  # leaf size out of range
    res = poll_all(srv, [t_big, t_bad])
    assert res[t_big][0] == M.OK
    assert res[t_bad][0] == M.EINVAL and res[t_bad][1] is None
    with pytest.raises(M.MPHFError):
        srv.poll(123456, 0)
    srv.close()


def test_destroy_with_queued_requests(torch):
    reqs = requests(torch, 6, 35)
    srv = M.Server(max_requests=2)
    for dk, leaf in reqs:
        srv.submit(dk, leaf, 500)
    srv.close()  # finishes the queue, frees unpolled results


def test_served_shockhash_and_fanout2_requests(torch, orc):
    """Requests with ShockHash leaves and the fanout-2 tree, mixed with
    rotation-fitting requests in one server, equal their plain builds."""
    specs = [(12000, 24, M.SHOCKHASH, M.TREE_FANOUT2), (8000, 16, M.SHOCKHASH, M.TREE_RECSPLIT),
             (9000, 12, M.ROTATION, M.TREE_RECSPLIT), (7000, 8, M.ROTATION, M.TREE_FANOUT2)]
    keys = [dev(torch, W.distinct_u64(n, 5200 + i)) for i, (n, *_r) in enumerate(specs)]
    srv = M.Server(max_requests=8)
    try:
        tickets = [srv.submit(k, leaf, 2000, bij, tree=tree)
                   for k, (n, leaf, bij, tree) in zip(keys, specs)]
        res = poll_all(srv, tickets)
        for t, k, (n, leaf, bij, tree) in zip(tickets, keys, specs):
            status, built, _ = res[t]
            assert status == M.OK
            alone = M.MPHF.build(k, leaf, 2000, bij, tree=tree)
            same(built, alone)
            assert built.info.tree_shape == tree and built.info.leaf_bijection == bij
            assert built.verify(k) == 0
    finally:
        srv.close()


def test_requests_join_a_running_search(torch):
    """A long request is on the device; short ones that arrive later are
    admitted while it runs, share the serving search with it and finish
    before it, each identical to its plain build."""
    big = dev(torch, W.distinct_u64(1_500_000, 36))
    small = [dev(torch, W.distinct_u64(20_000 + 5000 * i, 37 + i)) for i in range(4)]
    srv = M.Server(max_requests=64)
    try:
        t_big = srv.submit(big, 16, 2000)
        time.sleep(0.3)
        ts = [srv.submit(k, 12 if i % 2 else 8, 1000) for i, k in enumerate(small)]
        res = poll_all(srv, [t_big] + ts)
        big_done = res[t_big][2][2]
        for t, k, i in zip(ts, small, range(4)):
            st, built, (sub, adm, fin) = res[t]
            assert st == M.OK
            assert adm < big_done and fin < big_done, (adm, fin, big_done)
            same(built, M.MPHF.build(k, 12 if i % 2 else 8, 1000, True))
        assert res[t_big][0] == M.OK
        same(res[t_big][1], M.MPHF.build(big, 16, 2000, True))
    finally:
        srv.close()


def test_freed_request_slots_are_refilled(torch):
    """With room for two requests, the short ones take turns in the second
    slot while the long one keeps the first: each is admitted when the one
    before it finishes, all before the long request is done."""
    big = dev(torch, W.distinct_u64(1_200_000, 38))
    small = [dev(torch, W.distinct_u64(30_000, 39 + i)) for i in range(3)]
    srv = M.Server(max_requests=2)
    try:
        t_big = srv.submit(big, 16, 2000)
        ts = [srv.submit(k, 8, 1000) for k in small]
        res = poll_all(srv, [t_big] + ts)
        big_done = res[t_big][2][2]
        times = [res[t][2] for t in ts]
        for (sub, adm, fin) in times:
            assert fin < big_done
        for prev, nxt in zip(times, times[1:]):
            assert nxt[1] >= prev[2] - 1e-3  # admitted once the previous one freed its slot
        for t, k in zip(ts, small):
            same(res[t][1], M.MPHF.build(k, 8, 1000, True))
    finally:
        srv.close()


def test_search_blocks_leave_after_their_wait_bound_and_the_server_recovers(torch):
    """With a 1 ms bound on a serving-search block's wait for work, blocks
    leave whenever the queue is empty for that long (between requests, and
    while a request is being prepared); the server launches the search again
    for the next work, and every result still equals its plain build."""
    reqs = requests(torch, 6, 41)
    srv = M.Server(max_requests=2, idle_ms=1)
    try:
        tickets = []
        for dk, leaf in reqs:
            tickets.append(srv.submit(dk, leaf, 500))
            time.sleep(0.02)  # gaps longer than the bound
        res = poll_all(srv, tickets)
        for t, (dk, leaf) in zip(tickets, reqs):
            st, built, _ = res[t]
            assert st == M.OK
            same(built, M.MPHF.build(dk, leaf, 500, True))
    finally:
        srv.close()
