"""Multi-process host logic of the benchmark on CPU (gloo, world size 2):
every rank builds its own independent key set (weak scaling, no collective
on the data path), the job's time is the slowest rank's, and the reported
value counts the keys of all ranks.  Builds here use the CPU oracle."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    from oracle import oracle as O
    from paper_2212_09562_b300 import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = W.Workload("small", 20_000, 8, 100, 8, True, 4242)
    keys = bench.rank_keys(w, rank)
    h = O.build_mphf(keys, w.leaf, w.bucket, w.rotation)
    ok = np.array_equal(np.sort(h.query(keys)), np.arange(w.n, dtype=np.uint64))
    my_ms = 100.0 * (rank + 1)  # a stand-in per-rank time
    slowest = bench.max_over_ranks(my_ms, world, device="cpu")
    value = bench.weak_scaling_value(world, 3, w.n, slowest)
    np.save(os.path.join(out_dir, f"r{rank}.npy"),
            np.array([ok, slowest, value, int(keys[0]), int(keys[-1])], dtype=np.float64))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_build_independently_and_reduce_the_time(tmp_path):
    from oracle import oracle as O
    O.build()
    world, port = 2, _free_port()
    mp.spawn(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    r0, r1 = (np.load(tmp_path / f"r{r}.npy") for r in range(world))
    assert r0[0] == 1 and r1[0] == 1                  # both builds are bijections
    assert r0[1] == r1[1] == 200.0                    # the slowest rank's time
    assert r0[2] == pytest.approx(2 * 3 * 20_000 / 0.2)
    assert (r0[3], r0[4]) != (r1[3], r1[4])           # independent inputs per rank
