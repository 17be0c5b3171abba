#!/usr/bin/env python3
"""RecSplit construction benchmark on one node.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one complete build (fingerprint, bucket sort, split and leaf
searches with rotation fitting, Golomb-Rice / Elias-Fano packing) of the
10,000,000-key workload with leaf size 16 and bucket size 2000, keys already
resident in device memory.  Prints one JSON line (rank 0).  N > 1 builds one
function over N x 10,000,000 keys (each rank holds its own 10^7), sharded by
bucket ranges across the GPUs (Section 5.2): one all-to-all of keys, one
all-gather of the packed shards (weak scaling: keys per GPU fixed).

--impl reference times the CPU oracle on the host cores on a bounded bucket
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2212_09562_b300 import workloads as W  # noqa: E402

METRIC = "MPHF build keys/s + seed trials/s vs IMAD peak (ℓ=16,b=2000), batched vs plain"
WORKLOAD = "rot_l16"
# Integer-multiply (IMAD pipe) work of one key-hash evaluation at a full
# lower-level node, by instruction form: the two 64 x 64 -> 64-bit multiplies
# of the SplitMix64 remix on 32-bit lanes (each one 32 x 32 -> 64 wide
# multiply-add and two 32-bit multiply-adds), and the remainder of the digit
# sum that gives the child's counter index (h >> a) mod D (one multiply-high,
# one multiply-subtract; D = 7 and 35 at l = 16).  Each form is weighted by
# its issue cost relative to mad.lo.u32, measured in the same run by the
# integer microbenchmark (peaks/int_peaks.cu).
IMAD_FORMS_PER_EVAL = {"mad.wide.u32": 2, "mad.lo.u32": 5, "mad.hi.u32": 1}
# All integer instructions one evaluation needs at least on 32-bit lanes:
# 64-bit add (2), the remix's first two 64-bit xor-shifts (4 each), two
# 64 x 64-bit multiplies (3 each), the digits of h >> a read from the value
# before the last xor-shift, and their sum (5), their remainder (2 multiply
# forms + 1 shift), the counter (table load and add, 2).
OPS_PER_EVAL = 2 + 8 + 6 + 5 + 3 + 2
# DRAM bytes the search kernel moves per key (lo word and rotation bit read
# once per bucket, plus the keys of nodes given to other blocks), from
# dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of k_search
# on 3,000,000 keys of rot_l16 (a multi-wave launch): 28,173,568 B.  The
# traffic of a launch grows with its key count.
SEARCH_DRAM_BYTES_PER_KEY = 28_173_568 / 3_000_000
# Pipe utilisation of k_search over the elapsed cycles of the same capture
# (sm__pipe_fmaheavy_cycles_active, sm__pipe_alu_cycles_active,
# smsp__issue_active; .avg.pct_of_peak_sustained_elapsed).
SEARCH_NCU_PIPES = {"fmaheavy_busy_of_elapsed": 0.701, "alu_busy_of_elapsed": 0.749,
                    "issue_busy_of_elapsed": 0.686, "instructions_per_eval": 29.1,
                    "capture": "ncu, k_search on 3e6 keys of rot_l16 (multi-wave), current kernel"}
LEAF_NAMES = {0: "brute force", 1: "rotation fitting", 2: "ShockHash"}


def measured_int_peaks() -> dict:
    """Integer issue rates of this GPU measured now (full grid, CUDA events):
    mad.lo.u32, mad.wide.u32, mad.hi.u32 and the mixed IMAD + LOP3 issue rate."""
    from paper_2212_09562_b300 import intpeaks as P
    return {k: P.measure(k, reps=3, target_ms=20.0) for k in ("imad", "imad_wide", "imad_hi",
                                                              "imad+lop3", "mul64")}


def search_roofline(peaks: dict, evals_per_launch: float, launch_ms: float, bench_mhz,
                    traffic) -> dict:
    """Roofline of the search kernel against the measured integer-multiply peak.
    achieved = IMAD-equivalent operations per launch / launch time; the peak is
    mad.lo.u32 over a full grid, scaled to the SM clock of the timed region."""
    imad = peaks["imad"]
    scale = (bench_mhz / imad["sm_mhz"]) if (bench_mhz and imad["sm_mhz"]) else 1.0
    peak = imad["per_s"] * scale
    w = {"mad.lo.u32": 1.0, "mad.wide.u32": imad["per_s"] / peaks["imad_wide"]["per_s"],
         "mad.hi.u32": imad["per_s"] / peaks["imad_hi"]["per_s"]}
    eq = sum(IMAD_FORMS_PER_EVAL[k] * w[k] for k in IMAD_FORMS_PER_EVAL)
    raw = sum(IMAD_FORMS_PER_EVAL.values())
    evals_per_s = evals_per_launch / (launch_ms / 1e3)
    achieved = evals_per_s * eq
    issue = peaks["imad+lop3"]["per_s"] * scale
    return {"bound": "alu", "kernel": "k_search", "unit": "T IMAD-equivalents/s",
            "achieved": achieved / 1e12, "peak": peak / 1e12, "frac": achieved / peak,
            "peak_basis": (f"measured in this run (of measured): mad.lo.u32 over a full grid, "
                           f"{imad['per_s'] / 1e12:.3f} T/s at {imad['sm_mhz']:.0f} MHz, "
                           f"scaled to the timed region's {bench_mhz} MHz"),
            "imad_forms_per_eval": IMAD_FORMS_PER_EVAL,
            "measured_weights": {k: round(v, 3) for k, v in w.items()},
            "imad_equivalents_per_eval": eq,
            "mul64_check": {"predicted_equiv": w["mad.wide.u32"] + 2,
                            "measured_equiv": imad["per_s"] / peaks["mul64"]["per_s"]},
            "frac_unweighted": evals_per_s * raw / peak,
            "issue": {"ops_per_eval": OPS_PER_EVAL,
                      "peak_T_per_s": issue / 1e12,
                      "basis": "measured mixed mad.lo.u32 + lop3.b32 issue rate (of measured)",
                      "frac": evals_per_s * OPS_PER_EVAL / issue},
            "evals_per_launch": evals_per_launch, "launch_ms": launch_ms,
            "traffic": traffic,
            "traffic_basis": "ncu DRAM bytes of k_search at 3e6 keys of rot_l16, scaled by n",
            "ncu_pipes": SEARCH_NCU_PIPES}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(W.WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=0, help="override the key count (profiling runs)")
    ap.add_argument("--mode", choices=["build", "serve", "batch", "peaks"], default="build")
    ap.add_argument("--requests", type=int, default=24, help="serve mode: requests per run")
    ap.add_argument("--no-tune", action="store_true",
                    help="build with the library's default search shape (profiling runs)")
    ap.add_argument("--serve-requests", type=int, default=16,
                    help="requests of the serve leg in the default run (0 = skip)")
    ap.add_argument("--rate", type=float, default=200.0, help="serve mode: Poisson arrivals per second")
    ap.add_argument("--batch-builds", type=int, default=128,
                    help="builds in the batched-vs-plain comparison (0 = skip); batch mode: 4096")
    ap.add_argument("--batch-max-exp", type=float, default=6.0,
                    help="batch mode: key counts floor(10^U(3, this))")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)], stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait(timeout=10)
        self.file.flush()
        self.file.seek(0)
        rows = [l.strip().split(",") for l in self.file.read().splitlines() if l.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for name, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def bucket_index(hi: np.ndarray, nb: int) -> np.ndarray:
    """floor(hi * nb / 2^64) exactly, on 32-bit halves (nb < 2^32)."""
    h, l = hi >> np.uint64(32), hi & np.uint64(0xFFFFFFFF)
    nbu = np.uint64(nb)
    return ((h * nbu + ((l * nbu) >> np.uint64(32))) >> np.uint64(32)).astype(np.int64)


def cpu_baseline(w, keys, budget_s: float) -> dict:
    """The oracle as it stands, on all host cores, on a bounded bucket sample."""
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    nb = (w.n + w.bucket - 1) // w.bucket
    # size the sample from one bucket's single-thread time
    probe = W.sample_buckets(nb, 1, w.seed + 99)
    t0 = time.perf_counter()
    O.build_sample(keys, w.leaf, w.bucket, w.rotation, probe, threads=1, tree=w.tree)
    one = time.perf_counter() - t0
    count = int(max(1, min(nb, round(budget_s * cores / max(one, 1e-3)))))
    count = min(nb, max(cores, count - count % cores))  # at least one bucket per core
    sample = W.sample_buckets(nb, count, w.seed + 100)
    t0 = time.perf_counter()
    vals, counts, st = O.build_sample(keys, w.leaf, w.bucket, w.rotation, sample, threads=cores,
                                      tree=w.tree)
    dt = time.perf_counter() - t0
    hi, _ = O.fingerprint(keys)
    sample_keys = int(np.isin(bucket_index(hi, nb), sample.astype(np.int64)).sum())
    trials = sum(v[0] for v in st.values())
    return {"value": sample_keys / dt, "unit": "keys/s", "cores": cores, "kind": "oracle",
            "sample": f"{count} of {nb} buckets ({sample_keys} keys) of {w.name}, seeded",
            "seconds": dt, "trials_per_s": trials / dt}


def same_function(a, b) -> bool:
    """Word-for-word equality of two built functions: node values, offsets,
    Golomb-Rice and Elias-Fano words."""
    x, y = a.host_arrays(), b.host_arrays()
    return all(np.array_equal(x[k], y[k]) for k in ("values", "node_off", "cum_keys", "bit_pos",
                                                     "gr", "ef"))


def batch_vs_plain(M, torch, count: int, hi_exp: float = 5.0) -> dict:
    """The same independent builds (batch workload distribution, sizes
    10^3..10^hi_exp) through one batched call and through one call per build."""
    inst = W.batch_instances(count=count, lo_exp=3.0, hi_exp=hi_exp)
    keys = [torch.from_numpy(W.distinct_u64(x.n, x.seed).view(np.int64)).cuda() for x in inst]
    leaves = [x.leaf for x in inst]
    total = sum(x.n for x in inst)
    for g in M.build_batch(keys[:4], leaves[:4], bucket_size=2000):
        g.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batched = M.build_batch(keys, leaves, bucket_size=2000)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    t0 = time.perf_counter()
    plain = [M.MPHF.build(k, l, 2000, True, tuned=True) for k, l in zip(keys, leaves)]
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    identical = all(same_function(a, b) for a, b in zip(batched, plain))
    graph = graph_batch(M, torch, keys, leaves, batched, reps=3 if count <= 512 else 1)
    for g in batched + plain:
        g.close()
    return {"builds": count, "keys": total,
            "sizes": f"floor(10^U(3,{hi_exp:g})), leaf in {{8,12,16}}, b=2000",
            "batched_keys_per_s": total / t_batch, "plain_keys_per_s": total / t_plain,
            "batched_over_plain": t_plain / t_batch, "identical": identical,
            "graph": graph}


def graph_batch(M, torch, keys, leaves, batched, reps: int = 3) -> dict:
    """The same builds as prepared members of one batch (mphf_batch_*),
    captured once in a CUDA graph and replayed: keys/s per replay (plus the
    host's read of every build's totals) and equality with the batched call."""
    from paper_2212_09562_b300.autotune import tuned as cached_shape
    spt = {l: cached_shape(l, True, M.TREE_RECSPLIT)[2] for l in set(leaves)}

    def prepare(ks, ls):
        return [M.MPHF.prepare(int(k.shape[0]), l, 2000, True, seeds_per_thread=spt[l])
                for k, l in zip(ks, ls)]

    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    # an eager run of a small batch first: lazy module loading stays outside the capture
    small = sorted(range(len(keys)), key=lambda i: int(keys[i].shape[0]))[:2]
    warm = prepare([keys[i] for i in small], [leaves[i] for i in small])
    wb = M.PreparedBatch(warm)
    wb.enqueue([keys[i] for i in small], stream=s)
    wb.finish(stream=s)
    wb.close()
    for m in warm:
        m.close()
    members = prepare(keys, leaves)
    pb = M.PreparedBatch(members)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pb.enqueue(keys, stream=s)
    times = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(s):
            g.replay()
        pb.finish(stream=s)
        times.append(time.perf_counter() - t0)
    identical = all(same_function(a, b) for a, b in zip(members, batched))
    total = sum(int(k.shape[0]) for k in keys)
    pb.close()
    del g
    for m in members:
        m.close()
    return {"replays": reps, "graph_keys_per_s": total / min(times),
            "graph_ms": 1e3 * min(times), "identical": identical}


def serve_run(M, torch, keys, leaf, arrivals, plain=None) -> dict:
    """Requests submitted at their arrival times to one server; with `plain`
    (a list of functions built one by one from the same keys), every served
    function is compared with its plain build word for word."""
    srv = M.Server()
    tickets = []
    start = time.perf_counter()
    for dk, at in zip(keys, arrivals):
        delay = at - (time.perf_counter() - start)
        if delay > 0:
            time.sleep(delay)
        tickets.append(srv.submit(dk, leaf, 2000))
    res = {}
    while len(res) < len(tickets):
        for t in tickets:
            if t not in res:
                r = srv.poll(t, 50)
                if r is not None:
                    res[t] = r
    lat = sorted(r[2][2] - r[2][0] for r in res.values())
    first = min(r[2][0] for r in res.values())
    last = max(r[2][2] for r in res.values())
    ok = all(r[0] == M.OK for r in res.values())
    bad = sum(r[1].verify(dk) if r[1] is not None else 1
              for r, dk in zip((res[t] for t in tickets), keys))
    identical = None
    if plain is not None:
        identical = all(res[t][1] is not None and same_function(res[t][1], g)
                        for t, g in zip(tickets, plain))
    for r in res.values():
        if r[1] is not None:
            r[1].close()
    srv.close()
    n = sum(int(k.shape[0]) for k in keys)
    return {"requests": len(keys), "keys": n, "keys_per_s": n / (last - first),
            "requests_per_s": len(keys) / (last - first), "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "all_ok": ok and bad == 0,
            "identical_to_plain": identical}


def serve_leg(M, torch, requests: int, rate: float) -> dict:
    """The serve workload (Poisson arrivals at `rate`, 16-byte keys, n =
    floor(10^U(4,7)), l = 16, b = 2000), keys resident on the device: the
    same requests built one by one with plain builds, then served at the
    offered rate and again paced at 0.8x the served capacity; every served
    function equals its plain build."""
    seed = W.SEED_BASE + 5
    sizes = W.serve_sizes(requests, seed)
    keys = [torch.from_numpy(W.distinct_bytes16(int(n), seed * 1000 + i)).cuda()
            for i, n in enumerate(sizes)]
    warm = M.Server()
    t = warm.submit(keys[0][:5000], 16, 2000)
    while warm.poll(t, 100) is None:
        pass
    warm.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = [M.MPHF.build(k, 16, 2000, True) for k in keys]
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    n = sum(int(k.shape[0]) for k in keys)
    offered = serve_run(M, torch, keys, 16, W.poisson_arrivals(requests, rate, seed), plain)
    rate2 = 0.8 * offered["requests_per_s"]
    paced = serve_run(M, torch, keys, 16, W.poisson_arrivals(requests, rate2, seed + 1), plain)
    for g in plain:
        g.close()
    return {"requests": requests, "keys": n, "rate_per_s": rate,
            "sizes": "floor(10^U(4,7)) 16-byte keys, l=16, b=2000",
            "served_keys_per_s": offered["keys_per_s"], "plain_keys_per_s": n / t_plain,
            "served_over_plain": offered["keys_per_s"] / (n / t_plain),
            "p50_s": offered["p50_s"], "p99_s": offered["p99_s"],
            "identical": bool(offered["identical_to_plain"] and paced["identical_to_plain"]),
            "offered_rate": offered, "paced_at_0.8x_capacity": dict(paced, rate_per_s=rate2)}


def run_serve(args):
    """Serve workload alone (bench.py --mode serve)."""
    import torch
    from paper_2212_09562_b300 import mphf as M
    M.lib()
    sampler = ClockSampler(0)
    sampler.start()
    r = serve_leg(M, torch, args.requests, args.rate)
    clocks = sampler.stop()
    out = {"metric": "served MPHF build keys/s (l=16, b=2000, 16-byte keys, Poisson arrivals)",
           "value": r["served_keys_per_s"], "unit": "keys/s", "n_gpus": 1, "higher_is_better": True,
           "dtype": "u64", "data": "synthetic",
           "config": {"workload": "serve", "requests": args.requests, "rate_per_s": args.rate,
                      "sizes": r["sizes"]},
           "serve": r, "clocks": clocks}
    print(json.dumps(out), flush=True)


def run_batch(args):
    """Batched workload: independent builds with log-uniform key counts and a
    leaf size drawn per build, through one mphf_build_batch call and through
    one build call each; identical outputs checked."""
    import torch
    from paper_2212_09562_b300 import mphf as M
    M.lib()
    count = args.batch_builds if args.batch_builds != 128 else 4096
    sampler = ClockSampler(0)
    sampler.start()
    r = batch_vs_plain(M, torch, count, args.batch_max_exp)
    clocks = sampler.stop()
    out = {"metric": "batched MPHF build keys/s (b=2000, leaf in {8,12,16}, rotation fitting)",
           "value": r["batched_keys_per_s"], "unit": "keys/s", "n_gpus": 1,
           "higher_is_better": True, "dtype": "u64", "data": "synthetic",
           "config": {"workload": "batch", "builds": r["builds"], "keys": r["keys"],
                      "sizes": r["sizes"]},
           "plain_keys_per_s": r["plain_keys_per_s"], "batched_over_plain": r["batched_over_plain"],
           "identical": r["identical"], "graph": r["graph"], "clocks": clocks}
    print(json.dumps(out), flush=True)


def run_peaks(args):
    """Integer issue rates of this GPU, one instruction class at a time
    (paper_2212_09562_b300/peaks/int_peaks.cu), with the SM clock each ran at."""
    import torch
    from paper_2212_09562_b300 import intpeaks as P
    torch.cuda.set_device(0)
    sampler = ClockSampler(0)
    sampler.start()
    rows = {k: P.measure(k, reps=5, target_ms=40.0) for k in P.KINDS}
    clocks = sampler.stop()
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    for r in rows.values():
        # thread-level operations per SM per clock at the clock the kernel ran at
        r["per_sm_per_clock"] = r["per_s"] / (sms * r["sm_mhz"] * 1e6) if r["sm_mhz"] else None
    out = {"metric": "integer issue rates (thread ops per SM per clock)", "mode": "peaks",
           "device": props.name, "sms": sms, "rates": rows, "clocks": clocks}
    print(json.dumps(out), flush=True)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = workload(args)
    keys = W.keys_for(w)
    for _ in range(max(0, args.warmup)):  # untimed warm-up steps, about a second each
        cpu_baseline(w, keys, 1.0)
    vals, secs = [], []
    for _ in range(args.steps):
        r = cpu_baseline(w, keys, args.cpu_seconds / max(1, args.steps))
        vals.append(r["value"])
        secs.append(r["seconds"])
    v = statistics.mean(vals)
    out = {"metric": METRIC, "value": v, "unit": "keys/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * statistics.mean(secs),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": w.name, "n": w.n, "leaf": w.leaf, "bucket": w.bucket,
                      "rotation": int(w.rotation) == 1, "leaves": LEAF_NAMES[int(w.rotation)],
                      "tree": "fanout 2" if w.tree else "lower aggregation levels",
                      "key_bytes": w.key_bytes, "sample": r["sample"]},
           "cpu_baseline": {"value": v, "unit": "keys/s", "cores": r["cores"], "kind": "oracle",
                            "sample": r["sample"]},
           "e2e": {"value": v, "unit": "keys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def graph_vs_eager(M, torch, reps: int = 20) -> dict:
    """Small builds, where launches, allocation and host reads dominate: the
    plain_l8 workload (10^5 keys, l = 8, b = 100) built eagerly, and as a
    prepared build captured once in a CUDA graph and replayed on new keys
    copied into its input buffer; every replay's function equals the eager one."""
    w = W.WORKLOADS["plain_l8"]
    sets = [W.distinct_u64(w.n, w.seed + 10 + i) for i in range(4)]
    dsets = [torch.from_numpy(k.view(np.int64)).cuda() for k in sets]
    buf = torch.empty_like(dsets[0])
    s = torch.cuda.Stream()
    p = M.MPHF.prepare(w.n, w.leaf, w.bucket, w.rotation)
    buf.copy_(dsets[0])
    torch.cuda.synchronize()
    p.enqueue(buf, stream=s)
    p.finish(stream=s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        p.enqueue(buf, stream=s)
    identical = True
    for k in dsets:  # correctness first: replays on new keys equal eager builds
        buf.copy_(k)
        graph.replay()
        p.finish()
        e = M.MPHF.build(k, w.leaf, w.bucket, w.rotation)
        identical = identical and same_function(p, e)
        e.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(reps):
        M.MPHF.build(dsets[i % 4], w.leaf, w.bucket, w.rotation).close()
    torch.cuda.synchronize()
    t_eager = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    for i in range(reps):
        buf.copy_(dsets[i % 4])
        graph.replay()
        p.finish()  # host read of status and totals: the function is usable after each
    torch.cuda.synchronize()
    t_graph = (time.perf_counter() - t0) / reps
    p.close()
    return {"workload": w.name, "n": w.n, "eager_keys_per_s": w.n / t_eager,
            "graph_keys_per_s": w.n / t_graph, "eager_ms": 1e3 * t_eager, "graph_ms": 1e3 * t_graph,
            "identical": bool(identical)}


def query_throughput(torch, g, dkeys, stream, reps: int = 5) -> dict:
    """Queries of every built key through mphf_query, keys and results on the device."""
    out = torch.empty(dkeys.shape[0], dtype=torch.int64, device="cuda")
    g.query(dkeys, out=out)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(reps):
        g.query(dkeys, out=out)
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1) / reps
    return {"keys": int(dkeys.shape[0]), "ms": ms, "queries_per_s": dkeys.shape[0] / (ms / 1000.0)}


def rank_keys(w, rank: int) -> np.ndarray:
    """Each rank's own slice of the key set (weak scaling: w.n keys per rank)."""
    return W.keys_for(w) if rank == 0 else W.random_keys(w.n, w.key_bytes, w.seed + rank)


def max_over_ranks(value: float, world: int, device: str = "cuda") -> float:
    """The slowest rank's time decides the whole job's time."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(world: int, steps: int, n: int, total_ms: float) -> float:
    """Keys built by all ranks per second of the slowest rank."""
    return world * steps * n / (total_ms / 1000.0)


def workload(args):
    w = W.WORKLOADS[args.workload]
    if args.n:
        w = W.Workload(w.name + f"_n{args.n}", args.n, w.leaf, w.bucket, w.key_bytes, w.rotation,
                       w.seed, w.tree)
    return w


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2212_09562_b300 import mphf as M
    M.lib()
    w = workload(args)
    keys = rank_keys(w, rank)
    dkeys = torch.from_numpy(keys.view(np.int64) if keys.ndim == 1 else keys).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 126 MB L2
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2212_09562_b300 import shard as S

    # launch shape and seeds per thread from the autotuner (tuned now if this
    # device has no cached choice for the workload's leaf size)
    from paper_2212_09562_b300 import autotune as A
    if not args.no_tune and A.tuned(w.leaf, w.rotation, w.tree) == A.DEFAULT:
        # tuned on the workload's own size up to 3e6 keys (the best shape depends on it)
        A.tune(w.leaf, w.rotation, n=min(w.n, 3_000_000), bucket=w.bucket, tree=w.tree)
    shape = A.DEFAULT if args.no_tune else A.tuned(w.leaf, w.rotation, w.tree)

    def one_build(k):
        """(function, the part this rank searched): the whole build on one GPU,
        else one function over all ranks' keys in bucket-range shards."""
        if world == 1:
            g = M.MPHF.build(k, w.leaf, w.bucket, w.rotation, tree=w.tree, tuned=not args.no_tune)
            return g, g
        return S.build_sharded(k, w.leaf, w.bucket, w.rotation, tree=w.tree)

    def close(g, sh):
        if sh is not g:
            sh.close()
        g.close()

    for i in range(args.warmup):
        close(*one_build(dkeys))
    peaks = measured_int_peaks()  # before the timed region, on this GPU
    sampler = ClockSampler(local)
    sampler.start()
    step_ms, search_ms, evals, trials, my_evals, launches = [], [], 0, 0, 0, 0
    leaf_k_trials, leaf_evals = 0, 0
    barrier()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)  # evict the previous step's data from L2 (outside the step's events)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = M.kernel_launches()
        ev0.record(stream)
        g, sh = one_build(dkeys)
        ev1.record(stream)
        ev1.synchronize()
        launches += M.kernel_launches() - l0
        step_ms.append(ev0.elapsed_time(ev1))
        st, mine = g.stats(), sh.stats()
        search_ms.append(mine["ms"]["search"])
        evals += sum(st[k][1] for k in ("leaf", "lower1", "lower2", "upper"))  # all ranks'
        trials += sum(st[k][0] for k in ("leaf", "lower1", "lower2", "upper"))
        my_evals += sum(mine[k][1] for k in ("leaf", "lower1", "lower2", "upper"))
        leaf_k_trials += st["leaf"][0]
        leaf_evals += st["leaf"][1]
        if i == args.steps - 1:
            bad = g.verify(dkeys)
            assert bad == 0, f"built function is not injective on this rank's keys ({bad} bad keys)"
            stages = mine["ms"]
            query = query_throughput(torch, g, dkeys, stream)
        close(g, sh)
    barrier()
    wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    total_ms = max_over_ranks(sum(step_ms), world)
    keys_per_s = weak_scaling_value(world, args.steps, w.n, total_ms)

    # end to end through the public API from pinned host keys: one GPU calls
    # mphf_build_host; N GPUs copy their keys in and build the sharded function;
    # the packed function comes back to the host
    e2e = None
    if args.e2e_steps > 0:
        pinned = torch.from_numpy(keys.view(np.int64) if keys.ndim == 1 else keys).pin_memory()
        host_view = pinned.numpy().view(np.uint64) if keys.ndim == 1 else pinned.numpy()
        times, d2h = [], 0
        for _ in range(args.e2e_steps):
            barrier()
            t0 = time.perf_counter()
            if world == 1:
                g = M.MPHF.build_host(host_view, w.leaf, w.bucket, w.rotation, tree=w.tree)
                sh = g
            else:
                g, sh = one_build(pinned.cuda(non_blocking=True))
            blob = g.serialize()
            times.append(max_over_ranks(time.perf_counter() - t0, world))
            d2h = len(blob)
            close(g, sh)
        e2e = {"value": world * w.n / statistics.mean(times), "unit": "keys/s",
               "h2d_bytes_per_step": int(keys.nbytes) * world, "d2h_bytes_per_step": int(d2h)}

    if rank != 0:
        return
    mean_search = statistics.mean(search_ms)
    evals_per_build = my_evals / args.steps  # this rank's search launch
    roof = search_roofline(peaks, evals_per_build, mean_search, clocks.get("sm_mhz"),
                           SEARCH_DRAM_BYTES_PER_KEY * w.n if w.name.startswith("rot_l16") else None)
    out = {"metric": METRIC, "value": keys_per_s, "unit": "keys/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
           "data": "synthetic",
           "config": {"workload": w.name, "n": w.n, "leaf": w.leaf, "bucket": w.bucket,
                      "rotation": int(w.rotation) == 1, "leaves": LEAF_NAMES[int(w.rotation)],
                      "tree": "fanout 2" if w.tree else "lower aggregation levels",
                      "key_bytes": w.key_bytes,
                      "l2": "flushed between steps (256 MB write)",
                      "search_shape": {"threads_per_block": shape[0], "blocks_per_sm": shape[1],
                                       "seeds_per_thread": shape[2],
                                       "source": "autotuner (0 = library default)"},
                      "parallelism": ("1 GPU" if world == 1 else
                                      f"{world} GPUs: one function of {world} x {w.n} keys in "
                                      "bucket-range shards (all-to-all of keys, all-gather of shards)")},
           "trials_per_s": trials / (total_ms / 1000.0),
           # rotation fitting: one leaf trial is one k (m seeds k m + r at once); its
           # plain-equivalent count is m per trial, which is the leaves' evaluation count
           "leaf_trials": {"per_s": leaf_k_trials / (total_ms / 1000.0),
                           "plain_equivalent_per_s": leaf_evals / (total_ms / 1000.0)},
           "evals_per_s": evals / (total_ms / 1000.0),
           "search_ms": mean_search, "wall_s": wall, "stage_ms": stages, "query": query,
           "roofline": roof, "e2e": e2e, "gpu_launches": launches, "clocks": clocks}
    if world == 1 and args.batch_builds > 0:
        out["batch"] = batch_vs_plain(M, torch, args.batch_builds)
    if world == 1 and args.serve_requests > 0:
        out["serve"] = serve_leg(M, torch, args.serve_requests, args.rate)
    if world == 1 and args.batch_builds > 0:
        out["graph"] = graph_vs_eager(M, torch)
    if world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(w, keys, args.cpu_seconds)
        out["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "serve":
        run_serve(args)
    elif args.mode == "batch":
        run_batch(args)
    elif args.mode == "peaks":
        run_peaks(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
