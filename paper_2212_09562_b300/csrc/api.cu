// api.cu -- the C ABI of libmphf (declared in include/mphf.h).
//
// One build, all on the device (Section 2.2 of Bez et al. 2212.09562 in the
// order of its parallel form, Section 5.3):
//   fingerprint + histogram -> plan (nodes per bucket) -> prefix sums
//   -> [host reads: node total, largest bucket, status]
//   -> scatter by bucket -> persistent search kernel (splits, leaves)
//   -> Golomb-Rice lengths -> prefix sums -> [host reads: bit total]
//   -> Golomb-Rice bits, Elias-Fano sequences, rank directories, statistics.
// The two host reads size the output buffers; the build returns after a
// final stream synchronisation with the device status mapped to an error.
//
// This file holds the per-device tables, the engine's phases (build_engine.h),
// builds, batches, queries, verification, serialisation and loading.  The
// sharded-build entry points are in shard.cu, the prepared (graph-capturable)
// build in graph_build.cu, the server in serve.cu.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "build_engine.h"
#include "common.cuh"
#include "engine.h"
#include "handle.h"
#include "mphf.h"
#include "tables.h"

using namespace rs;

namespace rs {

// Per-device copy of the exact-remainder constants per node size.
int device_mod_tables(int dev, uint32_t **c, uint64_t **M) {
    static std::mutex mu;
    static std::map<int, std::pair<uint32_t *, uint64_t *>> cache;
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(dev);
    if (it == cache.end()) {
        const ModTables &t = mod_tables();
        uint32_t *dc = nullptr;
        uint64_t *dM = nullptr;
        int rc = MPHF_OK;
        if (cudaMalloc(&dc, sizeof(t.c)) != cudaSuccess || cudaMalloc(&dM, sizeof(t.M)) != cudaSuccess)
            rc = MPHF_ENOMEM;
        else if (cudaMemcpy(dc, t.c, sizeof(t.c), cudaMemcpyHostToDevice) != cudaSuccess ||
                 cudaMemcpy(dM, t.M, sizeof(t.M), cudaMemcpyHostToDevice) != cudaSuccess)
            rc = MPHF_ECUDA;
        if (rc != MPHF_OK) {
            cudaGetLastError();
            cudaFree(dc);
            cudaFree(dM);
            return rc;
        }
        it = cache.emplace(dev, std::make_pair(dc, dM)).first;
    }
    *c = it->second.first;
    *M = it->second.second;
    return MPHF_OK;
}

// Per-device copies of the per-size tables; live until the process exits.
// level_salt(L) for L < kSaltLevels on one device, kept: the query walk reads
// a fanout-2 level's salt instead of computing its remix.
static int device_salts(int dev, const uint64_t **out) {
    static std::mutex mu;
    static std::map<int, uint64_t *> cache;
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) {
        *out = it->second;
        return MPHF_OK;
    }
    uint64_t h[kSaltLevels];
    for (uint32_t L = 0; L < kSaltLevels; L++) h[L] = level_salt(L);
    uint64_t *d = nullptr;
    if (cudaMalloc(&d, sizeof(h)) != cudaSuccess) {
        cudaGetLastError();
        return MPHF_ENOMEM;
    }
    if (cudaMemcpy(d, h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d);
        return MPHF_ECUDA;
    }
    cache[dev] = d;
    *out = d;
    return MPHF_OK;
}

int device_tables(int dev, uint32_t leaf, uint32_t bij, uint32_t tree, DevTables *out) {
    static std::mutex mu;
    static std::map<uint64_t, DevTables> cache;
    std::lock_guard<std::mutex> g(mu);
    uint64_t key = ((uint64_t)dev << 32) | (tree << 16) | (leaf << 2) | bij;
    auto it = cache.find(key);
    if (it != cache.end()) {
        *out = it->second;
        return MPHF_OK;
    }
    const SizeTables &t = size_tables(leaf, bij, tree);
    DevTables d;
    int rc = MPHF_OK;
    if (cudaMalloc(&d.tau, sizeof(t.tau)) != cudaSuccess || cudaMalloc(&d.nodes, sizeof(t.nodes)) != cudaSuccess ||
        cudaMalloc(&d.fixed, sizeof(t.fixed)) != cudaSuccess || cudaMalloc(&d.left, sizeof(t.left)) != cudaSuccess)
        rc = MPHF_ENOMEM;
    else if (cudaMemcpy(d.tau, t.tau, sizeof(t.tau), cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(d.nodes, t.nodes, sizeof(t.nodes), cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(d.fixed, t.fixed, sizeof(t.fixed), cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(d.left, t.left, sizeof(t.left), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = MPHF_ECUDA;
    if (rc == MPHF_OK) rc = device_mod_tables(dev, &d.mod_c, &d.mod_M);
    if (rc == MPHF_OK) rc = device_salts(dev, &d.salts);
    if (rc != MPHF_OK) {  // nothing is cached: free what this call allocated
        cudaGetLastError();
        cudaFree(d.tau);
        cudaFree(d.nodes);
        cudaFree(d.fixed);
        cudaFree(d.left);
        return rc;
    }
    cache[key] = d;
    *out = d;
    return MPHF_OK;
}

// Rotation tables for leaves of m <= 16 keys, all m in one array (m's table
// at offset 2^m - 4): canonical rotation (the smallest r giving the smallest
// rot_m^r(x)) and rotation period of every m-bit word.  Per device, kept.
int device_rot_tables(int dev, const uint8_t **canon, const uint8_t **period) {
    static std::mutex mu;
    static std::map<int, std::pair<uint8_t *, uint8_t *>> cache;
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) {
        *canon = it->second.first;
        *period = it->second.second;
        return MPHF_OK;
    }
    const size_t total = (1u << 17) - 4;  // sum over m = 2..16 of 2^m
    std::vector<uint8_t> c(total), pr(total);
    for (uint32_t m = 2; m <= 16; m++) {
        const uint32_t full = (1u << m) - 1, base = (1u << m) - 4;
        for (uint32_t x = 0; x <= full; x++) {
            uint32_t best = x, br = 0, per = m;
            for (uint32_t r = 1; r < m; r++) {
                uint32_t y = ((x << r) | (x >> (m - r))) & full;
                if (y < best) {
                    best = y;
                    br = r;
                }
                if (y == x && per == m) per = r;
            }
            c[base + x] = (uint8_t)br;
            pr[base + x] = (uint8_t)per;
        }
    }
    uint8_t *dc = nullptr, *dp = nullptr;
    int rc = MPHF_OK;
    if (cudaMalloc(&dc, total) != cudaSuccess || cudaMalloc(&dp, total) != cudaSuccess)
        rc = MPHF_ENOMEM;
    else if (cudaMemcpy(dc, c.data(), total, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(dp, pr.data(), total, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = MPHF_ECUDA;
    if (rc != MPHF_OK) {
        cudaGetLastError();
        cudaFree(dc);
        cudaFree(dp);
        return rc;
    }
    cache[dev] = {dc, dp};
    *canon = dc;
    *period = dp;
    return MPHF_OK;
}

// Serialised form: a header of kHeadWords words starting with kMagic (the
// bytes "RMPFPH01" read as a little-endian word), then the Golomb-Rice and
// Elias-Fano words.
constexpr size_t kHeadWords = 16;
constexpr uint64_t kMagic = 0x3130485046504D52ull;



}  // namespace rs

// Frees a handle's arrays in the order of stream st (the build's stream while
// a build fails; the legacy stream after a device synchronisation otherwise).
void rs::release(mphf_t *h, cudaStream_t st) {
    if (!h) return;
    Mem mem{h->has_alloc ? &h->alloc : nullptr, st};
    release_plan(h, mem);
    void *ptrs[] = {h->values, h->node_off, h->cum_keys, h->bit_pos, h->gr, h->ef, h->ef_dir};
    for (void *p : ptrs) mem.put(p);
    delete h;
}

// Sizes of the packed function (Golomb-Rice words, the two Elias-Fano
// sequences over nb + 1 bucket offsets, their rank and select directories)
// and its arrays from the handle's allocator.  Nothing is written yet.
int rs::alloc_packed(mphf_t *h, uint64_t nb, uint64_t n, uint64_t gr_bits, Mem &jm) {
    h->info.gr_bits = gr_bits;
    h->info.gr_words = (gr_bits + 63) / 64;
    EfDims e0 = ef_dims(nb + 1, n), e1 = ef_dims(nb + 1, gr_bits);
    h->info.ef_low_bits[0] = e0.L;
    h->info.ef_low_bits[1] = e1.L;
    h->info.ef_seq_words[0] = e0.low_words;
    h->info.ef_seq_words[1] = e0.high_words;
    h->info.ef_seq_words[2] = e1.low_words;
    h->info.ef_seq_words[3] = e1.high_words;
    h->info.ef_words = e0.low_words + e0.high_words + e1.low_words + e1.high_words;
    h->ef_dir_len[0] = e0.high_words + 1;
    h->ef_dir_len[1] = e1.high_words + 1;
    h->ef_sel_len = (nb + 1 + 63) / 64;  // one entry per 64 elements of a sequence
    h->gr = (uint64_t *)jm.get(h->info.gr_words * 8 + 8);
    h->ef = (uint64_t *)jm.get(h->info.ef_words * 8 + 8);
    h->ef_dir = (uint64_t *)jm.get((h->ef_dir_len[0] + h->ef_dir_len[1] + 2 * h->ef_sel_len) * 8);
    return h->gr && h->ef && h->ef_dir ? MPHF_OK : MPHF_ENOMEM;
}

// Elias-Fano sequences of the key and bit offsets (Section 2.2,
// "Representation") into the zeroed h->ef, and their query directories.
void rs::write_ef_dirs(mphf_t *h, uint64_t nb, uint64_t *scan_tmp, cudaStream_t st) {
    const mphf_info &I = h->info;
    uint64_t *lo0 = h->ef, *hi0 = lo0 + I.ef_seq_words[0], *lo1 = hi0 + I.ef_seq_words[1],
             *hi1 = lo1 + I.ef_seq_words[2];
    launch_ef_write(h->cum_keys, nb + 1, I.ef_low_bits[0], lo0, hi0, st);
    launch_ef_write(h->bit_pos, nb + 1, I.ef_low_bits[1], lo1, hi1, st);
    uint64_t *rank0 = h->ef_dir, *rank1 = rank0 + h->ef_dir_len[0];
    uint64_t *sel0 = rank1 + h->ef_dir_len[1], *sel1 = sel0 + h->ef_sel_len;
    launch_rank_dir(hi0, I.ef_seq_words[1], rank0, scan_tmp, st);
    launch_rank_dir(hi1, I.ef_seq_words[3], rank1, scan_tmp, st);
    launch_select_dir(I.ef_seq_words[1], rank0, sel0, st);
    launch_select_dir(I.ef_seq_words[3], rank1, sel1, st);
}

extern "C" {

void mphf_default_params(mphf_build_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->leaf_size = 16;
    p->bucket_size = 2000;
    p->key_bytes = 8;
    p->leaf_bijection = MPHF_BIJECTION_ROTATION;
    p->max_value = MPHF_DEFAULT_MAX_VALUE;
    p->leaf_method = MPHF_LEAF_LOCKSTEP;
}

const char *mphf_strerror(int code) {
    switch (code) {
        case MPHF_OK: return "ok";
        case MPHF_EINVAL: return "invalid argument";
        case MPHF_ENOMEM: return "out of memory";
        case MPHF_ECUDA: return "CUDA runtime error";
        case MPHF_EDUPLICATE: return "duplicate keys (equal fingerprint lo word in one bucket)";
        case MPHF_ESEARCH_LIMIT: return "a node needs a value above max_value";
        case MPHF_EBUSY: return "busy";
        case MPHF_EBUCKET: return "a bucket holds more than 4096 keys";
        case MPHF_ENOTIMPL: return "not implemented";
        case MPHF_ETIMEOUT: return "a bounded device wait timed out";
        case MPHF_ECAPACITY: return "the packed function outgrew the space reserved for the prepared build";
        default: return "unknown error";
    }
}

int mphf_tau_table(uint32_t leaf_size, uint32_t leaf_bijection, uint32_t tree_shape, uint32_t max_m,
                   uint8_t *h_out) {
    if (!h_out || leaf_size < 2 || leaf_size > MPHF_MAX_LEAF || max_m > MPHF_MAX_BUCKET ||
        leaf_bijection > MPHF_BIJECTION_SHOCKHASH || tree_shape > MPHF_TREE_FANOUT2)
        return MPHF_EINVAL;
    const SizeTables &t = size_tables(leaf_size, leaf_bijection, tree_shape);
    memcpy(h_out, t.tau, max_m + 1);
    return MPHF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The build engine: any number of independent builds ("jobs") go through the
// same phases on one stream, with one host read between phases for all of
// them and ONE persistent search launch over the buckets of every job
// (largest buckets first across jobs, mixed leaf sizes in the same launch).
namespace rs {

thread_local PinnedWords t_pinned;


// Parameters of a build apart from where its keys are.
int check_shape(uint64_t n, const mphf_build_params *p) {
    if (!p) return MPHF_EINVAL;
    if (p->leaf_size < 2 || p->leaf_size > MPHF_MAX_LEAF || p->bucket_size < 1 ||
        p->bucket_size > MPHF_MAX_BUCKET_SIZE || (p->key_bytes != 8 && p->key_bytes != 16) ||
        n >= (1ull << 32))
        return MPHF_EINVAL;
    if (p->threads_per_block &&
        (p->threads_per_block % 32 || p->threads_per_block > 512 || p->threads_per_block < 64))
        return MPHF_EINVAL;
    if (p->leaf_method > MPHF_LEAF_TABLE || p->leaf_bijection > MPHF_BIJECTION_SHOCKHASH ||
        p->tree_shape > MPHF_TREE_FANOUT2)
        return MPHF_EINVAL;
    if (p->seeds_per_thread != 0 && p->seeds_per_thread != 1 && p->seeds_per_thread != 2 &&
        p->seeds_per_thread != 4)
        return MPHF_EINVAL;
    return MPHF_OK;
}

int check_params(const void *d_keys, uint64_t n, const mphf_build_params *p) {
    if ((n > 0 && !d_keys) || ((uintptr_t)d_keys & 7)) return MPHF_EINVAL;
    return check_shape(n, p);
}

void free_job_scratch(Job &j, Mem &mem) {
    mem.put(j.lo_s);
    mem.put(j.bb_s);
    mem.put(j.cursor);
    mem.put(j.small);
    mem.put(j.node_m);
    mem.put(j.counters);
    mem.put(j.blk);
    j.blk = nullptr;
    j.lo_s = j.counters = nullptr;
    j.bb_s = nullptr;
    j.cursor = j.small = nullptr;
    j.node_m = nullptr;
}

void fail_job(Job &j, int rc, Mem &mem) {
    if (j.rc == MPHF_OK) j.rc = rc;
    free_job_scratch(j, mem);
    if (j.h) {
        release(j.h, mem.st);
        j.h = nullptr;
    }
}

#define CU(x)                     \
    do {                          \
        if ((x) != cudaSuccess) { \
            cudaGetLastError();   \
            return MPHF_ECUDA;    \
        }                         \
    } while (0)

// Phase 1 (fingerprints, bucket sizes, plan, offsets) of every live job, then
// one host read of each job's node total, largest bucket and status.
// Jobs that fail get rc set; the return value is a failure of all of them.
int phase_plan(std::vector<Job *> &jobs, EngineCtx &c) {
    const cudaStream_t st = c.mem.st;
    for (Job *jp : jobs) {
        Job &j = *jp;
        if (j.rc) continue;
        mphf_t *h = j.h;
        Mem jm{h->has_alloc ? &h->alloc : nullptr, st};
        const uint64_t nb = j.nb;
        h->cum_keys = (uint64_t *)jm.get((nb + 1) * 8);
        h->node_off = (uint64_t *)jm.get((nb + 1) * 8);
        h->bit_pos = (uint64_t *)jm.get((nb + 1) * 8);
        j.cursor = (uint32_t *)c.mem.get((nb + 1) * 4);
        j.small = (uint32_t *)c.mem.get(64);
        j.lo_s = (uint64_t *)c.mem.get(j.n * 8);
        j.bb_s = (uint8_t *)c.mem.get(j.n);
        j.counters = (uint64_t *)c.mem.get(64);
        j.sort_g = sort_blocks(j.n, nb);
        if (j.sort_g) j.blk = (uint32_t *)c.mem.get((uint64_t)j.sort_g * nb * 4);
        if (!h->cum_keys || !h->node_off || !h->bit_pos || !j.cursor || !j.small || !j.lo_s ||
            !j.bb_s || !j.counters || (j.sort_g && !j.blk)) {
            fail_job(j, MPHF_ENOMEM, c.mem);
            continue;
        }
        CU(cudaMemsetAsync(h->cum_keys, 0, (nb + 1) * 8, st));
        CU(cudaMemsetAsync(h->node_off, 0, (nb + 1) * 8, st));
        CU(cudaMemsetAsync(j.cursor, 0, (nb + 1) * 4, st));
        CU(cudaMemsetAsync(j.small, 0, 64, st));
        CU(cudaMemsetAsync(j.counters, 0, 64, st));
        if (j.sort_g)
            launch_fp_hist_blk(j.d_keys, j.n, j.p.key_bytes, nb, j.range, j.sort_g, h->cum_keys, j.blk,
                               j.small, st);
        else
            launch_fp_hist(j.d_keys, j.n, j.p.key_bytes, nb, j.range, h->cum_keys, j.small, st);
        launch_plan(h->cum_keys, nb, h->tabs.nodes, h->node_off, j.small, j.small + 1, c.size_hist, st);
        j.planned = true;
        launch_exclusive_scan(h->cum_keys, nb + 1, c.scan_tmp, st);
        launch_exclusive_scan(h->node_off, nb + 1, c.scan_tmp, st);
        CU(cudaGetLastError());
    }
    for (size_t i = 0; i < jobs.size(); i++) {
        Job &j = *jobs[i];
        if (j.rc) continue;
        CU(cudaMemcpyAsync(c.host + 4 * i, j.h->node_off + j.nb, 8, cudaMemcpyDeviceToHost, st));
        CU(cudaMemcpyAsync(c.host + 4 * i + 1, j.small, 8, cudaMemcpyDeviceToHost, st));
    }
    CU(cudaStreamSynchronize(st));
    for (size_t i = 0; i < jobs.size(); i++) {
        Job &j = *jobs[i];
        if (j.rc) continue;
        j.n_nodes = c.host[4 * i];
        const uint32_t status = (uint32_t)c.host[4 * i + 1];
        j.max_m = (uint32_t)(c.host[4 * i + 1] >> 32);
        j.h->info.n_nodes = j.n_nodes;
        j.h->info.max_bucket = j.max_m;
        if (status) fail_job(j, status_code(status), c.mem);
    }
    return MPHF_OK;
}

// Phase 2: keys grouped by bucket and the search descriptor of every live job.
int phase_scatter(std::vector<Job *> &jobs, EngineCtx &c) {
    const cudaStream_t st = c.mem.st;
    for (Job *jp : jobs) {
        Job &j = *jp;
        if (j.rc) continue;
        mphf_t *h = j.h;
        Mem jm{h->has_alloc ? &h->alloc : nullptr, st};
        h->values = (uint64_t *)jm.get(j.n_nodes * 8);
        j.node_m = (uint16_t *)c.mem.get(j.n_nodes * 2);
        if (!h->values || !j.node_m) {
            fail_job(j, MPHF_ENOMEM, c.mem);
            continue;
        }
        if (j.sort_g)
            launch_scatter_blk(j.d_keys, j.n, j.p.key_bytes, j.nb, j.range, j.sort_g, h->cum_keys,
                               j.blk, j.lo_s, j.bb_s, j.small, st);
        else
            launch_scatter(j.d_keys, j.n, j.p.key_bytes, j.nb, j.range, h->cum_keys, j.cursor, j.lo_s,
                           j.bb_s, j.small, st);
        InstDesc &d = j.desc;
        memset(&d, 0, sizeof(d));
        d.lo = j.lo_s;
        d.bb = j.bb_s;
        d.bucket_off = h->cum_keys;
        d.node_off = h->node_off;
        d.nodes_tab = h->tabs.nodes;
        d.values = h->values;
        d.node_m = j.node_m;
        d.status = j.small;
        d.max_value = j.maxv;
        d.leaf = j.p.leaf_size;
        d.bij = j.p.leaf_bijection;
        d.tree = j.p.tree_shape;
        d.nb = (uint32_t)j.nb;
        d.red_leaf = (uint32_t)((1ull << 32) % j.p.leaf_size);
        d.leaf_method = j.p.leaf_method;
        d.spt = j.p.seeds_per_thread ? j.p.seeds_per_thread : (j.p.leaf_size >= 16 ? 2u : 1u);
        d.mod_c = h->tabs.mod_c;
        d.mod_M = h->tabs.mod_M;
        d.rot_canon = d.rot_period = nullptr;
        if (j.p.leaf_method == MPHF_LEAF_TABLE &&
            device_rot_tables(h->device, &d.rot_canon, &d.rot_period) != MPHF_OK) {
            fail_job(j, MPHF_ENOMEM, c.mem);
            continue;
        }
        CU(cudaGetLastError());
    }
    return MPHF_OK;
}

// Phases 3 and 4 of every live job whose search has finished: Golomb-Rice
// lengths and offsets, one host read of the bit totals and statuses, then
// the Golomb-Rice bits, Elias-Fano sequences, directories and statistics.
int phase_pack(std::vector<Job *> &jobs, EngineCtx &c) {
    const cudaStream_t st = c.mem.st;
    for (size_t i = 0; i < jobs.size(); i++) {
        Job &j = *jobs[i];
        if (j.rc) continue;
        mphf_t *h = j.h;
        CU(cudaMemsetAsync(h->bit_pos, 0, (j.nb + 1) * 8, st));
        launch_gr_lengths(h->values, j.node_m, h->node_off, j.nb, h->tabs.tau, j.p.leaf_size,
                          j.p.leaf_bijection, h->bit_pos, st);
        launch_exclusive_scan(h->bit_pos, j.nb + 1, c.scan_tmp, st);
        CU(cudaGetLastError());
        CU(cudaMemcpyAsync(c.host + 4 * i, h->bit_pos + j.nb, 8, cudaMemcpyDeviceToHost, st));
        CU(cudaMemcpyAsync(c.host + 4 * i + 1, j.small, 8, cudaMemcpyDeviceToHost, st));
    }
    CU(cudaStreamSynchronize(st));
    for (size_t i = 0; i < jobs.size(); i++) {
        Job &j = *jobs[i];
        if (j.rc) continue;
        mphf_t *h = j.h;
        const uint32_t status = (uint32_t)c.host[4 * i + 1];
        if (status) {
            fail_job(j, status_code(status), c.mem);
            continue;
        }
        const uint64_t gr_bits = c.host[4 * i];
        Mem jm{h->has_alloc ? &h->alloc : nullptr, st};
        if (alloc_packed(h, j.nb, j.n, gr_bits, jm) != MPHF_OK) {
            fail_job(j, MPHF_ENOMEM, c.mem);
            continue;
        }
        CU(cudaMemsetAsync(h->gr, 0, h->info.gr_words * 8 + 8, st));
        CU(cudaMemsetAsync(h->ef, 0, h->info.ef_words * 8 + 8, st));
        launch_gr_write(h->values, j.node_m, h->node_off, h->bit_pos, j.nb, h->tabs.tau,
                        h->tabs.fixed, h->cum_keys, j.p.leaf_size, j.p.leaf_bijection, h->gr, st);
        write_ef_dirs(h, j.nb, c.scan_tmp, st);
        launch_stats(h->values, j.node_m, j.n_nodes, j.p.leaf_size, j.p.leaf_bijection,
                     j.p.tree_shape, j.counters, st);
        CU(cudaGetLastError());
    }
    std::vector<uint64_t> hc(8 * (jobs.size() ? jobs.size() : 1));
    for (size_t i = 0; i < jobs.size(); i++)
        if (!jobs[i]->rc) CU(cudaMemcpyAsync(&hc[8 * i], jobs[i]->counters, 64, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    for (size_t i = 0; i < jobs.size(); i++) {
        Job &j = *jobs[i];
        if (j.rc) continue;
        for (int k = 0; k < 4; k++) {
            j.h->stats.trials[k] = hc[8 * i + k];
            j.h->stats.evals[k] = hc[8 * i + 4 + k];
        }
    }
    return MPHF_OK;
}
#undef CU

// Default block size of a search: the lower-level nodes of l >= 14 need
// hundreds of thousands of trials and fill 512 threads; smaller leaves and
// the fanout-2 tree do better with 256 (B300: l = 8 0.19 vs 0.30 ms, l = 12
// 15.6 both, fanout-2 l = 24 24.8 vs 28.3 ms; l = 16 8.85 s at 512 threads,
// two blocks per SM, against 9.22 s with one).
uint32_t default_threads(const std::vector<Job *> &jobs) {
    for (const Job *j : jobs)
        if (!j->rc && j->p.tree_shape == MPHF_TREE_RECSPLIT && j->p.leaf_size >= 14) return 512u;
    return 256u;
}

// Runs every job; afterwards each job has rc set and, if rc is OK, h built.
// Returns a code for failures that affect all jobs (CUDA errors), else OK.
// All jobs share each phase and ONE persistent search launch over all of
// their buckets (largest first across jobs).
int run_jobs(std::vector<Job> &jobs, cudaStream_t st, const mphf_allocator *shared_alloc,
             uint32_t threads, uint32_t blocks_per_sm) {
    EngineCtx c{Mem{shared_alloc, st}};
    std::vector<Job *> jp;
    uint64_t max_nb = 0, total_slots = 0;
    for (auto &j : jobs) {
        jp.push_back(&j);
        max_nb = j.nb > max_nb ? j.nb : max_nb;
    }
    uint32_t *head = nullptr;
    InstDesc *d_inst = nullptr;
    WorkItem *items = nullptr;
    StealQueue *steal = nullptr;
    std::vector<InstDesc> hinst;
    std::vector<uint32_t> inst_job;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    uint32_t max_m = 0;
    float ms[4] = {0, 0, 0, 0};
    int grc = c.reserve(jobs.size(), max_nb);
    for (auto &e : ev) cudaEventCreate(&e);
    cudaEventRecord(ev[0], st);
    head = (uint32_t *)c.mem.get(64);
    if (grc == MPHF_OK && !head) grc = MPHF_ENOMEM;
    if (grc == MPHF_OK) grc = c.clear_order();
    if (grc == MPHF_OK && cudaMemsetAsync(head, 0, 64, st) != cudaSuccess) grc = MPHF_ECUDA;
    if (grc == MPHF_OK) grc = phase_plan(jp, c);
    cudaEventRecord(ev[1], st);
    if (grc == MPHF_OK) {
        for (Job *j : jp)
            if (j->planned) total_slots += j->nb;  // every bucket in size_hist gets a slot
        grc = phase_scatter(jp, c);
    }
    if (grc == MPHF_OK) {
        for (size_t i = 0; i < jp.size(); i++) {
            if (jp[i]->rc) continue;
            inst_job.push_back((uint32_t)i);
            hinst.push_back(jp[i]->desc);
            max_m = jp[i]->max_m > max_m ? jp[i]->max_m : max_m;
        }
        if (total_slots > 0xFFFFFFFFull) grc = MPHF_EINVAL;
    }
    if (grc == MPHF_OK && !hinst.empty() && total_slots > 0) {
        // slots of jobs that failed after their plan stay empty (all-ones: skipped)
        launch_exclusive_scan(c.size_hist, 4098, c.scan_tmp, st);
        d_inst = (InstDesc *)c.mem.get(hinst.size() * sizeof(InstDesc));
        items = (WorkItem *)c.mem.get(total_slots * sizeof(WorkItem));
        steal = (StealQueue *)c.mem.get(kStealBytes);
        if (!d_inst || !items || !steal) {
            grc = MPHF_ENOMEM;
        } else if (cudaMemsetAsync(items, 0xFF, total_slots * sizeof(WorkItem), st) != cudaSuccess ||
                   cudaMemsetAsync(steal, 0, kStealBytes, st) != cudaSuccess ||
                   cudaMemcpyAsync(d_inst, hinst.data(), hinst.size() * sizeof(InstDesc),
                                   cudaMemcpyHostToDevice, st) != cudaSuccess) {
            grc = MPHF_ECUDA;
        } else {
            for (size_t k = 0; k < inst_job.size(); k++) {
                Job &j = *jp[inst_job[k]];
                launch_items_by_size(j.h->cum_keys, j.nb, c.size_hist, c.size_cursor, items,
                                     (uint32_t)k, st);
            }
            if (!threads) threads = default_threads(jp);
            SearchLaunch L = plan_search_launch(max_m, (uint32_t)total_slots, threads, blocks_per_sm);
            cudaEventRecord(ev[2], st);
            launch_search(d_inst, (uint32_t)hinst.size(), items, (uint32_t)total_slots, head, L, steal, st);
            if (cudaGetLastError() != cudaSuccess) grc = MPHF_ECUDA;
        }
    } else {
        cudaEventRecord(ev[2], st);
    }
    cudaEventRecord(ev[3], st);
    if (grc == MPHF_OK) grc = phase_pack(jp, c);
    cudaEventRecord(ev[4], st);
    if (grc == MPHF_OK) {
        cudaEventSynchronize(ev[4]);
        cudaEventElapsedTime(&ms[0], ev[0], ev[1]);
        cudaEventElapsedTime(&ms[1], ev[2], ev[3]);
        cudaEventElapsedTime(&ms[2], ev[3], ev[4]);
        cudaEventElapsedTime(&ms[3], ev[0], ev[4]);
        for (Job *j : jp) {
            if (j->rc) continue;
            j->h->stats.ms_plan = ms[0];
            j->h->stats.ms_search = ms[1];
            j->h->stats.ms_pack = ms[2];
            j->h->stats.ms_total = ms[3];
        }
    }
    cudaStreamSynchronize(st);
    for (auto &j : jobs) {
        free_job_scratch(j, c.mem);
        if (grc != MPHF_OK && j.rc == MPHF_OK) fail_job(j, grc, c.mem);
    }
    c.mem.put(head);
    c.mem.put(d_inst);
    c.mem.put(items);
    c.mem.put(steal);
    c.release();
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
    return grc;
}

// Creates the handle of a job (parameters checked, tables ready).
void start_job(Job &j, const void *d_keys, uint64_t n, const mphf_build_params &p) {
    j.d_keys = d_keys;
    j.n = n;
    j.p = p;
    j.rc = check_params(d_keys, n, &p);
    if (j.rc) return;
    mphf_t *h = new (std::nothrow) mphf;
    if (!h) {
        j.rc = MPHF_ENOMEM;
        return;
    }
    cudaGetDevice(&h->device);
    if (p.allocator) {
        h->alloc = *p.allocator;
        h->has_alloc = true;
    }
    j.h = h;
    j.nb = (n + p.bucket_size - 1) / p.bucket_size;
    j.range = BucketRange{j.nb, 0};
    j.maxv = p.max_value ? p.max_value : MPHF_DEFAULT_MAX_VALUE;
    h->info.n = n;
    h->info.nb = j.nb;
    h->info.leaf_size = p.leaf_size;
    h->info.bucket_size = p.bucket_size;
    h->info.key_bytes = p.key_bytes;
    h->info.leaf_bijection = p.leaf_bijection;
    h->info.tree_shape = p.tree_shape;
    int rc = device_tables(h->device, p.leaf_size, h->info.leaf_bijection, h->info.tree_shape,
                           &h->tabs);
    if (rc) {
        release(h, 0);
        j.h = nullptr;
        j.rc = rc;
    }
}

}  // namespace rs

extern "C" {

int mphf_build_ex(const void *d_keys, uint64_t n, const mphf_build_params *p, void *stream,
                  mphf_t **out) {
    if (!out || !p) return MPHF_EINVAL;
    *out = nullptr;
    std::vector<Job> jobs(1);
    start_job(jobs[0], d_keys, n, *p);
    if (jobs[0].rc) return jobs[0].rc;
    int grc = run_jobs(jobs, (cudaStream_t)stream, p->allocator, p->threads_per_block,
                       p->blocks_per_sm);
    if (grc) return grc;
    if (jobs[0].rc) return jobs[0].rc;
    *out = jobs[0].h;
    return MPHF_OK;
}

int mphf_build(const void *d_keys, uint64_t n, uint32_t leaf_size, uint32_t bucket_size,
               void *stream, mphf_t **out) {
    mphf_build_params p;
    mphf_default_params(&p);
    p.leaf_size = leaf_size;
    p.bucket_size = bucket_size;
    return mphf_build_ex(d_keys, n, &p, stream, out);
}

int mphf_build_host(const void *h_keys, uint64_t n, const mphf_build_params *p, void *stream,
                    mphf_t **out) {
    if (!out || (n > 0 && !h_keys)) return MPHF_EINVAL;
    *out = nullptr;
    int rc = check_shape(n, p);  // before copying n keys to the device
    if (rc != MPHF_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Mem mem{p->allocator, st};
    void *d = mem.get(n * p->key_bytes);
    if (!d) return MPHF_ENOMEM;
    if (n && cudaMemcpyAsync(d, h_keys, n * p->key_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        mem.put(d);
        return MPHF_ECUDA;
    }
    rc = mphf_build_ex(d, n, p, stream, out);
    mem.put(d);
    return rc;
}

static QueryView view_of(const mphf_t *h) {
    QueryView q;
    const mphf_info &I = h->info;
    q.gr = h->gr;
    q.ef_low[0] = h->ef;
    q.ef_high[0] = h->ef + I.ef_seq_words[0];
    q.ef_low[1] = q.ef_high[0] + I.ef_seq_words[1];
    q.ef_high[1] = q.ef_low[1] + I.ef_seq_words[2];
    q.ef_dir[0] = h->ef_dir;
    q.ef_dir[1] = h->ef_dir + h->ef_dir_len[0];
    q.ef_sel[0] = q.ef_dir[1] + h->ef_dir_len[1];
    q.ef_sel[1] = q.ef_sel[0] + h->ef_sel_len;
    q.ef_L[0] = I.ef_low_bits[0];
    q.ef_L[1] = I.ef_low_bits[1];
    q.tau = h->tabs.tau;
    q.nodes_tab = h->tabs.nodes;
    q.fixed_tab = h->tabs.fixed;
    q.left_tab = h->tabs.left;
    q.mod_c = h->tabs.mod_c;
    q.mod_M = h->tabs.mod_M;
    q.salts = h->tabs.salts;
    const Shape shp = make_shape(I.leaf_size, I.tree_shape);
    q.lower1 = shp.lower1;
    q.lower2 = shp.lower2;
    q.magic_leaf = unit_magic(shp.leaf);
    q.magic_l1 = unit_magic(shp.lower1);
    q.nb = I.nb;
    q.leaf = I.leaf_size;
    q.bij = I.leaf_bijection;
    q.key_bytes = I.key_bytes;
    q.tree = I.tree_shape;
    return q;
}

// Checks shared by the entry points that query: keys 8-byte aligned, the
// function built on the current device and not empty.
static int query_args(const mphf_t *h, const void *d_keys, uint64_t n) {
    if (!h || (n > 0 && !d_keys) || ((uintptr_t)d_keys & 7)) return MPHF_EINVAL;
    if (n == 0) return MPHF_OK;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return MPHF_ECUDA;
    }
    if (dev != h->device || h->info.n == 0 || h->shard || !h->ready) return MPHF_EINVAL;
    return MPHF_OK;
}

int mphf_query(const mphf_t *h, const void *d_keys, uint64_t n, uint64_t *d_out, void *stream) {
    if (n > 0 && (!d_out || ((uintptr_t)d_out & 7))) return MPHF_EINVAL;
    int rc = query_args(h, d_keys, n);
    if (rc != MPHF_OK || n == 0) return rc;
    launch_query(view_of(h), d_keys, n, d_out, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? MPHF_OK : MPHF_ECUDA;
}

int mphf_verify(const mphf_t *h, const void *d_keys, uint64_t n, uint64_t *n_bad, void *stream) {
    if (!n_bad) return MPHF_EINVAL;
    *n_bad = 0;
    int rc0 = query_args(h, d_keys, n);
    if (rc0 != MPHF_OK || n == 0) return rc0;
    cudaStream_t st = (cudaStream_t)stream;
    Mem mem{h->has_alloc ? &h->alloc : nullptr, st};
    uint64_t *vals = (uint64_t *)mem.get(n * 8);
    uint64_t words = (n + 31) / 32;
    uint32_t *bitmap = (uint32_t *)mem.get(words * 4 + 8);
    unsigned long long *bad = (unsigned long long *)mem.get(8);
    int rc = MPHF_OK;
    if (!vals || !bitmap || !bad) {
        rc = MPHF_ENOMEM;
    } else if (cudaMemsetAsync(bitmap, 0, words * 4 + 8, st) != cudaSuccess ||
               cudaMemsetAsync(bad, 0, 8, st) != cudaSuccess) {
        cudaGetLastError();  // an uncleared bitmap would give a wrong count
        rc = MPHF_ECUDA;
    } else {
        rc = mphf_query(h, d_keys, n, vals, stream);
        if (rc == MPHF_OK) {
            launch_mark(vals, n, bitmap, bad, st);
            unsigned long long hb = 0;
            if (cudaMemcpyAsync(&hb, bad, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                rc = MPHF_ECUDA;
            *n_bad = hb;
        }
    }
    mem.put(vals);
    mem.put(bitmap);
    mem.put(bad);
    cudaStreamSynchronize(st);
    return rc;
}

int mphf_get_info(const mphf_t *h, mphf_info *info) {
    if (!h || !info) return MPHF_EINVAL;
    *info = h->info;
    return MPHF_OK;
}

int mphf_get_values(const mphf_t *h, const uint64_t **d_values, const uint64_t **d_node_off,
                    const uint64_t **d_cum_keys, const uint64_t **d_bit_pos) {
    if (!h) return MPHF_EINVAL;
    if (d_values) *d_values = h->values;
    if (d_node_off) *d_node_off = h->node_off;
    if (d_cum_keys) *d_cum_keys = h->cum_keys;
    if (d_bit_pos) *d_bit_pos = h->bit_pos;
    return MPHF_OK;
}

int mphf_get_bits(const mphf_t *h, const uint64_t **d_gr, uint64_t *gr_bits, const uint64_t **d_ef,
                  uint64_t *ef_words) {
    if (!h) return MPHF_EINVAL;
    if (d_gr) *d_gr = h->gr;
    if (gr_bits) *gr_bits = h->info.gr_bits;
    if (d_ef) *d_ef = h->ef;
    if (ef_words) *ef_words = h->info.ef_words;
    return MPHF_OK;
}

int mphf_get_stats(const mphf_t *h, mphf_stats *s) {
    if (!h || !s) return MPHF_EINVAL;
    *s = h->stats;
    return MPHF_OK;
}

int mphf_serialize(const mphf_t *h, void *h_buf, size_t *len, void *stream) {
    if (!h || !len || h->shard || !h->ready) return MPHF_EINVAL;
    const size_t head = sizeof(uint64_t) * kHeadWords;
    const size_t need = head + (h->info.gr_words + h->info.ef_words) * 8;
    if (!h_buf) {
        *len = need;
        return MPHF_OK;
    }
    if (*len < need) {
        *len = need;
        return MPHF_EINVAL;
    }
    uint64_t hd[kHeadWords] = {kMagic, h->info.n, h->info.nb,
                       h->info.leaf_size | ((uint64_t)h->info.tree_shape << 16),
                       h->info.bucket_size, h->info.key_bytes,
                       h->info.leaf_bijection, h->info.gr_bits, h->info.gr_words,
                       h->info.ef_words, h->info.ef_low_bits[0], h->info.ef_low_bits[1],
                       h->info.ef_seq_words[0], h->info.ef_seq_words[1], h->info.ef_seq_words[2],
                       h->info.ef_seq_words[3]};
    memcpy(h_buf, hd, head);
    cudaStream_t st = (cudaStream_t)stream;
    uint8_t *dst = (uint8_t *)h_buf + head;
    if (h->info.gr_words &&
        cudaMemcpyAsync(dst, h->gr, h->info.gr_words * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return MPHF_ECUDA;
    if (h->info.ef_words && cudaMemcpyAsync(dst + h->info.gr_words * 8, h->ef, h->info.ef_words * 8,
                                            cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return MPHF_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return MPHF_ECUDA;
    *len = need;
    return MPHF_OK;
}

int mphf_free(mphf_t *h) {
    if (!h) return MPHF_EINVAL;
    int cur = h->device;
    if (cudaGetDevice(&cur) != cudaSuccess) cur = h->device;
    const int dev = h->device;
    if (cur != dev) cudaSetDevice(dev);
    cudaDeviceSynchronize();  // work still in flight on any stream may read these arrays
    release(h, 0);
    if (cur != dev) cudaSetDevice(cur);
    return MPHF_OK;
}

uint64_t mphf_kernel_launches(void) { return launches_total(); }

int mphf_build_batch(const mphf_build_desc *descs, uint32_t count, void *stream, mphf_t **outs,
                     int *statuses) {
    if (count && (!descs || !outs)) return MPHF_EINVAL;
    if (count == 0) return MPHF_OK;  // nothing to build, nothing to allocate
    std::vector<Job> jobs(count);
    for (uint32_t i = 0; i < count; i++) {
        mphf_build_params p;
        mphf_default_params(&p);
        p.leaf_size = descs[i].leaf_size;
        p.bucket_size = descs[i].bucket_size;
        p.key_bytes = descs[i].key_bytes;
        p.leaf_bijection = descs[i].leaf_bijection;
        p.tree_shape = descs[i].tree_shape;
        p.max_value = descs[i].max_value ? descs[i].max_value : MPHF_DEFAULT_MAX_VALUE;
        p.seeds_per_thread = descs[i].seeds_per_thread;
        outs[i] = nullptr;
        start_job(jobs[i], descs[i].d_keys, descs[i].n, p);
    }
    int grc = run_jobs(jobs, (cudaStream_t)stream, nullptr, 0, 0);
    int first = grc;
    for (uint32_t i = 0; i < count; i++) {
        int rc = jobs[i].rc ? jobs[i].rc : grc;
        if (statuses) statuses[i] = rc;
        if (rc == MPHF_OK) outs[i] = jobs[i].h;
        if (rc && first == MPHF_OK) first = rc;
    }
    return first;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Loading a serialised function.  The Golomb-Rice words and the two
// Elias-Fano sequences are the whole function (Section 2.2,
// "Representation"); the per-size tables and the query directories are
// recomputed.  A blob may be corrupt, and the query kernel trusts the
// structure it walks, so the host decodes all of it first: the header's
// sizes must agree with each other, the Elias-Fano sequences must decode to
// bucket offsets, and every bucket's code must hold exactly its nodes'
// fixed parts and unary terminators within its own bits.
namespace {

// Bits [pos, pos + w) of a little-endian word stream, w <= 64; the caller
// guarantees pos + w <= 64 * (words in the stream).
uint64_t host_bits(const uint64_t *words, uint64_t pos, uint32_t w) {
    if (w == 0) return 0;
    const uint64_t i = pos >> 6;
    const uint32_t s = (uint32_t)(pos & 63);
    uint64_t v = words[i] >> s;
    if (s + w > 64) v |= words[i + 1] << (64 - s);
    return w == 64 ? v : v & ((1ull << w) - 1);
}

// First set bit in [pos, end), or end.
uint64_t next_one(const uint64_t *words, uint64_t pos, uint64_t end) {
    while (pos < end) {
        const uint64_t w = words[pos >> 6] >> (pos & 63);
        if (w) {
            const uint64_t p = pos + (uint64_t)__builtin_ctzll(w);
            return p < end ? p : end;
        }
        pos = (pos | 63) + 1;
    }
    return end;
}

// Elias-Fano sequence of k values: low parts of L bits, then the high bit
// vector, which must hold exactly k ones.
bool ef_decode(const uint64_t *low, const uint64_t *high, uint64_t high_words, uint32_t L,
               uint64_t k, std::vector<uint64_t> &out) {
    out.assign(k, 0);
    uint64_t i = 0;
    for (uint64_t w = 0; w < high_words; w++) {
        for (uint64_t x = high[w]; x; x &= x - 1) {
            if (i == k) return false;
            const uint64_t hv = w * 64 + (uint64_t)__builtin_ctzll(x) - i;
            if (L && hv > (~0ull >> L)) return false;
            out[i] = (hv << L) | host_bits(low, i * L, L);
            i++;
        }
    }
    return i == k;
}

// Node sizes of the subtree of m keys in preorder (nodes of >= 2 keys).
void preorder_sizes(const Shape &s, uint32_t m, std::vector<uint32_t> &out) {
    std::vector<uint32_t> stack{m};
    while (!stack.empty()) {
        const uint32_t q = stack.back();
        stack.pop_back();
        if (q < 2) continue;
        out.push_back(q);
        if (q > s.leaf)
            for (uint32_t c = num_parts(s, q); c-- > 0;) stack.push_back(part_size(s, q, c));
    }
}

// A blob decoded on the host.
struct Decoded {
    mphf_info info{};
    const uint64_t *gr = nullptr, *ef = nullptr;  // inside the blob's words
    std::vector<uint64_t> copy;                   // the blob, when the caller's buffer is unaligned
    std::vector<uint64_t> cum, pos, node_off, values;
};

int decode_blob(const void *buf, size_t len, bool full, Decoded &d) {
    if (!buf || len < kHeadWords * 8) return MPHF_EINVAL;
    if ((uintptr_t)buf & 7) {
        d.copy.assign(len / 8, 0);
        memcpy(d.copy.data(), buf, d.copy.size() * 8);
        buf = d.copy.data();
    }
    const uint64_t *hd = (const uint64_t *)buf;
    mphf_info &I = d.info;
    if (hd[0] != kMagic || hd[1] >= (1ull << 32) || (hd[3] >> 32) || ((hd[3] >> 16) & 0xFFFF) > 1 ||
        (hd[3] & 0xFFFF) < 2 || (hd[3] & 0xFFFF) > MPHF_MAX_LEAF || hd[4] < 1 ||
        hd[4] > MPHF_MAX_BUCKET_SIZE || (hd[5] != 8 && hd[5] != 16) || hd[6] > MPHF_BIJECTION_SHOCKHASH)
        return MPHF_EINVAL;
    I.n = hd[1];
    I.nb = hd[2];
    I.leaf_size = (uint32_t)(hd[3] & 0xFFFF);
    I.tree_shape = (uint32_t)(hd[3] >> 16);
    I.bucket_size = (uint32_t)hd[4];
    I.key_bytes = (uint32_t)hd[5];
    I.leaf_bijection = (uint32_t)hd[6];
    I.gr_bits = hd[7];
    I.gr_words = hd[8];
    I.ef_words = hd[9];
    const uint64_t room = (len - kHeadWords * 8) / 8;  // payload words present
    if (I.nb != (I.n + I.bucket_size - 1) / I.bucket_size || I.gr_words > room ||
        I.ef_words > room - I.gr_words || I.gr_words != I.gr_bits / 64 + (I.gr_bits % 64 != 0))
        return MPHF_EINVAL;
    const EfDims e0 = ef_dims(I.nb + 1, I.n), e1 = ef_dims(I.nb + 1, I.gr_bits);
    if (hd[10] != e0.L || hd[11] != e1.L || hd[12] != e0.low_words || hd[13] != e0.high_words ||
        hd[14] != e1.low_words || hd[15] != e1.high_words ||
        I.ef_words != e0.low_words + e0.high_words + e1.low_words + e1.high_words)
        return MPHF_EINVAL;
    I.ef_low_bits[0] = e0.L;
    I.ef_low_bits[1] = e1.L;
    I.ef_seq_words[0] = e0.low_words;
    I.ef_seq_words[1] = e0.high_words;
    I.ef_seq_words[2] = e1.low_words;
    I.ef_seq_words[3] = e1.high_words;
    d.gr = hd + kHeadWords;
    d.ef = d.gr + I.gr_words;
    const uint64_t *lo0 = d.ef, *hi0 = lo0 + e0.low_words, *lo1 = hi0 + e0.high_words,
                   *hi1 = lo1 + e1.low_words;
    const uint64_t k = I.nb + 1;
    if (!ef_decode(lo0, hi0, e0.high_words, e0.L, k, d.cum) ||
        !ef_decode(lo1, hi1, e1.high_words, e1.L, k, d.pos))
        return MPHF_EINVAL;
    if (d.cum[0] != 0 || d.cum[I.nb] != I.n || d.pos[0] != 0 || d.pos[I.nb] != I.gr_bits)
        return MPHF_EINVAL;
    const SizeTables &t = size_tables(I.leaf_size, I.leaf_bijection, I.tree_shape);
    const Shape s = make_shape(I.leaf_size, I.tree_shape);
    const bool shock = I.leaf_bijection == MPHF_BIJECTION_SHOCKHASH;
    d.node_off.assign(k, 0);
    if (full) d.values.clear();
    std::vector<uint32_t> sizes;
    I.max_bucket = 0;
    for (uint64_t b = 0; b < I.nb; b++) {
        if (d.cum[b + 1] < d.cum[b] || d.cum[b + 1] - d.cum[b] > MPHF_MAX_BUCKET ||
            d.pos[b + 1] < d.pos[b])
            return MPHF_EINVAL;
        const uint32_t m = (uint32_t)(d.cum[b + 1] - d.cum[b]);
        const uint64_t start = d.pos[b], end = d.pos[b + 1];
        I.max_bucket = m > I.max_bucket ? m : I.max_bucket;
        d.node_off[b + 1] = d.node_off[b] + t.nodes[m];
        if (end - start < (uint64_t)t.fixed[m] + t.nodes[m]) return MPHF_EINVAL;
        sizes.clear();
        preorder_sizes(s, m, sizes);
        uint64_t fpos = start, upos = start + t.fixed[m];
        for (uint32_t q : sizes) {
            const uint32_t tq = t.tau[q];
            const bool sh_leaf = shock && q <= I.leaf_size;
            const uint64_t low = host_bits(d.gr, fpos, tq);
            fpos += tq;
            const uint64_t z = sh_leaf ? host_bits(d.gr, fpos, q) : 0;
            fpos += sh_leaf ? q : 0;
            const uint64_t one = next_one(d.gr, upos, end);
            if (one == end) return MPHF_EINVAL;  // the unary code runs past its bucket
            const uint64_t high = one - upos;
            upos = one + 1;
            if (tq >= 64 || high > (~0ull >> tq)) return MPHF_EINVAL;
            const uint64_t coded = (high << tq) | low;
            if (sh_leaf && coded > MPHF_SH_MASK) return MPHF_EINVAL;
            if (full) d.values.push_back(sh_leaf ? coded | (z << MPHF_SH_BITS) : coded);
        }
        if (upos != end) return MPHF_EINVAL;  // bits left over after the last terminator
    }
    I.n_nodes = d.node_off[I.nb];
    return MPHF_OK;
}

}  // namespace

extern "C" {

int mphf_load_info(const void *h_buf, size_t len, mphf_info *info) {
    if (!info) return MPHF_EINVAL;
    Decoded d;
    const int rc = decode_blob(h_buf, len, false, d);
    if (rc == MPHF_OK) *info = d.info;
    return rc;
}

int mphf_load(const void *h_buf, size_t len, const mphf_allocator *allocator, void *stream,
              mphf_t **out) {
    if (!out) return MPHF_EINVAL;
    *out = nullptr;
    Decoded d;
    int rc = decode_blob(h_buf, len, true, d);
    if (rc != MPHF_OK) return rc;
    mphf_t *h = new (std::nothrow) mphf;
    if (!h) return MPHF_ENOMEM;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return MPHF_ECUDA;
    }
    if (allocator) {
        h->alloc = *allocator;
        h->has_alloc = true;
    }
    h->info = d.info;
    rc = device_tables(h->device, d.info.leaf_size, d.info.leaf_bijection, d.info.tree_shape, &h->tabs);
    if (rc != MPHF_OK) {
        release(h, 0);
        return rc;
    }
    cudaStream_t st = (cudaStream_t)stream;
    Mem mem{allocator, st};
    const mphf_info &I = d.info;
    const uint64_t k = I.nb + 1, hw0 = I.ef_seq_words[1], hw1 = I.ef_seq_words[3];
    h->ef_dir_len[0] = hw0 + 1;
    h->ef_dir_len[1] = hw1 + 1;
    h->ef_sel_len = (k + 63) / 64;
    h->cum_keys = (uint64_t *)mem.get(k * 8);
    h->node_off = (uint64_t *)mem.get(k * 8);
    h->bit_pos = (uint64_t *)mem.get(k * 8);
    h->values = (uint64_t *)mem.get(I.n_nodes * 8);
    h->gr = (uint64_t *)mem.get(I.gr_words * 8 + 8);
    h->ef = (uint64_t *)mem.get(I.ef_words * 8 + 8);
    h->ef_dir = (uint64_t *)mem.get((h->ef_dir_len[0] + h->ef_dir_len[1] + 2 * h->ef_sel_len) * 8);
    const uint64_t tmp_words = scan_tmp_words((hw0 > hw1 ? hw0 : hw1) + 1) + 64;
    uint64_t *tmp = (uint64_t *)mem.get(tmp_words * 8);
    rc = MPHF_OK;
    if (!h->cum_keys || !h->node_off || !h->bit_pos || !h->values || !h->gr || !h->ef || !h->ef_dir || !tmp) {
        rc = MPHF_ENOMEM;
    } else {
        struct Copy {
            void *dst;
            const void *src;
            size_t bytes;
        } copies[] = {{h->cum_keys, d.cum.data(), k * 8},
                      {h->node_off, d.node_off.data(), k * 8},
                      {h->bit_pos, d.pos.data(), k * 8},
                      {h->values, d.values.data(), I.n_nodes * 8},
                      {h->gr, d.gr, I.gr_words * 8},
                      {h->ef, d.ef, I.ef_words * 8}};
        // the word after each packed array is read past the end by bit readers
        if (cudaMemsetAsync(h->gr + I.gr_words, 0, 8, st) != cudaSuccess ||
            cudaMemsetAsync(h->ef + I.ef_words, 0, 8, st) != cudaSuccess)
            rc = MPHF_ECUDA;
        for (const Copy &c : copies)
            if (rc == MPHF_OK && c.bytes &&
                cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
                rc = MPHF_ECUDA;
        if (rc == MPHF_OK) {
            const uint64_t *hi0 = h->ef + I.ef_seq_words[0];
            const uint64_t *hi1 = hi0 + hw0 + I.ef_seq_words[2];
            uint64_t *rank0 = h->ef_dir, *rank1 = rank0 + h->ef_dir_len[0];
            uint64_t *sel0 = rank1 + h->ef_dir_len[1], *sel1 = sel0 + h->ef_sel_len;
            launch_rank_dir(hi0, hw0, rank0, tmp, st);
            launch_rank_dir(hi1, hw1, rank1, tmp, st);
            launch_select_dir(hw0, rank0, sel0, st);
            launch_select_dir(hw1, rank1, sel1, st);
            if (cudaGetLastError() != cudaSuccess) rc = MPHF_ECUDA;
        }
        // the host arrays are read by the copies: wait before they go away
        if (cudaStreamSynchronize(st) != cudaSuccess) rc = MPHF_ECUDA;
    }
    if (rc != MPHF_OK) cudaGetLastError();
    mem.put(tmp);
    if (rc != MPHF_OK) {
        cudaStreamSynchronize(st);
        release(h, st);
        return rc;
    }
    *out = h;
    return MPHF_OK;
}

}  // extern "C"

