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
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"
#include "engine.h"
#include "mphf.h"
#include "tables.h"

using namespace rs;

#ifndef MPHF_LPT
#define MPHF_LPT 1
#endif

namespace {

struct DevTables {
    uint8_t *tau = nullptr;
    uint32_t *nodes = nullptr;
    uint32_t *fixed = nullptr;
};

// Per-device copies of the per-size tables; live until the process exits.
int device_tables(int dev, uint32_t leaf, uint32_t rotation, DevTables *out) {
    static std::mutex mu;
    static std::map<uint64_t, DevTables> cache;
    std::lock_guard<std::mutex> g(mu);
    uint64_t key = ((uint64_t)dev << 32) | (leaf << 1) | (rotation ? 1 : 0);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *out = it->second;
        return MPHF_OK;
    }
    const SizeTables &t = size_tables(leaf, rotation);
    DevTables d;
    if (cudaMalloc(&d.tau, sizeof(t.tau)) != cudaSuccess) return MPHF_ENOMEM;
    if (cudaMalloc(&d.nodes, sizeof(t.nodes)) != cudaSuccess) return MPHF_ENOMEM;
    if (cudaMalloc(&d.fixed, sizeof(t.fixed)) != cudaSuccess) return MPHF_ENOMEM;
    if (cudaMemcpy(d.tau, t.tau, sizeof(t.tau), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d.nodes, t.nodes, sizeof(t.nodes), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d.fixed, t.fixed, sizeof(t.fixed), cudaMemcpyHostToDevice) != cudaSuccess)
        return MPHF_ECUDA;
    cache[key] = d;
    *out = d;
    return MPHF_OK;
}

struct Mem {
    const mphf_allocator *a;
    cudaStream_t st;
    void *get(size_t bytes) {
        if (bytes == 0) bytes = 8;
        if (a) return a->alloc(bytes, st, a->ctx);
        void *p = nullptr;
        if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return p;
    }
    void put(void *p) {
        if (!p) return;
        if (a)
            a->free(p, st, a->ctx);
        else
            cudaFreeAsync(p, st);
    }
};

struct EfDims {
    uint32_t L;
    uint64_t low_words, high_words;
};

EfDims ef_dims(uint64_t k, uint64_t last) {
    EfDims d;
    d.L = 0;
    if (last >= k) {
        uint64_t q = last / k;
        while (q >>= 1) d.L++;
    }
    d.low_words = (k * d.L + 63) / 64;
    d.high_words = ((last >> d.L) + k + 63) / 64;
    return d;
}

int status_code(uint32_t st) {
    if (st & ST_BUCKET) return MPHF_EBUCKET;
    if (st & ST_DUPLICATE) return MPHF_EDUPLICATE;
    if (st & ST_LIMIT) return MPHF_ESEARCH_LIMIT;
    if (st & ST_TIMEOUT) return MPHF_ETIMEOUT;
    return MPHF_OK;
}

__global__ void k_items(WorkItem *items, uint32_t count, uint32_t inst) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        items[i] = WorkItem{inst, i};
}

}  // namespace

struct mphf {
    int device = 0;
    mphf_info info{};
    mphf_allocator alloc{};
    bool has_alloc = false;
    uint64_t *values = nullptr, *node_off = nullptr, *cum_keys = nullptr, *bit_pos = nullptr;
    uint64_t *gr = nullptr, *ef = nullptr, *ef_dir = nullptr;
    uint64_t ef_dir_len[2] = {0, 0};
    DevTables tabs;
    mphf_stats stats{};
};

static void release(mphf_t *h) {
    if (!h) return;
    Mem mem{h->has_alloc ? &h->alloc : nullptr, 0};
    void *ptrs[] = {h->values, h->node_off, h->cum_keys, h->bit_pos, h->gr, h->ef, h->ef_dir};
    for (void *p : ptrs) mem.put(p);
    delete h;
}

extern "C" {

void mphf_default_params(mphf_build_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->leaf_size = 16;
    p->bucket_size = 2000;
    p->key_bytes = 8;
    p->rotation_fitting = 1;
    p->max_value = MPHF_DEFAULT_MAX_VALUE;
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
        default: return "unknown error";
    }
}

int mphf_tau_table(uint32_t leaf_size, uint32_t rotation_fitting, uint32_t max_m, uint8_t *h_out) {
    if (!h_out || leaf_size < 2 || leaf_size > MPHF_MAX_LEAF || max_m > MPHF_MAX_BUCKET)
        return MPHF_EINVAL;
    const SizeTables &t = size_tables(leaf_size, rotation_fitting ? 1 : 0);
    memcpy(h_out, t.tau, max_m + 1);
    return MPHF_OK;
}

int mphf_build_ex(const void *d_keys, uint64_t n, const mphf_build_params *p, void *stream,
                  mphf_t **out) {
    if (!out || !p) return MPHF_EINVAL;
    *out = nullptr;
    if (p->leaf_size < 2 || p->leaf_size > MPHF_MAX_LEAF || p->bucket_size < 1 ||
        p->bucket_size > MPHF_MAX_BUCKET_SIZE || (p->key_bytes != 8 && p->key_bytes != 16) ||
        n >= (1ull << 32) || (n > 0 && !d_keys) || ((uintptr_t)d_keys & 7))
        return MPHF_EINVAL;
    if (p->threads_per_block && (p->threads_per_block % 32 || p->threads_per_block > 512 ||
                                 p->threads_per_block < 64))
        return MPHF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    mphf_t *h = new (std::nothrow) mphf;
    if (!h) return MPHF_ENOMEM;
    cudaGetDevice(&h->device);
    if (p->allocator) {
        h->alloc = *p->allocator;
        h->has_alloc = true;
    }
    Mem mem{h->has_alloc ? &h->alloc : nullptr, st};
    const uint32_t leaf = p->leaf_size, rot = p->rotation_fitting ? 1 : 0;
    const uint64_t nb = (n + p->bucket_size - 1) / p->bucket_size;
    const uint64_t maxv = p->max_value ? p->max_value : MPHF_DEFAULT_MAX_VALUE;
    h->info.n = n;
    h->info.nb = nb;
    h->info.leaf_size = leaf;
    h->info.bucket_size = p->bucket_size;
    h->info.key_bytes = p->key_bytes;
    h->info.rotation_fitting = rot;
    int rc = device_tables(h->device, leaf, rot, &h->tabs);
    if (rc) {
        release(h);
        return rc;
    }

    // temporaries
    uint64_t *node_cnt = nullptr, *scan_tmp = nullptr, *lo_s = nullptr, *counters = nullptr;
    uint8_t *bb_s = nullptr;
    uint32_t *cursor = nullptr, *small = nullptr;
    uint16_t *node_m = nullptr;
    InstDesc *d_inst = nullptr;
    WorkItem *items = nullptr;
    uint64_t *host_small = nullptr;
    uint64_t *size_hist = nullptr;
    uint32_t *size_cursor = nullptr;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    for (auto &e : ev) cudaEventCreate(&e);
    cudaEventRecord(ev[0], st);

    const uint64_t scan_words = scan_tmp_words(nb + 2 > 4096 ? nb + 2 : 4096) + 64;
#define CK(x)                   \
    do {                        \
        if (!(x)) {             \
            rc = MPHF_ENOMEM;   \
            goto done;          \
        }                       \
    } while (0)
#define CU(x)                                   \
    do {                                        \
        if ((x) != cudaSuccess) {               \
            cudaGetLastError();                 \
            rc = MPHF_ECUDA;                    \
            goto done;                          \
        }                                       \
    } while (0)
    {
        CK(h->cum_keys = (uint64_t *)mem.get((nb + 1) * 8));
        CK(h->node_off = (uint64_t *)mem.get((nb + 1) * 8));
        CK(h->bit_pos = (uint64_t *)mem.get((nb + 1) * 8));
        CK(node_cnt = h->node_off);
        CK(scan_tmp = (uint64_t *)mem.get(scan_words * 8));
        CK(cursor = (uint32_t *)mem.get((nb + 1) * 4));
        CK(small = (uint32_t *)mem.get(64));
        CK(lo_s = (uint64_t *)mem.get(n * 8));
        CK(bb_s = (uint8_t *)mem.get(n));
        CK(counters = (uint64_t *)mem.get(8 * 8));
        CK(size_hist = (uint64_t *)mem.get(4098 * 8));
        CK(size_cursor = (uint32_t *)mem.get(4097 * 4));
        CU(cudaMemsetAsync(size_hist, 0, 4098 * 8, st));
        CU(cudaMemsetAsync(size_cursor, 0, 4097 * 4, st));
        CU(cudaMallocHost(&host_small, 64));
        CU(cudaMemsetAsync(h->cum_keys, 0, (nb + 1) * 8, st));
        CU(cudaMemsetAsync(h->node_off, 0, (nb + 1) * 8, st));
        CU(cudaMemsetAsync(cursor, 0, (nb + 1) * 4, st));
        CU(cudaMemsetAsync(small, 0, 64, st));
        CU(cudaMemsetAsync(counters, 0, 64, st));

        // fingerprints, bucket sizes, plan, offsets
        launch_fp_hist(d_keys, n, p->key_bytes, nb, h->cum_keys, st);
        launch_plan(h->cum_keys, nb, h->tabs.nodes, node_cnt, small, small + 1, size_hist, st);
        launch_exclusive_scan(h->cum_keys, nb + 1, scan_tmp, st);
        launch_exclusive_scan(node_cnt, nb + 1, scan_tmp, st);
        launch_exclusive_scan(size_hist, 4098, scan_tmp, st);
        CU(cudaGetLastError());
        CU(cudaMemcpyAsync(host_small, node_cnt + nb, 8, cudaMemcpyDeviceToHost, st));
        CU(cudaMemcpyAsync(host_small + 1, small, 8, cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        cudaEventRecord(ev[1], st);
        const uint64_t n_nodes = host_small[0];
        const uint32_t status0 = (uint32_t)host_small[1], max_m = (uint32_t)(host_small[1] >> 32);
        h->info.n_nodes = n_nodes;
        h->info.max_bucket = max_m;
        if (status0) {
            rc = status_code(status0);
            goto done;
        }

        // group keys by bucket, search every bucket
        CK(h->values = (uint64_t *)mem.get(n_nodes * 8));
        CK(node_m = (uint16_t *)mem.get(n_nodes * 2));
        launch_scatter(d_keys, n, p->key_bytes, nb, h->cum_keys, cursor, lo_s, bb_s, st);
        if (nb > 0) {
            CK(items = (WorkItem *)mem.get(nb * sizeof(WorkItem)));
            CK(d_inst = (InstDesc *)mem.get(sizeof(InstDesc)));
            InstDesc hd;
            hd.lo = lo_s;
            hd.bb = bb_s;
            hd.bucket_off = h->cum_keys;
            hd.node_off = h->node_off;
            hd.nodes_tab = h->tabs.nodes;
            hd.values = h->values;
            hd.node_m = node_m;
            hd.status = small;
            hd.max_value = maxv;
            hd.leaf = leaf;
            hd.rotation = rot;
            hd.nb = (uint32_t)nb;
            hd.k30 = 1u << 2;
            hd.k27 = 1u << 5;
            hd.k31 = 1u << 1;
            {
                Shape shp = make_shape(leaf);
                hd.red[0] = (uint32_t)((1ull << 32) % leaf);
                hd.red[1] = (uint32_t)((1ull << 32) % shp.lower1);
                hd.red[2] = (uint32_t)((1ull << 32) % shp.lower2);
            }
            CU(cudaMemcpyAsync(d_inst, &hd, sizeof(hd), cudaMemcpyHostToDevice, st));
#if MPHF_LPT
            launch_items_by_size(h->cum_keys, nb, size_hist, size_cursor, items, 0, st);
#else
            k_items<<<(uint32_t)((nb + 255) / 256 < 4096 ? (nb + 255) / 256 : 4096), 256, 0, st>>>(
                items, (uint32_t)nb, 0);
            note_launches(1);
#endif
            SearchLaunch L = plan_search_launch(max_m, (uint32_t)nb, p->threads_per_block,
                                                p->blocks_per_sm);
            cudaEventRecord(ev[2], st);
            launch_search(d_inst, items, (uint32_t)nb, small + 2, L, st);
            CU(cudaGetLastError());
        } else {
            cudaEventRecord(ev[2], st);
        }
        cudaEventRecord(ev[3], st);

        // Golomb-Rice lengths and offsets
        CU(cudaMemsetAsync(h->bit_pos, 0, (nb + 1) * 8, st));
        launch_gr_lengths(h->values, node_m, h->node_off, nb, h->tabs.tau, h->bit_pos, st);
        launch_exclusive_scan(h->bit_pos, nb + 1, scan_tmp, st);
        CU(cudaGetLastError());
        CU(cudaMemcpyAsync(host_small, h->bit_pos + nb, 8, cudaMemcpyDeviceToHost, st));
        CU(cudaMemcpyAsync(host_small + 1, small, 8, cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        const uint64_t gr_bits = host_small[0];
        const uint32_t status1 = (uint32_t)host_small[1];
        if (status1) {
            rc = status_code(status1);
            goto done;
        }
        h->info.gr_bits = gr_bits;
        h->info.gr_words = (gr_bits + 63) / 64;
        CK(h->gr = (uint64_t *)mem.get(h->info.gr_words * 8 + 8));
        CU(cudaMemsetAsync(h->gr, 0, h->info.gr_words * 8 + 8, st));
        launch_gr_write(h->values, node_m, h->node_off, h->bit_pos, nb, h->tabs.tau,
                        h->tabs.fixed, h->cum_keys, h->gr, st);

        // Elias-Fano over bucket prefix sums and bucket bit positions
        EfDims e0 = ef_dims(nb + 1, n), e1 = ef_dims(nb + 1, gr_bits);
        h->info.ef_low_bits[0] = e0.L;
        h->info.ef_low_bits[1] = e1.L;
        h->info.ef_seq_words[0] = e0.low_words;
        h->info.ef_seq_words[1] = e0.high_words;
        h->info.ef_seq_words[2] = e1.low_words;
        h->info.ef_seq_words[3] = e1.high_words;
        h->info.ef_words = e0.low_words + e0.high_words + e1.low_words + e1.high_words;
        CK(h->ef = (uint64_t *)mem.get(h->info.ef_words * 8 + 8));
        CU(cudaMemsetAsync(h->ef, 0, h->info.ef_words * 8 + 8, st));
        uint64_t *lo0 = h->ef, *hi0 = lo0 + e0.low_words, *lo1 = hi0 + e0.high_words,
                 *hi1 = lo1 + e1.low_words;
        launch_ef_write(h->cum_keys, nb + 1, e0.L, lo0, hi0, st);
        launch_ef_write(h->bit_pos, nb + 1, e1.L, lo1, hi1, st);
        h->ef_dir_len[0] = e0.high_words + 1;
        h->ef_dir_len[1] = e1.high_words + 1;
        CK(h->ef_dir = (uint64_t *)mem.get((h->ef_dir_len[0] + h->ef_dir_len[1]) * 8));
        launch_rank_dir(hi0, e0.high_words, h->ef_dir, scan_tmp, st);
        launch_rank_dir(hi1, e1.high_words, h->ef_dir + h->ef_dir_len[0], scan_tmp, st);
        launch_stats(h->values, node_m, n_nodes, leaf, rot, counters, st);
        CU(cudaGetLastError());
        cudaEventRecord(ev[4], st);
        uint64_t hc[8];
        CU(cudaMemcpyAsync(host_small, counters, 64, cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        memcpy(hc, host_small, 64);
        for (int k = 0; k < 4; k++) {
            h->stats.trials[k] = hc[k];
            h->stats.evals[k] = hc[4 + k];
        }
        cudaEventElapsedTime(&h->stats.ms_plan, ev[0], ev[1]);
        cudaEventElapsedTime(&h->stats.ms_search, ev[2], ev[3]);
        cudaEventElapsedTime(&h->stats.ms_pack, ev[3], ev[4]);
        cudaEventElapsedTime(&h->stats.ms_total, ev[0], ev[4]);
        rc = MPHF_OK;
    }
done:
#undef CK
#undef CU
    mem.put(scan_tmp);
    mem.put(cursor);
    mem.put(small);
    mem.put(lo_s);
    mem.put(bb_s);
    mem.put(counters);
    mem.put(node_m);
    mem.put(items);
    mem.put(d_inst);
    mem.put(size_hist);
    mem.put(size_cursor);
    if (host_small) {
        cudaStreamSynchronize(st);
        cudaFreeHost(host_small);
    }
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
    if (rc != MPHF_OK) {
        cudaStreamSynchronize(st);
        release(h);
        return rc;
    }
    *out = h;
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
    if (!p || !out || (n > 0 && !h_keys) || (p->key_bytes != 8 && p->key_bytes != 16))
        return MPHF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    Mem mem{p->allocator, st};
    void *d = mem.get(n * p->key_bytes);
    if (!d) return MPHF_ENOMEM;
    if (n && cudaMemcpyAsync(d, h_keys, n * p->key_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        mem.put(d);
        return MPHF_ECUDA;
    }
    int rc = mphf_build_ex(d, n, p, stream, out);
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
    q.ef_high_words[0] = I.ef_seq_words[1];
    q.ef_high_words[1] = I.ef_seq_words[3];
    q.ef_L[0] = I.ef_low_bits[0];
    q.ef_L[1] = I.ef_low_bits[1];
    q.tau = h->tabs.tau;
    q.nodes_tab = h->tabs.nodes;
    q.fixed_tab = h->tabs.fixed;
    q.nb = I.nb;
    q.leaf = I.leaf_size;
    q.rotation = I.rotation_fitting;
    q.key_bytes = I.key_bytes;
    q.pad = 0;
    return q;
}

int mphf_query(const mphf_t *h, const void *d_keys, uint64_t n, uint64_t *d_out, void *stream) {
    if (!h || (n > 0 && (!d_keys || !d_out))) return MPHF_EINVAL;
    if (n == 0) return MPHF_OK;
    if (h->info.n == 0) return MPHF_EINVAL;
    launch_query(view_of(h), d_keys, n, d_out, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? MPHF_OK : MPHF_ECUDA;
}

int mphf_verify(const mphf_t *h, const void *d_keys, uint64_t n, uint64_t *n_bad, void *stream) {
    if (!h || !n_bad || (n > 0 && !d_keys)) return MPHF_EINVAL;
    *n_bad = 0;
    if (n == 0) return MPHF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    Mem mem{h->has_alloc ? &h->alloc : nullptr, st};
    uint64_t *vals = (uint64_t *)mem.get(n * 8);
    uint64_t words = (n + 31) / 32;
    uint32_t *bitmap = (uint32_t *)mem.get(words * 4 + 8);
    unsigned long long *bad = (unsigned long long *)mem.get(8);
    int rc = MPHF_OK;
    if (!vals || !bitmap || !bad) {
        rc = MPHF_ENOMEM;
    } else {
        cudaMemsetAsync(bitmap, 0, words * 4 + 8, st);
        cudaMemsetAsync(bad, 0, 8, st);
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
    if (!h || !len) return MPHF_EINVAL;
    const size_t head = sizeof(uint64_t) * 16;
    const size_t need = head + (h->info.gr_words + h->info.ef_words) * 8;
    if (!h_buf) {
        *len = need;
        return MPHF_OK;
    }
    if (*len < need) {
        *len = need;
        return MPHF_EINVAL;
    }
    uint64_t hd[16] = {0x3130485046504D52ull /* "RMPHF01" */, h->info.n, h->info.nb,
                       h->info.leaf_size, h->info.bucket_size, h->info.key_bytes,
                       h->info.rotation_fitting, h->info.gr_bits, h->info.gr_words,
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
    cudaDeviceSynchronize();
    release(h);
    return MPHF_OK;
}

uint64_t mphf_kernel_launches(void) { return launches_total(); }

int mphf_build_batch(const mphf_build_desc *descs, uint32_t count, void *stream, mphf_t **outs,
                     int *statuses) {
    if ((count && (!descs || !outs)) ) return MPHF_EINVAL;
    int first = MPHF_OK;
    for (uint32_t i = 0; i < count; i++) {
        mphf_build_params p;
        mphf_default_params(&p);
        p.leaf_size = descs[i].leaf_size;
        p.bucket_size = descs[i].bucket_size;
        p.key_bytes = descs[i].key_bytes;
        p.rotation_fitting = descs[i].rotation_fitting;
        p.max_value = descs[i].max_value ? descs[i].max_value : MPHF_DEFAULT_MAX_VALUE;
        int rc = mphf_build_ex(descs[i].d_keys, descs[i].n, &p, stream, &outs[i]);
        if (statuses) statuses[i] = rc;
        if (rc && first == MPHF_OK) first = rc;
    }
    return first;
}

}  // extern "C"
