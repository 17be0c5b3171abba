// graph_build.cu -- a build split into prepare / enqueue / finish, so that
// its device work can be captured once in a CUDA graph and replayed.
//
// A plain build reads two totals back to the host (the node count and the
// code length) to size its outputs, which a graph cannot do.  A prepared
// build sizes everything by upper bounds instead: at most n - 1 stored nodes
// per n keys, and a reserved code length (16 bits per key, 128 per bucket
// and 4096 more by default, about ten times what any leaf method needs); the
// Elias-Fano sizes and offsets that follow from the code length are computed
// on the device.  enqueue() then issues only memsets and kernels, on one
// stream, with no allocation and no host synchronisation; a code longer than
// reserved raises a device status bit and is not written.  finish() reads the
// totals and the status and fills the handle's sizes, after which it is an
// ordinary function (queries, serialisation, arrays) until the next enqueue.
// The stored words are those of mphf_build_ex on the same keys.
//
// A batch (mphf_batch_*) runs many prepared builds through ONE persistent
// search launch, as mphf_build_batch does: every member's plan counts its
// buckets into the batch's size histogram, one work order covers all of them
// largest first, and after the members' packing one kernel gathers every
// member's status and totals into one array, so that finishing the batch is
// one copy to the host.  The batch holds the launch's shared scratch; each
// member keeps its own search scratch too (about 0.7 MB, mostly its steal
// queue), unused while it builds inside a batch.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "handle.h"

namespace rs {

struct BuildPlan {
    mphf_build_params p{};
    uint64_t n = 0, nb = 0, cap_bits = 0, max_low1 = 0, max_high1 = 0;
    uint32_t sort_g = 0;
    SearchLaunch L{};
    // scratch kept across replays
    uint64_t *lo_s = nullptr, *counters = nullptr, *scan_tmp = nullptr, *size_hist = nullptr;
    uint8_t *bb_s = nullptr;
    uint32_t *cursor = nullptr, *small = nullptr, *blk = nullptr, *size_cursor = nullptr, *head = nullptr;
    uint16_t *node_m = nullptr;
    WorkItem *items = nullptr;
    InstDesc *d_inst = nullptr;
    EfPlan *efp = nullptr;
    StealQueue *steal = nullptr;
    uint64_t *host = nullptr;  // pinned: status word, node total, bit total, 8 counters
};

void release_plan(mphf_t *h, Mem &mem) {
    BuildPlan *b = h ? h->plan : nullptr;
    if (!b) return;
    void *ptrs[] = {b->lo_s, b->counters, b->scan_tmp, b->size_hist, b->bb_s, b->cursor, b->small,
                    b->blk, b->size_cursor, b->head, b->node_m, b->items, b->d_inst, b->efp,
                    b->steal};
    for (void *p : ptrs) mem.put(p);
    if (b->host) cudaFreeHost(b->host);
    delete b;
    h->plan = nullptr;
}

namespace {

bool on_device(int want) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return dev == want;
}

// The scratch that one search launch shares over all of its builds: the
// bucket-size histogram and cursors of the work order, the queue head, the
// steal queue.
int zero_shared(uint64_t *size_hist, uint32_t *size_cursor, uint32_t *head, StealQueue *steal,
                cudaStream_t st) {
    if (cudaMemsetAsync(size_hist, 0, 4098 * 8, st) != cudaSuccess ||
        cudaMemsetAsync(size_cursor, 0, 4097 * 4, st) != cudaSuccess ||
        cudaMemsetAsync(head, 0, 64, st) != cudaSuccess ||
        cudaMemsetAsync(steal, 0, kStealBytes, st) != cudaSuccess) {
        cudaGetLastError();
        return MPHF_ECUDA;
    }
    return MPHF_OK;
}

// A build's own outputs and scratch, cleared before it is enqueued again.
int zero_build(mphf_t *h, cudaStream_t st) {
    BuildPlan &b = *h->plan;
    const uint64_t n = b.n, k = b.nb + 1;
    const EfDims e0 = ef_dims(k, n);
    h->ready = false;
    struct Zero {
        void *p;
        size_t bytes;
    } zeros[] = {{h->cum_keys, k * 8},
                 {h->node_off, k * 8},
                 {h->bit_pos, k * 8},
                 {b.cursor, k * 4},
                 {b.small, 64},
                 {b.counters, 64},
                 {h->gr, (b.cap_bits / 64 + 2) * 8},
                 {h->ef, (e0.low_words + e0.high_words + b.max_low1 + b.max_high1 + 1) * 8},
                 {h->ef_dir, (h->ef_dir_len[0] + h->ef_dir_len[1] + 2 * h->ef_sel_len) * 8}};
    for (const Zero &z : zeros)
        if (cudaMemsetAsync(z.p, 0, z.bytes, st) != cudaSuccess) {
            cudaGetLastError();
            return MPHF_ECUDA;
        }
    return MPHF_OK;
}

// a1-a3 of one build: fingerprints, bucket sizes (counted into size_hist,
// which may be shared with other builds of the same search launch), plan,
// offsets, and its keys grouped by bucket.
void enqueue_front(mphf_t *h, const void *d_keys, uint64_t *size_hist, cudaStream_t st) {
    BuildPlan &b = *h->plan;
    const uint64_t n = b.n, nb = b.nb, k = nb + 1;
    const uint32_t kb = b.p.key_bytes;
    const BucketRange R{nb, 0};
    if (b.sort_g)
        launch_fp_hist_blk(d_keys, n, kb, nb, R, b.sort_g, h->cum_keys, b.blk, b.small, st);
    else
        launch_fp_hist(d_keys, n, kb, nb, R, h->cum_keys, b.small, st);
    launch_plan(h->cum_keys, nb, h->tabs.nodes, h->node_off, b.small, b.small + 1, size_hist, st);
    launch_exclusive_scan(h->cum_keys, k, b.scan_tmp, st);
    launch_exclusive_scan(h->node_off, k, b.scan_tmp, st);
    if (b.sort_g)
        launch_scatter_blk(d_keys, n, kb, nb, R, b.sort_g, h->cum_keys, b.blk, b.lo_s, b.bb_s, b.small, st);
    else
        launch_scatter(d_keys, n, kb, nb, R, h->cum_keys, b.cursor, b.lo_s, b.bb_s, b.small, st);
}

// a8 of one searched build: Golomb-Rice lengths and bits, Elias-Fano from the
// device totals, query directories, search counters.
void enqueue_back(mphf_t *h, cudaStream_t st) {
    BuildPlan &b = *h->plan;
    const uint64_t n = b.n, nb = b.nb, k = nb + 1;
    const uint32_t leaf = b.p.leaf_size, bij = b.p.leaf_bijection;
    const EfDims e0 = ef_dims(k, n);
    launch_gr_lengths(h->values, b.node_m, h->node_off, nb, h->tabs.tau, leaf, bij, h->bit_pos, st);
    launch_exclusive_scan(h->bit_pos, k, b.scan_tmp, st);
    launch_gr_write(h->values, b.node_m, h->node_off, h->bit_pos, nb, h->tabs.tau, h->tabs.fixed,
                    h->cum_keys, leaf, bij, h->gr, st, b.cap_bits, b.small);
    uint64_t *rank0 = h->ef_dir, *rank1 = rank0 + h->ef_dir_len[0];
    uint64_t *sel0 = rank1 + h->ef_dir_len[1], *sel1 = sel0 + h->ef_sel_len;
    launch_ef_planned(h->cum_keys, h->bit_pos, nb, b.cap_bits, b.efp, h->ef, b.max_high1, rank1,
                      b.scan_tmp, st);
    launch_rank_dir(h->ef + e0.low_words, e0.high_words, rank0, b.scan_tmp, st);
    launch_select_dir(e0.high_words, rank0, sel0, st);
    launch_select_dir(b.max_high1, rank1, sel1, st);
    launch_stats(h->values, b.node_m, n, leaf, bij, b.p.tree_shape, b.counters, st, h->node_off + nb);
}

// Makes h a usable function from its totals read back to the host: w[0] the
// status word, w[1] stored nodes, w[2] code bits, w[8..15] search counters.
int finish_from(mphf_t *h, const uint64_t *w) {
    BuildPlan &b = *h->plan;
    const uint64_t nb = b.nb;
    const uint32_t status = (uint32_t)w[0];
    if (status) return status_code(status);
    mphf_info &I = h->info;
    I.max_bucket = (uint32_t)(w[0] >> 32);
    I.n_nodes = w[1];
    I.gr_bits = w[2];
    I.gr_words = (I.gr_bits + 63) / 64;
    const EfDims e0 = ef_dims(nb + 1, b.n), e1 = ef_dims(nb + 1, I.gr_bits);
    I.ef_low_bits[0] = e0.L;
    I.ef_low_bits[1] = e1.L;
    I.ef_seq_words[0] = e0.low_words;
    I.ef_seq_words[1] = e0.high_words;
    I.ef_seq_words[2] = e1.low_words;
    I.ef_seq_words[3] = e1.high_words;
    I.ef_words = e0.low_words + e0.high_words + e1.low_words + e1.high_words;
    for (int k = 0; k < 4; k++) {
        h->stats.trials[k] = w[8 + k];
        h->stats.evals[k] = w[12 + k];
    }
    h->ready = true;
    return MPHF_OK;
}

}  // namespace

}  // namespace rs

using namespace rs;

// A batch of prepared builds searched by one persistent launch: the work
// order over all of their buckets, the launch's shared scratch, and one array
// of every build's totals.
struct mphf_batch {
    int device = 0;
    std::vector<mphf_t *> hs;
    uint64_t slots = 0;  // buckets of all builds
    mphf_allocator alloc{};
    bool has_alloc = false;
    SearchLaunch L{};
    uint64_t *size_hist = nullptr, *scan_tmp = nullptr, *totals = nullptr;
    uint32_t *size_cursor = nullptr, *head = nullptr;
    WorkItem *items = nullptr;
    InstDesc *d_inst = nullptr;
    StealQueue *steal = nullptr;
    BuildTotalsSrc *src = nullptr;
    uint64_t *host = nullptr;  // pinned: 16 words per build
};

namespace {

void release_batch(mphf_batch *b) {
    if (!b) return;
    Mem mem{b->has_alloc ? &b->alloc : nullptr, 0};
    void *ptrs[] = {b->size_hist, b->scan_tmp, b->totals, b->size_cursor, b->head,
                    b->items, b->d_inst, b->steal, b->src};
    cudaDeviceSynchronize();
    for (void *p : ptrs) mem.put(p);
    cudaStreamSynchronize(0);
    if (b->host) cudaFreeHost(b->host);
    cudaGetLastError();
    delete b;
}

}  // namespace


extern "C" {

int mphf_build_prepare(uint64_t n, const mphf_build_params *p, uint64_t gr_capacity_bits,
                       mphf_t **out) {
    if (!out || !p) return MPHF_EINVAL;
    *out = nullptr;
    // the shape checks of a plain build (mphf_build_ex), without keys yet
    if (p->leaf_size < 2 || p->leaf_size > MPHF_MAX_LEAF || p->bucket_size < 1 ||
        p->bucket_size > MPHF_MAX_BUCKET_SIZE || (p->key_bytes != 8 && p->key_bytes != 16) ||
        n == 0 || n >= (1ull << 32) || p->leaf_method > MPHF_LEAF_TABLE ||
        p->leaf_bijection > MPHF_BIJECTION_SHOCKHASH || p->tree_shape > MPHF_TREE_FANOUT2 ||
        (p->threads_per_block &&
         (p->threads_per_block % 32 || p->threads_per_block > 512 || p->threads_per_block < 64)) ||
        (p->seeds_per_thread != 0 && p->seeds_per_thread != 1 && p->seeds_per_thread != 2 &&
         p->seeds_per_thread != 4))
        return MPHF_EINVAL;
    mphf_t *h = new (std::nothrow) mphf;
    BuildPlan *b = new (std::nothrow) BuildPlan;
    if (!h || !b) {
        delete h;
        delete b;
        return MPHF_ENOMEM;
    }
    h->plan = b;
    h->ready = false;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        cudaGetLastError();
        release(h, 0);
        return MPHF_ECUDA;
    }
    if (p->allocator) {
        h->alloc = *p->allocator;
        h->has_alloc = true;
    }
    b->p = *p;
    b->n = n;
    b->nb = (n + p->bucket_size - 1) / p->bucket_size;
    const uint64_t nb = b->nb, k = nb + 1;
    b->cap_bits = gr_capacity_bits ? gr_capacity_bits : 16 * n + 128 * nb + 4096;
    const EfDims e0 = ef_dims(k, n), emax = ef_dims(k, b->cap_bits);
    b->max_low1 = emax.low_words;
    b->max_high1 = (3 * k + 63) / 64 + 1;  // (U >> L) < 2k for every U
    mphf_info &I = h->info;
    I.n = n;
    I.nb = nb;
    I.leaf_size = p->leaf_size;
    I.bucket_size = p->bucket_size;
    I.key_bytes = p->key_bytes;
    I.leaf_bijection = p->leaf_bijection;
    I.tree_shape = p->tree_shape;
    int rc = device_tables(h->device, p->leaf_size, p->leaf_bijection, p->tree_shape, &h->tabs);
    if (rc != MPHF_OK) {
        release(h, 0);
        return rc;
    }
    Mem mem{p->allocator, 0};
    b->sort_g = sort_blocks(n, nb);
    h->cum_keys = (uint64_t *)mem.get(k * 8);
    h->node_off = (uint64_t *)mem.get(k * 8);
    h->bit_pos = (uint64_t *)mem.get(k * 8);
    h->values = (uint64_t *)mem.get(n * 8);
    h->gr = (uint64_t *)mem.get((b->cap_bits / 64 + 2) * 8);
    h->ef = (uint64_t *)mem.get((e0.low_words + e0.high_words + b->max_low1 + b->max_high1 + 1) * 8);
    h->ef_dir_len[0] = e0.high_words + 1;
    h->ef_dir_len[1] = b->max_high1 + 1;
    h->ef_sel_len = (k + 63) / 64;
    h->ef_dir = (uint64_t *)mem.get((h->ef_dir_len[0] + h->ef_dir_len[1] + 2 * h->ef_sel_len) * 8);
    b->lo_s = (uint64_t *)mem.get(n * 8);
    b->bb_s = (uint8_t *)mem.get(n);
    b->node_m = (uint16_t *)mem.get(n * 2);
    b->cursor = (uint32_t *)mem.get(k * 4);
    b->small = (uint32_t *)mem.get(64);
    b->counters = (uint64_t *)mem.get(64);
    const uint64_t tmp_len = (k + 1 > 4098 ? k + 1 : 4098) > b->max_high1 + 1 ? (k + 1 > 4098 ? k + 1 : 4098)
                                                                              : b->max_high1 + 1;
    b->scan_tmp = (uint64_t *)mem.get((scan_tmp_words(tmp_len) + 64) * 8);
    b->size_hist = (uint64_t *)mem.get(4098 * 8);
    b->size_cursor = (uint32_t *)mem.get(4097 * 4);
    b->head = (uint32_t *)mem.get(64);
    b->items = (WorkItem *)mem.get(nb * sizeof(WorkItem));
    b->d_inst = (InstDesc *)mem.get(sizeof(InstDesc));
    b->efp = (EfPlan *)mem.get(sizeof(EfPlan));
    b->steal = (StealQueue *)mem.get(kStealBytes);
    if (b->sort_g) b->blk = (uint32_t *)mem.get((uint64_t)b->sort_g * nb * 4);
    bool ok = h->cum_keys && h->node_off && h->bit_pos && h->values && h->gr && h->ef && h->ef_dir &&
              b->lo_s && b->bb_s && b->node_m && b->cursor && b->small && b->counters && b->scan_tmp &&
              b->size_hist && b->size_cursor && b->head && b->items && b->d_inst && b->efp && b->steal &&
              (!b->sort_g || b->blk);
    if (!ok) {
        cudaStreamSynchronize(0);
        release(h, 0);
        return MPHF_ENOMEM;
    }
    if (cudaMallocHost(&b->host, 16 * 8) != cudaSuccess) {
        cudaGetLastError();
        b->host = nullptr;
        release(h, 0);
        return MPHF_ECUDA;
    }
    // the search descriptor never changes between replays: the arrays stay put
    InstDesc d;
    memset(&d, 0, sizeof(d));
    d.lo = b->lo_s;
    d.bb = b->bb_s;
    d.bucket_off = h->cum_keys;
    d.node_off = h->node_off;
    d.nodes_tab = h->tabs.nodes;
    d.values = h->values;
    d.node_m = b->node_m;
    d.status = b->small;
    d.max_value = p->max_value ? p->max_value : MPHF_DEFAULT_MAX_VALUE;
    d.leaf = p->leaf_size;
    d.bij = p->leaf_bijection;
    d.tree = p->tree_shape;
    d.nb = (uint32_t)nb;
    d.red_leaf = (uint32_t)((1ull << 32) % p->leaf_size);
    d.leaf_method = p->leaf_method;
    d.spt = p->seeds_per_thread ? p->seeds_per_thread : (p->leaf_size >= 16 ? 2u : 1u);
    d.mod_c = h->tabs.mod_c;
    d.mod_M = h->tabs.mod_M;
    if (p->leaf_method == MPHF_LEAF_TABLE &&
        device_rot_tables(h->device, &d.rot_canon, &d.rot_period) != MPHF_OK) {
        release(h, 0);
        return MPHF_ENOMEM;
    }
    const bool wide = p->tree_shape == MPHF_TREE_RECSPLIT && p->leaf_size >= 14;
    b->L = plan_search_launch(MPHF_MAX_BUCKET, (uint32_t)nb,
                              p->threads_per_block ? p->threads_per_block : (wide ? 512u : 256u),
                              p->blocks_per_sm);
    if (cudaMemcpy(b->d_inst, &d, sizeof(d), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        release(h, 0);
        return MPHF_ECUDA;
    }
    *out = h;
    return MPHF_OK;
}

int mphf_build_enqueue(mphf_t *h, const void *d_keys, void *stream) {
    if (!h || !h->plan || !d_keys || ((uintptr_t)d_keys & 7)) return MPHF_EINVAL;
    if (!on_device(h->device)) return MPHF_EINVAL;
    BuildPlan &b = *h->plan;
    const cudaStream_t st = (cudaStream_t)stream;
    if (zero_shared(b.size_hist, b.size_cursor, b.head, b.steal, st) != MPHF_OK ||
        zero_build(h, st) != MPHF_OK)
        return MPHF_ECUDA;
    enqueue_front(h, d_keys, b.size_hist, st);
    launch_exclusive_scan(b.size_hist, 4098, b.scan_tmp, st);
    launch_items_by_size(h->cum_keys, b.nb, b.size_hist, b.size_cursor, b.items, 0, st);
    launch_search(b.d_inst, 1, b.items, (uint32_t)b.nb, b.head, b.L, b.steal, st);
    enqueue_back(h, st);
    return cudaGetLastError() == cudaSuccess ? MPHF_OK : MPHF_ECUDA;
}

int mphf_build_finish(mphf_t *h, void *stream) {
    if (!h || !h->plan) return MPHF_EINVAL;
    BuildPlan &b = *h->plan;
    const cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(b.host, b.small, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(b.host + 1, h->node_off + b.nb, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(b.host + 2, h->bit_pos + b.nb, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(b.host + 8, b.counters, 64, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return MPHF_ECUDA;
    }
    return finish_from(h, b.host);
}

int mphf_batch_prepare(mphf_t *const *handles, uint32_t count, uint32_t threads_per_block,
                       uint32_t blocks_per_sm, const mphf_allocator *allocator, mphf_batch_t **out) {
    if (!out) return MPHF_EINVAL;
    *out = nullptr;
    if (!handles || count == 0 ||
        (threads_per_block &&
         (threads_per_block % 32 || threads_per_block > 512 || threads_per_block < 64)))
        return MPHF_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return MPHF_ECUDA;
    }
    std::vector<mphf_t *> hs(handles, handles + count), sorted(hs);
    uint64_t slots = 0;
    bool wide = false;
    for (mphf_t *h : hs) {
        if (!h || !h->plan || h->device != dev) return MPHF_EINVAL;
        slots += h->plan->nb;
        wide |= h->plan->p.tree_shape == MPHF_TREE_RECSPLIT && h->plan->p.leaf_size >= 14;
    }
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return MPHF_EINVAL;
    if (slots > 0xFFFFFFFFull) return MPHF_EINVAL;
    mphf_batch *b = new (std::nothrow) mphf_batch;
    if (!b) return MPHF_ENOMEM;
    b->device = dev;
    b->hs = hs;
    b->slots = slots;
    if (allocator) {
        b->alloc = *allocator;
        b->has_alloc = true;
    }
    Mem mem{b->has_alloc ? &b->alloc : nullptr, 0};
    b->size_hist = (uint64_t *)mem.get(4098 * 8);
    b->scan_tmp = (uint64_t *)mem.get((scan_tmp_words(4098) + 64) * 8);
    b->totals = (uint64_t *)mem.get(16ull * count * 8);
    b->size_cursor = (uint32_t *)mem.get(4097 * 4);
    b->head = (uint32_t *)mem.get(64);
    b->items = (WorkItem *)mem.get(slots * sizeof(WorkItem));
    b->d_inst = (InstDesc *)mem.get(count * sizeof(InstDesc));
    b->steal = (StealQueue *)mem.get(kStealBytes);
    b->src = (BuildTotalsSrc *)mem.get(count * sizeof(BuildTotalsSrc));
    if (!b->size_hist || !b->scan_tmp || !b->totals || !b->size_cursor || !b->head || !b->items ||
        !b->d_inst || !b->steal || !b->src) {
        release_batch(b);
        return MPHF_ENOMEM;
    }
    if (cudaMallocHost(&b->host, 16ull * count * 8) != cudaSuccess) {
        cudaGetLastError();
        b->host = nullptr;
        release_batch(b);
        return MPHF_ECUDA;
    }
    // every build's search descriptor (fixed since its prepare) and the
    // places of its totals, in batch order
    std::vector<BuildTotalsSrc> src(count);
    bool ok = true;
    for (uint32_t i = 0; i < count && ok; i++) {
        mphf_t *h = hs[i];
        BuildPlan &p = *h->plan;
        src[i] = BuildTotalsSrc{p.small, h->node_off + p.nb, h->bit_pos + p.nb, p.counters};
        ok = cudaMemcpyAsync(b->d_inst + i, p.d_inst, sizeof(InstDesc), cudaMemcpyDeviceToDevice,
                             0) == cudaSuccess;
    }
    ok = ok && cudaMemcpyAsync(b->src, src.data(), count * sizeof(BuildTotalsSrc),
                               cudaMemcpyHostToDevice, 0) == cudaSuccess &&
         cudaDeviceSynchronize() == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        release_batch(b);
        return MPHF_ECUDA;
    }
    b->L = plan_search_launch(MPHF_MAX_BUCKET, (uint32_t)slots,
                              threads_per_block ? threads_per_block : (wide ? 512u : 256u),
                              blocks_per_sm);
    *out = b;
    return MPHF_OK;
}

int mphf_batch_enqueue(mphf_batch_t *b, const void *const *d_keys, void *stream) {
    if (!b || !d_keys) return MPHF_EINVAL;
    const uint32_t count = (uint32_t)b->hs.size();
    for (uint32_t i = 0; i < count; i++)
        if (!d_keys[i] || ((uintptr_t)d_keys[i] & 7)) return MPHF_EINVAL;
    if (!on_device(b->device)) return MPHF_EINVAL;
    for (mphf_t *h : b->hs)
        if (!h->plan) return MPHF_EINVAL;
    const cudaStream_t st = (cudaStream_t)stream;
    if (zero_shared(b->size_hist, b->size_cursor, b->head, b->steal, st) != MPHF_OK)
        return MPHF_ECUDA;
    for (uint32_t i = 0; i < count; i++) {
        if (zero_build(b->hs[i], st) != MPHF_OK) return MPHF_ECUDA;
        enqueue_front(b->hs[i], d_keys[i], b->size_hist, st);
    }
    // one work order over the buckets of all builds, largest first
    launch_exclusive_scan(b->size_hist, 4098, b->scan_tmp, st);
    for (uint32_t i = 0; i < count; i++)
        launch_items_by_size(b->hs[i]->cum_keys, b->hs[i]->plan->nb, b->size_hist, b->size_cursor,
                             b->items, i, st);
    launch_search(b->d_inst, count, b->items, (uint32_t)b->slots, b->head, b->L, b->steal, st);
    for (mphf_t *h : b->hs) enqueue_back(h, st);
    launch_gather_totals(b->src, count, b->totals, st);
    return cudaGetLastError() == cudaSuccess ? MPHF_OK : MPHF_ECUDA;
}

int mphf_batch_finish(mphf_batch_t *b, void *stream, int *statuses) {
    if (!b) return MPHF_EINVAL;
    const uint32_t count = (uint32_t)b->hs.size();
    const cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(b->host, b->totals, 16ull * count * 8, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return MPHF_ECUDA;
    }
    int first = MPHF_OK;
    for (uint32_t i = 0; i < count; i++) {
        const int rc = finish_from(b->hs[i], b->host + 16ull * i);
        if (statuses) statuses[i] = rc;
        if (rc && first == MPHF_OK) first = rc;
    }
    return first;
}

int mphf_batch_free(mphf_batch_t *b) {
    if (!b) return MPHF_EINVAL;
    int prev = -1;
    const bool have_prev = cudaGetDevice(&prev) == cudaSuccess;
    cudaGetLastError();
    if (cudaSetDevice(b->device) != cudaSuccess) {
        cudaGetLastError();
        return MPHF_ECUDA;
    }
    release_batch(b);
    if (have_prev) cudaSetDevice(prev);
    return MPHF_OK;
}

}  // extern "C"
