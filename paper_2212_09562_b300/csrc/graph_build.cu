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
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <new>

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

}  // namespace rs

using namespace rs;

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
    const Shape shp = make_shape(p->leaf_size);
    d.red[0] = (uint32_t)((1ull << 32) % p->leaf_size);
    d.red[1] = (uint32_t)((1ull << 32) % shp.lower1);
    d.red[2] = (uint32_t)((1ull << 32) % shp.lower2);
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
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return MPHF_ECUDA;
    }
    if (dev != h->device) return MPHF_EINVAL;
    BuildPlan &b = *h->plan;
    const cudaStream_t st = (cudaStream_t)stream;
    const uint64_t n = b.n, nb = b.nb, k = nb + 1;
    const uint32_t kb = b.p.key_bytes, leaf = b.p.leaf_size, bij = b.p.leaf_bijection;
    const BucketRange R{nb, 0};
    h->ready = false;
    const EfDims e0 = ef_dims(k, n);
    struct Zero {
        void *p;
        size_t bytes;
    } zeros[] = {{h->cum_keys, k * 8},
                 {h->node_off, k * 8},
                 {h->bit_pos, k * 8},
                 {b.cursor, k * 4},
                 {b.small, 64},
                 {b.counters, 64},
                 {b.size_hist, 4098 * 8},
                 {b.size_cursor, 4097 * 4},
                 {b.head, 64},
                 {b.steal, kStealBytes},
                 {h->gr, (b.cap_bits / 64 + 2) * 8},
                 {h->ef, (e0.low_words + e0.high_words + b.max_low1 + b.max_high1 + 1) * 8},
                 {h->ef_dir, (h->ef_dir_len[0] + h->ef_dir_len[1] + 2 * h->ef_sel_len) * 8}};
    for (const Zero &z : zeros)
        if (cudaMemsetAsync(z.p, 0, z.bytes, st) != cudaSuccess) {
            cudaGetLastError();
            return MPHF_ECUDA;
        }
    // a1-a3: fingerprints, bucket sizes, plan, offsets
    if (b.sort_g)
        launch_fp_hist_blk(d_keys, n, kb, nb, R, b.sort_g, h->cum_keys, b.blk, b.small, st);
    else
        launch_fp_hist(d_keys, n, kb, nb, R, h->cum_keys, b.small, st);
    launch_plan(h->cum_keys, nb, h->tabs.nodes, h->node_off, b.small, b.small + 1, b.size_hist, st);
    launch_exclusive_scan(h->cum_keys, k, b.scan_tmp, st);
    launch_exclusive_scan(h->node_off, k, b.scan_tmp, st);
    // keys by bucket, the work order, a4-a7: the searches
    if (b.sort_g)
        launch_scatter_blk(d_keys, n, kb, nb, R, b.sort_g, h->cum_keys, b.blk, b.lo_s, b.bb_s, b.small, st);
    else
        launch_scatter(d_keys, n, kb, nb, R, h->cum_keys, b.cursor, b.lo_s, b.bb_s, b.small, st);
    launch_exclusive_scan(b.size_hist, 4098, b.scan_tmp, st);
    launch_items_by_size(h->cum_keys, nb, b.size_hist, b.size_cursor, b.items, 0, st);
    launch_search(b.d_inst, 1, b.items, (uint32_t)nb, b.head, b.L, b.steal, st);
    // a8: Golomb-Rice lengths and bits, Elias-Fano from the device totals
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
    return cudaGetLastError() == cudaSuccess ? MPHF_OK : MPHF_ECUDA;
}

int mphf_build_finish(mphf_t *h, void *stream) {
    if (!h || !h->plan) return MPHF_EINVAL;
    BuildPlan &b = *h->plan;
    const cudaStream_t st = (cudaStream_t)stream;
    const uint64_t nb = b.nb;
    if (cudaMemcpyAsync(b.host, b.small, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(b.host + 1, h->node_off + nb, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(b.host + 2, h->bit_pos + nb, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(b.host + 8, b.counters, 64, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return MPHF_ECUDA;
    }
    const uint32_t status = (uint32_t)b.host[0];
    if (status) return status_code(status);
    mphf_info &I = h->info;
    I.max_bucket = (uint32_t)(b.host[0] >> 32);
    I.n_nodes = b.host[1];
    I.gr_bits = b.host[2];
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
        h->stats.trials[k] = b.host[8 + k];
        h->stats.evals[k] = b.host[12 + k];
    }
    h->ready = true;
    return MPHF_OK;
}

}  // extern "C"
