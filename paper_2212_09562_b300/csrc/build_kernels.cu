// build_kernels.cu -- device side of one or many RecSplit builds.
//
// Stages (Section 2.2 of Bez et al. 2212.09562, parallel form of Section 5.3):
//   k_fp_hist(_blk)   master hash of every key, bucket histogram (per-block
//                     histograms when nb <= 8192, global atomics above)
//   k_plan            stored-node count per bucket (from the bucket size alone)
//   k_scan_*          exclusive prefix sums (bucket offsets, node offsets, bits)
//   k_scatter(_blk)   keys grouped by bucket (lo word + rotation bit)
//   k_search          persistent kernel, one block per bucket at a time, largest
//                     first: split searches of the inner nodes (lower levels:
//                     all threads of the block try consecutive seeds; fanout-2
//                     nodes: one seed per warp), redistribution in shared
//                     memory, then leaf searches with one warp per leaf (plain,
//                     rotation fitting of Section 4, or ShockHash of Appendix C)
//   k_gr_*            Golomb-Rice lengths and bit writes (fixed parts, then unary
//                     parts, in preorder per bucket)
//   k_ef_write        Elias-Fano sequences; k_popcount + scan and k_select_dir
//                     build their rank and select directories
//   k_stats           trial / hash-evaluation counts from the stored values
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "common.cuh"
#include "engine.h"
#include "mphf.h"

namespace rs {

__device__ __forceinline__ void load_key(const void *keys, uint64_t i, uint32_t kb, uint64_t &w0,
                                         uint64_t &w1) {
    const uint64_t *p = (const uint64_t *)keys;
    if (kb == 8) {
        w0 = p[i];
        w1 = 0;
    } else {
        w0 = p[2 * i];
        w1 = p[2 * i + 1];
    }
}

// The same with the streaming hint (evict first): keys read for the last
// time, which should not push out of L2 the output lines still being filled.
__device__ __forceinline__ void load_key_last(const void *keys, uint64_t i, uint32_t kb, uint64_t &w0,
                                              uint64_t &w1) {
    const uint64_t *p = (const uint64_t *)keys;
    if (kb == 8) {
        w0 = __ldcs(p + i);
        w1 = 0;
    } else {
        w0 = __ldcs(p + 2 * i);
        w1 = __ldcs(p + 2 * i + 1);
    }
}

static unsigned long long g_launches = 0;
void note_launches(uint64_t k) { __atomic_fetch_add(&g_launches, (unsigned long long)k, __ATOMIC_RELAXED); }
uint64_t launches_total() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

static uint32_t grid_for(uint64_t n, uint32_t threads, uint32_t cap = 148u * 32u) {
    uint64_t g = (n + threads - 1) / threads;
    if (g > cap) g = cap;
    return g ? (uint32_t)g : 1u;
}

// ---------------------------------------------------------------------------
// Fingerprint + bucket histogram.
// A key's bucket is mulhi64(hi, R.nb_hash) - R.b_lo (R.b_lo = 0 and nb_hash =
// nb for a whole function; a shard holds the consecutive range [b_lo, b_lo +
// nb) of a function with nb_hash buckets, Section 5.2).  A key outside the
// range sets ST_RANGE and is not counted.
__device__ __forceinline__ bool local_bucket(const BucketRange &R, uint64_t hi, uint64_t nb,
                                             uint32_t *status, uint64_t &b) {
    b = mulhi64(hi, R.nb_hash) - R.b_lo;  // wraps to a huge value below b_lo
    if (b < nb) return true;
    atomicOr(status, ST_RANGE);
    return false;
}

__global__ void k_fp_hist(const void *keys, uint64_t n, uint32_t kb, uint64_t nb, BucketRange R,
                          unsigned long long *counts, uint32_t *status) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t w0, w1, hi, lo, b;
        load_key(keys, i, kb, w0, w1);
        fingerprint(w0, w1, hi, lo);
        if (local_bucket(R, hi, nb, status, b)) atomicAdd(&counts[b], 1ull);
    }
}

void launch_fp_hist(const void *keys, uint64_t n, uint32_t key_bytes, uint64_t nb,
                    const BucketRange &R, uint64_t *counts, uint32_t *status, cudaStream_t st) {
    if (n == 0) return;
    k_fp_hist<<<grid_for(n, 256), 256, 0, st>>>(keys, n, key_bytes, nb, R, (unsigned long long *)counts,
                                                status);
    note_launches(1);
}

// ---------------------------------------------------------------------------
// Two-level counting sort for builds with few buckets (nb <= kSmemBuckets):
// block g takes the contiguous chunk [g*C, (g+1)*C) of keys, counts its
// buckets in shared memory, and writes its counts as row g of blk[G][nb]
// (plus one global add per bucket for the totals).  A column pass turns row g
// into the block's first slot in every bucket, and the scatter re-reads the
// chunk and places keys through shared-memory cursors.  Global atomics drop
// from one per key to one per bucket and block.
constexpr uint32_t kSmemBuckets = 8192;
// Keys a thread loads before it hashes any: the chunk loops are bound by
// the latency of their key loads, so more loads in flight per thread raise
// the bandwidth (one coalesced load per key position, as before).
constexpr int kSortBatch = 4;

__global__ void k_fp_hist_blk(const void *keys, uint64_t n, uint32_t kb, uint32_t nb, BucketRange R,
                              uint64_t chunk, unsigned long long *counts, uint32_t *blk,
                              uint32_t *status) {
    extern __shared__ uint32_t hist[];
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const uint64_t beg = blockIdx.x * chunk, end = beg + chunk < n ? beg + chunk : n;
    const uint64_t T = blockDim.x;
    for (uint64_t i0 = beg + threadIdx.x; i0 < end; i0 += kSortBatch * T) {
        uint64_t w0[kSortBatch], w1[kSortBatch];
#pragma unroll
        for (int u = 0; u < kSortBatch; u++) {
            w0[u] = w1[u] = 0;
            if (i0 + u * T < end) load_key(keys, i0 + u * T, kb, w0[u], w1[u]);
        }
#pragma unroll
        for (int u = 0; u < kSortBatch; u++) {
            if (i0 + u * T >= end) continue;
            uint64_t hi, lo, b;
            fingerprint(w0[u], w1[u], hi, lo);
            if (local_bucket(R, hi, nb, status, b)) atomicAdd(&hist[b], 1u);
        }
    }
    __syncthreads();
    uint32_t *row = blk + (uint64_t)blockIdx.x * nb;
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) {
        const uint32_t c = hist[b];
        row[b] = c;
        if (c) atomicAdd(&counts[b], (unsigned long long)c);
    }
}

// blk[g][b] <- bucket_off[b] + sum of blk[g'][b] over g' < g: one warp per
// bucket, 32 rows at a time with a shuffle scan (the column is L2-resident).
__global__ void k_block_offsets(uint32_t *blk, uint32_t G, uint32_t nb, const uint64_t *bucket_off) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t b = warp; b < nb; b += nwarps) {
        uint32_t run = (uint32_t)bucket_off[b];
        for (uint32_t g0 = 0; g0 < G; g0 += 32) {
            const uint32_t g = g0 + lane;
            const uint32_t v = g < G ? blk[(uint64_t)g * nb + b] : 0;
            uint32_t incl = v;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= (uint32_t)d) incl += o;
            }
            if (g < G) blk[(uint64_t)g * nb + b] = run + incl - v;
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

__global__ void k_scatter_blk(const void *keys, uint64_t n, uint32_t kb, uint32_t nb, BucketRange R,
                              uint64_t chunk, const uint32_t *blk, uint64_t *lo_out, uint8_t *bb_out,
                              uint32_t *status) {
    extern __shared__ uint32_t cursor[];
    const uint32_t *row = blk + (uint64_t)blockIdx.x * nb;
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) cursor[b] = row[b];
    __syncthreads();
    const uint64_t beg = blockIdx.x * chunk, end = beg + chunk < n ? beg + chunk : n;
    const uint64_t T = blockDim.x;
    for (uint64_t i0 = beg + threadIdx.x; i0 < end; i0 += kSortBatch * T) {
        uint64_t w0[kSortBatch], w1[kSortBatch];
#pragma unroll
        for (int u = 0; u < kSortBatch; u++) {
            w0[u] = w1[u] = 0;
            if (i0 + u * T < end) load_key_last(keys, i0 + u * T, kb, w0[u], w1[u]);
        }
#pragma unroll
        for (int u = 0; u < kSortBatch; u++) {
            if (i0 + u * T >= end) continue;
            uint64_t hi, lo, b;
            fingerprint(w0[u], w1[u], hi, lo);
            if (!local_bucket(R, hi, nb, status, b)) continue;
            const uint32_t p = atomicAdd(&cursor[b], 1u);
            lo_out[p] = lo;
            bb_out[p] = (uint8_t)(hi & 1);
        }
    }
}

uint32_t sort_blocks(uint64_t n, uint64_t nb) {
    if (nb == 0 || nb > kSmemBuckets || n < 4096) return 0;  // use the global-atomic path
    uint64_t g = (n + 8191) / 8192;                          // at least 8192 keys per block
    return (uint32_t)(g > 2 * 148 ? 2 * 148 : g);
}

void launch_fp_hist_blk(const void *keys, uint64_t n, uint32_t key_bytes, uint64_t nb,
                        const BucketRange &R, uint32_t G, uint64_t *counts, uint32_t *blk,
                        uint32_t *status, cudaStream_t st) {
    const uint64_t chunk = (n + G - 1) / G;
    k_fp_hist_blk<<<G, 512, (uint32_t)nb * 4, st>>>(keys, n, key_bytes, (uint32_t)nb, R, chunk,
                                                    (unsigned long long *)counts, blk, status);
    note_launches(1);
}

void launch_scatter_blk(const void *keys, uint64_t n, uint32_t key_bytes, uint64_t nb,
                        const BucketRange &R, uint32_t G, const uint64_t *bucket_off, uint32_t *blk,
                        uint64_t *lo, uint8_t *bb, uint32_t *status, cudaStream_t st) {
    const uint64_t chunk = (n + G - 1) / G;
    k_block_offsets<<<(uint32_t)((nb * 32 + 255) / 256), 256, 0, st>>>(blk, G, (uint32_t)nb, bucket_off);
    note_launches(1);
    k_scatter_blk<<<G, 512, (uint32_t)nb * 4, st>>>(keys, n, key_bytes, (uint32_t)nb, R, chunk, blk, lo,
                                                    bb, status);
    note_launches(1);
}

// ---------------------------------------------------------------------------
// Plan (Section 2.2: the tree shape follows from the bucket size alone):
// nodes per bucket, oversized buckets, largest bucket, and a histogram
// of bucket sizes in descending order (size_hist[4096 - m]) for the work order.
__global__ void k_plan(const uint64_t *counts, uint64_t nb, const uint32_t *nodes_tab,
                       uint64_t *node_cnt, uint32_t *status, uint32_t *max_m,
                       unsigned long long *size_hist) {
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < nb;
         b += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t m = counts[b];
        if (m > 4096) {
            atomicOr(status, ST_BUCKET);
            node_cnt[b] = 0;
        } else {
            node_cnt[b] = nodes_tab[m];
            if (size_hist) atomicAdd(&size_hist[4096 - m], 1ull);
        }
        atomicMax(max_m, (uint32_t)(m > 0xFFFFFFFFull ? 0xFFFFFFFFull : m));
    }
}

void launch_plan(const uint64_t *counts, uint64_t nb, const uint32_t *nodes_tab, uint64_t *node_cnt,
                 uint32_t *status, uint32_t *max_m, uint64_t *size_hist, cudaStream_t st) {
    if (nb == 0) return;
    k_plan<<<grid_for(nb, 256), 256, 0, st>>>(counts, nb, nodes_tab, node_cnt, status, max_m,
                                               (unsigned long long *)size_hist);
    note_launches(1);
}

// Work order: buckets by decreasing size (longest first), from the scanned
// descending size histogram; the order among equal sizes is arbitrary.
__global__ void k_items_by_size(const uint64_t *bucket_off, uint64_t nb, const uint64_t *size_off,
                                uint32_t *size_cursor, WorkItem *items, uint32_t inst) {
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < nb;
         b += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t m = bucket_off[b + 1] - bucket_off[b];
        uint32_t k = m > 4096 ? 0 : 4096 - (uint32_t)m;
        uint64_t pos = size_off[k] + atomicAdd(&size_cursor[k], 1u);
        items[pos] = WorkItem{inst, (uint32_t)b};
    }
}

void launch_items_by_size(const uint64_t *bucket_off, uint64_t nb, const uint64_t *size_off,
                          uint32_t *size_cursor, WorkItem *items, uint32_t inst, cudaStream_t st) {
    if (nb == 0) return;
    k_items_by_size<<<grid_for(nb, 256), 256, 0, st>>>(bucket_off, nb, size_off, size_cursor, items,
                                                        inst);
    note_launches(1);
}

// ---------------------------------------------------------------------------
// Exclusive scan, reduce-then-scan over tiles of 2048 values.
constexpr uint32_t SCAN_T = 256, SCAN_PER = 8, SCAN_TILE = SCAN_T * SCAN_PER;

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v) {
    uint32_t lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= (uint32_t)d) v += o;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; returns the prefix,
// *total receives the block sum.
__device__ uint64_t block_excl_scan(uint64_t v, uint64_t *total) {
    __shared__ uint64_t warp_sums[32];
    uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    uint64_t incl = warp_incl_scan(v);
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint64_t s = lane < nw ? warp_sums[lane] : 0;
        uint64_t si = warp_incl_scan(s);
        if (lane < nw) warp_sums[lane] = si - s;
        if (lane == nw - 1) warp_sums[31] = si;
    }
    __syncthreads();
    uint64_t r = warp_sums[warp] + incl - v;
    if (total) *total = warp_sums[31];
    __syncthreads();
    return r;
}

__global__ void k_scan_reduce(const uint64_t *d, uint64_t len, uint64_t *sums) {
    uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    uint64_t s = 0;
    for (uint32_t j = 0; j < SCAN_PER; j++) {
        uint64_t i = base + (uint64_t)j * SCAN_T + threadIdx.x;
        if (i < len) s += d[i];
    }
    uint64_t total;
    block_excl_scan(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_scan_apply(uint64_t *d, uint64_t len, const uint64_t *offs) {
    uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_PER;
    uint64_t v[SCAN_PER];
    uint64_t s = 0;
#pragma unroll
    for (uint32_t j = 0; j < SCAN_PER; j++) {
        v[j] = base + j < len ? d[base + j] : 0;
        s += v[j];
    }
    uint64_t pre = block_excl_scan(s, nullptr) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
    for (uint32_t j = 0; j < SCAN_PER; j++) {
        if (base + j < len) d[base + j] = pre;
        pre += v[j];
    }
}

uint64_t scan_tmp_words(uint64_t len) {
    uint64_t tiles = (len + SCAN_TILE - 1) / SCAN_TILE;
    return tiles <= 1 ? 1 : tiles + scan_tmp_words(tiles);
}

void launch_exclusive_scan(uint64_t *data, uint64_t len, uint64_t *tmp, cudaStream_t st) {
    if (len == 0) return;
    uint64_t tiles = (len + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 1) {
        k_scan_apply<<<1, SCAN_T, 0, st>>>(data, len, nullptr);
        note_launches(1);
        return;
    }
    k_scan_reduce<<<(uint32_t)tiles, SCAN_T, 0, st>>>(data, len, tmp);
    note_launches(1);
    launch_exclusive_scan(tmp, tiles, tmp + tiles, st);
    k_scan_apply<<<(uint32_t)tiles, SCAN_T, 0, st>>>(data, len, tmp);
    note_launches(1);
}

// ---------------------------------------------------------------------------
// Scatter: lo word and rotation bit of every key to its bucket's range.
__global__ void k_scatter(const void *keys, uint64_t n, uint32_t kb, uint64_t nb, BucketRange R,
                          const uint64_t *bucket_off, uint32_t *cursor, uint64_t *lo_out,
                          uint8_t *bb_out, uint32_t *status) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t w0, w1, hi, lo, b;
        load_key(keys, i, kb, w0, w1);
        fingerprint(w0, w1, hi, lo);
        if (!local_bucket(R, hi, nb, status, b)) continue;
        uint64_t p = bucket_off[b] + atomicAdd(&cursor[b], 1u);
        lo_out[p] = lo;
        bb_out[p] = (uint8_t)(hi & 1);
    }
}

void launch_scatter(const void *keys, uint64_t n, uint32_t key_bytes, uint64_t nb,
                    const BucketRange &R, const uint64_t *bucket_off, uint32_t *cursor, uint64_t *lo,
                    uint8_t *bb, uint32_t *status, cudaStream_t st) {
    if (n == 0) return;
    k_scatter<<<grid_for(n, 256), 256, 0, st>>>(keys, n, key_bytes, nb, R, bucket_off, cursor, lo, bb,
                                                status);
    note_launches(1);
}

// ---------------------------------------------------------------------------
// The search kernel.
constexpr int STACK = 64;

// The item a block works on, for sharing a node search's seed range with
// idle blocks in the tail of a launch (full lower nodes only); q = nullptr:
// no sharing (the serving search).
struct HelpCtx {
    StealQueue *q;
    const uint32_t *bucket_head;
    uint32_t nitems, inst, bucket;
    uint32_t gbase, gpos;  // key offset within the bucket: of the item, of the node searched
    uint64_t *glo;         // the build's grouped keys
    uint64_t kbeg;         // the bucket's first key
};
constexpr uint32_t kStealReady = 1u << 31;
constexpr uint32_t kHelpMarker = 0xFFFFFFFEu;  // a steal item inviting a block to a shared search

// Quotient-indexed counter increments of the full lower nodes of the
// compiled leaf sizes (see DivNone, QIdx): for leaf size l, fanouts f1, f2 and
// nodes L1 = f1 l, L2 = f2 L1, a table of L1 >> ctz(l) entries (lower-1
// nodes, unit l) and one of L2 >> ctz(L1) entries (lower-2 nodes, unit L1).
__host__ __device__ constexpr uint32_t ctz_ce(uint32_t x) { return (x & 1u) ? 0u : 1u + ctz_ce(x >> 1); }
__host__ __device__ constexpr uint32_t fan1_ce(uint32_t l) { return (35u * l + 154u) / 100u < 2 ? 2 : (35u * l + 154u) / 100u; }
__host__ __device__ constexpr uint32_t fan2_ce(uint32_t l) { return (21u * l + 189u) / 100u < 2 ? 2 : (21u * l + 189u) / 100u; }
__host__ __device__ constexpr uint32_t lutq_len(uint32_t l, int level) {
    return level == 1 ? (fan1_ce(l) * l) >> ctz_ce(l)
                      : (fan2_ce(l) * fan1_ce(l) * l) >> ctz_ce(fan1_ce(l) * l);
}
// The leaf sizes with compiled paths (the cases of the kernels' leaf switch),
// in table order: 8, 12, 16; lutq_off of any other size is the total.
__host__ __device__ constexpr uint32_t lutq_pair(uint32_t l) { return lutq_len(l, 1) + lutq_len(l, 2); }
__host__ __device__ constexpr uint32_t lutq_off(uint32_t l, int level) {
    return (l == 8 ? 0u : l == 12 ? lutq_pair(8) : l == 16 ? lutq_pair(8) + lutq_pair(12)
                                               : lutq_pair(8) + lutq_pair(12) + lutq_pair(16)) +
           ((l == 8 || l == 12 || l == 16) && level == 2 ? lutq_len(l, 1) : 0u);
}
constexpr uint32_t kLutQ = 128;
static_assert(lutq_off(0, 1) <= kLutQ, "quotient tables too small");

struct BlockState {
    uint16_t st_off[STACK], st_m[STACK], st_pidx[STACK];
    uint8_t st_depth[STACK];
    int sp;
    uint32_t nleaves, leaf_next, flags, item;
    unsigned long long found, claim;
    int give;  // stack entries to give away now
    uint32_t want, hround, hstop, hgen;  // shared node search: open it / round / stop / generation
    HelpCtx hc;
    uint32_t cnt[16];
    unsigned long long lut64[16];  // child -> counter increment (last child: 0)
    uint32_t lut32[16];
    // full lower nodes of a compiled leaf size, unit U = 2^a b: the increment
    // by p >> a instead of by the child p / U = (p >> a) / b (see DivNone)
    unsigned long long lutq64[kLutQ];
    uint32_t lutq32[kLutQ];
    InstDesc desc;  // the serving search's current request (read at L2 by load_desc_shared)
};

struct SmemArrays {
    uint64_t *lo, *tlo;
    uint8_t *bb, *tbb;
    uint16_t *leaf_off, *leaf_pidx;
    uint8_t *leaf_m;
};

// Number of bits of x (x >= 1).
__host__ __device__ constexpr uint32_t bit_width_ce(uint32_t x) { return x ? 1 + bit_width_ce(x >> 1) : 0; }

// Width of a packed child counter field for parts of at most `unit` keys:
// the smallest w with 2^w >= unit + 2 (see search_lower for why).
__host__ __device__ constexpr uint32_t field_width(uint32_t unit) { return bit_width_ce(unit + 1); }

// A node of m keys with np parts has its counter fit 32 bits when the top
// counted field (np - 2) cannot push past bit 31 even with all m keys in it.
__host__ __device__ constexpr bool counter_fits32(uint32_t m, uint32_t w, uint32_t np) {
    return ((uint64_t)m << (w * (np - 2))) < (1ull << 32);
}

// The reduction's result to the index of the counter increment.  For the
// full lower nodes of the compiled leaf sizes the reduction (QIdx) already
// yields p >> a for a unit U = 2^a b, the index into S.lutq: the child is
// p / U = (p >> a) / b (floor of a floor), so that table holds the increment
// of child q / b at index q, and no division is left in the search loop.
struct DivNone {
    __device__ __forceinline__ uint32_t operator()(uint32_t p) const { return p; }
};
// Runtime units: the child p / U by a multiply-high (unit_magic).
struct DivRT {
    uint32_t magic;
    __device__ __forceinline__ uint32_t operator()(uint32_t p) const { return div_unit(p, magic); }
};

// ---------------------------------------------------------------------------
// The node hash (Section 2.2, "a hash function modulo l"): h = mix64(x + s),
// handed on as its two 32-bit halves for the reduction modulo the node size.
struct Mixer {
    __device__ __forceinline__ void operator()(uint64_t z, uint32_t &hl, uint32_t &hh) const {
        const uint64_t h = mix64(z);
        hl = (uint32_t)h;
        hh = (uint32_t)(h >> 32);
    }
    // the halves of y = mix64_pre(z), for reductions that read the bits of
    // h = y ^ (y >> 31) they need straight from y (QIdx)
    __device__ __forceinline__ void pre(uint64_t z, uint32_t &yl, uint32_t &yh) const {
        const uint64_t y = mix64_pre(z);
        yl = (uint32_t)y;
        yh = (uint32_t)(y >> 32);
    }
};

// h mod m from the halves of h (same reduction as ModRT / ModCT).
__device__ __forceinline__ uint32_t mod_halves(const ModRT &r, uint32_t hl, uint32_t hh) {
    uint64_t t = (uint64_t)hh * r.c + hl;
    uint64_t u = (uint64_t)(uint32_t)(t >> 32) * r.c + (uint32_t)t;
    uint32_t v = (uint32_t)(u >> 32) * r.c + (uint32_t)u;
    return (uint32_t)__umul64hi(r.M * v, r.m);
}
// Compile-time modulus (the full leaves) with the reduction constant
// c = 2^32 mod MM held in a register, read from the instance descriptor so
// that the compiler keeps the wide multiply-add on the IMAD pipe instead of
// turning it into ALU shift/add chains.  A power-of-two MM (8, 16) is the low
// bits of h; for MM = 12, c = 4 and the fold below applies.  The last step
// v mod MM keeps the constant divisor.
template <uint32_t MM>
struct ModCTR {
    uint32_t c;
};
template <uint32_t MM>
__device__ __forceinline__ uint32_t mod_halves(const ModCTR<MM> &r, uint32_t hl, uint32_t hh) {
    if constexpr ((MM & (MM - 1)) == 0) {
        return hl & (MM - 1);
    } else {
        const uint32_t c = r.c;
        uint64_t t = (uint64_t)hh * c + hl;
        // c = 2^k for every full node size of the benchmarks (32 at 112, 256
        // at 560, 16 at 60 and 240, 64 at 96): fold t = th 2^32 + tl as
        // tl + th 2^k on the ALU, with the carry folded once more
        constexpr uint32_t cc = (uint32_t)((1ull << 32) % MM);
        if constexpr ((cc & (cc - 1)) == 0) {
            constexpr uint32_t k = bit_width_ce(cc) - 1;
            const uint32_t th = (uint32_t)(t >> 32), tl = (uint32_t)t;
            const uint32_t add = th << k;
            const uint32_t ul = tl + add;
            const uint32_t v = ul + (ul < add ? cc : 0u);  // carry out of 2^32 is worth c
            return v % MM;
        }
        uint64_t u = (uint64_t)(uint32_t)(t >> 32) * c + (uint32_t)t;
        uint32_t v = (uint32_t)(u >> 32) * c + (uint32_t)u;
        return v % MM;
    }
}
// The increment index of a full lower node straight from the hash, with no
// 64-bit remainder.  For a node of MM keys in parts of U = 2^A b keys the
// split search needs only p >> A, p = h mod MM (its entry in S.lutq).  As
// 2^A divides MM, p >> A = y mod D with y = h >> A and D = MM >> A.  Write
// D = 2^t D' (D' odd): y mod D = 2^t ((y >> t) mod D') + (y mod 2^t).  For
// z = y >> t, with k a multiple of the order e of 2 modulo D' (2^e = 1 mod
// D'), 2^k = 1 (mod D'), so z mod D' is the sum of z's k-bit digits mod D'
// (the digits taken from the two 32-bit halves of h at fixed bit positions).
// At l = 16: D = 7 (lower-1, two 30-bit digits) and 35 (lower-2, three
// 24-bit digits); at l = 12: 15 and 4 * 15 (32-bit digits, the carry of
// their sum folded back since 2^32 = 1 mod 15); at l = 8: 4 and 3.
__host__ __device__ constexpr uint32_t ord2_ce(uint32_t d, uint32_t e = 1, uint32_t p = 2) {
    return d <= 1 ? 1 : (p % d == 1 ? e : ord2_ce(d, e + 1, (p * 2) % d));
}
// The low word of y >> POS, y = yh 2^32 + yl (POS < 64).
template <uint32_t POS>
__device__ __forceinline__ uint32_t word_at(uint32_t yl, uint32_t yh) {
    if constexpr (POS >= 32) return yh >> (POS - 32);
    else if constexpr (POS == 0) return yl;
    else return __funnelshift_r(yl, yh, POS);
}
// Bits [POS, POS + W) of h = y ^ (y >> 31) (the remix's last xor-shift),
// read from y: bit i of h is y_i ^ y_(i+31), so a field of h is the field of
// y xor the field 31 bits higher (zero past bit 63), and h itself is never
// formed (W <= 32, POS + W <= 64).
template <uint32_t POS, uint32_t W>
__device__ __forceinline__ uint32_t hbits_of(uint32_t yl, uint32_t yh) {
    static_assert(W >= 1 && W <= 32 && POS + W <= 64, "bit field out of range");
    uint32_t v = word_at<POS>(yl, yh);
    if constexpr (POS + 31 < 64) v ^= word_at<POS + 31>(yl, yh);
    if constexpr (W < 32) v &= (1u << W) - 1u;
    return v;
}
template <uint32_t MM, uint32_t A>
struct QIdx {
    static constexpr uint32_t D = MM >> A;
    static constexpr uint32_t t = ctz_ce(D);
    static constexpr uint32_t Dp = D >> t;  // odd part
    static constexpr uint32_t Z = A + t;    // z = h >> Z
    static constexpr uint32_t e = ord2_ce(Dp);
    static constexpr uint32_t k = (32 / e) * e;  // digit width
    static_assert(((MM >> A) << A) == MM, "2^A must divide the node size");
    static_assert(Dp == 1 || e <= 32, "no digit width for this modulus");
};
// The index from the halves of y = mix64_pre(x + s) (round_counts passes y,
// not h, for this reduction; see hbits_of).
template <uint32_t MM, uint32_t A>
__device__ __forceinline__ uint32_t mod_halves(const QIdx<MM, A> &, uint32_t yl, uint32_t yh) {
    using Q = QIdx<MM, A>;
    uint32_t r = 0;  // z mod D'
    if constexpr (Q::Dp > 1) {
        constexpr uint32_t Z = Q::Z, k = Q::k;
        uint32_t s;
        if constexpr (k == 32) {
            // two digits (z has at most 64 bits); 2^32 = 1 (mod D'): a carry adds 1
            const uint32_t d0 = hbits_of<Z, (64 - Z < 32 ? 64 - Z : 32)>(yl, yh);
            if constexpr (Z + 32 < 64) {
                const uint32_t d1 = hbits_of<Z + 32, 32 - Z>(yl, yh);
                const uint32_t sum = d0 + d1;
                s = sum + (sum < d0 ? 1u : 0u);  // no overflow: with a carry, sum <= 2^32 - 2
            } else {
                s = d0;
            }
        } else {
            static_assert(64 - Z <= 3 * k && k <= 30, "digit sum must fit 32 bits");
            s = hbits_of<Z, k>(yl, yh);
            if constexpr (Z + k < 64) s += hbits_of<Z + k, (64 - Z - k < k ? 64 - Z - k : k)>(yl, yh);
            if constexpr (Z + 2 * k < 64) s += hbits_of<Z + 2 * k, 64 - Z - 2 * k>(yl, yh);
        }
        r = s % Q::Dp;
    }
    if constexpr (Q::t > 0) return (r << Q::t) | hbits_of<A, Q::t>(yl, yh);
    return r;
}
// Reductions that take y = mix64_pre(x + s) instead of the hash itself.
template <class M>
struct TakesPre : std::false_type {};
template <uint32_t MM, uint32_t A>
struct TakesPre<QIdx<MM, A>> : std::true_type {};

// The constant comes from the instance descriptor in device memory, so the
// compiler cannot fold it back into an immediate.
template <uint32_t MM>
__device__ __forceinline__ ModCTR<MM> make_modct(uint32_t c_from_memory) {
    return ModCTR<MM>{c_from_memory};
}

// Lower aggregation split: all threads of the block test consecutive seeds.
// Each thread counts the keys of every child but the last in w-bit fields of
// one word (the increment of child c is lut[c] = 2^(w c), the last child's is
// 0: its count is m minus the others).  The seed is valid iff the word equals
// sum_{c < np-1} p_c 2^(w c).  No wrong count can match: as long as no field
// carries past the word (counter_fits32 / 64-bit words), equal words mean the
// normalised digits of the counts equal the p_c, each carry lowers the digit
// sum by 2^w - 1, so any carry would need the last child to hold p_last -
// (2^w - 1) < 0 keys (p_last <= unit <= 2^w - 2).
// The whole chunk of seeds is decided before the next one starts, so the
// smallest working seed wins.
constexpr int kKeyUnroll = 8;  // key-loop unroll factor of the split search

// SPT seeds per thread and round: independent hash chains per key load (the
// descriptor's spt: 2 by default where trials are many, the full nodes of
// l = 16; 1 keeps the round, and the work past the winning seed, small
// elsewhere; the autotuner may pick another per device).
// The counters of one round: seeds s0 + j T (j < SPT) over the node's keys.
template <int SPT, class Cnt, class Mod, class Div>
__device__ __forceinline__ void round_counts(const uint64_t *xs, uint32_t m, Mod mod, Div div,
                                             const Cnt *lut, const Mixer &mx, uint64_t s0,
                                             Cnt (&cnt)[SPT]) {
    const uint32_t T = blockDim.x;
#pragma unroll
    for (int j = 0; j < SPT; j++) cnt[j] = 0;
    auto eval = [&](uint64_t x) {
#pragma unroll
        for (int j = 0; j < SPT; j++) {
            uint32_t hl, hh;
            if constexpr (TakesPre<Mod>::value)
                mx.pre(x + s0 + (uint64_t)j * T, hl, hh);
            else
                mx(x + s0 + (uint64_t)j * T, hl, hh);
            cnt[j] += lut[div(mod_halves(mod, hl, hh))];
        }
    };
    // xs is 16-byte aligned: two keys per shared-memory load
    const ulonglong2 *xs2 = (const ulonglong2 *)xs;
#pragma unroll kKeyUnroll
    for (uint32_t i = 0; i < m / 2; i++) {
        const ulonglong2 q = xs2[i];
        eval(q.x);
        eval(q.y);
    }
    if (m & 1) eval(xs[m - 1]);
}


// Thread 0: share the current node search now (idle blocks wait, no bucket left).
__device__ __forceinline__ bool help_wanted(const HelpCtx &h) {
    return h.q && blockIdx.x < kHelpCap && atomicAdd(&h.q->idle, 0u) > 0 &&
           atomicAdd((unsigned int *)h.bucket_head, 0u) >= h.nitems;
}

// Rounds of the shared search of node `rec`, claimed in order by the owner
// and any helpers: a round whose first seed is above the best found so far,
// or above maxv, is not evaluated (it cannot hold the smallest), and a block
// stops at the first such round.  Every round below the best round was
// claimed before it and is evaluated by its claimer, so once all blocks have
// left, rec->best is the smallest valid seed.
template <int SPT, class Cnt, class Mod, class Div>
__device__ __forceinline__ void shared_rounds(const uint64_t *xs, uint32_t m, Mod mod, Div div, const Cnt *lut,
                                           Cnt expected, uint64_t maxv, HelpRec *rec, uint32_t gen,
                                           bool owner, BlockState &S) {
    const uint32_t T = blockDim.x;
    const uint64_t step = (uint64_t)T * SPT;
    const Mixer mx{};
    for (;;) {
        if (threadIdx.x == 0) {
            bool stop = false;
            uint32_t r = 0;
            if (!owner && (atomicAdd(&rec->state, 0u) != 1u || atomicAdd(&rec->gen, 0u) != gen)) {
                stop = true;
            } else {
                r = atomicAdd(&rec->next_round, 1u);
                const unsigned long long b = atomicAdd(&rec->best, 0ull);
                const uint64_t first = (uint64_t)r * step;
                stop = first > b || first > maxv;
            }
            S.hround = r;
            S.hstop = stop;
        }
        __syncthreads();
        if (S.hstop) break;
        const uint64_t s0 = (uint64_t)S.hround * step + threadIdx.x;
        Cnt cnt[SPT];
        round_counts<SPT>(xs, m, mod, div, lut, mx, s0, cnt);
        uint64_t best = ~0ull;
#pragma unroll
        for (int j = SPT - 1; j >= 0; j--)
            if (cnt[j] == expected && s0 + (uint64_t)j * T <= maxv) best = s0 + (uint64_t)j * T;
        const bool ok = best != ~0ull;
        if (__syncthreads_or(ok) && ok) atomicMin(&rec->best, (unsigned long long)best);
    }
    __syncthreads();
}

// The owner opens its node to helpers from round `first` on: the node's
// salted keys go to the build's grouped-key array at the node's place (a
// helper copies them from there), then the record, then a few help items in
// the steal queue for the idle blocks.  After its last round it closes the
// record, waits (bounded) for the helpers to leave and takes the best seed.
template <int SPT, class Cnt, class Mod, class Div>
__device__ __forceinline__ uint64_t open_help(const uint64_t *xs, uint32_t m, Mod mod, Div div, const Cnt *lut,
                                           Cnt expected, uint64_t maxv, bool &limit, BlockState &S,
                                           const HelpCtx &h, uint32_t first) {
    HelpRec *rec = &help_recs(h.q)[blockIdx.x];
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) h.glo[h.kbeg + h.gpos + i] = xs[i];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        rec->inst = h.inst;
        rec->bucket = h.bucket;
        rec->gpos = h.gpos;
        rec->m = m;
        rec->best = ~0ull;
        rec->next_round = first;
        const uint32_t gen = atomicAdd(&rec->gen, 0u);
        S.hgen = gen;
        __threadfence();
        atomicExch(&rec->state, 1u);
        uint32_t want = atomicAdd(&h.q->idle, 0u);
        want = want > 16 ? 16 : want;
        for (uint32_t k = 0; k < want; k++) {  // invitations: (marker, owner block, generation)
            const uint32_t slot = atomicAdd(&h.q->tail, 1u);
            if (slot >= kStealCap) break;
            unsigned int *w = h.q->items[slot].w;
            __stcg(w + 0, kHelpMarker);
            __stcg(w + 1, blockIdx.x);
            __stcg(w + 2, gen);
            __threadfence();
            atomicExch(w + 3, kStealReady);
        }
    }
    __syncthreads();
    shared_rounds<SPT>(xs, m, mod, div, lut, expected, maxv, rec, S.hgen, true, S);
    if (threadIdx.x == 0) {
        atomicExch(&rec->state, 2u);
        __threadfence();
        unsigned long long t0, now;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
        while (atomicAdd(&rec->helpers, 0u) != 0) {  // helpers finish their round and leave
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
            if (now - t0 > 10000000000ull) {  // 10 s: cannot happen unless the device misbehaves
                S.flags |= ST_TIMEOUT;
                break;
            }
            __nanosleep(1000);
        }
        __threadfence();
        S.found = atomicAdd(&rec->best, 0ull);
        atomicAdd(&rec->gen, 1u);
        atomicExch(&rec->state, 0u);
    }
    __syncthreads();
    const uint64_t x = S.found;
    if (x == ~0ull) {
        limit = true;
        return 0;
    }
    return x;
}

template <int SPT, class Cnt, class Mod, class Div>
__device__ __forceinline__ uint64_t search_lower(const uint64_t *xs, uint32_t m, Mod mod, Div div,
                                                 const Cnt *lut, Cnt expected, const Mixer &mx,
                                                 uint64_t maxv, bool &limit, BlockState &S,
                                                 bool share = false) {
    const uint32_t T = blockDim.x;
    if (threadIdx.x == 0) S.want = 0;  // read after the first round's barrier
    uint32_t round = 0;
    for (uint64_t base = 0;; base += (uint64_t)T * SPT, round++) {
        Cnt cnt[SPT];
        const uint64_t s0 = base + threadIdx.x;
        round_counts<SPT>(xs, m, mod, div, lut, mx, s0, cnt);
        uint64_t best = ~0ull;
#pragma unroll
        for (int j = SPT - 1; j >= 0; j--)
            if (cnt[j] == expected && s0 + (uint64_t)j * T <= maxv) best = s0 + (uint64_t)j * T;
        const bool ok = best != ~0ull;
        // shared only once a search has run a while, and only where a round is long
        // (at least 2^16 evaluations): the per-round claim would not pay below that
        if (share && threadIdx.x == 0 && (round & 7) == 7 && round >= 15 &&
            (uint64_t)T * SPT * m >= (1u << 16))
            S.want = help_wanted(S.hc);
        if (__syncthreads_or(ok)) {
            if (ok) atomicMin(&S.found, (unsigned long long)best);
            __syncthreads();
            return S.found;
        }
        if (base + (uint64_t)T * SPT > maxv) {
            limit = true;
            return 0;
        }
        if (share && S.want)  // from the next round on, with the idle blocks
            return open_help<SPT>(xs, m, mod, div, lut, expected, maxv, limit, S, S.hc, round + 1);
    }
}

// Fanout-2 split (Section 2.2, "Splitting Trees": fanout 2 above the lower
// levels; the whole tree in Appendix C): the number of keys hashed below
// `left` must be `left`.
// One seed per warp and round, the lanes sharing the node's keys, so a round
// tests 16 seeds (512 threads): a fanout-2 split of m keys needs about
// sqrt(pi m / 2) trials, far fewer than one seed per thread would test.
template <class Mod>
__device__ __forceinline__ uint64_t search_upper(const uint64_t *xs, uint32_t m, Mod mod, uint32_t left,
                                 const Mixer &mx, uint64_t maxv, bool &limit, BlockState &S) {
    const uint32_t lane = threadIdx.x & 31, W = blockDim.x >> 5;
    for (uint64_t base = 0;; base += W) {
        const uint64_t s = base + (threadIdx.x >> 5);
        uint32_t cnt = 0;
        for (uint32_t i = lane; i < m; i += 32) {
            uint32_t hl, hh;
            mx(xs[i] + s, hl, hh);
            cnt += mod_halves(mod, hl, hh) < left;
        }
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        const bool ok = cnt == left && s <= maxv;  // the same in every lane of the warp
        if (__syncthreads_or(ok)) {
            if (ok && lane == 0) atomicMin(&S.found, (unsigned long long)s);
            __syncthreads();
            return S.found;
        }
        if (base + W > maxv) {
            limit = true;
            return 0;
        }
    }
}

// Leaf, plain brute force (Section 2.2 "Bijections"): one warp, lane = seed.
// MT = m known at compile time (full leaves: the key loop unrolls), 0 = runtime m.
template <uint32_t MT, class Mod>
__device__ __forceinline__ uint64_t leaf_plain(const uint64_t *xs, uint32_t m_rt, Mod mod,
                                               const Mixer &mx, uint64_t maxv, bool &limit,
                                               uint32_t lane) {
    const uint32_t m = MT ? MT : m_rt;
    const uint32_t full = (1u << m) - 1;
    for (uint64_t s0 = 0;; s0 += 32) {
        uint64_t s = s0 + lane;
        uint32_t mask = 0;
#pragma unroll
        for (uint32_t i = 0; i < (MT ? MT : 32u); i++) {
            if (!MT && i >= m) break;
            uint32_t hl, hh;
            mx(xs[i] + s, hl, hh);
            mask |= 1u << mod_halves(mod, hl, hh);
        }
        uint32_t ball = __ballot_sync(0xffffffffu, mask == full);
        if (ball) {
            uint64_t x = s0 + (uint32_t)(__ffs(ball) - 1);
            if (x > maxv) limit = true;
            return x;
        }
        if (s0 + 32 > maxv) {
            limit = true;
            return 0;
        }
    }
}

// Leaf with rotation fitting (Section 4): lane = k, seed k*m; keys of A set
// bits of a, keys of B bits of b; the smallest r with a | rot_m^r(b) full.
// The lowest lane with a hit has the smallest k, hence the smallest k*m + r.
// bmask has bit i set for the keys of B.
template <uint32_t MT, class Mod>
__device__ __forceinline__ uint64_t leaf_rotation(const uint64_t *xs, uint32_t bmask, uint32_t m_rt,
                                                  Mod mod, const Mixer &mx, uint64_t maxv,
                                                  bool &limit, uint32_t lane) {
    const uint32_t m = MT ? MT : m_rt;
    const uint32_t full = (1u << m) - 1;
    const uint32_t nb = __popc(bmask);
    const uint32_t na = m - nb;
    for (uint64_t k0 = 0;; k0 += 32) {
        uint64_t s = (k0 + lane) * m;
        uint32_t a = 0, b = 0;
#pragma unroll
        for (uint32_t i = 0; i < (MT ? MT : 32u); i++) {
            if (!MT && i >= m) break;
            uint32_t hl, hh;
            mx(xs[i] + s, hl, hh);
            uint32_t bit = 1u << mod_halves(mod, hl, hh);
            if ((bmask >> i) & 1)
                b |= bit;
            else
                a |= bit;
        }
        int rf = -1;
        if (__popc(a) == (int)na && __popc(b) == (int)nb) {
            for (uint32_t r = 0; r < m; r++) {
                uint32_t rot = r == 0 ? b : (((b << r) | (b >> (m - r))) & full);
                if ((a | rot) == full) {
                    rf = (int)r;
                    break;
                }
            }
        }
        uint32_t ball = __ballot_sync(0xffffffffu, rf >= 0);
        if (ball) {
            uint64_t x = __shfl_sync(0xffffffffu, s + (uint64_t)(rf < 0 ? 0 : rf), __ffs(ball) - 1);
            if (x > maxv) limit = true;
            return x;
        }
        if ((k0 + 32) * m > maxv) {
            limit = true;
            return 0;
        }
    }
}

// Leaf search with early rejection (the early-exit brute force that the
// paper's hash-evaluation counts of Appendix C assume).  Lane L tries its own
// trials L, L + 32, L + 64, ... (seed t for plain leaves, t*m for rotation
// fitting).  All lanes walk the leaf's keys cyclically in lock step, so every
// key load is a broadcast; a lane abandons a trial at its first collision
// (within A or within B for rotation fitting) and starts its next trial at the
// next key.  A trial that places all m keys without collision is a bijection
// (plain) or leaves only the rotation to find (Section 4).  A lane stops after
// its first candidate or once its trials cannot beat the warp's best value, so
// the warp's minimum is the smallest stored value, as with the lock-step form.
// With a lookup table (m <= 16) the rotation comes from canonical rotations:
// r = (t[~b] - t[a]) mod m, reduced modulo the period of ~b to the smallest
// working rotation (Section 4, "Lookup Tables").
template <bool ROT, class Mod>
__device__ __forceinline__ uint64_t leaf_cyclic(const uint64_t *xs, const uint8_t *bbs, uint32_t m,
                                                Mod mod, const Mixer &mx, uint64_t maxv,
                                                bool &limit, uint32_t lane,
                                                const uint8_t *canon, const uint8_t *period) {
    const uint32_t full = (1u << m) - 1;
    const uint64_t step = ROT ? m : 1;
    uint64_t t = lane;  // this lane's current trial
    uint32_t a = 0, b = 0, prog = 0;
    uint64_t best = ~0ull;  // warp-uniform
    bool active = true;
    uint32_t i = 0;  // warp-uniform key index
    for (;;) {
        if (active && (t * step > best || t * step > maxv)) active = false;
        if (!__any_sync(0xffffffffu, active)) break;
        uint64_t cand = ~0ull;
        if (active) {
            uint32_t hl, hh;
            mx(xs[i] + t * step, hl, hh);
            const uint32_t bit = 1u << mod_halves(mod, hl, hh);
            bool coll;
            if (ROT && bbs[i]) {
                coll = (b & bit) != 0;
                b |= bit;
            } else {
                coll = (a & bit) != 0;
                a |= bit;
            }
            if (coll) {
                t += 32;
                a = b = 0;
                prog = 0;
            } else if (++prog == m) {
                if (!ROT) {
                    cand = t;
                    active = false;
                } else {
                    int rf = -1;
                    if (canon) {
                        const uint32_t nb_ = ~b & full;
                        uint32_t r = (canon[nb_] + m - canon[a]) % m;
                        r %= period[nb_];
                        const uint32_t rot = r == 0 ? b : (((b << r) | (b >> (m - r))) & full);
                        if ((a | rot) == full) rf = (int)r;
                    } else {
                        for (uint32_t r = 0; r < m; r++) {
                            const uint32_t rot = r == 0 ? b : (((b << r) | (b >> (m - r))) & full);
                            if ((a | rot) == full) {
                                rf = (int)r;
                                break;
                            }
                        }
                    }
                    if (rf >= 0) {
                        cand = t * m + (uint32_t)rf;
                        active = false;
                    } else {
                        t += 32;
                        a = b = 0;
                        prog = 0;
                    }
                }
            }
        }
        if (__any_sync(0xffffffffu, cand != ~0ull)) {
            uint64_t c = cand;
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const uint64_t y = __shfl_xor_sync(0xffffffffu, c, o);
                c = y < c ? y : c;
            }
            best = c < best ? c : best;
        }
        i = i + 1 == m ? 0 : i + 1;
    }
    if (best > maxv) limit = true;
    return best;
}

// ShockHash leaf (Appendix C), one warp per leaf.  Under seed s key i has
// the cells c0 = lo32(h) mod m and c1 = hi32(h) mod m; the keys are the
// edges of a multigraph on the m cells, and a bijection choosing one cell
// per key exists iff no component gets more keys than cells.  Lanes screen
// seeds and run their own union-find over the edges (shock_trial,
// leaf_shock); the smallest accepted seed gets its canonical bits
// (leaf_shock_bits) and retrieval vector (leaf_shock_solve) from the whole
// warp, and the first with a solvable system is stored, with the vector in
// bits MPHF_SH_BITS and up.
__device__ __forceinline__ uint32_t leaf_shock_bits(uint32_t c0, uint32_t c1, uint64_t lo, uint32_t m,
                                                    uint32_t lane) {
    const bool key = lane < m;
    uint32_t deg = 0;  // lane = cell
    for (uint32_t i = 0; i < m; i++) {
        const uint32_t u = __shfl_sync(0xffffffffu, c0, i), v = __shfl_sync(0xffffffffu, c1, i);
        deg += (u == lane) + (v == lane);
    }
    bool alive = key;  // lane = key
    uint32_t beta = 0;
    // trees: a cell of degree one takes its only remaining key
    for (uint32_t it = 0; it < m; it++) {
        const uint32_t ones = __ballot_sync(0xffffffffu, key && deg == 1);
        if (!ones) break;
        const uint32_t c = __ffs(ones) - 1;
        const uint32_t eb = __ballot_sync(0xffffffffu, alive && (c0 == c || c1 == c));
        if (!eb) break;
        const uint32_t e = __ffs(eb) - 1;
        const uint32_t ue = __shfl_sync(0xffffffffu, c0, e), ve = __shfl_sync(0xffffffffu, c1, e);
        if (lane == e) {
            beta = c0 == c ? 0u : 1u;
            alive = false;
        }
        const uint32_t other = ue == c ? ve : ue;
        if (lane == c) deg = 0;
        if (lane == other) deg -= 1;
    }
    // cycles: walked from the key with the smallest lo word, which takes c0
    for (uint32_t it = 0; it < m; it++) {
        if (!__any_sync(0xffffffffu, alive)) break;
        unsigned long long best = alive ? lo : ~0ull;
        for (int d = 16; d; d >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, d);
            best = o < best ? o : best;
        }
        const uint32_t e0 = __ffs(__ballot_sync(0xffffffffu, alive && lo == best)) - 1;
        const uint32_t start = __shfl_sync(0xffffffffu, c0, e0);
        uint32_t cur = __shfl_sync(0xffffffffu, c1, e0);
        if (lane == e0) {
            beta = 0;
            alive = false;
        }
        for (uint32_t k = 0; k < m && cur != start; k++) {
            const uint32_t eb = __ballot_sync(0xffffffffu, alive && (c0 == cur || c1 == cur));
            if (!eb) break;
            const uint32_t e = __ffs(eb) - 1;
            const uint32_t ue = __shfl_sync(0xffffffffu, c0, e), ve = __shfl_sync(0xffffffffu, c1, e);
            if (lane == e) {
                beta = c0 == cur ? 0u : 1u;
                alive = false;
            }
            cur = ue == cur ? ve : ue;
        }
    }
    return beta;
}

// The retrieval vector of a ShockHash leaf (Appendix C; one bit per key).
// Gauss-Jordan over GF(2), lane i < m holding row i and its bit: columns in
// increasing order, the lowest remaining lane with the column's bit as pivot.
// The reduced row echelon form is unique, so the solution with zero
// non-pivot coordinates does not depend on the order of the keys.
__device__ __forceinline__ bool leaf_shock_solve(uint32_t row, uint32_t rhs, uint32_t m, uint32_t lane,
                                                 uint32_t &z) {
    const bool key = lane < m;
    bool piv = false;
    uint32_t pcol = 0;
    for (uint32_t j = 0; j < m; j++) {
        const uint32_t cand = __ballot_sync(0xffffffffu, key && !piv && ((row >> j) & 1));
        if (!cand) continue;
        const uint32_t p = __ffs(cand) - 1;
        const uint32_t rp = __shfl_sync(0xffffffffu, row, p), bp = __shfl_sync(0xffffffffu, rhs, p);
        if (lane != p && ((row >> j) & 1)) {
            row ^= rp;
            rhs ^= bp;
        }
        if (lane == p) {
            piv = true;
            pcol = j;
        }
    }
    if (__any_sync(0xffffffffu, key && !piv && rhs)) return false;
    z = __reduce_or_sync(0xffffffffu, (piv && rhs) ? (1u << pcol) : 0u);
    return true;
}

// Component labels of up to 24 cells, one byte per cell in NW <= 6
// registers (cell c in byte c & 3 of w[c >> 2]); a component's label is one
// of its cells.  Relabelling compares all bytes at once.
template <int NW>
struct CellLabels {
    uint32_t w[NW];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int i = 0; i < NW; i++) w[i] = 0x03020100u + 0x04040404u * (uint32_t)i;
    }
    __device__ __forceinline__ uint32_t get(uint32_t c) const {
        const uint32_t r = c >> 2;
        uint32_t x = w[0];
#pragma unroll
        for (int i = 1; i < NW; i++) x = r == (uint32_t)i ? w[i] : x;
        return (x >> ((c & 3) * 8)) & 0xFFu;
    }
    // every byte equal to `from` becomes `to`.  Labels are below 128, so a
    // byte of t = w ^ from is zero iff adding 0x7F leaves its top bit clear
    // (no carry crosses bytes); a sign-replicating byte permute turns those
    // top bits into byte masks.
    __device__ __forceinline__ void relabel(uint32_t from, uint32_t to) {
        const uint32_t bf = from * 0x01010101u, diff = bf ^ (to * 0x01010101u);
#pragma unroll
        for (int i = 0; i < NW; i++) {
            const uint32_t t = w[i] ^ bf;
            const uint32_t zero_hi = ~(t + 0x7F7F7F7Fu) & 0x80808080u;
            uint32_t mask;
            asm("prmt.b32 %0, %1, %2, 0xBA98;" : "=r"(mask) : "r"(zero_hi), "r"(0u));
            w[i] ^= mask & diff;
        }
    }
};

// One lane's trial: true iff the cells of the m keys under seed s admit a
// bijection.  `cyc` marks the labels of components that hold their cycle.
template <uint32_t MT>
__device__ __forceinline__ bool shock_trial(const uint64_t *xs, uint32_t m_rt, uint64_t s,
                                            const Mixer &mx, const ModRT &mod) {
    const uint32_t m = MT ? MT : m_rt;
    constexpr int NW = MT ? (int)((MT + 3) / 4) : 6;
    CellLabels<NW> L;
    L.init();
    uint32_t cyc = 0;
    for (uint32_t i = 0; i < m; i++) {
        uint32_t hl, hh;
        mx(xs[i] + s, hl, hh);
        uint32_t c0, c1;
        if constexpr (MT != 0) {
            c0 = hl % MT;
            c1 = hh % MT;
        } else {
            c0 = mod32(mod, hl);
            c1 = mod32(mod, hh);
        }
        const uint32_t a = L.get(c0), b = L.get(c1);
        if (a == b) {  // closes the component's cycle
            if ((cyc >> a) & 1) return false;
            cyc |= 1u << a;
        } else {
            const uint32_t ca = (cyc >> a) & 1, cb = (cyc >> b) & 1;
            if (ca & cb) return false;
            L.relabel(b, a);
            cyc |= cb << a;
        }
    }
    return true;
}

// Not inlined: its label registers would otherwise push the split searches
// of the same kernel past the 64-register budget.
// Position of the k-th set bit (0-based, k < popcount) of a 32-bit mask.
__device__ __forceinline__ uint32_t select32(uint32_t x, uint32_t k) {
    uint32_t pos = 0, c = __popc(x & 0xFFFFu);
    if (k >= c) {
        k -= c;
        x >>= 16;
        pos = 16;
    }
    c = __popc(x & 0xFFu);
    if (k >= c) {
        k -= c;
        x >>= 8;
        pos += 8;
    }
    for (; k; k--) x &= x - 1;
    return pos + (uint32_t)(__ffs(x) - 1);
}

// Seeds are screened first by a necessary condition: a bijection occupies
// every cell, so every cell must be one of some key's two cells.  With 2m
// uniform choices all m cells are covered with probability about
// exp(-m e^-2) (4 % at m = 24), and the screen costs only the hashes.
// ShockHash leaf (Appendix C): the smallest seed whose two cells per key
// admit a bijection and whose retrieval system is solvable.
// Passing seeds queue up in increasing order, one per lane; the queue gets
// the union-find (one seed per lane) once it holds `batch` seeds, the round
// would overflow it, or the seeds are exhausted.  The first queued seed
// that admits a bijection and a solvable retrieval system is stored: every
// smaller seed either failed the screen or the union-find.
// Not inlined: its label registers would otherwise push the split searches
// of the same kernel past the 64-register budget.
template <uint32_t MT>
__device__ __noinline__ uint64_t leaf_shock(const uint64_t *xs, const uint64_t *los, uint32_t m_rt,
                                            ModRT mod, const Mixer &mx, uint64_t maxv,
                                            bool &limit, uint32_t lane) {
    const uint32_t m = MT ? MT : m_rt;
    const bool key = lane < m;
    const uint64_t x = key ? xs[lane] : 0;  // lo + salt(0)
    const uint64_t lo = key ? los[lane] : 0;
    const uint64_t row_salt = level_salt(MPHF_SH_ROW_LEVEL);
    const uint32_t full = (1u << m) - 1;
    // queue length: screening past the answer costs more than union-find
    // rounds with idle lanes (measured on l = 24: 8 seeds 28.3 ms, 16 30.8,
    // 32 39.0, 4 29.1 per 10^7 keys)
    const uint32_t batch = m >= 16 ? 8u : 4u;
    if (maxv > MPHF_SH_MASK) maxv = MPHF_SH_MASK;
    uint64_t queued = 0;  // lane j: the j-th queued seed
    uint32_t count = 0;   // queued seeds (the same in every lane)
    // union-find on the queued seeds, then the warp's bits and solve in order
    auto drain = [&](uint64_t &found) -> bool {
        const bool ok = lane < count && shock_trial<MT>(xs, m, queued, mx, mod);
        uint32_t ball = __ballot_sync(0xffffffffu, ok);
        count = 0;
        while (ball) {
            const uint32_t src = __ffs(ball) - 1;
            ball &= ball - 1;
            const uint64_t s = __shfl_sync(0xffffffffu, queued, src);
            uint32_t hl, hh;
            mx(x + s, hl, hh);
            const uint32_t c0 = key ? mod32(mod, hl) : 0u, c1 = key ? mod32(mod, hh) : 0u;
            const uint32_t beta = leaf_shock_bits(c0, c1, lo, m, lane);
            const uint64_t r = mix64(lo + row_salt + s);
            const uint32_t row = key ? ((uint32_t)r & ((1u << m) - 1)) : 0u;
            uint32_t z;
            if (leaf_shock_solve(row, key ? beta : 0u, m, lane, z)) {
                found = s | ((uint64_t)z << MPHF_SH_BITS);
                return true;
            }
        }
        return false;
    };
    uint64_t found = 0;
    for (uint64_t s0 = 0;; s0 += 32) {
        const uint64_t mine = s0 + lane;
        bool pass = false;
        if (mine <= maxv) {
            uint32_t cover = 0;
            for (uint32_t i = 0; i < m; i++) {
                uint32_t hl, hh;
                mx(xs[i] + mine, hl, hh);
                if constexpr (MT != 0)
                    cover |= (1u << (hl % MT)) | (1u << (hh % MT));
                else
                    cover |= (1u << mod32(mod, hl)) | (1u << mod32(mod, hh));
            }
            pass = cover == full;
        }
        const uint32_t pb = __ballot_sync(0xffffffffu, pass);
        const uint32_t np = __popc(pb);
        const bool last = s0 + 32 > maxv;
        if (count + np > 32 && drain(found)) return found;
        // append this round's passing seeds behind the queue, in seed order
        const uint32_t t = lane - count;  // rank of the seed this lane receives
        const uint32_t src = (lane >= count && t < np) ? select32(pb, t) : 0u;
        const uint64_t v = __shfl_sync(0xffffffffu, mine, src);
        if (lane >= count && t < np) queued = v;
        count += np;
        if ((count >= batch || (last && count)) && drain(found)) return found;
        if (last) {
            limit = true;
            return 0;
        }
    }
}

// Any two equal lo words among keys [0, m) of the block's bucket.
__device__ __forceinline__ bool block_has_duplicate(const uint64_t *lo, uint32_t m) {
    bool dup = false;
    for (uint32_t i = threadIdx.x; i < m && !dup; i += blockDim.x)
        for (uint32_t j = i + 1; j < m; j++)
            if (lo[i] == lo[j]) {
                dup = true;
                break;
            }
    return __syncthreads_or(dup);
}

// The packed child counters of a lower node of m keys (see search_lower):
// the per-child increments in S.lut32 / S.lut64 and the expected word.
__device__ __forceinline__ uint64_t lower_counters(const Shape &sh, uint32_t m, BlockState &S) {
    const uint32_t np = num_parts(sh, m);
    const uint32_t w = field_width(lower_unit(sh, m));
    uint64_t expected = 0;
    for (uint32_t c = 0; c + 1 < np; c++) expected += (uint64_t)part_size(sh, m, c) << (w * c);
    if (threadIdx.x < 16) {
        const uint64_t inc = threadIdx.x + 1 < np ? 1ull << (w * threadIdx.x) : 0;
        S.lut64[threadIdx.x] = inc;
        S.lut32[threadIdx.x] = (uint32_t)inc;
    }
    return expected;
}

// One inner node (Section 2.2, "Splitting Trees"; Section 5.3, "Splittings":
// a thread block tries seeds, then regroups the node's keys): search its
// smallest valid seed, store it in preorder, regroup its keys by child in
// shared memory and push the children.
template <int LEAF>
__device__ __forceinline__ void split_node(const InstDesc &d, const Shape &sh, uint32_t off, uint32_t m,
                           uint32_t depth, uint32_t pidx, uint64_t nbase, uint32_t bucket_m,
                           const SmemArrays &A, BlockState &S) {
    const uint32_t T = blockDim.x, tid = threadIdx.x;
    const uint32_t kind = node_kind(sh, m);
    const uint64_t salt = level_salt(salt_level(sh, m, depth));
    // salted keys of the node at the start of the (16-byte aligned) scratch area
    for (uint32_t i = tid; i < m; i += T) A.tlo[i] = A.lo[off + i] + salt;
    if (tid == 0) S.found = ~0ull;
    __syncthreads();
    const uint64_t *xs = A.tlo;
    const uint32_t np = num_parts(sh, m);
    uint64_t x = 0;
    bool limit = false;
    const ModRT mrt{m, d.mod_c[m], d.mod_M[m]};  // from the table: no divisions per node
    const Mixer mx{};
    if (kind == NODE_UPPER) {
        x = search_upper(xs, m, mrt, upper_left(sh, m), mx, d.max_value, limit, S);
    } else {
        const uint32_t unit = lower_unit(sh, m);
        const uint32_t w = field_width(unit);
        const uint64_t expected = lower_counters(sh, m, S);
        if (tid == 0) S.hc.gpos = S.hc.gbase + off;  // where the node's keys sit in the bucket
        __syncthreads();
        const bool share = S.hc.q != nullptr;
        bool done = false;
        if constexpr (LEAF != 0) {
            // full lower-1 and lower-2 nodes: the counter index from a digit sum (QIdx),
            // compile-time unit and counter width
            constexpr uint32_t f1 = ((35u * LEAF + 154u) / 100u) < 2 ? 2 : (35u * LEAF + 154u) / 100u;
            constexpr uint32_t f2 = ((21u * LEAF + 189u) / 100u) < 2 ? 2 : (21u * LEAF + 189u) / 100u;
            constexpr uint32_t L1 = f1 * LEAF, L2 = f2 * L1;
            constexpr bool n1 = counter_fits32(L1, field_width(LEAF), f1);
            constexpr bool n2 = counter_fits32(L2, field_width(L1), f2);
            using C1 = typename std::conditional<n1, uint32_t, unsigned long long>::type;
            using C2 = typename std::conditional<n2, uint32_t, unsigned long long>::type;
            // seeds per thread from the descriptor (the autotuner's choice)
            constexpr uint32_t a1 = ctz_ce(LEAF), a2 = ctz_ce(L1);
            if (m == L1) {
                const C1 *lut = n1 ? (const C1 *)(S.lutq32 + lutq_off(LEAF, 1)) : (const C1 *)(S.lutq64 + lutq_off(LEAF, 1));
                const QIdx<L1, a1> mod{};  // the table index p >> a1 straight from the hash
                const DivNone dv{};
                x = d.spt == 4 ? search_lower<4, C1>(xs, m, mod, dv, lut, (C1)expected, mx, d.max_value, limit, S, share)
                  : d.spt == 2 ? search_lower<2, C1>(xs, m, mod, dv, lut, (C1)expected, mx, d.max_value, limit, S, share)
                               : search_lower<1, C1>(xs, m, mod, dv, lut, (C1)expected, mx, d.max_value, limit, S, share);
                done = true;
            } else if (m == L2) {
                const C2 *lut = n2 ? (const C2 *)(S.lutq32 + lutq_off(LEAF, 2)) : (const C2 *)(S.lutq64 + lutq_off(LEAF, 2));
                const QIdx<L2, a2> mod{};
                const DivNone dv{};
                x = d.spt == 4 ? search_lower<4, C2>(xs, m, mod, dv, lut, (C2)expected, mx, d.max_value, limit, S, share)
                  : d.spt == 2 ? search_lower<2, C2>(xs, m, mod, dv, lut, (C2)expected, mx, d.max_value, limit, S, share)
                               : search_lower<1, C2>(xs, m, mod, dv, lut, (C2)expected, mx, d.max_value, limit, S, share);
                done = true;
            }
        }
        if (!done) {
            const DivRT dv{unit_magic(unit)};
            if (counter_fits32(m, w, np))
                x = search_lower<1, uint32_t>(xs, m, mrt, dv, S.lut32, (uint32_t)expected, mx,
                                           d.max_value, limit, S);
            else
                x = search_lower<1, unsigned long long>(xs, m, mrt, dv, S.lut64, expected, mx,
                                                     d.max_value, limit, S);
        }
    }
    if (limit) {  // uniform: decided after a block-wide vote
        bool dup = block_has_duplicate(A.lo, bucket_m);
        if (tid == 0) S.flags |= dup ? ST_DUPLICATE : ST_LIMIT;
        __syncthreads();
        return;
    }
    if (tid == 0) {
        d.values[nbase + pidx] = x;
        d.node_m[nbase + pidx] = (uint16_t)m;
    }
    // regroup the node's keys by child with the seed found
    if (tid < np) S.cnt[tid] = 0;
    __syncthreads();
    const bool upper = kind == NODE_UPPER;
    const uint32_t left = upper ? upper_left(sh, m) : 0;
    const uint32_t unit = upper ? 1 : lower_unit(sh, m);
    const uint32_t um = upper ? 0 : unit_magic(unit);
    for (uint32_t i = tid; i < m; i += T) {
        uint32_t p = mrt(mix64(xs[i] + x));
        uint32_t c = upper ? (p < left ? 0u : 1u) : div_unit(p, um);
        uint32_t start = upper ? (c ? left : 0u) : c * unit;
        uint32_t dst = off + start + atomicAdd(&S.cnt[c], 1u);
        A.lo[dst] = xs[i] - salt;
        A.tbb[dst] = A.bb[off + i];
    }
    __syncthreads();
    for (uint32_t i = tid; i < m; i += T) A.bb[off + i] = A.tbb[off + i];
    if (tid == 0) {
        uint32_t coff = off, cp = pidx + 1;
        for (uint32_t c = 0; c < np; c++) {
            uint32_t q = part_size(sh, m, c);
            if (q >= 2) {
                if (q <= sh.leaf) {
                    uint32_t j = S.nleaves++;
                    A.leaf_off[j] = (uint16_t)coff;
                    A.leaf_m[j] = (uint8_t)q;
                    A.leaf_pidx[j] = (uint16_t)cp;
                } else {
                    int k = S.sp++;
                    S.st_off[k] = (uint16_t)coff;
                    S.st_m[k] = (uint16_t)q;
                    S.st_depth[k] = (uint8_t)(depth + 1);
                    S.st_pidx[k] = (uint16_t)cp;
                }
            }
            cp += d.nodes_tab[q];
            coff += q;
        }
    }
    __syncthreads();
}

template <int LEAF>
__device__ __forceinline__ void leaf_phase(const InstDesc &d, uint64_t nbase, const SmemArrays &A, BlockState &S) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t salt = level_salt(0);
    const Mixer mx{};
    for (;;) {
        uint32_t j = 0;
        if (lane == 0) j = atomicAdd(&S.leaf_next, 1u);
        j = __shfl_sync(0xffffffffu, j, 0);
        if (j >= S.nleaves) break;
        const uint32_t off = A.leaf_off[j], m = A.leaf_m[j];
        // equal lo words can never be separated: refuse the bucket
        bool dup = false;
        if (lane < m)
            for (uint32_t i = lane + 1; i < m; i++) dup |= A.lo[off + lane] == A.lo[off + i];
        if (__any_sync(0xffffffffu, dup)) {
            if (lane == 0) atomicOr(&S.flags, ST_DUPLICATE);
            continue;
        }
        if (lane < m) A.tlo[off + lane] = A.lo[off + lane] + salt;
        __syncwarp();
        const uint64_t *xs = A.tlo + off;
        const ModRT mleaf{m, d.mod_c[m], d.mod_M[m]};
        bool limit = false;
        uint64_t x;
        bool done = false;
        if (d.bij == MPHF_BIJECTION_SHOCKHASH) {
            if constexpr (LEAF != 0) {
                if (m == (uint32_t)LEAF) {
                    x = leaf_shock<LEAF>(xs, A.lo + off, m, mleaf, mx, d.max_value, limit, lane);
                    done = true;
                }
            } else {
                // full leaves of l = 24 (the size ShockHash makes affordable) get a
                // compile-time copy of the leaf search without one of the whole kernel
                if (m == 24 && d.leaf == 24) {
                    x = leaf_shock<24>(xs, A.lo + off, m, mleaf, mx, d.max_value, limit, lane);
                    done = true;
                }
            }
            if (!done) x = leaf_shock<0>(xs, A.lo + off, m, mleaf, mx, d.max_value, limit, lane);
        } else if (d.leaf_method == 0) {  // lock-step: every lane hashes all m keys per trial
            uint32_t bmask = 0;
            for (uint32_t i = 0; i < m; i++) bmask |= (uint32_t)A.bb[off + i] << i;
            if constexpr (LEAF != 0) {
                if (m == (uint32_t)LEAF) {  // full leaf: compile-time m and modulus
                    x = d.bij ? leaf_rotation<LEAF>(xs, bmask, m, make_modct<LEAF>(d.red_leaf), mx, d.max_value, limit, lane)
                                   : leaf_plain<LEAF>(xs, m, make_modct<LEAF>(d.red_leaf), mx, d.max_value, limit, lane);
                    done = true;
                }
            }
            if (!done)
                x = d.bij ? leaf_rotation<0>(xs, bmask, m, mleaf, mx, d.max_value, limit, lane)
                               : leaf_plain<0>(xs, m, mleaf, mx, d.max_value, limit, lane);
        } else {  // early rejection (1), with the rotation lookup table (2)
            const bool use_lut = d.leaf_method == 2 && m <= 16 && d.rot_canon;
            const uint8_t *canon = use_lut ? d.rot_canon + ((1u << m) - 4) : nullptr;
            const uint8_t *period = use_lut ? d.rot_period + ((1u << m) - 4) : nullptr;
            if constexpr (LEAF != 0) {
                if (m == (uint32_t)LEAF) {
                    x = d.bij ? leaf_cyclic<true>(xs, A.bb + off, m, make_modct<LEAF>(d.red_leaf), mx, d.max_value, limit, lane, canon, period)
                                   : leaf_cyclic<false>(xs, A.bb + off, m, make_modct<LEAF>(d.red_leaf), mx, d.max_value, limit, lane, nullptr, nullptr);
                    done = true;
                }
            }
            if (!done)
                x = d.bij ? leaf_cyclic<true>(xs, A.bb + off, m, mleaf, mx, d.max_value, limit, lane, canon, period)
                               : leaf_cyclic<false>(xs, A.bb + off, m, mleaf, mx, d.max_value, limit, lane, nullptr, nullptr);
        }
        if (lane == 0) {
            if (limit) {
                atomicOr(&S.flags, ST_LIMIT);
            } else {
                d.values[nbase + A.leaf_pidx[j]] = x;
                d.node_m[nbase + A.leaf_pidx[j]] = (uint16_t)m;
            }
        }
    }
}

// Giving subtrees away (the tail of a search).  Buckets take random times
// (geometric trial counts), so when the bucket queue runs dry the blocks
// finish one by one and idle while the last ones work.  From then on a block
// whose stack holds two or more inner nodes not yet started, while some
// block is idle, gives all but the next one away: it writes their keys back
// to the build's grouped-key array and publishes (build, bucket, key offset,
// size, depth, preorder index) in the steal queue; an idle block takes one,
// loads its keys and processes it like a bucket.  Every node is still
// searched by one block with the same keys and salt, so the stored values
// do not change.  A published node is never lost: a block leaves only when
// the queue is empty and no block is busy, and a block that published nodes
// takes from the queue itself after its own work.
struct StealCtx {
    StealQueue *q;           // nullptr: no stealing (the serving search)
    const uint32_t *bucket_head;
    uint32_t nitems, cap;
};
// Thread 0: the number of bottom stack entries to give away now.
__device__ __forceinline__ int donation(const StealCtx &X, const BlockState &S) {
    if (!X.q || S.sp < 2) return 0;
    if (atomicAdd(&X.q->idle, 0u) == 0) return 0;
    if (atomicAdd((unsigned int *)X.bucket_head, 0u) < X.nitems) return 0;  // buckets still queued
    return S.sp - 1;
}

template <int LEAF>
__device__ __forceinline__ void give_away(const InstDesc &d, uint32_t inst, uint32_t bucket, uint64_t kbeg,
                                          uint32_t goff, const SmemArrays &A, BlockState &S,
                                          const StealCtx &X) {
    const uint32_t tid = threadIdx.x, T = blockDim.x;
    const int give = S.give;
    uint64_t *glo = (uint64_t *)d.lo;  // the build's grouped-key scratch
    uint8_t *gbb = (uint8_t *)d.bb;
    for (int e = 0; e < give; e++) {
        const uint32_t off = S.st_off[e], m = S.st_m[e];
        for (uint32_t i = tid; i < m; i += T) {
            glo[kbeg + goff + off + i] = A.lo[off + i];
            gbb[kbeg + goff + off + i] = A.bb[off + i];
        }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        int kept = 0;
        for (int e = 0; e < give; e++) {
            const uint32_t slot = atomicAdd(&X.q->tail, 1u);
            if (slot >= X.cap) {  // queue full: keep the node
                S.st_off[kept] = S.st_off[e];
                S.st_m[kept] = S.st_m[e];
                S.st_depth[kept] = S.st_depth[e];
                S.st_pidx[kept] = S.st_pidx[e];
                kept++;
                continue;
            }
            unsigned int *w = X.q->items[slot].w;
            __stcg(w + 0, inst);
            __stcg(w + 1, bucket);
            __stcg(w + 2, (goff + S.st_off[e]) | ((uint32_t)S.st_m[e] << 16));
            __threadfence();
            atomicExch(w + 3, (uint32_t)S.st_pidx[e] | ((uint32_t)S.st_depth[e] << 16) | kStealReady);
        }
        const int top = S.sp - 1;  // the node this block takes next stays
        S.st_off[kept] = S.st_off[top];
        S.st_m[kept] = S.st_m[top];
        S.st_depth[kept] = S.st_depth[top];
        S.st_pidx[kept] = S.st_pidx[top];
        S.sp = kept + 1;
    }
    __syncthreads();
}

// One unit of search work (Section 2.2): the subtree of m0 keys at key offset
// goff of a bucket (a whole bucket: goff = 0, m0 = its size), its inner nodes
// depth first, then every leaf's bijection search, values written in preorder.
template <int LEAF>
__device__ __forceinline__ void process_item(const InstDesc &d, uint32_t inst, uint32_t bucket, uint32_t goff,
                                             uint32_t m0, uint32_t depth0, uint32_t pidx0,
                                             const SmemArrays &A, BlockState &S, const StealCtx &X) {
    const uint32_t tid = threadIdx.x, T = blockDim.x;
    const Shape sh = make_shape(LEAF ? (uint32_t)LEAF : d.leaf, d.tree);
    // a build's arrays are read past L1 (ld.global.cg): a serving search runs
    // across requests whose arrays may reuse the addresses of earlier ones,
    // and keys given away were written by another block of this launch
    const uint64_t kbeg = __ldcg(d.bucket_off + bucket);
    const uint64_t nbase = __ldcg(d.node_off + bucket);
    if (m0 <= 1 || m0 > 4096) return;  // nothing stored / refused by the plan
    for (uint32_t i = tid; i < m0; i += T) {
        A.lo[i] = __ldcg(d.lo + kbeg + goff + i);
        A.bb[i] = __ldcg(d.bb + kbeg + goff + i);
    }
    if (tid == 0) {
        S.sp = 0;
        S.nleaves = 0;
        S.leaf_next = 0;
        S.flags = 0;
        S.hc = HelpCtx{X.q, X.bucket_head, X.nitems, inst, bucket, goff, goff, (uint64_t *)d.lo, kbeg};
        if (m0 <= sh.leaf) {
            A.leaf_off[0] = 0;
            A.leaf_m[0] = (uint8_t)m0;
            A.leaf_pidx[0] = (uint16_t)pidx0;
            S.nleaves = 1;
        } else {
            S.st_off[0] = 0;
            S.st_m[0] = (uint16_t)m0;
            S.st_depth[0] = (uint8_t)depth0;
            S.st_pidx[0] = (uint16_t)pidx0;
            S.sp = 1;
        }
    }
    __syncthreads();
    for (;;) {
        if (S.sp == 0 || S.flags) break;
        if (tid == 0) S.give = donation(X, S);
        __syncthreads();
        if (S.give) give_away<LEAF>(d, inst, bucket, kbeg, goff, A, S, X);
        const int k = S.sp - 1;
        const uint32_t off = S.st_off[k], m = S.st_m[k], depth = S.st_depth[k], pidx = S.st_pidx[k];
        __syncthreads();
        if (tid == 0) S.sp = k;
        split_node<LEAF>(d, sh, off, m, depth, pidx, nbase, m0, A, S);
    }
    if (!S.flags) leaf_phase<LEAF>(d, nbase, A, S);
    __syncthreads();
    if (tid == 0 && S.flags) atomicOr(d.status, S.flags);
    __syncthreads();
}

template <int LEAF>
__device__ __forceinline__ void process_bucket(const InstDesc &d, uint32_t bucket, const SmemArrays &A,
                                               BlockState &S) {
    const uint32_t m = (uint32_t)(__ldcg(d.bucket_off + bucket + 1) - __ldcg(d.bucket_off + bucket));
    process_item<LEAF>(d, 0, bucket, 0, m > 4096 ? 4097u : m, 0, 0, A, S, StealCtx{nullptr, nullptr, 0, 0});
}

// A helper's part of a shared node search (open_help): the node's salted
// keys from the build's grouped-key array, the same counters, modulus and
// seeds per thread as the owner, then rounds until the owner's search ends.
template <int LEAF>
__device__ __forceinline__ void help_node(const InstDesc &d, HelpRec *rec, uint32_t gen,
                                          const SmemArrays &A, BlockState &S) {
    if constexpr (LEAF != 0) {
        const Shape sh = make_shape((uint32_t)LEAF, d.tree);
        const uint32_t m = __ldcg(&rec->m), bucket = __ldcg(&rec->bucket), gpos = __ldcg(&rec->gpos);
        const uint64_t kbeg = __ldcg(d.bucket_off + bucket);
        for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) A.tlo[i] = __ldcg(d.lo + kbeg + gpos + i);
        const uint64_t expected = lower_counters(sh, m, S);
        __syncthreads();
        constexpr uint32_t f1 = ((35u * LEAF + 154u) / 100u) < 2 ? 2 : (35u * LEAF + 154u) / 100u;
        constexpr uint32_t f2 = ((21u * LEAF + 189u) / 100u) < 2 ? 2 : (21u * LEAF + 189u) / 100u;
        constexpr uint32_t L1 = f1 * LEAF, L2 = f2 * L1;
        constexpr bool n1 = counter_fits32(L1, field_width(LEAF), f1);
        constexpr bool n2 = counter_fits32(L2, field_width(L1), f2);
        using C1 = typename std::conditional<n1, uint32_t, unsigned long long>::type;
        using C2 = typename std::conditional<n2, uint32_t, unsigned long long>::type;
        const uint64_t *xs = A.tlo;
        const DivNone dv1{}, dv2{};
        if (d.tree == MPHF_TREE_RECSPLIT && m == L1) {
            const C1 *lut = n1 ? (const C1 *)(S.lutq32 + lutq_off(LEAF, 1)) : (const C1 *)(S.lutq64 + lutq_off(LEAF, 1));
            const QIdx<L1, ctz_ce(LEAF)> mod{};
            if (d.spt == 4) shared_rounds<4>(xs, m, mod, dv1, lut, (C1)expected, d.max_value, rec, gen, false, S);
            else if (d.spt == 2) shared_rounds<2>(xs, m, mod, dv1, lut, (C1)expected, d.max_value, rec, gen, false, S);
            else shared_rounds<1>(xs, m, mod, dv1, lut, (C1)expected, d.max_value, rec, gen, false, S);
        } else if (d.tree == MPHF_TREE_RECSPLIT && m == L2) {
            const C2 *lut = n2 ? (const C2 *)(S.lutq32 + lutq_off(LEAF, 2)) : (const C2 *)(S.lutq64 + lutq_off(LEAF, 2));
            const QIdx<L2, ctz_ce(L1)> mod{};
            if (d.spt == 4) shared_rounds<4>(xs, m, mod, dv2, lut, (C2)expected, d.max_value, rec, gen, false, S);
            else if (d.spt == 2) shared_rounds<2>(xs, m, mod, dv2, lut, (C2)expected, d.max_value, rec, gen, false, S);
            else shared_rounds<1>(xs, m, mod, dv2, lut, (C2)expected, d.max_value, rec, gen, false, S);
        }
    }
    __syncthreads();
}

// Thread 0 of an idle block: a node from the steal queue, or ~0u when the
// queue is empty and no block is busy (nothing more can be given away).
// Waits are bounded: leaving is always safe, since a block that gave nodes
// away takes from the queue after its own work.
__device__ uint32_t steal_claim(const StealCtx &X, const InstDesc *insts, uint32_t ninst) {
    StealQueue *Q = X.q;
    atomicAdd(&Q->idle, 1u);
    uint32_t got = ~0u;
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (uint32_t spin = 0; spin < (1u << 24); spin++) {
        const uint32_t h = atomicAdd(&Q->head, 0u);
        uint32_t t = atomicAdd(&Q->tail, 0u);
        t = t < X.cap ? t : X.cap;
        if (h < t) {
            if (atomicCAS(&Q->head, h, h + 1) == h) {
                got = h;
                break;
            }
            continue;
        }
        if (atomicAdd(&Q->busy, 0u) == 0) {
            __threadfence();
            t = atomicAdd(&Q->tail, 0u);
            t = t < X.cap ? t : X.cap;
            if (atomicAdd(&Q->head, 0u) >= t) break;
            continue;
        }
        unsigned long long now;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
        if (now - t0 > 30000000000ull) break;  // 30 s
        __nanosleep(2000);
    }
    if (got != ~0u) {
        atomicAdd(&Q->busy, 1u);
        // the publisher's last store may still be on its way (bounded wait)
        bool ready = false;
        for (uint32_t spin = 0; spin < (1u << 22) && !ready; spin++) {
            ready = (atomicAdd(&Q->items[got].w[3], 0u) & kStealReady) != 0;
            if (!ready) __nanosleep(100);
        }
        if (!ready) {  // cannot happen unless the device misbehaves: fail every build of the launch
            for (uint32_t i = 0; i < ninst; i++)
                if (insts[i].status) atomicOr(insts[i].status, ST_TIMEOUT);
            atomicSub(&Q->busy, 1u);
            got = ~0u;
        }
        __threadfence();
    }
    atomicSub(&Q->idle, 1u);
    return got;
}

// Dynamic shared memory of the search kernel for buckets of at most `cap`
// keys.  The capacity is padded to 16 so that every array starts aligned:
// lo, tlo at 0 and 8P (u64), bb, tbb at 16P and 17P (u8), the leaf list at
// 18P (two u16 arrays of nl entries, then nl bytes).
struct SmemLayout {
    uint32_t P, nl, bytes;
    __host__ __device__ explicit SmemLayout(uint32_t cap) {
        P = (cap + 15u) & ~15u;
        nl = P / 2 + 1;
        bytes = 18u * P + 5u * nl;
    }
};

// The persistent search (the brute-force searches of Section 2.2 in the
// parallel form of Section 5.3): blocks take buckets from a device queue,
// largest first, and run process_bucket on each.
// All quotient-indexed increment tables of one block (before its first
// barrier, once per launch).
template <uint32_t UNIT, uint32_t NP, uint32_t M>
__device__ __forceinline__ void fill_lutq(BlockState &S, uint32_t off) {
    constexpr uint32_t a = ctz_ce(UNIT), b = UNIT >> a, w = field_width(UNIT);
    for (uint32_t q = threadIdx.x; q < (M >> a); q += blockDim.x) {
        const uint32_t c = q / b;
        const uint64_t inc = c + 1 < NP ? 1ull << (w * c) : 0;  // the last child is implied
        S.lutq64[off + q] = inc;
        S.lutq32[off + q] = (uint32_t)inc;
    }
}
template <uint32_t LEAF>
__device__ __forceinline__ void fill_lutq_leaf(BlockState &S) {
    constexpr uint32_t f1 = fan1_ce(LEAF), f2 = fan2_ce(LEAF), L1 = f1 * LEAF, L2 = f2 * L1;
    fill_lutq<LEAF, f1, L1>(S, lutq_off(LEAF, 1));
    fill_lutq<L1, f2, L2>(S, lutq_off(LEAF, 2));
}
__device__ __forceinline__ void init_lutq(BlockState &S) {
    fill_lutq_leaf<8>(S);
    fill_lutq_leaf<12>(S);
    fill_lutq_leaf<16>(S);
}

__global__ void __launch_bounds__(512) k_search(const InstDesc *insts, uint32_t ninst, const WorkItem *items,
                                                uint32_t nitems, uint32_t *head, uint32_t cap,
                                                StealQueue *steal, uint32_t steal_cap) {
    extern __shared__ __align__(16) uint8_t dyn[];
    __shared__ BlockState S;
    const SmemLayout lay(cap);
    SmemArrays A;
    A.lo = (uint64_t *)dyn;
    A.tlo = A.lo + lay.P;
    A.bb = dyn + 16u * lay.P;
    A.tbb = A.bb + lay.P;
    A.leaf_off = (uint16_t *)(dyn + 18u * lay.P);
    A.leaf_pidx = A.leaf_off + lay.nl;
    A.leaf_m = (uint8_t *)(A.leaf_pidx + lay.nl);
    const StealCtx X{steal, head, nitems, steal_cap};
    init_lutq(S);  // published by the first barrier below
    for (;;) {
        if (threadIdx.x == 0) {
            S.item = atomicAdd(head, 1u);
            if (S.item < nitems && steal) atomicAdd(&steal->busy, 1u);
            const uint32_t g = S.item < nitems || !steal ? ~0u : steal_claim(X, insts, ninst);
            S.claim = g < steal_cap ? (unsigned long long)g : ~0ull;  // ~0: nothing was claimed
        }
        __syncthreads();
        const uint32_t it = S.item;
        const unsigned long long got = S.claim;
        __syncthreads();
        uint32_t inst, bucket, goff = 0, m0 = 0, depth = 0, pidx = 0;
        if (it < nitems) {  // a whole bucket
            const WorkItem w = items[it];
            inst = w.inst;
            bucket = w.bucket;
            if (inst != 0xFFFFFFFFu) {  // else an empty slot (its build failed its plan)
                const InstDesc &dd = insts[inst];
                const uint64_t mm = __ldcg(dd.bucket_off + bucket + 1) - __ldcg(dd.bucket_off + bucket);
                m0 = mm > 4096 ? 4097u : (uint32_t)mm;
            }
        } else if (got != ~0ull) {  // a subtree another block gave away, or an invitation
            const unsigned int *w = steal->items[got].w;
            inst = __ldcg(w + 0);
            bucket = __ldcg(w + 1);
            const uint32_t w2 = __ldcg(w + 2), w3 = __ldcg(w + 3);
            if (inst == kHelpMarker) {  // join block w1's search of one node, generation w2
                HelpRec *rec = &help_recs(steal)[bucket];
                if (threadIdx.x == 0) {
                    atomicAdd(&rec->helpers, 1u);
                    __threadfence();
                    S.hstop = !(atomicAdd(&rec->state, 0u) == 1u && atomicAdd(&rec->gen, 0u) == w2);
                }
                __syncthreads();
                if (!S.hstop) {
                    const InstDesc d = insts[__ldcg(&rec->inst)];
                    switch (d.leaf) {
                        case 8: help_node<8>(d, rec, w2, A, S); break;
                        case 12: help_node<12>(d, rec, w2, A, S); break;
                        case 16: help_node<16>(d, rec, w2, A, S); break;
                        default: break;
                    }
                }
                if (threadIdx.x == 0) {
                    __threadfence();
                    atomicSub(&rec->helpers, 1u);
                    atomicSub(&steal->busy, 1u);
                }
                __syncthreads();
                continue;
            }
            goff = w2 & 0xFFFFu;
            m0 = w2 >> 16;
            pidx = w3 & 0xFFFFu;
            depth = (w3 >> 16) & 0xFFu;
        } else {
            break;
        }
        if (inst != 0xFFFFFFFFu) {
            const InstDesc d = insts[inst];
            switch (d.leaf) {
                case 8: process_item<8>(d, inst, bucket, goff, m0, depth, pidx, A, S, X); break;
                case 12: process_item<12>(d, inst, bucket, goff, m0, depth, pidx, A, S, X); break;
                case 16: process_item<16>(d, inst, bucket, goff, m0, depth, pidx, A, S, X); break;
                default: process_item<0>(d, inst, bucket, goff, m0, depth, pidx, A, S, X); break;
            }
        }
        if (threadIdx.x == 0 && steal) atomicSub(&steal->busy, 1u);
    }
}

// ---------------------------------------------------------------------------
// The serving search: the same bucket work as k_search, but the work items
// arrive while it runs.  The host appends items to a ring and then raises
// ctl->tail; a block claims the next item by advancing ctl->head.  After a
// bucket, its build's done counter is raised.  A block that finds the ring
// empty sleeps and looks again; it leaves when the host sets ctl->stop (no
// request left) or, as a bound on the wait, after idle_ns without work (the
// host is gone or stalled; ctl->err records it).  The second block that
// lands on each of the first reserved_sms SMs exits at once, which leaves
// room there for the preparation and packing kernels of other requests.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ unsigned long long serve_claim(ServeCtl *c, unsigned long long idle_ns) {
    const unsigned long long t0 = global_ns();
    for (uint32_t spin = 0; spin < (1u << 22); spin++) {  // bounded: about a minute of sleeps at most
        const unsigned long long h = atomicAdd(&c->head, 0ull);  // reads at L2, where the host's copies land
        const unsigned long long t = atomicAdd(&c->tail, 0ull);
        if (h < t) {
            if (atomicCAS(&c->head, h, h + 1) == h) return h;
            continue;
        }
        if (atomicAdd(&c->stop, 0u)) return ~0ull;
        if (global_ns() - t0 > idle_ns) break;
        __nanosleep(20000);
    }
    atomicOr(&c->err, 1u);  // waited the limit: leave, the host relaunches if work remains
    return ~0ull;
}

// A request's descriptor, written by the host while the kernel runs, is read
// at L2 (never a stale L1 line of a reused slot) into shared memory by the
// first threads; the caller's barrier publishes it.  Held there rather than in
// registers, it leaves the search loops their registers.
__device__ __forceinline__ void load_desc_shared(const InstDesc *p, InstDesc &out) {
    static_assert(sizeof(InstDesc) % 8 == 0, "descriptor is copied as 64-bit words");
    const unsigned long long *src = (const unsigned long long *)p;
    unsigned long long *dst = (unsigned long long *)&out;
    if (threadIdx.x < sizeof(InstDesc) / 8) dst[threadIdx.x] = __ldcg(src + threadIdx.x);
}

__global__ void __launch_bounds__(512) k_serve(const InstDesc *insts, const WorkItem *ring,
                                               uint32_t ring_cap, ServeCtl *ctl, unsigned int *done,
                                               unsigned int *sm_count, uint32_t reserved_sms,
                                               unsigned long long idle_ns, uint32_t cap) {
    extern __shared__ __align__(16) uint8_t dyn[];
    __shared__ BlockState S;
    const SmemLayout lay(cap);
    SmemArrays A;
    A.lo = (uint64_t *)dyn;
    A.tlo = A.lo + lay.P;
    A.bb = dyn + 16u * lay.P;
    A.tbb = A.bb + lay.P;
    A.leaf_off = (uint16_t *)(dyn + 18u * lay.P);
    A.leaf_pidx = A.leaf_off + lay.nl;
    A.leaf_m = (uint8_t *)(A.leaf_pidx + lay.nl);
    if (threadIdx.x == 0) {
        uint32_t smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        const uint32_t before = atomicAdd(&sm_count[smid & (kServeMaxSms - 1)], 1u);
        S.item = smid < reserved_sms && before >= 1;
    }
    init_lutq(S);  // published by the barrier below
    __syncthreads();
    if (S.item) return;
    for (;;) {
        if (threadIdx.x == 0) S.claim = serve_claim(ctl, idle_ns);
        __syncthreads();
        const unsigned long long it = S.claim;
        __syncthreads();
        if (it == ~0ull) break;
        const unsigned long long raw = __ldcg((const unsigned long long *)(ring + it % ring_cap));
        const WorkItem w{(uint32_t)raw, (uint32_t)(raw >> 32)};
        load_desc_shared(insts + w.inst, S.desc);  // every thread has left the previous bucket
        __syncthreads();
        const InstDesc &d = S.desc;
        switch (d.leaf) {
            case 8: process_bucket<8>(d, w.bucket, A, S); break;
            case 12: process_bucket<12>(d, w.bucket, A, S); break;
            case 16: process_bucket<16>(d, w.bucket, A, S); break;
            default: process_bucket<0>(d, w.bucket, A, S); break;
        }
        if (threadIdx.x == 0) {
            __threadfence();  // the bucket's values before its completion
            atomicAdd(&done[w.inst], 1u);
        }
    }
}

ServeLaunch plan_serve_launch(uint32_t threads, uint32_t reserved_sms) {
    ServeLaunch L;
    L.cap = 4096;  // any bucket a build accepts
    L.threads = threads ? threads : 512;
    L.smem_bytes = SmemLayout(L.cap).bytes;
    int dev = 0, sms = 148, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_serve, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem_bytes);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_serve, L.threads, L.smem_bytes);
    if (occ < 1) occ = 1;
    L.blocks = (uint32_t)sms * (uint32_t)occ;
    L.working_blocks = L.blocks - (occ > 1 ? (reserved_sms < (uint32_t)sms ? reserved_sms : sms) : 0);
    return L;
}

void launch_serve(const InstDesc *insts, const WorkItem *ring, uint32_t ring_cap, ServeCtl *ctl,
                  unsigned int *done, unsigned int *sm_count, uint32_t reserved_sms,
                  unsigned long long idle_ns, const ServeLaunch &L, cudaStream_t st) {
    k_serve<<<L.blocks, L.threads, L.smem_bytes, st>>>(insts, ring, ring_cap, ctl, done, sm_count,
                                                       reserved_sms, idle_ns, L.cap);
    note_launches(1);
}

static uint32_t search_smem(uint32_t cap) { return SmemLayout(cap).bytes; }

SearchLaunch plan_search_launch(uint32_t max_m, uint32_t items, uint32_t threads,
                                uint32_t blocks_per_sm) {
    SearchLaunch L;
    L.cap = max_m < 2 ? 2 : max_m;
    L.threads = threads ? threads : 512;
    L.smem_bytes = search_smem(L.cap);
    int dev = 0, sms = 148, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // the limit is the kernel's, not this launch's: it stays at the largest
    // bucket any launch may hold, so that a smaller launch planned later does
    // not refuse a larger one planned earlier (a prepared build, a captured graph)
    const uint32_t limit = search_smem(MPHF_MAX_BUCKET);
    cudaFuncSetAttribute(k_search, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(L.smem_bytes > limit ? L.smem_bytes : limit));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_search, L.threads, L.smem_bytes);
    if (occ < 1) occ = 1;
    uint32_t per_sm = blocks_per_sm ? (blocks_per_sm < (uint32_t)occ ? blocks_per_sm : occ) : occ;
    uint64_t g = (uint64_t)sms * per_sm;
    if (g > items) g = items;
    L.blocks = g ? (uint32_t)g : 1;
    return L;
}

void launch_search(const InstDesc *d_inst, uint32_t ninst, const WorkItem *d_items, uint32_t items,
                   uint32_t *d_head, const SearchLaunch &L, StealQueue *steal, cudaStream_t st) {
    if (items == 0) return;
    k_search<<<L.blocks, L.threads, L.smem_bytes, st>>>(d_inst, ninst, d_items, items, d_head, L.cap,
                                                        steal, kStealCap);
    note_launches(1);
}

// ---------------------------------------------------------------------------
// Golomb-Rice: per-bucket lengths, then the bits (one warp per bucket).
// A node codes its value with its size's parameter tau; a ShockHash leaf
// codes its seed and appends its m-bit retrieval vector to the fixed part.
struct GrPiece {
    uint64_t fixed;  // fixed-part bits, LSB first
    uint32_t width;  // their number
    uint64_t high;   // unary part: zeros before the one
};
__device__ __forceinline__ GrPiece gr_piece(uint64_t v, uint32_t m, uint32_t t, uint32_t leaf, uint32_t bij) {
    GrPiece g;
    const bool shock = bij == MPHF_BIJECTION_SHOCKHASH && m <= leaf;
    const uint64_t coded = shock ? (v & MPHF_SH_MASK) : v;
    const uint64_t low = t ? (coded & ((t == 64) ? ~0ull : ((1ull << t) - 1))) : 0;
    g.fixed = shock ? (low | ((v >> MPHF_SH_BITS) << t)) : low;
    g.width = shock ? t + m : t;
    g.high = coded >> t;
    return g;
}

// Golomb-Rice code length of each bucket (Section 2.1, "Golomb-Rice";
// Section 2.2, "Representation"): fixed parts plus unary parts of its nodes.
__global__ void k_gr_len(const uint64_t *values, const uint16_t *node_m, const uint64_t *node_off,
                         uint64_t nb, const uint8_t *tau, uint32_t leaf, uint32_t bij,
                         uint64_t *bucket_bits) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t b = warp; b < nb; b += nwarps) {
        uint64_t bits = 0;
        for (uint64_t j = node_off[b] + lane; j < node_off[b + 1]; j += 32) {
            const uint32_t m = node_m[j];
            const GrPiece g = gr_piece(values[j], m, tau[m], leaf, bij);
            bits += g.width + 1 + g.high;
        }
        for (int d = 16; d; d >>= 1) bits += __shfl_xor_sync(0xffffffffu, bits, d);
        if (lane == 0) bucket_bits[b] = bits;
    }
}

void launch_gr_lengths(const uint64_t *values, const uint16_t *node_m, const uint64_t *node_off,
                       uint64_t nb, const uint8_t *tau, uint32_t leaf, uint32_t bij,
                       uint64_t *bucket_bits, cudaStream_t st) {
    if (nb == 0) return;
    k_gr_len<<<grid_for(nb * 32, 256), 256, 0, st>>>(values, node_m, node_off, nb, tau, leaf, bij,
                                                       bucket_bits);
    note_launches(1);
}

__device__ __forceinline__ void or_bits(uint64_t *w, uint64_t pos, uint64_t v, uint32_t len) {
    if (len == 0 || v == 0) return;
    uint32_t sh = (uint32_t)(pos & 63);
    atomicOr((unsigned long long *)&w[pos >> 6], (unsigned long long)(v << sh));
    if (sh + len > 64) atomicOr((unsigned long long *)&w[(pos >> 6) + 1], (unsigned long long)(v >> (64 - sh)));
}

// Golomb-Rice bits of each bucket (Section 2.2, "Representation"): all
// fixed parts of its nodes in preorder, then all unary parts.
__global__ void k_gr_write(const uint64_t *values, const uint16_t *node_m, const uint64_t *node_off,
                           const uint64_t *bit_pos, uint64_t nb, const uint8_t *tau,
                           const uint32_t *fixed_tab, const uint64_t *bucket_off, uint32_t leaf,
                           uint32_t bij, uint64_t *gr, uint64_t cap_bits, uint32_t *status) {
    // a prepared build reserved cap_bits: a longer code is refused, not written
    if (bit_pos[nb] > cap_bits) {
        if (status && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, ST_OVERFLOW);
        return;
    }
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t b = warp; b < nb; b += nwarps) {
        const uint64_t m = bucket_off[b + 1] - bucket_off[b];
        const uint64_t start = bit_pos[b];
        const uint64_t ustart = start + fixed_tab[m <= 4096 ? m : 0];
        uint64_t frun = 0, urun = 0;
        for (uint64_t j0 = node_off[b]; j0 < node_off[b + 1]; j0 += 32) {
            const uint64_t j = j0 + lane;
            const bool valid = j < node_off[b + 1];
            GrPiece g{0, 0, 0};
            if (valid) {
                const uint32_t mj = node_m[j];
                g = gr_piece(values[j], mj, tau[mj], leaf, bij);
            }
            const uint64_t ulen = valid ? g.high + 1 : 0;
            const uint64_t it = warp_incl_scan(g.width), iu = warp_incl_scan(ulen);
            if (valid) {
                or_bits(gr, start + frun + it - g.width, g.fixed, g.width);
                uint64_t up = ustart + urun + iu - 1;
                atomicOr((unsigned long long *)&gr[up >> 6], 1ull << (up & 63));
            }
            frun += __shfl_sync(0xffffffffu, it, 31);
            urun += __shfl_sync(0xffffffffu, iu, 31);
        }
    }
}

void launch_gr_write(const uint64_t *values, const uint16_t *node_m, const uint64_t *node_off,
                     const uint64_t *bit_pos, uint64_t nb, const uint8_t *tau,
                     const uint32_t *fixed_tab, const uint64_t *bucket_off, uint32_t leaf,
                     uint32_t bij, uint64_t *gr, cudaStream_t st, uint64_t cap_bits,
                     uint32_t *status) {
    if (nb == 0) return;
    k_gr_write<<<grid_for(nb * 32, 256), 256, 0, st>>>(values, node_m, node_off, bit_pos, nb, tau,
                                                         fixed_tab, bucket_off, leaf, bij, gr,
                                                         cap_bits, status);
    note_launches(1);
}

// ---------------------------------------------------------------------------
// Elias-Fano (Section 2.1): low L bits of v_i at [iL, iL + L), a one at
// (v_i >> L) + i in the high bits.
__global__ void k_ef_write(const uint64_t *v, uint64_t k, uint32_t L, uint64_t *low,
                           uint64_t *high) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < k;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t x = v[i];
        if (L) or_bits(low, i * L, x & ((L == 64) ? ~0ull : ((1ull << L) - 1)), L);
        uint64_t hb = (x >> L) + i;
        atomicOr((unsigned long long *)&high[hb >> 6], 1ull << (hb & 63));
    }
}

void launch_ef_write(const uint64_t *v, uint64_t k, uint32_t L, uint64_t *low, uint64_t *high,
                     cudaStream_t st) {
    if (k == 0) return;
    k_ef_write<<<grid_for(k, 256), 256, 0, st>>>(v, k, L, low, high);
    note_launches(1);
}

__global__ void k_popcount(const uint64_t *words, uint64_t n, uint64_t *out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = __popcll(words[i]);
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = 0;
}

// Stats: trials up to the stored value, and hash evaluations, per node kind
// (the smallest stored value is the number of failed trials, Section 5.1).
__global__ void k_stats(const uint64_t *values, const uint16_t *node_m, uint64_t n_nodes,
                        const uint64_t *n_nodes_dev, uint32_t leaf, uint32_t bij, uint32_t tree,
                        unsigned long long *counters) {
    __shared__ unsigned long long acc[8];
    if (threadIdx.x < 8) acc[threadIdx.x] = 0;
    if (n_nodes_dev && *n_nodes_dev < n_nodes) n_nodes = *n_nodes_dev;  // counted on the device
    __syncthreads();
    const Shape sh = make_shape(leaf, tree);
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n_nodes;
         j += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t m = node_m[j];
        uint32_t kind = node_kind(sh, m);
        uint64_t x = values[j];
        uint64_t trials = x + 1;
        if (kind == NODE_LEAF && bij == MPHF_BIJECTION_ROTATION) trials = x / m + 1;
        if (kind == NODE_LEAF && bij == MPHF_BIJECTION_SHOCKHASH) trials = (x & MPHF_SH_MASK) + 1;
        uint32_t idx = kind == NODE_LEAF ? 0 : kind == NODE_LOWER1 ? 1 : kind == NODE_LOWER2 ? 2 : 3;
        atomicAdd(&acc[idx], (unsigned long long)trials);
        atomicAdd(&acc[4 + idx], (unsigned long long)(trials * m));
    }
    __syncthreads();
    if (threadIdx.x < 8) atomicAdd(&counters[threadIdx.x], acc[threadIdx.x]);
}

void launch_stats(const uint64_t *values, const uint16_t *node_m, uint64_t n_nodes, uint32_t leaf,
                  uint32_t bij, uint32_t tree, uint64_t *counters, cudaStream_t st,
                  const uint64_t *n_nodes_dev) {
    if (n_nodes == 0) return;
    k_stats<<<grid_for(n_nodes, 256, 1024), 256, 0, st>>>(values, node_m, n_nodes, n_nodes_dev, leaf, bij,
                                                          tree, (unsigned long long *)counters);
    note_launches(1);
}

// ---------------------------------------------------------------------------
// Elias-Fano for a prepared build, whose code length is known only on the
// device: the sizes and word offsets of both sequences from the device totals
// (the same ef_dims as the host), then the writers and the popcounts of the
// second high-bit vector read them from there.
__global__ void k_ef_plan(const uint64_t *cum_keys, const uint64_t *bit_pos, uint64_t nb,
                          uint64_t cap_bits, EfPlan *p) {
    if (blockIdx.x || threadIdx.x) return;
    // a code longer than reserved was refused (k_gr_write); its Elias-Fano
    // sizes would not fit the arrays sized for cap_bits either, so nothing is written
    p->ok = bit_pos[nb] <= cap_bits;
    const EfDims a = ef_dims(nb + 1, cum_keys[nb]), b = ef_dims(nb + 1, p->ok ? bit_pos[nb] : 0);
    p->L[0] = a.L;
    p->L[1] = b.L;
    p->off[0] = 0;                                      // low words of the key offsets
    p->off[1] = a.low_words;                            // their high words
    p->off[2] = a.low_words + a.high_words;             // low words of the bit offsets
    p->off[3] = a.low_words + a.high_words + b.low_words;  // their high words
    p->high[0] = a.high_words;
    p->high[1] = b.high_words;
}

__global__ void k_ef_write_plan(const uint64_t *v, uint64_t k, const EfPlan *p, uint32_t which,
                                uint64_t *ef) {
    if (!p->ok) return;
    const uint32_t L = p->L[which];
    uint64_t *low = ef + p->off[2 * which], *high = ef + p->off[2 * which + 1];
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < k;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t x = v[i];
        if (L) or_bits(low, i * L, x & ((L == 64) ? ~0ull : ((1ull << L) - 1)), L);
        uint64_t hb = (x >> L) + i;
        atomicOr((unsigned long long *)&high[hb >> 6], 1ull << (hb & 63));
    }
}

// out[w] = ones in word w of the bit offsets' high vector for w < max_words
// (zero past its end: the buffer is zeroed up to the reserved size), out[max_words] = 0.
__global__ void k_popcount_plan(const uint64_t *ef, const EfPlan *p, uint64_t max_words, uint64_t *out) {
    const uint64_t *high = ef + p->off[3];
    const uint64_t words = p->ok ? p->high[1] : 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= max_words;
         i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = i < words ? __popcll(high[i]) : 0;
}

void launch_ef_planned(const uint64_t *cum_keys, const uint64_t *bit_pos, uint64_t nb, uint64_t cap_bits,
                       EfPlan *p, uint64_t *ef, uint64_t max_high1, uint64_t *rank1, uint64_t *tmp,
                       cudaStream_t st) {
    k_ef_plan<<<1, 32, 0, st>>>(cum_keys, bit_pos, nb, cap_bits, p);
    k_ef_write_plan<<<grid_for(nb + 1, 256), 256, 0, st>>>(cum_keys, nb + 1, p, 0, ef);
    k_ef_write_plan<<<grid_for(nb + 1, 256), 256, 0, st>>>(bit_pos, nb + 1, p, 1, ef);
    k_popcount_plan<<<grid_for(max_high1 + 1, 256), 256, 0, st>>>(ef, p, max_high1, rank1);
    note_launches(4);
    launch_exclusive_scan(rank1, max_high1 + 1, tmp, st);
}

// Rank directory of a bit vector: out[w] = ones in words [0, w) (select support).
void launch_rank_dir(const uint64_t *words, uint64_t nwords, uint64_t *dir, uint64_t *tmp,
                     cudaStream_t st) {
    k_popcount<<<grid_for(nwords + 1, 256), 256, 0, st>>>(words, nwords, dir);
    note_launches(1);
    launch_exclusive_scan(dir, nwords + 1, tmp, st);
}

// For the select_1 queries of Section 2.2, "Query", on the Elias-Fano high
// bits.  Select directory of a bit vector: sel[j] = the word holding one number
// 64 j.  Word w holds the ones dir[w] .. dir[w + 1] - 1, so it writes every
// multiple of 64 in that range (each entry exactly once).
__global__ void k_select_dir(uint64_t nwords, const uint64_t *dir, uint64_t *sel) {
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < nwords;
         w += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t first = dir[w], end = dir[w + 1];
        for (uint64_t j = (first + 63) >> 6; (j << 6) < end; j++) sel[j] = w;
    }
}

void launch_select_dir(uint64_t nwords, const uint64_t *dir, uint64_t *sel, cudaStream_t st) {
    if (nwords == 0) return;
    k_select_dir<<<grid_for(nwords, 256), 256, 0, st>>>(nwords, dir, sel);
    note_launches(1);
}

// ---------------------------------------------------------------------------
// The totals of a batch of prepared builds in one array, so that one copy to
// the host finishes them all: per build 16 words, [0] its status word (status
// bits, largest bucket above bit 32), [1] stored nodes, [2] code bits, [8..15]
// its search counters; the other words are zero.
__global__ void k_gather_totals(const BuildTotalsSrc *src, uint32_t count, uint64_t *out) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < 16ull * count;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const BuildTotalsSrc &s = src[t >> 4];
        const uint32_t j = (uint32_t)(t & 15);
        uint64_t v = 0;
        if (j == 0) v = ((uint64_t)s.status[1] << 32) | s.status[0];
        else if (j == 1) v = *s.nodes;
        else if (j == 2) v = *s.bits;
        else if (j >= 8) v = s.counters[j - 8];
        out[t] = v;
    }
}

void launch_gather_totals(const BuildTotalsSrc *src, uint32_t count, uint64_t *out, cudaStream_t st) {
    if (count == 0) return;
    k_gather_totals<<<grid_for(16ull * count, 256), 256, 0, st>>>(src, count, out);
    note_launches(1);
}

}  // namespace rs
