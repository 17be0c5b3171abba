// engine.h -- internal interface between the C-ABI layer and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rs {

// Device status bits of one build (host maps them to error codes with the
// precedence bucket size > duplicate > search cap > wait timeout).
enum : uint32_t {
    ST_BUCKET = 1u, ST_DUPLICATE = 2u, ST_LIMIT = 4u, ST_TIMEOUT = 8u, ST_RANGE = 16u,
    ST_OVERFLOW = 32u  // a prepared build's packed words outgrew the space reserved for them
};

// Buckets a build covers: the consecutive range [b_lo, b_lo + nb) of a function
// whose keys hash to nb_hash buckets (b_lo = 0, nb_hash = nb for a whole function).
struct BucketRange {
    uint64_t nb_hash, b_lo;
};

// Per-build descriptor read by the search kernel (one per instance of a batch).
struct InstDesc {
    const uint64_t *lo;          // fingerprint lo words, grouped by bucket
    const uint8_t *bb;           // B bit (hi & 1) of the same keys
    const uint64_t *bucket_off;  // nb + 1 key offsets
    const uint64_t *node_off;    // nb + 1 node offsets
    const uint32_t *nodes_tab;   // stored nodes per subtree size
    uint64_t *values;            // node values, preorder per bucket
    uint16_t *node_m;            // node sizes, same order
    uint32_t *status;            // ST_* bits
    uint64_t max_value;
    uint32_t leaf, bij;          // bij: MPHF_BIJECTION_* leaf method
    uint32_t tree;               // MPHF_TREE_*: lower aggregation levels or fanout 2 everywhere
    uint32_t nb;
    uint32_t red_leaf;           // 2^32 mod l, for the remainders of full leaves
    uint32_t leaf_method;        // 0 lock-step, 1 early rejection, 2 early rejection + table
    uint32_t spt;                // seeds per thread of full lower-level split searches (1, 2, 4)
    const uint8_t *rot_canon;    // per m <= 16 at offset 2^m - 4: canonical rotation of x
    const uint8_t *rot_period;   // same layout: rotation period of x
    const uint32_t *mod_c;       // exact remainder constants per node size (ModRT)
    const uint64_t *mod_M;
};

// One unit of work: a bucket of an instance (inst = all ones: an empty slot).
struct WorkItem {
    uint32_t inst, bucket;
};

struct SearchLaunch {
    uint32_t threads;        // per block
    uint32_t blocks;         // persistent grid size
    uint32_t smem_bytes;     // dynamic shared memory
    uint32_t cap;            // largest bucket the blocks hold
};

// The serving search's queue: items [head, tail) of the ring are published
// and not yet claimed; stop asks idle blocks to leave; err records a block
// that gave up waiting on a contended claim.
struct ServeCtl {
    unsigned long long head, tail;
    unsigned int stop, err;
};
constexpr uint32_t kServeMaxSms = 1024;  // entries of the per-SM block counter (power of two)

struct ServeLaunch {
    uint32_t threads, blocks, smem_bytes, cap;
    uint32_t working_blocks;  // blocks left after the reserved SMs' second blocks exit
};

// Kernels launched by this library in this process (every launcher adds its count).
void note_launches(uint64_t k);
uint64_t launches_total();

// Stage launchers (all asynchronous on `st`).
void launch_fp_hist(const void *keys, uint64_t n, uint32_t key_bytes, uint64_t nb,
                    const BucketRange &R, uint64_t *counts, uint32_t *status, cudaStream_t st);
// Two-level counting sort (nb <= 8192): number of blocks for n keys, 0 when
// the build must use launch_fp_hist / launch_scatter instead.  blk holds
// G * nb counters.
uint32_t sort_blocks(uint64_t n, uint64_t nb);
void launch_fp_hist_blk(const void *keys, uint64_t n, uint32_t key_bytes, uint64_t nb,
                        const BucketRange &R, uint32_t G, uint64_t *counts, uint32_t *blk,
                        uint32_t *status, cudaStream_t st);
void launch_scatter_blk(const void *keys, uint64_t n, uint32_t key_bytes, uint64_t nb,
                        const BucketRange &R, uint32_t G, const uint64_t *bucket_off, uint32_t *blk,
                        uint64_t *lo, uint8_t *bb, uint32_t *status, cudaStream_t st);
void launch_plan(const uint64_t *counts, uint64_t nb, const uint32_t *nodes_tab, uint64_t *node_cnt,
                 uint32_t *status, uint32_t *max_m, uint64_t *size_hist, cudaStream_t st);
// Work items of one instance ordered by decreasing bucket size; size_off is
// the exclusive scan of the size histogram (4097 + 1 entries), size_cursor
// 4097 zeroed counters.
void launch_items_by_size(const uint64_t *bucket_off, uint64_t nb, const uint64_t *size_off,
                          uint32_t *size_cursor, WorkItem *items, uint32_t inst, cudaStream_t st);
// Exclusive scan of n + 1 values in place (the last input should be 0; the
// last output is then the total).  tmp needs scan_tmp_words(n + 1) words.
uint64_t scan_tmp_words(uint64_t len);
void launch_exclusive_scan(uint64_t *data, uint64_t len, uint64_t *tmp, cudaStream_t st);
void launch_scatter(const void *keys, uint64_t n, uint32_t key_bytes, uint64_t nb,
                    const BucketRange &R, const uint64_t *bucket_off, uint32_t *cursor, uint64_t *lo,
                    uint8_t *bb, uint32_t *status, cudaStream_t st);
SearchLaunch plan_search_launch(uint32_t max_m, uint32_t items, uint32_t threads, uint32_t blocks_per_sm);
// Nodes given away by busy blocks to idle ones at the end of a search (see
// k_search): a node is (build, bucket, key offset | size << 16, preorder
// index | depth << 16 | ready bit); zero it (kStealBytes) before each launch.
struct StealItem {
    unsigned int w[4];
};
struct StealQueue {
    unsigned int tail, head, idle, busy;
    StealItem items[1];  // kStealCap entries, then kHelpCap HelpRec (help_recs())
};
// A node search shared with idle blocks by seed range (see k_search): rounds
// of blockDim * seeds-per-thread consecutive seeds are claimed in order from
// next_round; the smallest valid seed any block finds goes to best.
struct HelpRec {
    unsigned int state;       // 0 closed, 1 open to helpers, 2 closing
    unsigned int helpers;     // helper blocks inside the search
    unsigned int gen;         // raised at every closing
    unsigned int next_round;
    unsigned int inst, bucket, gpos, m;  // the node: build, bucket, key offset in the bucket, size
    unsigned long long best;
};
constexpr uint32_t kStealCap = 32768;
constexpr uint32_t kHelpCap = 4096;  // one record per block of the launch (more blocks: no sharing)
constexpr size_t kStealItemsEnd = 16 + sizeof(StealItem) * kStealCap;
constexpr size_t kStealBytes = kStealItemsEnd + sizeof(HelpRec) * kHelpCap;
__host__ __device__ inline HelpRec *help_recs(StealQueue *q) {
    return (HelpRec *)((char *)q + kStealItemsEnd);
}
void launch_search(const InstDesc *d_inst, uint32_t ninst, const WorkItem *d_items, uint32_t items,
                   uint32_t *d_head, const SearchLaunch &L, StealQueue *steal, cudaStream_t st);
// The serving search (reads work from a ring the host appends to; see k_serve).
ServeLaunch plan_serve_launch(uint32_t threads, uint32_t reserved_sms);
void launch_serve(const InstDesc *insts, const WorkItem *ring, uint32_t ring_cap, ServeCtl *ctl,
                  unsigned int *done, unsigned int *sm_count, uint32_t reserved_sms,
                  unsigned long long idle_ns, const ServeLaunch &L, cudaStream_t st);
// Golomb-Rice coding of the stored values (a ShockHash leaf codes its seed
// and appends its retrieval vector to the fixed part).
void launch_gr_lengths(const uint64_t *values, const uint16_t *node_m, const uint64_t *node_off,
                       uint64_t nb, const uint8_t *tau, uint32_t leaf, uint32_t bij,
                       uint64_t *bucket_bits, cudaStream_t st);
// cap_bits / status: a prepared build's reserved code length; a longer code
// sets ST_OVERFLOW and writes nothing.
void launch_gr_write(const uint64_t *values, const uint16_t *node_m, const uint64_t *node_off,
                     const uint64_t *bit_pos, uint64_t nb, const uint8_t *tau,
                     const uint32_t *fixed_tab, const uint64_t *bucket_off, uint32_t leaf,
                     uint32_t bij, uint64_t *gr, cudaStream_t st, uint64_t cap_bits = ~0ull,
                     uint32_t *status = nullptr);
void launch_ef_write(const uint64_t *v, uint64_t k, uint32_t L, uint64_t *low, uint64_t *high,
                     cudaStream_t st);
// dir[w] = ones in words [0, w), w in [0, nwords]; tmp: scan_tmp_words(nwords + 1).
void launch_rank_dir(const uint64_t *words, uint64_t nwords, uint64_t *dir, uint64_t *tmp,
                     cudaStream_t st);
// sel[j] = the word holding one number 64 j (0-based), from the rank directory.
void launch_select_dir(uint64_t nwords, const uint64_t *dir, uint64_t *sel, cudaStream_t st);
// n_nodes bounds the grid; n_nodes_dev (if given) is the count on the device.
void launch_stats(const uint64_t *values, const uint16_t *node_m, uint64_t n_nodes, uint32_t leaf,
                  uint32_t bij, uint32_t tree, uint64_t *counters, cudaStream_t st,
                  const uint64_t *n_nodes_dev = nullptr);
// Elias-Fano of a prepared build (code length known only on the device): the
// sizes and word offsets of both sequences, as ef_dims gives them.
struct EfPlan {
    uint32_t ok;       // the code fits the reserved length (else nothing is written)
    uint32_t L[2];
    uint64_t off[4];   // low and high words of the key offsets, then of the bit offsets
    uint64_t high[2];  // high words of each sequence
};
// Writes both sequences into the zeroed ef (sized for the largest possible
// code), and rank1 = the rank directory of the bit offsets' high vector over
// max_high1 words (tmp: scan_tmp_words(max_high1 + 1)).
void launch_ef_planned(const uint64_t *cum_keys, const uint64_t *bit_pos, uint64_t nb, uint64_t cap_bits,
                       EfPlan *p, uint64_t *ef, uint64_t max_high1, uint64_t *rank1, uint64_t *tmp,
                       cudaStream_t st);

// Where a prepared build keeps its totals on the device (status word, stored
// nodes, code bits, search counters); k_gather_totals packs them 16 words per
// build.
struct BuildTotalsSrc {
    const uint32_t *status;  // [0] status bits, [1] largest bucket
    const uint64_t *nodes;
    const uint64_t *bits;
    const uint64_t *counters;  // 8 words
};
void launch_gather_totals(const BuildTotalsSrc *src, uint32_t count, uint64_t *out, cudaStream_t st);

// Building one function on several GPUs (bucket ranges, Section 5.2).
// Keys grouped by the rank owning their bucket (nb buckets, `world` ranges):
// counts[r] += keys of rank r; then each key to cursor[r]++ in `out`.
void launch_route_count(const uint64_t *keys, uint64_t n, uint32_t kb, uint64_t nb, uint32_t world,
                        uint64_t *counts, cudaStream_t st);
void launch_route_scatter(const uint64_t *keys, uint64_t n, uint32_t kb, uint64_t nb, uint32_t world,
                          uint64_t *cursor, uint64_t *out, cudaStream_t st);
void launch_shard_offsets(const uint64_t *in, uint64_t count, uint64_t base, uint64_t *out,
                          cudaStream_t st);
void launch_shard_bits(const uint64_t *in, uint64_t bits, uint64_t at, uint64_t *out, cudaStream_t st);

// Query side.
constexpr uint32_t kSaltLevels = 64;  // salt levels kept in a table (a walk uses at most 16)
struct QueryView {
    const uint64_t *gr;
    const uint64_t *ef_low[2], *ef_high[2];
    const uint64_t *ef_dir[2];   // ones before each high word
    const uint64_t *ef_sel[2];   // the high word holding element 64 j, per j
    uint32_t ef_L[2];
    const uint8_t *tau;
    const uint32_t *nodes_tab, *fixed_tab;
    const uint16_t *left_tab;   // left part per fanout-2 node size
    const uint32_t *mod_c;      // exact remainder constants per node size
    const uint64_t *mod_M;
    const uint64_t *salts;      // level_salt(L) for L < kSaltLevels
    uint64_t nb;
    uint32_t leaf, bij, key_bytes, tree;
    uint32_t magic_leaf, magic_l1;  // ceil(2^32 / l), ceil(2^32 / lower-1 size)
    uint32_t lower1, lower2;
};
void launch_query(const QueryView &q, const void *keys, uint64_t n, uint64_t *out, cudaStream_t st);
void launch_mark(const uint64_t *vals, uint64_t n, uint32_t *bitmap, unsigned long long *bad,
                 cudaStream_t st);

}  // namespace rs
