/*
 * mphf.h -- C ABI of the B300 RecSplit construction library (libmphf.so).
 *
 * Builds a RecSplit minimal perfect hash function (MPHF) with rotation
 * fitting (or plain brute-force or ShockHash leaves) on one CUDA device, after Bez, Kurpicz, Lehmann and Sanders,
 * "High Performance Construction of RecSplit Based Minimal Perfect Hash
 * Functions" (arXiv 2212.09562).  The problem (Section 1): given a set S of
 * n distinct keys, build h with h bijective from S onto [0, n); outside S the
 * value is arbitrary.
 *
 * Conventions for every entry point:
 *   - Pointers prefixed d_ are device pointers, h_ are host pointers.
 *   - Streams are cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Work is ordered on the given stream.  Functions that return
 *     a device-side error code (build, verify) synchronise the stream
 *     before returning; mphf_query does not.
 *   - Keys are caller-owned, 8-byte aligned, and must stay valid until the
 *     call returns.  A misaligned key or output pointer gives MPHF_EINVAL
 *     before any device work.
 *     A key is 8 bytes (one little-endian 64-bit word) or 16 bytes (two
 *     words, the first is w0).  Keys must be distinct.
 *   - A function lives on the device that was current when it was built
 *     or loaded; query and verify it with that device current (else
 *     MPHF_EINVAL).
 *   - Everything a build allocates belongs to the returned mphf_t and is
 *     released by mphf_free.  Device memory comes from the allocator in the
 *     build parameters, or from cudaMallocAsync on the stream.
 *   - Every function returns MPHF_OK (0) or a negative error code below.  No
 *     exception crosses the ABI and no device code traps: device errors are
 *     reported through a status word that the host reads.
 */
#ifndef MPHF_H
#define MPHF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPHF_OK 0
#define MPHF_EINVAL (-1)         /* bad argument: leaf_size, bucket_size, key_bytes, n, NULL  */
#define MPHF_ENOMEM (-2)         /* an allocation failed                                     */
#define MPHF_ECUDA (-3)          /* a CUDA runtime call failed                               */
#define MPHF_EDUPLICATE (-4)     /* two keys of one bucket share the fingerprint's lo word   */
#define MPHF_ESEARCH_LIMIT (-5)  /* some node needs a value above max_value                  */
#define MPHF_EBUSY (-6)          /* server full (no free slot or device memory)              */
#define MPHF_EBUCKET (-7)        /* a bucket holds more than MPHF_MAX_BUCKET keys            */
#define MPHF_ENOTIMPL (-8)       /* not supported by this build of the library               */
#define MPHF_ETIMEOUT (-9)       /* a bounded device wait gave up                            */
#define MPHF_ECAPACITY (-10)     /* a prepared build's packed function outgrew the space
                                    reserved for it (build it with mphf_build_ex instead)    */

#define MPHF_MAX_BUCKET 4096u    /* largest bucket a build accepts (keys)                    */
#define MPHF_MAX_LEAF 24u        /* leaf sizes 2..24                                          */
#define MPHF_MAX_BUCKET_SIZE 3000u /* bucket_size parameter b in 1..3000                      */
#define MPHF_DEFAULT_MAX_VALUE 0xFFFFFFFFFFull /* 2^40 - 1                                    */

typedef struct mphf mphf_t;

/* Device allocator hooks.  alloc returns NULL on failure. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*free)(void *ptr, void *stream, void *ctx);
    void *ctx;
} mphf_allocator;

/* Build parameters.  Fields left 0 by mphf_default_params take defaults.
 *   leaf_size        l, 2..24 (Section 2.2: leaves of l keys).
 *   bucket_size      b, 1..3000; nb = ceil(n / b) buckets.
 *   key_bytes        8 or 16.
 *   leaf_bijection   how a leaf's bijection is found (the stored values
 *                    differ between the three):
 *                    MPHF_BIJECTION_PLAIN     brute force over seeds (Section
 *                                             2.2, "Bijections");
 *                    MPHF_BIJECTION_ROTATION  rotation fitting (Section 4);
 *                    MPHF_BIJECTION_SHOCKHASH ShockHash (Appendix C): a seed
 *                                             whose two cells per key admit a
 *                                             bijection, one retrieved bit per
 *                                             key choosing the cell.
 *   max_value        largest value any node may store; a node that needs
 *                    more fails the build with MPHF_ESEARCH_LIMIT.
 *   threads_per_block, blocks_per_sm
 *                    launch shape of the search kernel; 0 = the default:
 *                    512 threads when a build of the launch has lower
 *                    aggregation levels with l >= 14, else 256, and as many
 *                    blocks per SM as fit.
 *   tree_shape       MPHF_TREE_RECSPLIT: leaves under two lower aggregation
 *                    levels with fanouts f1, f2 of l, fanout 2 above (Section
 *                    2.2, "Splitting Trees"); MPHF_TREE_FANOUT2: fanout 2 for
 *                    the entire tree, each left part a multiple of l (the
 *                    configuration Appendix C uses with ShockHash leaves).
 *   seeds_per_thread seeds each thread tests per round in the split search of
 *                    full lower-level nodes (each key load feeds that many
 *                    independent hash chains): 1, 2 or 4; 0 = the default
 *                    (2 for l >= 16, else 1).  The result does not depend on
 *                    it; the autotuner picks it per device and leaf size.
 *   leaf_method      how plain and rotation leaves are searched (same result
 *                    every time; ShockHash leaves have one search):
 *                    MPHF_LEAF_LOCKSTEP  every trial hashes all m keys
 *                                        (default, the fastest measured);
 *                    MPHF_LEAF_EARLY     a trial stops at its first collision;
 *                    MPHF_LEAF_TABLE     as EARLY, the rotation from a table of
 *                                        canonical rotations (leaves of <= 16
 *                                        keys; Section 4, "Lookup Tables"). */
#define MPHF_TREE_RECSPLIT 0u
#define MPHF_TREE_FANOUT2 1u
#define MPHF_BIJECTION_PLAIN 0u
#define MPHF_BIJECTION_ROTATION 1u
#define MPHF_BIJECTION_SHOCKHASH 2u
/* A ShockHash leaf of m keys stores its seed in bits 0..39 of the value and
 * its m-bit retrieval vector Z in bits 40..: key x takes its second cell iff
 * parity(row(x) & Z) = 1.  Its seed is capped at 2^40 - 1 whatever max_value. */
#define MPHF_SH_SEED_BITS 40u
#define MPHF_LEAF_LOCKSTEP 0u
#define MPHF_LEAF_EARLY 1u
#define MPHF_LEAF_TABLE 2u
typedef struct {
    uint32_t leaf_size;
    uint32_t bucket_size;
    uint32_t key_bytes;
    uint32_t leaf_bijection;
    uint64_t max_value;
    const mphf_allocator *allocator;
    uint32_t threads_per_block;
    uint32_t blocks_per_sm;
    uint32_t leaf_method;
    uint32_t tree_shape;
    uint32_t seeds_per_thread;
    uint32_t reserved;           /* 0 */
} mphf_build_params;

/* Sizes and parameters of a built function. */
typedef struct {
    uint64_t n, nb;            /* keys, buckets                                    */
    uint32_t leaf_size, bucket_size, key_bytes, leaf_bijection;
    uint64_t n_nodes;          /* stored values (nodes with >= 2 keys)              */
    uint64_t gr_bits;          /* Golomb-Rice bit length                           */
    uint64_t gr_words;         /* 64-bit words holding them                        */
    uint64_t ef_words;         /* words of the two Elias-Fano sequences            */
    uint32_t ef_low_bits[2];   /* L of the key-count / bit-position sequences      */
    uint64_t ef_seq_words[4];  /* low, high words of sequence 0, then sequence 1   */
    uint32_t max_bucket;       /* largest bucket seen                              */
    uint32_t tree_shape;       /* MPHF_TREE_*                                      */
} mphf_info;

/* Work done by the searches, per node kind (0 leaf, 1 lower-1 split, 2 lower-2
 * split, 3 fanout-2 split): trials = candidate values up to and including the
 * stored one (one k counts once for rotation leaves); evals = trials * m. */
typedef struct {
    uint64_t trials[4];
    uint64_t evals[4];
    /* device time: fingerprint/plan up to the first host read, the search
     * kernel alone, the packing after it, and the whole build */
    float ms_plan, ms_search, ms_pack, ms_total;
} mphf_stats;

/* Fills *p with leaf 16, bucket 2000, 8-byte keys, rotation fitting on,
 * max_value MPHF_DEFAULT_MAX_VALUE, default allocator and launch shape,
 * MPHF_LEAF_LOCKSTEP leaves. */
void mphf_default_params(mphf_build_params *p);

/* Builds the function of the n keys at d_keys (Section 2.2, the whole
 * construction: fingerprint, bucket sort, split and leaf searches, preorder
 * Golomb-Rice and Elias-Fano packing, all on the device).  Shorthand for
 * mphf_build_ex with 8-byte keys and rotation fitting on.  n = 0 gives a
 * valid empty function.  On success *out owns the result.  Synchronises
 * the stream. */
int mphf_build(const void *d_keys, uint64_t n, uint32_t leaf_size, uint32_t bucket_size,
               void *stream, mphf_t **out);

/* The same with every parameter explicit (mphf_build_params; start from
 * mphf_default_params).  Keys: n keys of params->key_bytes bytes at d_keys,
 * read only.  Errors (on any error *out is NULL and nothing stays allocated):
 *   MPHF_EINVAL         a parameter out of range, n >= 2^32, d_keys NULL or
 *                       not 8-byte aligned with n > 0, out or params NULL;
 *   MPHF_ENOMEM         a device allocation failed;
 *   MPHF_EDUPLICATE     two keys of one bucket share the fingerprint's lo
 *                       word (equal keys, or a 2^-64 accident);
 *   MPHF_EBUCKET        a bucket holds more than MPHF_MAX_BUCKET keys;
 *   MPHF_ESEARCH_LIMIT  a node needs a value above max_value;
 *   MPHF_ECUDA          a CUDA runtime call failed. */
int mphf_build_ex(const void *d_keys, uint64_t n, const mphf_build_params *params, void *stream,
                  mphf_t **out);

/* Same as mphf_build_ex with the keys in host memory: the keys are copied
 * to the device inside the call (pinned host memory gives the fastest copy).
 * The parameters and n are checked before anything is allocated or copied. */
int mphf_build_host(const void *h_keys, uint64_t n, const mphf_build_params *params,
                    void *stream, mphf_t **out);

/* ---------------------------------------------------------------------------
 * A build in three calls, whose device work can be captured once in a CUDA
 * graph and replayed on new keys (the paper has no counterpart).  A plain
 * build reads its node count and code length back to the host to size its
 * outputs; a prepared build reserves upper bounds instead (n values, and
 * gr_capacity_bits of Golomb-Rice code: 0 = 16 bits per key + 128 per bucket
 * + 4096, about ten times what any leaf method needs), so enqueueing it
 * involves no allocation and no host synchronisation.  The stored words are
 * those of mphf_build_ex on the same keys. */

/* Allocates a build of exactly n keys (1 <= n < 2^32) with params (as for
 * mphf_build_ex) on the current device, through params->allocator if given.
 * *out is not a usable function until mphf_build_finish succeeds.  Errors:
 * MPHF_EINVAL (bad parameters or n = 0), MPHF_ENOMEM, MPHF_ECUDA.
 * Synchronises the device. */
int mphf_build_prepare(uint64_t n, const mphf_build_params *params, uint64_t gr_capacity_bits,
                       mphf_t **out);

/* Issues the whole build of the n keys at d_keys (device, 8-byte aligned,
 * key_bytes each) on the stream: memsets and kernels only, so it may run
 * inside stream capture; a captured graph rebuilds from whatever keys are at
 * d_keys when it is launched.  The previous contents of h are overwritten.
 * MPHF_EINVAL for a handle not made by mphf_build_prepare, a bad pointer or
 * another device current than h's. */
int mphf_build_enqueue(mphf_t *h, const void *d_keys, void *stream);

/* Waits for the stream, then reads the build's status and totals back and
 * makes h a usable function.  Returns the build's error, if any
 * (MPHF_EDUPLICATE, MPHF_EBUCKET, MPHF_ESEARCH_LIMIT, or MPHF_ECAPACITY when
 * the code outgrew gr_capacity_bits), in which case h stays unusable until
 * the next successful enqueue and finish. */
int mphf_build_finish(mphf_t *h, void *stream);

/* Prepared builds searched together: the buckets of all of them go through
 * ONE persistent search launch (the work order of mphf_build_batch), and the
 * whole batch is enqueued without allocation or host synchronisation, so
 * that it, too, can be captured in a CUDA graph.  The batch refers to the
 * handles (it does not own them): they must stay allocated while the batch
 * is used, and no handle may be enqueued elsewhere while the batch's work on
 * it is in flight. */
typedef struct mphf_batch mphf_batch_t;

/* Makes a batch of count >= 1 distinct handles from mphf_build_prepare, all
 * on the current device.  threads_per_block (0 = 512 when some build has
 * RecSplit lower levels of leaf size >= 14, else 256; otherwise a multiple of
 * 32 in [64, 512]) and blocks_per_sm (0 = the occupancy limit) shape the
 * search launch.  The batch's own scratch comes from allocator (NULL =
 * stream-ordered cudaMallocAsync).  Errors: MPHF_EINVAL (a NULL, repeated,
 * unprepared or other-device handle, a bad launch shape, 2^32 or more buckets
 * in all), MPHF_ENOMEM, MPHF_ECUDA.  Synchronises the device. */
int mphf_batch_prepare(mphf_t *const *handles, uint32_t count, uint32_t threads_per_block,
                       uint32_t blocks_per_sm, const mphf_allocator *allocator,
                       mphf_batch_t **out);

/* Issues every build of the batch on the stream: handle i builds from the
 * keys at d_keys[i] (a host array of count device pointers, each 8-byte
 * aligned, holding that handle's n keys; the pointers are read now, the keys
 * when the work runs).  Memsets and kernels only.  MPHF_EINVAL for a bad
 * pointer or another device current than the batch's. */
int mphf_batch_enqueue(mphf_batch_t *b, const void *const *d_keys, void *stream);

/* Waits for the stream, reads all builds' totals back in one copy and
 * finishes each handle as mphf_build_finish would.  statuses (may be NULL)
 * receives each build's code; the return value is MPHF_OK if all succeeded,
 * else the first failure (the failed handles stay unusable). */
int mphf_batch_finish(mphf_batch_t *b, void *stream, int *statuses);

/* Releases the batch's scratch (not its handles).  Synchronises its device.
 * MPHF_EINVAL for NULL. */
int mphf_batch_free(mphf_batch_t *b);

/* ---------------------------------------------------------------------------
 * One function built on several GPUs (Section 5.2, "Multi-Threading": each
 * worker builds a consecutive range of buckets; the local Golomb-Rice
 * sequences and bucket offsets are concatenated).  Rank r of `world` owns
 * buckets [floor(r nb / world), floor((r + 1) nb / world)) of the function
 * over n_total keys, nb = ceil(n_total / bucket_size).  The steps:
 *   1. mphf_shard_route on each rank's own keys: keys grouped by owner rank;
 *   2. an exchange of keys between ranks (the caller's collective, e.g. an
 *      all-to-all) so that each rank holds exactly its buckets' keys;
 *   3. mphf_build_shard on each rank: the rank's buckets, searched and packed;
 *   4. mphf_shard_pack, and a gather of every rank's pack (the caller's
 *      collective) to wherever the whole function is wanted;
 *   5. mphf_shard_concat: the whole function, word for word the one that
 *      mphf_build_ex makes from all n_total keys on one device. */
#define MPHF_MAX_SHARDS 1024u

/* Groups the n keys at d_keys (device, key_bytes each, 8-byte aligned) by
 * the rank that owns their bucket: d_out (n keys, device) receives rank 0's
 * keys, then rank 1's, ...; h_counts[r] (host, world entries) the number of
 * keys for rank r.  The order within a rank's keys is unspecified (builds do
 * not depend on it).  Errors: MPHF_EINVAL for bad sizes or pointers
 * (n <= n_total < 2^32, world <= MPHF_MAX_SHARDS), MPHF_ENOMEM, MPHF_ECUDA.
 * Synchronises the stream. */
int mphf_shard_route(const void *d_keys, uint64_t n, uint32_t key_bytes, uint64_t n_total,
                     uint32_t bucket_size, uint32_t world, void *d_out, uint64_t *h_counts,
                     void *stream);

/* Builds rank `rank`'s buckets of the function over n_total keys from the n
 * keys at d_keys, which must be exactly the keys of those buckets (any other
 * key gives MPHF_EINVAL).  params as for mphf_build_ex.  The shard holds the
 * range's node values, local offsets (starting at 0) and its own Golomb-Rice
 * sequence (mphf_get_values, mphf_get_bits, mphf_get_stats work); it cannot
 * be queried, verified or serialised (MPHF_EINVAL).  Free with mphf_free. */
int mphf_build_shard(const void *d_keys, uint64_t n, uint64_t n_total,
                     const mphf_build_params *params, uint32_t rank, uint32_t world,
                     void *stream, mphf_t **out);

/* Writes a shard into the device buffer d_buf (8-byte aligned) of *len bytes:
 * 24 header words (magic "RMPFSHD1", n, the range's bucket count, its first
 * bucket, n_total, node count, Golomb-Rice bits, leaf_size | tree_shape << 16,
 * bucket_size, key_bytes, leaf_bijection, largest bucket, 4 zero words, the
 * 4 trial and 4 evaluation counters of mphf_stats), then cum_keys, node_off,
 * bit_pos (nb + 1 words each), the node values and the Golomb-Rice words.
 * With d_buf NULL, *len receives the size needed.  MPHF_EINVAL for a handle
 * that is not a shard or a buffer too small.  Synchronises the stream. */
int mphf_shard_pack(const mphf_t *shard, void *d_buf, size_t *len, void *stream);

/* Builds the whole function on the current device from the packs of ranks
 * 0..count-1 (device memory, lens[i] bytes each, in rank order): node values
 * and offsets concatenated, Golomb-Rice sequences joined at their bit
 * offsets, the Elias-Fano sequences and query directories built once.  The
 * statistics are the sums of the shards'.  MPHF_EINVAL unless the packs are
 * the ranks of one function in order.  Device memory from allocator (NULL:
 * cudaMallocAsync).  Synchronises the stream. */
int mphf_shard_concat(const void *const *d_parts, const size_t *lens, uint32_t count,
                      const mphf_allocator *allocator, void *stream, mphf_t **out);

/* Evaluates h on n keys (Section 2.2, "Query"; Section 4 for the rotation
 * of the keys in B; Appendix C for the retrieved cell of a ShockHash leaf).
 * d_out[i] = h(key i) in [0, n_built) for keys of the built set; d_out holds
 * n 8-byte-aligned words.  Asynchronous on the stream.  Errors: MPHF_EINVAL
 * for a NULL or misaligned pointer with n > 0, a function with no keys, or
 * another device current than the function's. */
int mphf_query(const mphf_t *h, const void *d_keys, uint64_t n, uint64_t *d_out, void *stream);

/* Checks on the device that h maps the n keys at d_keys bijectively onto
 * [0, n) (queries them, marks a bitmap).  *n_bad = keys whose value was out
 * of range or already taken; 0 means a bijection.  Scratch comes from h's
 * allocator.  Errors: those of mphf_query, MPHF_ENOMEM.  Synchronises. */
int mphf_verify(const mphf_t *h, const void *d_keys, uint64_t n, uint64_t *n_bad, void *stream);

/* The same check without allocating: it uses a fixed scratch area that the
 * library reserves in device memory (about 8.5 MB on every GPU where the
 * library is loaded, held until the process exits).  For callers that cannot
 * allocate device memory at this point: memory owned and budgeted by another
 * allocator, latency-critical paths where allocation may stall the device,
 * or code where allocation is not permitted.  The paper has no counterpart;
 * this is a service of the library.
 *   n <= MPHF_VERIFY_STATIC_MAX_KEYS, else MPHF_EINVAL (nothing is run).
 *   Every call shares the scratch: calls whose work overlaps on the device
 *   race and must be serialised.  The first call on a device looks up the
 *   scratch address; make it before any stream capture.  The address is
 *   kept until the process exits: do not call this on a device after a
 *   cudaDeviceReset of it.  Synchronises. */
#define MPHF_VERIFY_STATIC_MAX_KEYS 1048576u
int mphf_verify_static(const mphf_t *h, const void *d_keys, uint64_t n, uint64_t *n_bad,
                       void *stream);

/* Copies h's sizes and parameters to *info (host memory).  MPHF_EINVAL if
 * either pointer is NULL. */
int mphf_get_info(const mphf_t *h, mphf_info *info);

/* Device arrays of a built function, owned by h:
 *   d_values   n_nodes stored values; bucket i's nodes in preorder at
 *              [d_node_off[i], d_node_off[i+1]).  A rotation leaf of m keys
 *              stores k*m + r (seed k*m, rotation r); a ShockHash leaf its
 *              seed and retrieval vector (MPHF_SH_SEED_BITS).
 *   d_node_off nb + 1 offsets.
 *   d_cum_keys nb + 1 bucket prefix sums of key counts.
 *   d_bit_pos  nb + 1 start bits of each bucket's Golomb-Rice code. */
int mphf_get_values(const mphf_t *h, const uint64_t **d_values, const uint64_t **d_node_off,
                    const uint64_t **d_cum_keys, const uint64_t **d_bit_pos);

/* Packed function: Golomb-Rice words (bit i of the stream is bit i % 64 of
 * word i / 64) and the Elias-Fano words (low and high words of the key-count
 * sequence, then of the bit-position sequence). */
int mphf_get_bits(const mphf_t *h, const uint64_t **d_gr, uint64_t *gr_bits, const uint64_t **d_ef,
                  uint64_t *ef_words);

/* Copies the build's search statistics and stage times (mphf_stats) to
 * *stats; all zero for a loaded function. */
int mphf_get_stats(const mphf_t *h, mphf_stats *stats);

/* Golomb-Rice parameter per node size m in [0, max_m] as the library uses it
 * (Section 2.2, "Representation": one parameter per tree layer, precomputed).
 * Writes max_m + 1 bytes to host memory. */
int mphf_tau_table(uint32_t leaf_size, uint32_t leaf_bijection, uint32_t tree_shape, uint32_t max_m,
                   uint8_t *h_out);

/* Copies the function to host memory: a header of 16 64-bit words, then the
 * Golomb-Rice and Elias-Fano words.  The header holds, in order: the magic
 * (the ASCII bytes "RMPFPH01" in little-endian order), n, nb,
 * leaf_size | tree_shape << 16, bucket_size, key_bytes, leaf_bijection,
 * gr_bits, gr_words, ef_words, the two Elias-Fano low-bit counts, and the
 * four Elias-Fano sequence word counts.  With h_buf NULL, *len receives the
 * size needed. */
int mphf_serialize(const mphf_t *h, void *h_buf, size_t *len, void *stream);

/* Checks the len bytes at h_buf as mphf_serialize wrote them, on the host
 * alone (no device is needed), and fills *info.  The Golomb-Rice and
 * Elias-Fano words are the whole function (Section 2.2, "Representation"),
 * so the check decodes all of them:
 *   - the header's sizes must agree with one another and with len (bytes
 *     after the function are ignored);
 *   - both Elias-Fano sequences must decode to nb + 1 nondecreasing values,
 *     from 0 to n (key counts, at most MPHF_MAX_BUCKET keys a bucket) and
 *     from 0 to gr_bits (bit positions);
 *   - each bucket's bits must hold exactly the fixed parts and unary
 *     terminators of its nodes, in preorder.
 * A blob that fails any check gives MPHF_EINVAL.  h_buf needs no alignment. */
int mphf_load_info(const void *h_buf, size_t len, mphf_info *info);

/* Rebuilds a function on the current device from a blob that passes
 * mphf_load_info's checks (else MPHF_EINVAL, nothing allocated).  The node
 * values, offsets and packed words equal the serialised function's; the
 * per-size tables and query directories are recomputed; the statistics are
 * zero.  Device memory comes from allocator (NULL: cudaMallocAsync on the
 * stream).  On success *out owns the function.  Synchronises the stream. */
int mphf_load(const void *h_buf, size_t len, const mphf_allocator *allocator, void *stream,
              mphf_t **out);

/* Releases h.  Synchronises h's device first (queries of h may still be in
 * flight on any stream); the current device is left as it was. */
int mphf_free(mphf_t *h);

const char *mphf_strerror(int code);

/* Number of CUDA kernels this library has launched in the process so far
 * (all builds, queries and verifications). */
uint64_t mphf_kernel_launches(void);

/* ---------------------------------------------------------------------------
 * Batched builds: many independent functions through one persistent search
 * launch (buckets of all builds share one device work queue).  Results are
 * identical to building each alone.  statuses[i] receives each build's code;
 * the return value is MPHF_OK if all succeeded, else the first failure. */
typedef struct {
    const void *d_keys;
    uint64_t n;
    uint32_t leaf_size;
    uint32_t bucket_size;
    uint32_t key_bytes;
    uint32_t leaf_bijection;  /* MPHF_BIJECTION_* */
    uint64_t max_value;       /* 0 = MPHF_DEFAULT_MAX_VALUE */
    uint32_t tree_shape;      /* MPHF_TREE_* */
    uint32_t seeds_per_thread; /* as in mphf_build_params (0 = default) */
} mphf_build_desc;

int mphf_build_batch(const mphf_build_desc *descs, uint32_t count, void *stream, mphf_t **outs,
                     int *statuses);

/* ---------------------------------------------------------------------------
 * Serving: a build server with continuous batching (the paper has no
 * counterpart; its builds are one at a time).  One serving search kernel
 * stays on the device while there is work and takes buckets from a queue in
 * device memory.  A control thread admits queued requests in arrival order
 * while a request slot and device memory are free, prepares them (the
 * fingerprint, bucket sort and plan kernels run beside the search on the SM
 * room it leaves), feeds their buckets into the queue a few at a time from
 * each running request in turn, and packs each request as soon as its own
 * last bucket is done.  So requests that arrive while others are on the
 * device join the running search, and each completes on its own.  Results
 * are identical to building each request alone.  The search leaves the
 * device when no request is left.  Every device wait is bounded (a search
 * block waits at most idle_ms for work); every host wait is bounded by the
 * caller's timeout. */
typedef struct mphf_server mphf_server_t;

#define MPHF_SERVER_MAX_REQUESTS 1024u

typedef struct {
    uint32_t max_requests;       /* requests on the device at once (default 64, at most
                                    MPHF_SERVER_MAX_REQUESTS)                           */
    uint32_t reserved_sms;       /* SMs on which the search keeps one block slot free for
                                    the other requests' preparation and packing (default 4
                                    when the whole cfg is NULL; 0 allowed)              */
    uint64_t hbm_reserve_bytes;  /* device memory kept free (default 1 GiB)             */
    uint32_t idle_ms;            /* bound on a search block's wait for work while the server
                                    is silent (default 10000, at most 600000); the server
                                    stops the search itself whenever no request is left */
    uint32_t threads;            /* search block size, a multiple of 32 in 64..512
                                    (default 512)                                       */
} mphf_server_cfg;

/* Submit/admit/finish times of a request, seconds since the server started. */
typedef struct {
    double submitted, admitted, finished;
} mphf_request_times;

/* cfg NULL = defaults.  The server uses the current device. */
int mphf_server_create(const mphf_server_cfg *cfg, mphf_server_t **out);

/* Queues a build.  The keys (device memory) must stay valid until the
 * request is finished.  *ticket identifies it for mphf_server_poll. */
int mphf_server_submit(mphf_server_t *s, const mphf_build_desc *desc, uint64_t *ticket);

/* Waits up to timeout_ms for the request (0 = do not wait).  Returns
 * MPHF_ETIMEOUT if it is not finished yet, else MPHF_OK with *status the
 * build's code and, on success, *out the built function (owned by the caller
 * from now on).  A finished ticket can be polled once. */
int mphf_server_poll(mphf_server_t *s, uint64_t ticket, uint32_t timeout_ms, mphf_t **out,
                     int *status, mphf_request_times *times);

/* Finishes every queued request, then stops the executors.  Functions built
 * but never polled are freed. */
int mphf_server_destroy(mphf_server_t *s);

#ifdef __cplusplus
}
#endif

#endif /* MPHF_H */
