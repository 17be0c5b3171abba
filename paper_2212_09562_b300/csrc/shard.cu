// shard.cu -- device side of building one function across several GPUs.
//
// Section 5.2 of Bez et al. 2212.09562 builds the buckets in consecutive
// ranges, one range per thread, and concatenates the ranges' local
// Golomb-Rice sequences and bucket offsets.  Here a range is a GPU (a rank):
//   k_route_count / k_route_scatter  group a rank's input keys by the rank
//                                    that owns their bucket (before the
//                                    exchange of keys between ranks)
//   k_shard_offsets                  a range's local prefix sums, shifted by
//                                    the keys / nodes / bits before the range
//   k_shard_bits                     a range's Golomb-Rice words, ORed into
//                                    the whole sequence at its bit offset
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "build_engine.h"
#include "common.cuh"
#include "engine.h"
#include "handle.h"
#include "mphf.h"

namespace rs {

// Owner of bucket b when nb buckets are cut into `world` consecutive ranges,
// range r = [floor(r nb / world), floor((r + 1) nb / world)): the largest r
// with floor(r nb / world) <= b, i.e. floor(((b + 1) world - 1) / nb).
__host__ __device__ __forceinline__ uint32_t bucket_owner(uint64_t b, uint64_t nb, uint32_t world) {
    return (uint32_t)(((b + 1) * world - 1) / nb);
}

__device__ __forceinline__ uint32_t key_owner(const uint64_t *k, uint64_t i, uint32_t kb, uint64_t nb,
                                              uint32_t world) {
    const uint64_t w0 = kb == 8 ? k[i] : k[2 * i], w1 = kb == 8 ? 0 : k[2 * i + 1];
    uint64_t hi, lo;
    fingerprint(w0, w1, hi, lo);
    return bucket_owner(mulhi64(hi, nb), nb, world);
}

__global__ void k_route_count(const uint64_t *keys, uint64_t n, uint32_t kb, uint64_t nb,
                              uint32_t world, unsigned long long *counts) {
    extern __shared__ unsigned long long part[];
    for (uint32_t r = threadIdx.x; r < world; r += blockDim.x) part[r] = 0;
    __syncthreads();
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        atomicAdd(&part[key_owner(keys, i, kb, nb, world)], 1ull);
    __syncthreads();
    for (uint32_t r = threadIdx.x; r < world; r += blockDim.x)
        if (part[r]) atomicAdd(&counts[r], part[r]);
}

// cursor[r] starts at the first output slot of rank r's keys.
__global__ void k_route_scatter(const uint64_t *keys, uint64_t n, uint32_t kb, uint64_t nb,
                                uint32_t world, unsigned long long *cursor, uint64_t *out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t p = atomicAdd(&cursor[key_owner(keys, i, kb, nb, world)], 1ull);
        if (kb == 8) {
            out[p] = keys[i];
        } else {
            out[2 * p] = keys[2 * i];
            out[2 * p + 1] = keys[2 * i + 1];
        }
    }
}

static uint32_t grid_of(uint64_t n) {
    uint64_t g = (n + 255) / 256;
    return (uint32_t)(g < 1 ? 1 : g > 148 * 16 ? 148 * 16 : g);
}

void launch_route_count(const uint64_t *keys, uint64_t n, uint32_t kb, uint64_t nb, uint32_t world,
                        uint64_t *counts, cudaStream_t st) {
    if (n == 0) return;
    k_route_count<<<grid_of(n), 256, world * 8, st>>>(keys, n, kb, nb, world,
                                                       (unsigned long long *)counts);
    note_launches(1);
}

void launch_route_scatter(const uint64_t *keys, uint64_t n, uint32_t kb, uint64_t nb, uint32_t world,
                          uint64_t *cursor, uint64_t *out, cudaStream_t st) {
    if (n == 0) return;
    k_route_scatter<<<grid_of(n), 256, 0, st>>>(keys, n, kb, nb, world, (unsigned long long *)cursor,
                                                 out);
    note_launches(1);
}

// out[i] = in[i] + base for i < count (a range's local offsets in the whole function).
__global__ void k_shard_offsets(const uint64_t *in, uint64_t count, uint64_t base, uint64_t *out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = in[i] + base;
}

void launch_shard_offsets(const uint64_t *in, uint64_t count, uint64_t base, uint64_t *out,
                          cudaStream_t st) {
    if (count == 0) return;
    k_shard_offsets<<<grid_of(count), 256, 0, st>>>(in, count, base, out);
    note_launches(1);
}

// Bits [0, bits) of `in` ORed into `out` at bit offset `at`; out must be zero
// there and one word longer than the last bit it receives.  Ranges occupy
// disjoint bits, so concurrent ranges may OR into a shared boundary word.
__global__ void k_shard_bits(const uint64_t *in, uint64_t bits, uint64_t at, uint64_t *out) {
    const uint64_t words = (bits + 63) / 64;
    const uint32_t sh = (uint32_t)(at & 63);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < words;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t v = in[i];
        if (i == words - 1 && (bits & 63)) v &= (1ull << (bits & 63)) - 1;
        if (!v) continue;
        const uint64_t w = (at >> 6) + i;
        atomicOr((unsigned long long *)&out[w], (unsigned long long)(v << sh));
        if (sh) atomicOr((unsigned long long *)&out[w + 1], (unsigned long long)(v >> (64 - sh)));
    }
}

void launch_shard_bits(const uint64_t *in, uint64_t bits, uint64_t at, uint64_t *out, cudaStream_t st) {
    if (bits == 0) return;
    k_shard_bits<<<grid_of((bits + 63) / 64), 256, 0, st>>>(in, bits, at, out);
    note_launches(1);
}

}  // namespace rs

using namespace rs;

extern "C" {

// The C ABI of sharded builds.
// One function built on several GPUs (Section 5.2: consecutive bucket
// ranges, local sequences concatenated).  Rank r of `world` owns buckets
// [floor(r nb / world), floor((r + 1) nb / world)) of the function over
// n_total keys (nb = ceil(n_total / bucket_size)).

// The pack of a shard: kShardHead header words, then its arrays.
constexpr size_t kShardHead = 24;
constexpr uint64_t kShardMagic = 0x3144485346504D52ull;  // "RMPFSHD1"

static void shard_range(uint64_t nb, uint32_t rank, uint32_t world, uint64_t *lo, uint64_t *hi) {
    *lo = nb * rank / world;
    *hi = nb * (rank + 1) / world;
}

int mphf_build_shard(const void *d_keys, uint64_t n, uint64_t n_total, const mphf_build_params *p,
                     uint32_t rank, uint32_t world, void *stream, mphf_t **out) {
    if (!out || !p) return MPHF_EINVAL;
    *out = nullptr;
    if (world == 0 || world > MPHF_MAX_SHARDS || rank >= world || n > n_total) return MPHF_EINVAL;
    int rc = check_shape(n_total, p);
    if (rc != MPHF_OK) return rc;
    std::vector<Job> jobs(1);
    Job &j = jobs[0];
    start_job(j, d_keys, n, *p);
    if (j.rc) return j.rc;
    const uint64_t nb_hash = (n_total + p->bucket_size - 1) / p->bucket_size;
    uint64_t b_lo, b_hi;
    shard_range(nb_hash, rank, world, &b_lo, &b_hi);
    j.nb = b_hi - b_lo;
    j.range = BucketRange{nb_hash, b_lo};
    j.h->info.nb = j.nb;
    j.h->shard = true;
    j.h->b_lo = b_lo;
    j.h->nb_hash = nb_hash;
    j.h->n_total = n_total;
    int grc = run_jobs(jobs, (cudaStream_t)stream, p->allocator, p->threads_per_block, p->blocks_per_sm);
    if (grc) return grc;
    if (j.rc) return j.rc;
    *out = j.h;
    return MPHF_OK;
}

int mphf_shard_route(const void *d_keys, uint64_t n, uint32_t key_bytes, uint64_t n_total,
                     uint32_t bucket_size, uint32_t world, void *d_out, uint64_t *h_counts,
                     void *stream) {
    if (!h_counts || world == 0 || world > MPHF_MAX_SHARDS || (key_bytes != 8 && key_bytes != 16) ||
        bucket_size < 1 || bucket_size > MPHF_MAX_BUCKET_SIZE || n > n_total || n_total >= (1ull << 32))
        return MPHF_EINVAL;
    if (n > 0 && (!d_keys || !d_out || ((uintptr_t)d_keys & 7) || ((uintptr_t)d_out & 7)))
        return MPHF_EINVAL;
    memset(h_counts, 0, world * sizeof(uint64_t));
    if (n == 0) return MPHF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t nb = (n_total + bucket_size - 1) / bucket_size;
    Mem mem{nullptr, st};
    uint64_t *d = (uint64_t *)mem.get(2 * world * sizeof(uint64_t));
    if (!d) return MPHF_ENOMEM;
    std::vector<uint64_t> cur(world);
    int rc = MPHF_OK;
    if (cudaMemsetAsync(d, 0, world * sizeof(uint64_t), st) != cudaSuccess) rc = MPHF_ECUDA;
    if (rc == MPHF_OK) {
        launch_route_count((const uint64_t *)d_keys, n, key_bytes, nb, world, d, st);
        if (cudaMemcpyAsync(h_counts, d, world * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = MPHF_ECUDA;
    }
    if (rc == MPHF_OK) {
        uint64_t run = 0;
        for (uint32_t r = 0; r < world; r++) {
            cur[r] = run;
            run += h_counts[r];
        }
        if (cudaMemcpyAsync(d + world, cur.data(), world * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
            rc = MPHF_ECUDA;
        else
            launch_route_scatter((const uint64_t *)d_keys, n, key_bytes, nb, world, d + world,
                                 (uint64_t *)d_out, st);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
            rc = MPHF_ECUDA;
    }
    if (rc != MPHF_OK) cudaGetLastError();
    mem.put(d);
    cudaStreamSynchronize(st);
    return rc;
}

static size_t shard_pack_bytes(const mphf_t *h) {
    const uint64_t nb = h->info.nb;
    return 8 * (kShardHead + 3 * (nb + 1) + h->info.n_nodes + h->info.gr_words);
}

int mphf_shard_pack(const mphf_t *h, void *d_buf, size_t *len, void *stream) {
    if (!h || !len || !h->shard) return MPHF_EINVAL;
    const size_t need = shard_pack_bytes(h);
    if (!d_buf) {
        *len = need;
        return MPHF_OK;
    }
    if (*len < need || ((uintptr_t)d_buf & 7)) {
        *len = need;
        return MPHF_EINVAL;
    }
    const mphf_info &I = h->info;
    uint64_t hd[kShardHead] = {kShardMagic, I.n, I.nb, h->b_lo, h->n_total, I.n_nodes, I.gr_bits,
                               I.leaf_size | ((uint64_t)I.tree_shape << 16), I.bucket_size,
                               I.key_bytes, I.leaf_bijection, I.max_bucket, 0, 0, 0, 0};
    for (int k = 0; k < 4; k++) {
        hd[16 + k] = h->stats.trials[k];
        hd[20 + k] = h->stats.evals[k];
    }
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t *w = (uint64_t *)d_buf;
    const uint64_t nb = I.nb;
    struct Part {
        const void *src;
        size_t words;
    } parts[] = {{hd, kShardHead}, {h->cum_keys, nb + 1}, {h->node_off, nb + 1},
                 {h->bit_pos, nb + 1}, {h->values, I.n_nodes}, {h->gr, I.gr_words}};
    int rc = MPHF_OK;
    for (const Part &q : parts) {
        if (q.words && cudaMemcpyAsync(w, q.src, q.words * 8, cudaMemcpyDefault, st) != cudaSuccess)
            rc = MPHF_ECUDA;
        w += q.words;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = MPHF_ECUDA;  // hd is read by the copy
    if (rc != MPHF_OK) cudaGetLastError();
    *len = need;
    return rc;
}

int mphf_shard_concat(const void *const *d_parts, const size_t *lens, uint32_t count,
                      const mphf_allocator *allocator, void *stream, mphf_t **out) {
    if (!out || !d_parts || !lens || count == 0 || count > MPHF_MAX_SHARDS) return MPHF_EINVAL;
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<uint64_t> hd(kShardHead * (size_t)count);
    for (uint32_t s = 0; s < count; s++) {
        if (!d_parts[s] || ((uintptr_t)d_parts[s] & 7) || lens[s] < kShardHead * 8) return MPHF_EINVAL;
        if (cudaMemcpyAsync(&hd[kShardHead * s], d_parts[s], kShardHead * 8, cudaMemcpyDefault, st) !=
            cudaSuccess) {
            cudaGetLastError();
            return MPHF_ECUDA;
        }
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return MPHF_ECUDA;
    }
    // the parts must be the ranks 0..count-1 of one function, in order
    const uint64_t *h0 = &hd[0];
    const uint64_t n_total = h0[4], bucket = h0[8];
    if (bucket < 1 || bucket > MPHF_MAX_BUCKET_SIZE || n_total >= (1ull << 32)) return MPHF_EINVAL;
    const uint64_t nb = (n_total + bucket - 1) / bucket;
    uint64_t keys = 0, nodes = 0, bits = 0, max_bucket = 0;
    for (uint32_t s = 0; s < count; s++) {
        const uint64_t *x = &hd[kShardHead * s];
        uint64_t lo, hi;
        shard_range(nb, s, count, &lo, &hi);
        if (x[0] != kShardMagic || x[4] != n_total || x[7] != h0[7] || x[8] != bucket ||
            x[9] != h0[9] || x[10] != h0[10] || x[3] != lo || x[2] != hi - lo || x[1] > n_total ||
            x[5] > 4096ull * (hi - lo))
            return MPHF_EINVAL;
        // the part must hold its arrays (no sum below can wrap)
        uint64_t room = lens[s] / 8 - kShardHead;
        if (x[2] + 1 > room / 3) return MPHF_EINVAL;
        room -= 3 * (x[2] + 1);
        if (x[5] > room) return MPHF_EINVAL;
        room -= x[5];
        if (x[6] > 64 * room) return MPHF_EINVAL;
        keys += x[1];
        nodes += x[5];
        bits += x[6];
        max_bucket = x[11] > max_bucket ? x[11] : max_bucket;
    }
    if (keys != n_total) return MPHF_EINVAL;
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
    mphf_info &I = h->info;
    I.n = n_total;
    I.nb = nb;
    I.leaf_size = (uint32_t)(h0[7] & 0xFFFF);
    I.tree_shape = (uint32_t)(h0[7] >> 16);
    I.bucket_size = (uint32_t)bucket;
    I.key_bytes = (uint32_t)h0[9];
    I.leaf_bijection = (uint32_t)h0[10];
    I.n_nodes = nodes;
    I.max_bucket = (uint32_t)max_bucket;
    int rc = device_tables(h->device, I.leaf_size, I.leaf_bijection, I.tree_shape, &h->tabs);
    if (rc != MPHF_OK) {
        release(h, 0);
        return rc;
    }
    Mem mem{allocator, st};
    h->cum_keys = (uint64_t *)mem.get((nb + 1) * 8);
    h->node_off = (uint64_t *)mem.get((nb + 1) * 8);
    h->bit_pos = (uint64_t *)mem.get((nb + 1) * 8);
    h->values = (uint64_t *)mem.get(nodes * 8);
    uint64_t *tmp = (uint64_t *)mem.get((scan_tmp_words(nb + 2 > 4098 ? nb + 2 : 4098) + 64) * 8);
    if (!h->cum_keys || !h->node_off || !h->bit_pos || !h->values || !tmp ||
        alloc_packed(h, nb, n_total, bits, mem) != MPHF_OK) {
        mem.put(tmp);
        cudaStreamSynchronize(st);
        release(h, st);
        return MPHF_ENOMEM;
    }
    const uint64_t last[3] = {n_total, nodes, bits};  // the closing entry of each offset array
    bool ok = cudaMemsetAsync(h->gr, 0, I.gr_words * 8 + 8, st) == cudaSuccess &&
              cudaMemsetAsync(h->ef, 0, I.ef_words * 8 + 8, st) == cudaSuccess &&
              cudaMemcpyAsync(h->cum_keys + nb, &last[0], 8, cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(h->node_off + nb, &last[1], 8, cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(h->bit_pos + nb, &last[2], 8, cudaMemcpyHostToDevice, st) == cudaSuccess;
    uint64_t k0 = 0, n0 = 0, g0 = 0;
    for (uint32_t s = 0; s < count && ok; s++) {
        const uint64_t *x = &hd[kShardHead * s];
        const uint64_t snb = x[2], b_lo = x[3], sn = x[5], sbits = x[6];
        const uint64_t *w = (const uint64_t *)d_parts[s] + kShardHead;
        const uint64_t *cum = w, *noff = cum + snb + 1, *bpos = noff + snb + 1, *vals = bpos + snb + 1;
        const uint64_t *gr = vals + sn;
        launch_shard_offsets(cum, snb, k0, h->cum_keys + b_lo, st);
        launch_shard_offsets(noff, snb, n0, h->node_off + b_lo, st);
        launch_shard_offsets(bpos, snb, g0, h->bit_pos + b_lo, st);
        if (sn && cudaMemcpyAsync(h->values + n0, vals, sn * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            ok = false;
        launch_shard_bits(gr, sbits, g0, h->gr, st);
        k0 += x[1];
        n0 += sn;
        g0 += sbits;
    }
    if (ok) write_ef_dirs(h, nb, tmp, st);
    for (uint32_t s = 0; s < count; s++)
        for (int k = 0; k < 4; k++) {
            h->stats.trials[k] += hd[kShardHead * s + 16 + k];
            h->stats.evals[k] += hd[kShardHead * s + 20 + k];
        }
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) ok = false;
    mem.put(tmp);
    if (!ok) {
        cudaGetLastError();
        cudaStreamSynchronize(st);
        release(h, st);
        return MPHF_ECUDA;
    }
    *out = h;
    return MPHF_OK;
}

}  // extern "C"
