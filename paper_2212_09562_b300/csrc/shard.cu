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

#include "common.cuh"
#include "engine.h"

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
