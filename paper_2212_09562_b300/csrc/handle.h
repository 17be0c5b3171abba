// handle.h -- what a function handle (mphf_t) holds, and the host helpers
// shared by the C-ABI entry points of libmphf.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "engine.h"
#include "mphf.h"

namespace rs {

// Per-device copies of the per-size tables of one (leaf size, leaf method,
// tree shape); cached for the life of the process.
struct DevTables {
    uint8_t *tau = nullptr;
    uint32_t *nodes = nullptr;
    uint32_t *fixed = nullptr;
    uint16_t *left = nullptr;
    uint32_t *mod_c = nullptr;
    uint64_t *mod_M = nullptr;
    const uint64_t *salts = nullptr;  // level_salt(L) for L < kSaltLevels (per device)
};

// Device memory from the caller's allocator hooks, else stream-ordered
// cudaMallocAsync / cudaFreeAsync on st.
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

// Error code of a build's device status bits (precedence: another shard's
// key, oversized bucket, duplicate, search cap, wait timeout, overflow).
inline int status_code(uint32_t st) {
    if (st & ST_RANGE) return MPHF_EINVAL;  // a shard was given a key of another shard
    if (st & ST_BUCKET) return MPHF_EBUCKET;
    if (st & ST_DUPLICATE) return MPHF_EDUPLICATE;
    if (st & ST_LIMIT) return MPHF_ESEARCH_LIMIT;
    if (st & ST_TIMEOUT) return MPHF_ETIMEOUT;
    if (st & ST_OVERFLOW) return MPHF_ECAPACITY;
    return MPHF_OK;
}

int device_tables(int dev, uint32_t leaf, uint32_t bij, uint32_t tree, DevTables *out);
int device_rot_tables(int dev, const uint8_t **canon, const uint8_t **period);

struct BuildPlan;  // arrays of a build prepared for replay (graph_build.cu)

}  // namespace rs

struct mphf {
    int device = 0;
    mphf_info info{};
    mphf_allocator alloc{};
    bool has_alloc = false;
    uint64_t *values = nullptr, *node_off = nullptr, *cum_keys = nullptr, *bit_pos = nullptr;
    uint64_t *gr = nullptr, *ef = nullptr, *ef_dir = nullptr;  // ef_dir: rank then select directories
    uint64_t ef_dir_len[2] = {0, 0};
    uint64_t ef_sel_len = 0;
    rs::DevTables tabs;
    mphf_stats stats{};
    // a shard: buckets [b_lo, b_lo + info.nb) of a function over n_total keys
    // hashed to nb_hash buckets (not queryable on its own)
    bool shard = false;
    uint64_t b_lo = 0, nb_hash = 0, n_total = 0;
    // a prepared build (mphf_build_prepare): its scratch and capacities; the
    // function is usable only after a successful mphf_build_finish
    rs::BuildPlan *plan = nullptr;
    bool ready = true;
};


namespace rs {

// Frees a handle's arrays in the order of stream st, then the handle.
void release(mphf_t *h, cudaStream_t st);
// Frees a prepared build's scratch (nothing if the handle has none).
void release_plan(mphf_t *h, Mem &mem);
// Sizes of the packed function (Golomb-Rice words, the two Elias-Fano
// sequences over nb + 1 bucket offsets, their rank and select directories)
// and its arrays from the handle's allocator.  Nothing is written yet.
int alloc_packed(mphf_t *h, uint64_t nb, uint64_t n, uint64_t gr_bits, Mem &jm);
// Elias-Fano sequences of the key and bit offsets into the zeroed h->ef, and
// their query directories.
void write_ef_dirs(mphf_t *h, uint64_t nb, uint64_t *scan_tmp, cudaStream_t st);

}  // namespace rs
