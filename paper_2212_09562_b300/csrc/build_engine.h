// build_engine.h -- the build engine shared by the C-ABI entry points of
// libmphf: jobs (one build each), the scratch of an engine pass, and its
// phases (plan, scatter, pack) around one persistent search.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "engine.h"
#include "handle.h"
#include "mphf.h"

namespace rs {

// One build going through the engine.
struct Job {
    const void *d_keys = nullptr;
    uint64_t n = 0;
    mphf_build_params p{};
    mphf_t *h = nullptr;
    int rc = MPHF_OK;
    uint64_t nb = 0, maxv = 0;
    BucketRange range{0, 0};  // the buckets this job builds (all of them unless a shard)
    uint64_t *lo_s = nullptr, *counters = nullptr;
    uint8_t *bb_s = nullptr;
    uint32_t *cursor = nullptr, *small = nullptr;  // small: status, max bucket, spare
    uint32_t *blk = nullptr;                         // per-block bucket counts (two-level sort)
    uint32_t sort_g = 0;
    uint16_t *node_m = nullptr;
    uint64_t n_nodes = 0;
    uint32_t max_m = 0;    // largest bucket
    bool planned = false;  // its buckets are counted in the pass's work-order histogram
    InstDesc desc{};       // what the search kernel reads about this job
};

// Pinned host words for the totals read between phases, one buffer per host
// thread, kept for the thread's life: cudaMallocHost / cudaFreeHost cost
// about as much as a whole small build, and cudaFreeHost synchronises.
struct PinnedWords {
    uint64_t *p = nullptr;
    size_t words = 0;
    ~PinnedWords() {
        if (p) cudaFreeHost(p);
    }
    uint64_t *get(size_t n) {
        if (n <= words) return p;
        if (p) cudaFreeHost(p);
        p = nullptr;
        words = 0;
        if (cudaMallocHost(&p, n * 8) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return nullptr;
        }
        words = n;
        return p;
    }
};
extern thread_local PinnedWords t_pinned;

// Scratch shared by the jobs of one engine pass: the prefix-sum scratch, the
// bucket-size histogram of the work order, and a pinned host buffer for the
// totals read between phases (four words per job).
struct EngineCtx {
    Mem mem;
    uint64_t *host = nullptr, *scan_tmp = nullptr, *size_hist = nullptr;
    uint32_t *size_cursor = nullptr;
    uint64_t cap_nb = 0;

    // Room for `jobs` jobs of at most max_nb buckets each.
    int reserve(size_t jobs, uint64_t max_nb) {
        host = t_pinned.get(4 * (jobs ? jobs : 1));
        if (!host) return MPHF_ECUDA;
        if (!scan_tmp || max_nb > cap_nb) {
            mem.put(scan_tmp);
            const uint64_t len = max_nb + 2 > 4098 ? max_nb + 2 : 4098;
            scan_tmp = (uint64_t *)mem.get((scan_tmp_words(len) + 64) * 8);
            cap_nb = max_nb;
        }
        if (!size_hist) size_hist = (uint64_t *)mem.get(4098 * 8);
        if (!size_cursor) size_cursor = (uint32_t *)mem.get(4097 * 4);
        return scan_tmp && size_hist && size_cursor ? MPHF_OK : MPHF_ENOMEM;
    }
    // The work-order histogram starts empty for every pass.
    int clear_order() {
        if (cudaMemsetAsync(size_hist, 0, 4098 * 8, mem.st) != cudaSuccess ||
            cudaMemsetAsync(size_cursor, 0, 4097 * 4, mem.st) != cudaSuccess) {
            cudaGetLastError();
            return MPHF_ECUDA;
        }
        return MPHF_OK;
    }
    void release() {
        mem.put(scan_tmp);
        mem.put(size_hist);
        mem.put(size_cursor);
        scan_tmp = size_hist = nullptr;
        size_cursor = nullptr;
        cudaStreamSynchronize(mem.st);
        host = nullptr;  // the thread's pinned words stay for its next build
        cap_nb = 0;
    }
};

// Parameters of a build apart from where its keys are; and with them.
int check_shape(uint64_t n, const mphf_build_params *p);
int check_params(const void *d_keys, uint64_t n, const mphf_build_params *p);
// Frees a job's scratch; fails it (first error kept) and releases its handle.
void free_job_scratch(Job &j, Mem &mem);
void fail_job(Job &j, int rc, Mem &mem);
// Creates the handle of a job (parameters checked, tables ready).
void start_job(Job &j, const void *d_keys, uint64_t n, const mphf_build_params &p);
// Phase 1 (fingerprints, bucket sizes, plan, offsets, one host read); phase
// 2 (keys by bucket, search descriptors); phases 3-4 (Golomb-Rice and
// Elias-Fano packing, statistics).  Jobs that fail get rc set; the return
// value is a failure of all of them.
int phase_plan(std::vector<Job *> &jobs, EngineCtx &c);
int phase_scatter(std::vector<Job *> &jobs, EngineCtx &c);
int phase_pack(std::vector<Job *> &jobs, EngineCtx &c);
// Default search block size for these jobs.
uint32_t default_threads(const std::vector<Job *> &jobs);
// Runs every job through all phases with one search launch over all of
// their buckets; each job ends with rc set and, if OK, h built.
int run_jobs(std::vector<Job> &jobs, cudaStream_t st, const mphf_allocator *shared_alloc,
             uint32_t threads, uint32_t blocks_per_sm);

}  // namespace rs
