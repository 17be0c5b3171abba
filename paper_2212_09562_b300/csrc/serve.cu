// serve.cu -- the build server of libmphf (mphf_server_*), with continuous
// batching through one serving search kernel on the device.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "build_engine.h"
#include "common.cuh"
#include "engine.h"
#include "handle.h"
#include "mphf.h"

using namespace rs;

// ---------------------------------------------------------------------------
// Build server with continuous batching.
//
// One serving search kernel (k_serve) stays on the device while there is
// work and takes buckets from a ring in device memory.  A control thread:
//   - admits queued requests in arrival order while a request slot and
//     device memory are free: it runs their fingerprint, bucket sort and plan
//     on the preparation stream (these kernels run beside the search, on the
//     SM room the search leaves free) and stages their work items;
//   - keeps the ring filled, a few items from each running request in turn,
//     so a request admitted while others are on the device gets blocks
//     within about one bucket's time;
//   - polls the per-request bucket counters and packs (Golomb-Rice, Elias-
//     Fano) each request as soon as its last bucket is done, while the others
//     keep searching; the request completes on its own, not with a batch.
// Every request goes through the same kernels as a plain build, so its
// function is identical.
namespace {

struct ServerRequest {
    uint64_t ticket = 0;
    mphf_build_desc desc{};
    mphf_request_times t{};
    int status = MPHF_OK;
    mphf_t *out = nullptr;
    bool done = false;
};

double seconds_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// Device memory a build needs besides its keys: grouped lo words and bits,
// node values and sizes, offsets, packed output (about 11 bytes per key).
uint64_t build_bytes(const mphf_build_desc &d) {
    uint64_t nb = d.bucket_size ? (d.n + d.bucket_size - 1) / d.bucket_size : 0;
    return 16 * d.n + 48 * nb + (1u << 20);
}

constexpr uint32_t kRing = 1u << 16;           // work items the ring holds
constexpr uint32_t kMaxSlots = MPHF_SERVER_MAX_REQUESTS;

// A request on the device.
struct Active {
    ServerRequest *r = nullptr;
    Job job;
    uint32_t slot = 0;
    WorkItem *staging = nullptr;  // its buckets' work items, largest first
    uint64_t nb = 0, published = 0;
    uint64_t reserve = 0;         // device bytes counted against the budget
};

}  // namespace

struct mphf_server {
    int device = 0;
    mphf_server_cfg cfg{};
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ServerRequest *> pending;
    std::unordered_map<uint64_t, ServerRequest *> requests;
    std::thread control;
    uint64_t next_ticket = 1;
    bool stop = false;
    int fatal = MPHF_OK;  // a CUDA failure of the server itself
    // device side
    cudaStream_t prep = nullptr, search = nullptr, poll = nullptr;
    ServeCtl *ctl = nullptr;
    WorkItem *ring = nullptr;
    InstDesc *insts = nullptr;
    unsigned int *done = nullptr, *sm_count = nullptr;
    uint64_t *pinned = nullptr;  // [0] new tail, [1] head seen, then done[] as 32-bit words
    ServeLaunch launch{};
};

namespace {

void finish(mphf_server_t *S, ServerRequest *r, int status, mphf_t *h) {
    std::lock_guard<std::mutex> g(S->mu);
    r->status = status;
    r->out = status == MPHF_OK ? h : nullptr;
    r->t.finished = seconds_since(S->t0);
    r->done = true;
    S->cv_done.notify_all();
}

// Fingerprints, sort, plan and work items of one request on the preparation
// stream; its descriptor goes to slot a.slot.  Returns a server-wide error
// (CUDA) or OK; a failure of the request alone is left in a.job.rc.
int prepare(mphf_server_t *S, EngineCtx &c, Active &a) {
    Job &j = a.job;
    std::vector<Job *> jp{&j};
    int rc = c.reserve(1, j.nb);
    if (rc != MPHF_OK) return rc;
    if ((rc = c.clear_order()) != MPHF_OK) return rc;
    if ((rc = phase_plan(jp, c)) != MPHF_OK) return rc;
    if (j.rc) return MPHF_OK;
    if ((rc = phase_scatter(jp, c)) != MPHF_OK) return rc;
    if (j.rc) return MPHF_OK;
    a.nb = j.nb;
    a.staging = (WorkItem *)c.mem.get(j.nb * sizeof(WorkItem) + 8);
    if (!a.staging) {
        fail_job(j, MPHF_ENOMEM, c.mem);
        return MPHF_OK;
    }
    const cudaStream_t st = c.mem.st;
    launch_exclusive_scan(c.size_hist, 4098, c.scan_tmp, st);
    launch_items_by_size(j.h->cum_keys, j.nb, c.size_hist, c.size_cursor, a.staging, a.slot, st);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(S->insts + a.slot, &j.desc, sizeof(InstDesc), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemsetAsync(S->done + a.slot, 0, sizeof(unsigned int), st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return MPHF_ECUDA;
    }
    return MPHF_OK;
}

// Sets the search's stop flag (copied from pinned memory, then synchronised).
int set_stop(mphf_server_t *S, uint32_t v) {
    uint32_t *p = (uint32_t *)S->pinned;
    p[0] = v;
    if (cudaMemcpyAsync(&S->ctl->stop, p, 4, cudaMemcpyHostToDevice, S->prep) != cudaSuccess ||
        cudaStreamSynchronize(S->prep) != cudaSuccess) {
        cudaGetLastError();
        return MPHF_ECUDA;
    }
    return MPHF_OK;
}

void release_active(EngineCtx &c, Active &a) {
    free_job_scratch(a.job, c.mem);
    c.mem.put(a.staging);
    a.staging = nullptr;
}

void server_control(mphf_server_t *S) {
    cudaSetDevice(S->device);
    EngineCtx c{Mem{nullptr, S->prep}};
    std::vector<Active *> active;
    std::vector<uint32_t> free_slots;
    for (uint32_t i = S->cfg.max_requests; i-- > 0;) free_slots.push_back(i);
    uint64_t tail = 0, head = 0;
    bool running = false;  // a serving search was launched and may still run
    size_t rr = 0;  // round-robin position over the active requests
    const uint64_t low_water = 2ull * S->launch.working_blocks;
    const unsigned long long idle_ns = (unsigned long long)S->cfg.idle_ms * 1000000ull;
    auto fatal = [&](int rc) {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->fatal == MPHF_OK) S->fatal = rc;
    };
    for (;;) {
        bool progress = false;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->fatal != MPHF_OK) {  // the device failed: every request gets the error
                const int rc = S->fatal;
                std::vector<ServerRequest *> left(S->pending.begin(), S->pending.end());
                S->pending.clear();
                lk.unlock();
                for (ServerRequest *r : left) finish(S, r, rc, nullptr);
                // the search may still read the active requests' arrays: stop it first
                set_stop(S, 1);
                cudaStreamSynchronize(S->search);
                cudaGetLastError();
                running = false;
                for (Active *a : active) {
                    if (a->job.h) fail_job(a->job, rc, c.mem);
                    release_active(c, *a);
                    finish(S, a->r, rc, nullptr);
                    delete a;
                }
                active.clear();
                break;
            }
        }
        // 1. admission, in arrival order, while a slot and memory are free
        for (;;) {
            ServerRequest *r = nullptr;
            {
                std::unique_lock<std::mutex> lk(S->mu);
                if (S->pending.empty() || free_slots.empty()) break;
                size_t free_b = 0, total_b = 0;
                if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
                    cudaGetLastError();
                    free_b = 0;
                }
                // memory of admitted requests is already allocated, so free_b counts it
                const int64_t budget = (int64_t)free_b - (int64_t)S->cfg.hbm_reserve_bytes;
                const uint64_t need = build_bytes(S->pending.front()->desc);
                // a request that never fits still runs when nothing else is on the device
                if ((int64_t)need > budget && !active.empty()) break;
                r = S->pending.front();
                S->pending.pop_front();
                r->t.admitted = seconds_since(S->t0);
            }
            progress = true;
            Active *a = new Active;
            a->r = r;
            a->slot = free_slots.back();
            free_slots.pop_back();
            mphf_build_params p;
            mphf_default_params(&p);
            p.leaf_size = r->desc.leaf_size;
            p.bucket_size = r->desc.bucket_size;
            p.key_bytes = r->desc.key_bytes;
            p.leaf_bijection = r->desc.leaf_bijection;
            p.tree_shape = r->desc.tree_shape;
            p.max_value = r->desc.max_value ? r->desc.max_value : MPHF_DEFAULT_MAX_VALUE;
            p.seeds_per_thread = r->desc.seeds_per_thread;
            start_job(a->job, r->desc.d_keys, r->desc.n, p);
            int rc = a->job.rc ? MPHF_OK : prepare(S, c, *a);
            if (rc != MPHF_OK) fatal(rc);
            if (rc != MPHF_OK || a->job.rc) {
                const int st = rc != MPHF_OK ? rc : a->job.rc;
                if (rc != MPHF_OK && a->job.h) fail_job(a->job, rc, c.mem);
                release_active(c, *a);
                free_slots.push_back(a->slot);
                finish(S, r, st, nullptr);
                delete a;
                continue;
            }
            active.push_back(a);
        }
        // 2. keep the ring filled: a few items of each request in turn
        if (!active.empty() && tail - head < low_water) {
            const uint64_t start = tail;
            bool any = true;
            while (tail - head < low_water + 64 && any) {
                any = false;
                for (size_t k = 0; k < active.size() && tail - head < low_water + 64; k++) {
                    Active &a = *active[(rr + k) % active.size()];
                    if (a.published >= a.nb) continue;
                    uint64_t take = a.nb - a.published;
                    take = take > 8 ? 8 : take;
                    take = take > kRing - (tail % kRing) ? kRing - (tail % kRing) : take;  // no wrap
                    if (cudaMemcpyAsync(S->ring + tail % kRing, a.staging + a.published,
                                        take * sizeof(WorkItem), cudaMemcpyDeviceToDevice,
                                        S->prep) != cudaSuccess)
                        fatal(MPHF_ECUDA);
                    a.published += take;
                    tail += take;
                    any = true;
                }
                rr++;
            }
            if (tail != start) {
                S->pinned[0] = tail;
                if (cudaMemcpyAsync(&S->ctl->tail, S->pinned, 8, cudaMemcpyHostToDevice, S->prep) !=
                        cudaSuccess ||
                    cudaStreamSynchronize(S->prep) != cudaSuccess) {
                    cudaGetLastError();
                    fatal(MPHF_ECUDA);
                }
                progress = true;
            }
        }
        // 3. the search must be on the device while items wait (its blocks
        // leave only when told to, or after the idle bound)
        if (tail > head) {
            if (running) {
                const cudaError_t q = cudaStreamQuery(S->search);
                if (q != cudaSuccess && q != cudaErrorNotReady) fatal(MPHF_ECUDA);
                cudaGetLastError();  // a search still running is not an error
                running = q != cudaSuccess;
            }
            if (!running) {
                if (cudaMemsetAsync(S->sm_count, 0, kServeMaxSms * 4, S->search) != cudaSuccess)
                    fatal(MPHF_ECUDA);
                launch_serve(S->insts, S->ring, kRing, S->ctl, S->done, S->sm_count,
                             S->cfg.reserved_sms, idle_ns, S->launch, S->search);
                if (cudaGetLastError() != cudaSuccess) fatal(MPHF_ECUDA);
                running = true;
            }
        }
        // 4. poll the queue head and the per-request bucket counters
        if (!active.empty()) {
            uint32_t *d32 = (uint32_t *)(S->pinned + 2);
            if (cudaMemcpyAsync(S->pinned + 1, &S->ctl->head, 8, cudaMemcpyDeviceToHost, S->poll) != cudaSuccess ||
                cudaMemcpyAsync(d32, S->done, S->cfg.max_requests * 4, cudaMemcpyDeviceToHost, S->poll) !=
                    cudaSuccess ||
                cudaStreamSynchronize(S->poll) != cudaSuccess) {
                cudaGetLastError();
                fatal(MPHF_ECUDA);
            }
            head = S->pinned[1] < tail ? S->pinned[1] : tail;
            // 5. pack every request whose buckets are all done
            for (size_t k = 0; k < active.size();) {
                Active &a = *active[k];
                if (a.published < a.nb || d32[a.slot] < a.nb) {
                    k++;
                    continue;
                }
                std::vector<Job *> jp{&a.job};
                int rc = phase_pack(jp, c);
                if (rc != MPHF_OK) fatal(rc);
                const int st = rc != MPHF_OK ? rc : a.job.rc;
                mphf_t *h = a.job.h;
                release_active(c, a);
                if (st != MPHF_OK && h) {
                    if (!a.job.rc) fail_job(a.job, st, c.mem);
                    h = nullptr;
                }
                free_slots.push_back(a.slot);
                finish(S, a.r, st, h);
                delete active[k];
                active.erase(active.begin() + (long)k);
                progress = true;
            }
        }
        // 6. nothing on the device: the search leaves, so that the next
        // request's preparation has the whole GPU
        if (running && active.empty()) {
            bool idle;
            {
                std::lock_guard<std::mutex> g(S->mu);
                idle = S->pending.empty();
            }
            if (idle) {
                if (set_stop(S, 1) != MPHF_OK || cudaStreamSynchronize(S->search) != cudaSuccess ||
                    set_stop(S, 0) != MPHF_OK) {
                    cudaGetLastError();
                    fatal(MPHF_ECUDA);
                }
                running = false;
                head = tail;  // every published item was claimed and done
            }
        }
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop && S->pending.empty() && active.empty()) break;
            if (!progress) {
                if (active.empty())
                    S->cv_work.wait_for(lk, std::chrono::milliseconds(20));
                else
                    S->cv_work.wait_for(lk, std::chrono::microseconds(300));
            }
        }
    }
    // no work left: the search's blocks leave, then the server's arrays can go
    set_stop(S, 1);
    cudaStreamSynchronize(S->search);
    cudaGetLastError();
    c.release();
}

}  // namespace

extern "C" {

int mphf_server_create(const mphf_server_cfg *cfg, mphf_server_t **out) {
    if (!out) return MPHF_EINVAL;
    *out = nullptr;
    mphf_server_t *S = new (std::nothrow) mphf_server;
    if (!S) return MPHF_ENOMEM;
    S->cfg.max_requests = cfg && cfg->max_requests ? cfg->max_requests : 64;
    S->cfg.reserved_sms = cfg ? cfg->reserved_sms : 4;
    S->cfg.hbm_reserve_bytes = cfg && cfg->hbm_reserve_bytes ? cfg->hbm_reserve_bytes : (1ull << 30);
    S->cfg.idle_ms = cfg && cfg->idle_ms ? cfg->idle_ms : 10000;
    S->cfg.threads = cfg && cfg->threads ? cfg->threads : 512;
    if (S->cfg.max_requests > kMaxSlots || S->cfg.idle_ms > 600000 || S->cfg.threads % 32 ||
        S->cfg.threads < 64 || S->cfg.threads > 512) {
        delete S;
        return MPHF_EINVAL;
    }
    S->t0 = std::chrono::steady_clock::now();
    int lo_prio = 0, hi_prio = 0;
    bool ok = cudaGetDevice(&S->device) == cudaSuccess &&
              cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio) == cudaSuccess &&
              cudaStreamCreateWithPriority(&S->prep, cudaStreamNonBlocking, hi_prio) == cudaSuccess &&
              cudaStreamCreateWithPriority(&S->search, cudaStreamNonBlocking, lo_prio) == cudaSuccess &&
              cudaStreamCreateWithFlags(&S->poll, cudaStreamNonBlocking) == cudaSuccess &&
              cudaMalloc(&S->ctl, sizeof(ServeCtl)) == cudaSuccess &&
              cudaMalloc(&S->ring, kRing * sizeof(WorkItem)) == cudaSuccess &&
              cudaMalloc(&S->insts, kMaxSlots * sizeof(InstDesc)) == cudaSuccess &&
              cudaMalloc(&S->done, kMaxSlots * sizeof(unsigned int)) == cudaSuccess &&
              cudaMalloc(&S->sm_count, kServeMaxSms * sizeof(unsigned int)) == cudaSuccess &&
              cudaMallocHost(&S->pinned, 8 * (2 + kMaxSlots / 2)) == cudaSuccess &&
              cudaMemset(S->ctl, 0, sizeof(ServeCtl)) == cudaSuccess &&
              cudaMemset(S->done, 0, kMaxSlots * sizeof(unsigned int)) == cudaSuccess &&
              cudaDeviceSynchronize() == cudaSuccess;
    if (ok) S->launch = plan_serve_launch(S->cfg.threads, S->cfg.reserved_sms);
    if (ok) {
        try {
            S->control = std::thread(server_control, S);
        } catch (...) {
            ok = false;
        }
    }
    if (!ok) {
        cudaGetLastError();
        cudaFree(S->ctl);
        cudaFree(S->ring);
        cudaFree(S->insts);
        cudaFree(S->done);
        cudaFree(S->sm_count);
        if (S->pinned) cudaFreeHost(S->pinned);
        for (cudaStream_t st : {S->prep, S->search, S->poll})
            if (st) cudaStreamDestroy(st);
        delete S;
        return MPHF_ECUDA;
    }
    *out = S;
    return MPHF_OK;
}

int mphf_server_submit(mphf_server_t *S, const mphf_build_desc *desc, uint64_t *ticket) {
    if (!S || !desc || !ticket) return MPHF_EINVAL;
    ServerRequest *r = new (std::nothrow) ServerRequest;
    if (!r) return MPHF_ENOMEM;
    r->desc = *desc;
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stop || S->fatal != MPHF_OK) {
        delete r;
        return S->fatal != MPHF_OK ? S->fatal : MPHF_EBUSY;
    }
    r->ticket = S->next_ticket++;
    r->t.submitted = seconds_since(S->t0);
    try {
        S->requests[r->ticket] = r;
        S->pending.push_back(r);
    } catch (...) {
        S->requests.erase(r->ticket);
        delete r;
        return MPHF_ENOMEM;
    }
    *ticket = r->ticket;
    S->cv_work.notify_one();
    return MPHF_OK;
}

int mphf_server_poll(mphf_server_t *S, uint64_t ticket, uint32_t timeout_ms, mphf_t **out,
                     int *status, mphf_request_times *times) {
    if (!S || !out || !status) return MPHF_EINVAL;
    *out = nullptr;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->requests.find(ticket);
    if (it == S->requests.end()) return MPHF_EINVAL;
    ServerRequest *r = it->second;
    if (!r->done)
        S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; });
    if (!r->done) return MPHF_ETIMEOUT;
    *out = r->out;
    *status = r->status;
    if (times) *times = r->t;
    S->requests.erase(it);
    delete r;
    return MPHF_OK;
}

int mphf_server_destroy(mphf_server_t *S) {
    if (!S) return MPHF_EINVAL;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->control.joinable()) S->control.join();
    cudaFree(S->ctl);
    cudaFree(S->ring);
    cudaFree(S->insts);
    cudaFree(S->done);
    cudaFree(S->sm_count);
    cudaFreeHost(S->pinned);
    for (cudaStream_t st : {S->prep, S->search, S->poll}) cudaStreamDestroy(st);
    for (auto &kv : S->requests) {
        if (kv.second->out) mphf_free(kv.second->out);
        delete kv.second;
    }
    delete S;
    return MPHF_OK;
}

}  // extern "C"
