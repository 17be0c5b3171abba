// noalloc.cu -- a bijection check that allocates no device memory.
//
// mphf_verify allocates its scratch (one value per key, a bitmap over [0, n)
// and a counter) on every call.  Some callers cannot do that where they want
// to check a function: a service whose device memory is owned and budgeted by
// another allocator (a framework's caching allocator), a latency-critical path
// where cudaMalloc / cudaFree may synchronise the device and stall other
// streams, or code that runs where allocation is not permitted at all.
// mphf_verify_static gives them the same check with a fixed scratch area that
// the library reserves in device memory on every GPU where it is loaded.
//
// The scratch is shared by every call: calls whose work overlaps on the
// device race on it and must be serialised (one stream, or wait for the
// previous call).  The first call on a device looks up the scratch address
// with cudaGetSymbolAddress; make that first call before any stream capture.
// The address is kept for the life of the process: a cudaDeviceReset (or any
// other teardown of the device's primary context) makes it stale, so the
// entry point must not be called on a device after it was reset.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "engine.h"
#include "mphf.h"

namespace {

constexpr uint64_t kMaxKeys = MPHF_VERIFY_STATIC_MAX_KEYS;
constexpr uint64_t kBitmapWords = kMaxKeys / 64;  // bitmap over [0, n) as 64-bit words
constexpr int kMaxDevices = 64;

// Per-key query values, then the bitmap, then the counter of bad keys.
static __device__ __align__(256) uint64_t g_verify_scratch[kMaxKeys + kBitmapWords + 1];

std::mutex g_mu;
uint64_t *g_scratch[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device (looked up once per
// device; the host-side symbol itself is not a device address).
int scratch_address(uint64_t **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return MPHF_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return MPHF_EINVAL;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_verify_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return MPHF_ECUDA;
        }
        g_scratch[dev] = (uint64_t *)p;
    }
    *out = g_scratch[dev];
    return MPHF_OK;
}

}  // namespace

extern "C" int mphf_verify_static(const mphf_t *h, const void *d_keys, uint64_t n, uint64_t *n_bad,
                                  void *stream) {
    if (!h || !n_bad || (n > 0 && !d_keys)) return MPHF_EINVAL;
    *n_bad = 0;
    if (n > kMaxKeys) return MPHF_EINVAL;  // more keys than the fixed scratch holds
    if ((uintptr_t)d_keys & 7) return MPHF_EINVAL;
    if (n == 0) return MPHF_OK;
    uint64_t *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != MPHF_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t *vals = base;
    uint32_t *bitmap = (uint32_t *)(base + kMaxKeys);
    unsigned long long *bad = (unsigned long long *)(base + kMaxKeys + kBitmapWords);
    // the previous call left its bitmap and count behind: clear what this call uses
    if (cudaMemsetAsync(bitmap, 0, ((n + 63) / 64) * 8, st) != cudaSuccess ||
        cudaMemsetAsync(bad, 0, sizeof(*bad), st) != cudaSuccess) {
        cudaGetLastError();
        return MPHF_ECUDA;
    }
    rc = mphf_query(h, d_keys, n, vals, stream);
    if (rc != MPHF_OK) return rc;
    rs::launch_mark(vals, n, bitmap, bad, st);
    unsigned long long hb = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return MPHF_ECUDA;
    }
    *n_bad = hb;
    return MPHF_OK;
}
