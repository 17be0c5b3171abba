// int_peaks.cu -- integer issue-rate microbenchmark of the GPU it runs on.
//
// The brute-force searches of the build are integer arithmetic (64-bit
// multiply-xorshift hashing and an exact remainder on 32-bit lanes), so
// their roofline is the rate at which an SM retires integer instructions,
// not memory bandwidth or tensor throughput.  This file measures that rate
// per instruction class with dependent-free chains: every thread runs eight
// independent chains of one instruction (sixteen for the mixed class), so
// latency is hidden and only the pipe's throughput limits the kernel.
//
//   kind 0  mad.lo.u32   32-bit multiply-add (the integer multiply pipe)
//   kind 1  mad.wide.u32 32x32 -> 64-bit multiply-add
//   kind 2  mad.hi.u32   high half of a 32x32 product plus an addend
//   kind 3  lop3.b32     three-input logic (the integer ALU pipe)
//   kind 4  shf.r.clamp  funnel shift (ALU)
//   kind 5  mixed        one mad.lo.u32 and one lop3.b32 per step
//   kind 6  evaluation   one key-hash evaluation of a lower-level split at
//                        l = 16 (node of 112 keys, 7 children of 16): the
//                        SplitMix64 remix, the child index (h mod 112) / 16
//                        = (h >> 4) mod 7 from the sum of two 30-bit digits
//                        (2^30 = 1 mod 7), and the packed counter update,
//                        keys and counters in registers
//   kind 7  mul64        64 x 64 -> 64-bit multiply by a runtime constant
//                        (mul.lo.u64 in inline PTX, so the chain stays one
//                        multiply per step)
//   kind 8  remix        the SplitMix64 output function on a 64-bit word
//
// Each timed launch also reads clock64 and %globaltimer in every block, so
// the result carries the SM clock the kernel actually ran at.  Used by the
// benchmark to put the search kernel's rate against a measured peak.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

extern "C" {
typedef struct {
    double ops;     // instructions (kinds 0-5) or evaluations (kind 6) per launch, all threads
    double ms;      // best launch time of the repetitions (CUDA events)
    double sm_mhz;  // SM clock during that launch (median over blocks of clock64 / globaltimer)
    double per_s;   // ops / (ms / 1000)
    uint32_t blocks, threads;
} ip_result;
}

namespace {

constexpr int kChains = 8;

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint64_t remix(uint64_t z) {  // SplitMix64 output function
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}

template <int KIND>
__device__ __forceinline__ void step(uint32_t (&x)[2 * kChains], uint64_t (&w)[kChains], uint32_t a,
                                     uint32_t b) {
#pragma unroll
    for (int c = 0; c < kChains; c++) {
        if constexpr (KIND == 0) {
            asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(a), "r"(b));
        } else if constexpr (KIND == 1) {
            const uint32_t lo = (uint32_t)w[c];
            asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(w[c]) : "r"(lo), "r"(a));
        } else if constexpr (KIND == 2) {
            asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(a), "r"(b));
        } else if constexpr (KIND == 3) {
            asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[c]) : "r"(a), "r"(b));
        } else if constexpr (KIND == 4) {
            asm volatile("shf.r.clamp.b32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(a), "r"(b));
        } else if constexpr (KIND == 5) {
            asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(a), "r"(b));
            asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[kChains + c]) : "r"(a), "r"(b));
        } else if constexpr (KIND == 7) {
            const uint64_t m = ((uint64_t)b << 32) | a;
            asm volatile("mul.lo.u64 %0, %0, %1;" : "+l"(w[c]) : "l"(m));
        } else if constexpr (KIND == 8) {
            w[c] = remix(w[c]);
        }
    }
}

template <int KIND>
__global__ void __launch_bounds__(512) k_peak(uint32_t a, uint32_t b, uint32_t iters, uint32_t *sink,
                                              unsigned long long *clk) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t x[2 * kChains];
    uint64_t w[kChains];
#pragma unroll
    for (int c = 0; c < 2 * kChains; c++) x[c] = tid * 2654435761u + (uint32_t)c;
#pragma unroll
    for (int c = 0; c < kChains; c++) w[c] = ((uint64_t)tid << 32) | (uint32_t)c;
    __syncthreads();
    const long long c0 = clock64();
    const uint64_t g0 = gtimer();
    for (uint32_t i = 0; i < iters; i++) step<KIND>(x, w, a, b);
    const long long c1 = clock64();
    const uint64_t g1 = gtimer();
    uint32_t r = 0;
#pragma unroll
    for (int c = 0; c < 2 * kChains; c++) r ^= x[c];
#pragma unroll
    for (int c = 0; c < kChains; c++) r ^= (uint32_t)w[c] ^ (uint32_t)(w[c] >> 32);
    sink[tid] = r;
    if (threadIdx.x == 0) {
        clk[2 * blockIdx.x] = (unsigned long long)(c1 - c0);
        clk[2 * blockIdx.x + 1] = g1 - g0;
    }
}

// One evaluation of a lower-1 split of l = 16 per key and seed: h = remix(x +
// s), child = (h mod 112) / 16 = (h >> 4) mod 7, taken as the sum of the two
// 30-bit digits of h >> 4 mod 7, and the child's packed counter field
// incremented (the last child's field implied, as in the build).  mask30 is
// 2^30 - 1, passed at run time like the build's table lookups.
__global__ void __launch_bounds__(512) k_eval(uint32_t mask30, uint32_t iters, uint32_t *sink,
                                              unsigned long long *clk) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t key[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) key[c] = remix(((uint64_t)tid << 8) + c);
    uint32_t cnt0 = 0, cnt1 = 0;
    __syncthreads();
    const long long c0 = clock64();
    const uint64_t g0 = gtimer();
    for (uint32_t s = 0; s < iters; s += 2) {
#pragma unroll
        for (int c = 0; c < kChains; c++) {
#pragma unroll
            for (int j = 0; j < 2; j++) {
                const uint64_t h = remix(key[c] + (uint64_t)(tid + (s + j) * 4096u));
                const uint32_t hl = (uint32_t)h, hh = (uint32_t)(h >> 32);
                const uint32_t d0 = __funnelshift_r(hl, hh, 4) & mask30, d1 = hh >> 2;
                const uint32_t child = (d0 + d1) % 7u;
                const uint32_t inc = child < 6 ? 1u << (5 * child) : 0u;
                if (j == 0)
                    cnt0 += inc;
                else
                    cnt1 += inc;
            }
        }
    }
    const long long c1 = clock64();
    const uint64_t g1 = gtimer();
    sink[tid] = cnt0 ^ (cnt1 * 3u);
    if (threadIdx.x == 0) {
        clk[2 * blockIdx.x] = (unsigned long long)(c1 - c0);
        clk[2 * blockIdx.x + 1] = g1 - g0;
    }
}

template <class F>
int time_kernel(F launch, uint32_t blocks, int reps, double *best_ms, double *mhz,
                unsigned long long *d_clk) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch();  // warm-up
    float best = 1e30f;
    std::vector<unsigned long long> clk(2 * (size_t)blocks);
    double best_mhz = 0;
    for (int r = 0; r < reps; r++) {
        cudaEventRecord(e0);
        launch();
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            cudaMemcpy(clk.data(), d_clk, clk.size() * 8, cudaMemcpyDeviceToHost);
            std::vector<double> f;
            for (uint32_t i = 0; i < blocks; i++)
                if (clk[2 * i + 1]) f.push_back(1e3 * (double)clk[2 * i] / (double)clk[2 * i + 1]);
            std::sort(f.begin(), f.end());
            best_mhz = f.empty() ? 0 : f[f.size() / 2];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *best_ms = best;
    *mhz = best_mhz;
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace

extern "C" {

// Runs instruction class `kind` (0-6, see the file comment) on the current
// device: a full grid (resident blocks of 512 threads on every SM), `reps`
// timed launches of about target_ms each after one calibration launch.
// Returns 0, -1 for a bad argument, -3 for a CUDA error.
int ip_run(int kind, int reps, double target_ms, ip_result *out) {
    if (!out || kind < 0 || kind > 8 || reps < 1 || !(target_ms > 0)) return -1;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return -3;
    }
    const void *fn = nullptr;
    switch (kind) {
        case 0: fn = (const void *)k_peak<0>; break;
        case 1: fn = (const void *)k_peak<1>; break;
        case 2: fn = (const void *)k_peak<2>; break;
        case 3: fn = (const void *)k_peak<3>; break;
        case 4: fn = (const void *)k_peak<4>; break;
        case 5: fn = (const void *)k_peak<5>; break;
        case 7: fn = (const void *)k_peak<7>; break;
        case 8: fn = (const void *)k_peak<8>; break;
        default: fn = (const void *)k_eval; break;
    }
    const uint32_t threads = 512;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, 0) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        return -3;
    }
    const uint32_t blocks = (uint32_t)sms * (uint32_t)occ;
    uint32_t *sink = nullptr;
    unsigned long long *clk = nullptr;
    if (cudaMalloc(&sink, (size_t)blocks * threads * 4) != cudaSuccess ||
        cudaMalloc(&clk, (size_t)blocks * 16) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(sink);
        return -3;
    }
    // kind 6: a loop step covers two seeds, each over kChains keys
    const double per_iter = kind == 5 ? 2.0 * kChains : kChains;
    uint32_t iters = kind >= 6 ? 64 : 1024;
    auto launch = [&]() {
        switch (kind) {
            case 0: k_peak<0><<<blocks, threads>>>(3u, 7u, iters, sink, clk); break;
            case 1: k_peak<1><<<blocks, threads>>>(3u, 7u, iters, sink, clk); break;
            case 2: k_peak<2><<<blocks, threads>>>(2654435761u, 7u, iters, sink, clk); break;
            case 3: k_peak<3><<<blocks, threads>>>(0x9E3779B9u, 0x7F4A7C15u, iters, sink, clk); break;
            case 4: k_peak<4><<<blocks, threads>>>(0x9E3779B9u, 5u, iters, sink, clk); break;
            case 5: k_peak<5><<<blocks, threads>>>(3u, 7u, iters, sink, clk); break;
            case 7: k_peak<7><<<blocks, threads>>>(0x1CE4E5B9u, 0xBF58476Du, iters, sink, clk); break;
            case 8: k_peak<8><<<blocks, threads>>>(0u, 0u, iters, sink, clk); break;
            default: k_eval<<<blocks, threads>>>((1u << 30) - 1u, iters, sink, clk); break;
        }
    };
    // calibrate the iteration count to about target_ms per launch
    double ms = 0, mhz = 0;
    int rc = time_kernel(launch, blocks, 1, &ms, &mhz, clk);
    if (rc == 0 && ms > 0) {
        double scale = target_ms / ms;
        double it = (double)iters * (scale < 1 ? 1 : scale);
        it = it > 4e6 ? 4e6 : it;
        iters = ((uint32_t)it + 1) & ~1u;
        rc = time_kernel(launch, blocks, reps, &ms, &mhz, clk);
    }
    cudaFree(sink);
    cudaFree(clk);
    if (rc) return rc;
    out->ops = (double)blocks * threads * (double)iters * per_iter;
    out->ms = ms;
    out->sm_mhz = mhz;
    out->per_s = out->ops / (ms / 1e3);
    out->blocks = blocks;
    out->threads = threads;
    return 0;
}

}  // extern "C"
