// query_kernels.cu -- evaluation of a built function on the device.
//
// Section 2.2 ("Query"): bucket of the key, two Elias-Fano lookups (keys
// before the bucket, start bit of its code), then a walk from the root:
// decode the node's value (fixed part in the bucket's fixed region, unary
// part found by select in its unary region), hash to the child, add the
// sizes of the children to its left and skip their subtrees (per-size
// tables give their node counts and fixed bits).  At the leaf: the position
// under the leaf's seed, plus the rotation r mod m for keys of B (Section 4),
// or the retrieved one of the key's two cells (ShockHash, Appendix C).
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "engine.h"
#include "mphf.h"

namespace rs {

__device__ __forceinline__ uint64_t read_bits(const uint64_t *w, uint64_t pos, uint32_t len) {
    if (len == 0) return 0;
    uint32_t sh = (uint32_t)(pos & 63);
    uint64_t v = w[pos >> 6] >> sh;
    if (sh + len > 64) v |= w[(pos >> 6) + 1] << (64 - sh);
    return len == 64 ? v : v & ((1ull << len) - 1);
}

// Position of the r-th one (0-based, r < popcount) of a word: narrow by
// the popcounts of halves, quarters and bytes, then clear at most 7 ones.
__device__ __forceinline__ uint32_t select_in_word(uint64_t word, uint32_t r) {
    uint32_t pos = 0;
    uint32_t x = (uint32_t)word, c = __popc(x);
    if (r >= c) {
        r -= c;
        x = (uint32_t)(word >> 32);
        pos = 32;
    }
    c = __popc(x & 0xFFFFu);
    if (r >= c) {
        r -= c;
        x >>= 16;
        pos += 16;
    }
    c = __popc(x & 0xFFu);
    if (r >= c) {
        r -= c;
        x >>= 8;
        pos += 8;
    }
    for (; r; r--) x &= x - 1;
    return pos + (uint32_t)(__ffs(x) - 1);
}

// Position of the j-th one (0-based) at or after bit `start`.
__device__ __forceinline__ uint64_t select_from(const uint64_t *w, uint64_t start, uint64_t j) {
    uint64_t wi = start >> 6;
    uint64_t word = w[wi] & (~0ull << (start & 63));
    for (;;) {
        uint32_t c = __popcll(word);
        if (j < c) return wi * 64 + select_in_word(word, (uint32_t)j);
        j -= c;
        word = w[++wi];
    }
}

// Element i of an Elias-Fano sequence.  The select directory gives the high
// word holding element 64 floor(i / 64); the rank directory (ones before each
// word) moves forward from there to the word holding element i, about one
// or two words since the high bits hold about two bits per element.  With
// `next` it also returns element i + 1, whose high-bit one is the next one.
__device__ __forceinline__ uint64_t ef_get(const uint64_t *low, const uint64_t *high,
                                           const uint64_t *dir, const uint64_t *seldir, uint32_t L,
                                           uint64_t i, uint64_t *next = nullptr) {
    uint64_t a = seldir[i >> 6];
    while (dir[a + 1] <= i) a++;
    uint64_t word = high[a];
    const uint32_t bit = select_in_word(word, (uint32_t)(i - dir[a]));
    const uint64_t sel = a * 64 + bit;
    if (next) {
        // the ones after element i's, in this word and then the next ones
        word = bit == 63 ? 0 : word & (~0ull << (bit + 1));
        uint64_t wi = a;
        while (!word) word = high[++wi];
        const uint64_t sel1 = wi * 64 + (uint64_t)(__ffsll((long long)word) - 1);
        *next = ((sel1 - i - 1) << L) | read_bits(low, (i + 1) * L, L);
    }
    return ((sel - i) << L) | read_bits(low, i * L, L);
}

// Unary parts of one bucket, read front to back: the walk visits nodes in
// increasing preorder index, so one cursor serves every level.  `pos` is the
// first bit of code `count` (after `count` ones from the region's start).
struct UnaryCursor {
    uint64_t pos, count;
    // the unary value (zeros before the one) of code idx >= count
    __device__ __forceinline__ uint64_t value(const uint64_t *gr, uint64_t idx) {
        const uint64_t begin = idx == count ? pos : select_from(gr, pos, idx - count - 1) + 1;
        const uint64_t end = select_from(gr, begin, 0);
        pos = end + 1;
        count = idx + 1;
        return end - begin;
    }
};

__device__ __forceinline__ uint64_t node_value(const uint64_t *gr, uint64_t fixed_pos, uint32_t tau,
                                               UnaryCursor &u, uint64_t idx) {
    const uint64_t fixed = read_bits(gr, fixed_pos, tau);
    return (u.value(gr, idx) << tau) | fixed;
}

// One thread per key (Section 2.2, "Query"; the walk is described at the
// top of this file).
// The walk reads every per-size constant from tables (remainder constants,
// fanout-2 left parts, the unit divisors' magic numbers): computing them in
// the kernel would cost 64-bit divisions at every level.
__global__ void k_query(QueryView q, const void *keys, uint64_t n, uint64_t *out) {
    const uint32_t leaf = q.leaf, lower1 = q.lower1, lower2 = q.lower2;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t *p = (const uint64_t *)keys;
        uint64_t w0 = q.key_bytes == 8 ? p[i] : p[2 * i];
        uint64_t w1 = q.key_bytes == 8 ? 0 : p[2 * i + 1];
        uint64_t hi, lo;
        fingerprint(w0, w1, hi, lo);
        uint64_t b = mulhi64(hi, q.nb);
        uint64_t nxt;
        const uint64_t cum = ef_get(q.ef_low[0], q.ef_high[0], q.ef_dir[0], q.ef_sel[0], q.ef_L[0], b,
                                    &nxt);
        const uint64_t start = ef_get(q.ef_low[1], q.ef_high[1], q.ef_dir[1], q.ef_sel[1], q.ef_L[1], b);
        uint32_t m = (uint32_t)(nxt - cum);
        if (m > 4096) {  // not a key of the built set (or a corrupt function)
            out[i] = cum;
            continue;
        }
        UnaryCursor ucur{start + q.fixed_tab[m], 0};
        uint64_t fpos = start, idx = 0, rank = 0;
        uint32_t depth = 0;
        while (m > leaf) {
            const uint32_t t = q.tau[m];
            const uint64_t x = node_value(q.gr, fpos, t, ucur, idx);
            const ModRT mod{m, q.mod_c[m], q.mod_M[m]};
            fpos += t;
            idx += 1;
            if (m > lower2) {  // fanout 2: salt 3 + depth
                const uint32_t L = 3 + depth;  // its salt from the table (a remix otherwise)
                const uint64_t salt = L < kSaltLevels ? q.salts[L] : level_salt(L);
                const uint32_t pos = mod(mix64(lo + salt + x));
                const uint32_t left = q.left_tab[m];
                if (pos < left) {
                    m = left;
                } else {
                    rank += left;
                    fpos += q.fixed_tab[left];
                    idx += q.nodes_tab[left];
                    m -= left;
                }
            } else {  // lower aggregation: children of `unit` keys, the last one smaller
                const bool l1 = m <= lower1;
                const uint32_t unit = l1 ? leaf : lower1;
                const uint32_t pos = mod(mix64(lo + level_salt(l1 ? 1 : 2) + x));
                const uint32_t c = div_unit(pos, l1 ? q.magic_leaf : q.magic_l1);
                // every child before c is a full unit
                rank += (uint64_t)c * unit;
                fpos += (uint64_t)c * q.fixed_tab[unit];
                idx += (uint64_t)c * q.nodes_tab[unit];
                m = min(unit, m - c * unit);
            }
            depth++;
        }
        if (m <= 1) {
            out[i] = cum + rank;
            continue;
        }
        const uint64_t x = node_value(q.gr, fpos, q.tau[m], ucur, idx);
        const ModRT mod{m, q.mod_c[m], q.mod_M[m]};
        uint64_t pos;
        if (q.bij == MPHF_BIJECTION_PLAIN) {
            pos = mod(mix64(lo + level_salt(0) + x));
        } else if (q.bij == MPHF_BIJECTION_SHOCKHASH) {
            // Appendix C: the retrieval vector follows the seed's tau bits;
            // parity(row & Z) says which of its two cells the key occupies
            const uint32_t z = (uint32_t)read_bits(q.gr, fpos + q.tau[m], m);
            const uint64_t h = mix64(lo + level_salt(0) + x);
            const uint32_t row = (uint32_t)mix64(lo + level_salt(MPHF_SH_ROW_LEVEL) + x) & ((1u << m) - 1);
            const uint32_t half = (__popc(row & z) & 1) ? (uint32_t)(h >> 32) : (uint32_t)h;
            pos = mod32(mod, half);
        } else {
            const uint32_t r = mod(x);  // x = k m + r
            pos = mod(mix64(lo + level_salt(0) + (x - r)));
            if (hi & 1) {  // keys of B move by r (Section 4)
                pos += r;
                if (pos >= m) pos -= m;
            }
        }
        out[i] = cum + rank + pos;
    }
}

void launch_query(const QueryView &q, const void *keys, uint64_t n, uint64_t *out, cudaStream_t st) {
    if (n == 0) return;
    uint64_t g = (n + 255) / 256;
    if (g > 148 * 64) g = 148 * 64;
    k_query<<<(uint32_t)g, 256, 0, st>>>(q, keys, n, out);
    note_launches(1);
}

// Bijection check (Section 1: h maps the n keys onto [0, n) one to one):
// every value below n and taken once.
__global__ void k_mark(const uint64_t *vals, uint64_t n, uint32_t *bitmap, unsigned long long *bad) {
    unsigned long long local = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t v = vals[i];
        if (v >= n) {
            local++;
            continue;
        }
        uint32_t bit = 1u << (v & 31);
        if (atomicOr(&bitmap[v >> 5], bit) & bit) local++;
    }
    if (local) atomicAdd(bad, local);
}

void launch_mark(const uint64_t *vals, uint64_t n, uint32_t *bitmap, unsigned long long *bad,
                 cudaStream_t st) {
    if (n == 0) return;
    uint64_t g = (n + 255) / 256;
    if (g > 148 * 64) g = 148 * 64;
    k_mark<<<(uint32_t)g, 256, 0, st>>>(vals, n, bitmap, bad);
    note_launches(1);
}

}  // namespace rs
