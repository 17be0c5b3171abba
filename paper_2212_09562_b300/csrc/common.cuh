// common.cuh -- hashing, tree shape and exact modulo helpers shared by the
// device kernels and the host planner of libmphf.
//
// Definitions (the method's, Section 2.2 of Bez et al. 2212.09562, with the
// readings the paper leaves open):
//   mix64       SplitMix64 output function (a bijection on 64-bit words).
//   fingerprint three Feistel rounds over mix64: (w0, w1) -> (hi, lo).
//   bucket      floor(hi * nb / 2^64).
//   shape       leaves of l keys; lower aggregation fanouts
//               f1 = max(2, ceil(0.35 l + 0.55)), f2 = max(2, ceil(0.21 l + 0.9));
//               fanout 2 above, left part a multiple of the lower-2 size.
//               The fanout-2 tree (Appendix C) has f1 = f2 = 1: every inner
//               node splits in two, its left part a multiple of l.
//   node hash   mix64(lo + salt(level) + s) mod m.
#pragma once
#include <stdint.h>

#define MPHF_GOLDEN 0x9E3779B97F4A7C15ull
#define MPHF_MAX_LEVELS 64
// ShockHash leaves (Appendix C): seed in the low 40 bits of the stored word,
// the retrieval vector above; retrieval rows hashed with the salt of level 63.
#define MPHF_SH_BITS 40
#define MPHF_SH_MASK ((1ull << MPHF_SH_BITS) - 1)
#define MPHF_SH_ROW_LEVEL 63u

namespace rs {

// The remix of the node hash (Section 2.2, "a hash function modulo l"):
// the SplitMix64 output function of Steele, Lea and Flood (OOPSLA 2014).
// mix64 without its last xor-shift: mix64(z) = y ^ (y >> 31), y = mix64_pre(z).
__host__ __device__ __forceinline__ uint64_t mix64_pre(uint64_t z) {
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    return z;
}
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = mix64_pre(z);
    return z ^ (z >> 31);
}

// The master hash code of a key (Section 2.2, the initial hash; Section 6
// uses random 128-bit codes): three Feistel rounds, invertible, so distinct
// keys never share a fingerprint.
__host__ __device__ __forceinline__ void fingerprint(uint64_t w0, uint64_t w1, uint64_t &hi,
                                                     uint64_t &lo) {
    uint64_t t1 = w1 ^ mix64(w0 + MPHF_GOLDEN);
    uint64_t t0 = w0 ^ mix64(t1 + 2 * MPHF_GOLDEN);
    t1 ^= mix64(t0 + 3 * MPHF_GOLDEN);
    hi = t0;
    lo = t1;
}

__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// Salt of a tree level: 0 leaves, 1 and 2 the lower aggregation levels,
// 3 + depth the fanout-2 nodes (depth 0 = bucket root).
__host__ __device__ __forceinline__ uint64_t level_salt(uint32_t level) {
    return mix64((uint64_t)(level + 1) * MPHF_GOLDEN);
}

enum NodeKind : uint32_t { NODE_NONE = 0, NODE_LEAF = 1, NODE_LOWER1 = 2, NODE_LOWER2 = 3, NODE_UPPER = 4 };

struct Shape {
    uint32_t leaf;    // l
    uint32_t lower1;  // f1 * l: largest node cut into leaves
    uint32_t lower2;  // f2 * f1 * l: largest node cut into lower-1 nodes
};

// tree: 0 = the two lower aggregation levels, 1 = fanout 2 everywhere.
__host__ __device__ __forceinline__ Shape make_shape(uint32_t leaf, uint32_t tree = 0) {
    uint32_t f1 = (35u * leaf + 154u) / 100u;  // ceil((35 l + 55) / 100)
    uint32_t f2 = (21u * leaf + 189u) / 100u;  // ceil((21 l + 90) / 100)
    f1 = f1 < 2 ? 2 : f1;
    f2 = f2 < 2 ? 2 : f2;
    if (tree) f1 = f2 = 1;
    Shape s;
    s.leaf = leaf;
    s.lower1 = f1 * leaf;
    s.lower2 = f2 * s.lower1;
    return s;
}

__host__ __device__ __forceinline__ uint32_t node_kind(const Shape &s, uint32_t m) {
    return m <= 1 ? NODE_NONE : m <= s.leaf ? NODE_LEAF : m <= s.lower1 ? NODE_LOWER1
         : m <= s.lower2 ? NODE_LOWER2 : NODE_UPPER;
}

// Left part of a fanout-2 node: the smallest multiple of lower2 >= m/2.
__host__ __device__ __forceinline__ uint32_t upper_left(const Shape &s, uint32_t m) {
    return ((m / 2 + s.lower2 - 1) / s.lower2) * s.lower2;
}

// Unit of a lower node (every part but the last has this size).
__host__ __device__ __forceinline__ uint32_t lower_unit(const Shape &s, uint32_t m) {
    return m <= s.lower1 ? s.leaf : s.lower1;
}

// Number of children and size of child c of an inner node.
__host__ __device__ __forceinline__ uint32_t num_parts(const Shape &s, uint32_t m) {
    if (m > s.lower2) return 2;
    uint32_t u = lower_unit(s, m);
    return (m + u - 1) / u;
}

__host__ __device__ __forceinline__ uint32_t part_size(const Shape &s, uint32_t m, uint32_t c) {
    if (m > s.lower2) {
        uint32_t left = upper_left(s, m);
        return c == 0 ? left : m - left;
    }
    uint32_t u = lower_unit(s, m);
    uint32_t rest = m - c * u;
    return rest < u ? rest : u;
}

__host__ __device__ __forceinline__ uint32_t salt_level(const Shape &s, uint32_t m, uint32_t depth) {
    uint32_t k = node_kind(s, m);
    return k == NODE_LEAF ? 0 : k == NODE_LOWER1 ? 1 : k == NODE_LOWER2 ? 2 : 3 + depth;
}

// ---------------------------------------------------------------------------
// Exact h mod m for a 64-bit h and 2 <= m <= 4096, without a 64-bit divide.
// With c = 2^32 mod m:
//   t = hi32(h) * c + lo32(h)      <  2^32 m         (so hi32(t) < m)
//   u = hi32(t) * c + lo32(t)      <  (m-1)^2 + 2^32
//   v = hi32(u) * c + lo32(u)      <  2^32           (hi32(u) = 1 forces lo32(u) < (m-1)^2)
// all congruent to h mod m; then v mod m by Lemire, Kaser and Kurz ("Faster
// remainder by direct computation", 2019): M = floor((2^64 - 1) / m) + 1,
// v mod m = hi64((M * v mod 2^64) * m), exact for every 32-bit v.
struct ModRT {
    uint32_t m, c;
    uint64_t M;
    __host__ __device__ __forceinline__ uint32_t operator()(uint64_t h) const {
        uint64_t t = (uint64_t)(uint32_t)(h >> 32) * c + (uint32_t)h;
        uint64_t u = (uint64_t)(uint32_t)(t >> 32) * c + (uint32_t)t;
        uint32_t v = (uint32_t)(u >> 32) * c + (uint32_t)u;
        uint64_t low = M * v;
        return (uint32_t)mulhi64(low, m);
    }
};

__host__ __device__ __forceinline__ ModRT make_mod(uint32_t m) {
    ModRT r;
    r.m = m;
    r.c = (uint32_t)((1ull << 32) % m);
    r.M = 0xFFFFFFFFFFFFFFFFull / m + 1;
    return r;
}

// ShockHash cells of a key: the two 32-bit halves of h, each mod m (Lemire,
// Kaser and Kurz's direct remainder, exact for 32-bit values).
__host__ __device__ __forceinline__ uint32_t mod32(const ModRT &r, uint32_t v) {
    return (uint32_t)mulhi64(r.M * v, r.m);
}

// Compile-time modulus: same reduction, the last step by the compiler's
// constant division; a power of two is a mask.
template <uint32_t MM>
struct ModCT {
    __device__ __forceinline__ uint32_t operator()(uint64_t h) const {
        if constexpr ((MM & (MM - 1)) == 0) {
            return (uint32_t)h & (MM - 1);
        } else {
            constexpr uint32_t c = (uint32_t)((1ull << 32) % MM);
            uint64_t t = (uint64_t)(uint32_t)(h >> 32) * c + (uint32_t)h;
            uint64_t u = (uint64_t)(uint32_t)(t >> 32) * c + (uint32_t)t;
            uint32_t v = (uint32_t)(u >> 32) * c + (uint32_t)u;
            return v % MM;
        }
    }
};

// floor(p / unit) for p < 4096 and 2 <= unit <= 4096: with g = ceil(2^32 / unit)
// and e = g * unit - 2^32 < unit, p * g / 2^32 = p / unit + p * e / (unit 2^32),
// and p * e < 2^24 keeps the error below 1 / unit, so hi32(p * g) is exact.
__host__ __device__ __forceinline__ uint32_t unit_magic(uint32_t unit) {
    return (uint32_t)(((1ull << 32) + unit - 1) / unit);
}

__device__ __forceinline__ uint32_t div_unit(uint32_t p, uint32_t magic) { return __umulhi(p, magic); }

// Field width of a packed child counter: enough bits for the largest part.
__host__ __device__ __forceinline__ uint32_t counter_width(uint32_t max_part) {
    uint32_t w = 1;
    while ((1u << w) <= max_part) w++;
    return w;
}

// Sizes of an Elias-Fano sequence of k values whose largest is `last`
// (Section 2.1): L low bits each, high bits in unary.
struct EfDims {
    uint32_t L;
    uint64_t low_words, high_words;
};

__host__ __device__ inline EfDims ef_dims(uint64_t k, uint64_t last) {
    EfDims d;
    d.L = 0;
    if (last >= k) {
        uint64_t q = last / k;
        while (q >>= 1) d.L++;
    }
    d.low_words = (k * d.L + 63) / 64;
    d.high_words = ((last >> d.L) + k + 63) / 64;
    return d;
}

}  // namespace rs
