/*
 * recsplit_oracle.c -- plain, sequential CPU oracle for RecSplit minimal
 * perfect hash construction with rotation fitting, after Bez, Kurpicz,
 * Lehmann and Sanders, "High Performance Construction of RecSplit Based
 * Minimal Perfect Hash Functions" (arXiv 2212.09562).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the correctness authority that
 * the CUDA path is checked against.  Only the test suite, the package smoke
 * check and the CPU-baseline / reference legs of the benchmark may load it.
 * The product library neither links it nor shares any code, header or table
 * with it; both sides implement the same definitions independently.
 *
 * Every step follows the paper in its own order, one key and one trial at a
 * time: no blocking, no fusion, no reordering, no early exits that the
 * definition does not have.  Where the paper is silent the readings below
 * are used (they are listed with reasons in the project design notes):
 *
 *   R1  mix64 is the SplitMix64 output function; the 128-bit fingerprint of
 *       a key (w0, w1) is three Feistel rounds over mix64, hi = t0, lo = t1.
 *   R2  nb = ceil(n / b) buckets, bucket(hi) = floor(hi * nb / 2^64).
 *   R3  tree shape: leaves of l keys, lower aggregation fanouts
 *       f1 = max(2, ceil(0.35 l + 0.55)), f2 = max(2, ceil(0.21 l + 0.9)) in
 *       integer arithmetic, fanout 2 above with the left part a multiple of
 *       the lower-2 node size.  The fanout-2 tree of Appendix C (used there
 *       with ShockHash leaves) has fanout 2 everywhere: f1 = f2 = 1, so every
 *       inner node splits in two with its left part a multiple of l.  In
 *       this file's interface a leaf size argument with ORC_TREE_FANOUT2
 *       set selects that tree.
 *   R4  the hash tried at a node is mix64(lo + salt(level) + s) mod m.
 *   R5  rotation fitting puts a key in B iff (hi & 1) = 1; a rotation by r
 *       moves bit p of B's mask to bit (p + r) mod m.
 *   R6  Golomb-Rice parameter per node from Kiely's rule for a geometric
 *       source; the success probability of a rotation leaf uses the bound of
 *       the Appendix A lemma.
 *   R7  ShockHash leaves (Appendix C): under seed s a key has the two cells
 *       (h mod 2^32) mod m and (h >> 32) mod m of h = mix64(lo + salt(0) + s).
 *       The cells of the m keys must admit a bijection, i.e. every connected
 *       component of the cuckoo graph has as many keys as cells.  The
 *       canonical choice: tree edges point away from the cycle; on each cycle
 *       the key with the smallest lo word takes its first cell.  The chosen
 *       bit of every key is retrieved through one GF(2) equation per key,
 *       row = mix64(lo + salt(63) + s) mod 2^m, value = parity(row & Z); Z is
 *       the solution whose non-pivot coordinates (reduced row echelon form,
 *       pivots at the lowest set bit) are zero.  The stored value is the
 *       smallest s for which the graph admits a bijection and the system is
 *       solvable, with Z in bits 40.. of the stored word.
 *
 * Parity pins: see the oracle test files (fixed points from the paper's
 * figures, closed forms, invariants, brute force on tiny inputs).  The
 * absolute seed values are fixed only by the definitions above; beyond the
 * brute-force minimality check they are "parity unpinned".
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_EDUPLICATE (-4)
#define ORC_ESEARCH_LIMIT (-5)
#define ORC_EBUCKET (-7)

#define ORC_MAX_BUCKET 4096u
#define ORC_TREE_FANOUT2 0x100u /* flag on a leaf size argument: fanout 2 everywhere */
#define ORC_MAX_LEAF 24u
#define ORC_MAX_PARTS 16u
#define ORC_GOLDEN 0x9E3779B97F4A7C15ull

/* leaf bijection methods */
#define ORC_BIJ_PLAIN 0
#define ORC_BIJ_ROTATION 1
#define ORC_BIJ_SHOCKHASH 2
#define ORC_SH_SEED_BITS 40 /* ShockHash: seed in bits 0..39, retrieval vector above */
#define ORC_SH_SEED_MASK ((1ull << ORC_SH_SEED_BITS) - 1)
#define ORC_SH_RETRIEVAL_LEVEL 63u

enum { KIND_NONE = 0, KIND_LEAF = 1, KIND_LOWER1 = 2, KIND_LOWER2 = 3, KIND_UPPER = 4 };
enum { ST_LEAF = 0, ST_LOWER1 = 1, ST_LOWER2 = 2, ST_UPPER = 3, ST_N = 4 };

/* ------------------------------------------------------------------------ */
/* R1: hashing.  SplitMix64 output function (Steele, Lea, Flood, OOPSLA     */
/* 2014).  The paper's initial hash (Section 2.2, "Splitting Trees"; master */
/* hash codes in Section 6) is only required to be of high quality.        */
/* ------------------------------------------------------------------------ */
uint64_t orc_mix64(uint64_t z) {
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}

static uint64_t load_le64(const uint8_t *p) {
    uint64_t v = 0;
    for (int i = 7; i >= 0; i--) v = (v << 8) | p[i];
    return v;
}

/* 128-bit master hash code of every key: three Feistel rounds, so distinct
 * keys always get distinct fingerprints. */
void orc_fingerprint(const uint8_t *keys, uint64_t n, uint32_t key_bytes, uint64_t *hi,
                     uint64_t *lo) {
    for (uint64_t i = 0; i < n; i++) {
        const uint8_t *k = keys + i * key_bytes;
        uint64_t w0 = load_le64(k);
        uint64_t w1 = key_bytes == 16 ? load_le64(k + 8) : 0;
        uint64_t t1 = w1 ^ orc_mix64(w0 + ORC_GOLDEN);
        uint64_t t0 = w0 ^ orc_mix64(t1 + 2 * ORC_GOLDEN);
        t1 ^= orc_mix64(t0 + 3 * ORC_GOLDEN);
        hi[i] = t0;
        lo[i] = t1;
    }
}

/* R2: bucket of a fingerprint (Section 2.2: objects go to buckets of
 * expected size b). */
uint64_t orc_bucket_of(uint64_t hi, uint64_t nb) {
    return (uint64_t)(((unsigned __int128)hi * nb) >> 64);
}

/* ------------------------------------------------------------------------ */
/* R3: splitting-tree shape (Section 2.2, "Splitting Trees").               */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint32_t leaf;   /* l                                   */
    uint32_t f1, f2; /* lower aggregation fanouts            */
    uint32_t lower1; /* largest node split into leaves: f1*l */
    uint32_t lower2; /* largest lower-2 node: f2*f1*l        */
} orc_shape;

/* Fanouts and unit sizes of the tree for leaf size l (Section 2.2,
 * "Splitting Trees"; reading R3, or R18 for the fanout-2 tree flag). */
static orc_shape shape_of(uint32_t leaf_arg) {
    orc_shape sh;
    uint32_t leaf = leaf_arg & 0xFFu;
    sh.leaf = leaf;
    if (leaf_arg & ORC_TREE_FANOUT2) {
        sh.f1 = sh.f2 = 1;
    } else {
        sh.f1 = (35 * leaf + 55 + 99) / 100; /* ceil(0.35 l + 0.55) */
        if (sh.f1 < 2) sh.f1 = 2;
        sh.f2 = (21 * leaf + 90 + 99) / 100; /* ceil(0.21 l + 0.90) */
        if (sh.f2 < 2) sh.f2 = 2;
    }
    sh.lower1 = sh.f1 * leaf;
    sh.lower2 = sh.f2 * sh.lower1;
    return sh;
}

void orc_fanouts(uint32_t leaf, uint32_t *f1, uint32_t *f2) {
    orc_shape sh = shape_of(leaf);
    *f1 = sh.f1;
    *f2 = sh.f2;
}

/* Kind of the node of m keys (Section 2.2): none (m <= 1), leaf (m <= l),
 * lower level 1 or 2, or fanout 2 above. */
static int kind_of(const orc_shape *sh, uint32_t m) {
    if (m <= 1) return KIND_NONE;
    if (m <= sh->leaf) return KIND_LEAF;
    if (m <= sh->lower1) return KIND_LOWER1;
    if (m <= sh->lower2) return KIND_LOWER2;
    return KIND_UPPER;
}

/* Part sizes of an inner node of m keys, left to right.  Lower levels cut
 * into units (l or f1*l) with the remainder last; upper levels cut in two. */
static uint32_t parts_of(const orc_shape *sh, uint32_t m, uint32_t *parts) {
    int kind = kind_of(sh, m);
    uint32_t np = 0;
    if (kind == KIND_LOWER1 || kind == KIND_LOWER2) {
        uint32_t unit = kind == KIND_LOWER1 ? sh->leaf : sh->lower1;
        uint32_t left = m;
        while (left > 0) {
            uint32_t p = left < unit ? left : unit;
            parts[np++] = p;
            left -= p;
        }
    } else if (kind == KIND_UPPER) {
        uint32_t half = m / 2;
        uint32_t left = ((half + sh->lower2 - 1) / sh->lower2) * sh->lower2;
        parts[np++] = left;
        parts[np++] = m - left;
    }
    return np;
}

uint32_t orc_parts(uint32_t leaf, uint32_t m, uint32_t *parts) {
    orc_shape sh = shape_of(leaf);
    return parts_of(&sh, m, parts);
}

/* Number of stored nodes (nodes with at least two keys) in the tree of m
 * (Section 2.2: one stored value per node of the splitting tree). */
static uint64_t count_nodes(const orc_shape *sh, uint32_t m) {
    if (m <= 1) return 0;
    if (m <= sh->leaf) return 1;
    uint32_t parts[ORC_MAX_PARTS];
    uint32_t np = parts_of(sh, m, parts);
    uint64_t c = 1;
    for (uint32_t i = 0; i < np; i++) c += count_nodes(sh, parts[i]);
    return c;
}

uint64_t orc_count_nodes(uint32_t leaf, uint32_t m) {
    orc_shape sh = shape_of(leaf);
    return count_nodes(&sh, m);
}

/* R4: the salt distinguishes the tree levels.  Level 0 = leaves, 1 = lower
 * aggregation level next to the leaves, 2 = the one above, 3 + depth for
 * the fanout-2 nodes (depth counted from the bucket's root, root = 0). */
uint64_t orc_salt(uint32_t level) { return orc_mix64((uint64_t)(level + 1) * ORC_GOLDEN); }

static uint32_t level_of(const orc_shape *sh, uint32_t m, uint32_t depth) {
    int kind = kind_of(sh, m);
    if (kind == KIND_LEAF) return 0;
    if (kind == KIND_LOWER1) return 1;
    if (kind == KIND_LOWER2) return 2;
    return 3 + depth;
}

/* Child index of hash position pos in [0, m) for an inner node. */
static uint32_t child_of(const orc_shape *sh, uint32_t m, const uint32_t *parts, uint64_t pos) {
    int kind = kind_of(sh, m);
    if (kind == KIND_UPPER) return pos < parts[0] ? 0 : 1;
    uint32_t unit = kind == KIND_LOWER1 ? sh->leaf : sh->lower1;
    return (uint32_t)(pos / unit);
}

/* ------------------------------------------------------------------------ */
/* Statistics (trials = candidate values tested, evals = key hashes).       */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t trials[ST_N];
    uint64_t evals[ST_N];
} orc_stats;

/* ------------------------------------------------------------------------ */
/* Split search (Section 2.2 "Splitting Trees"; Section 5.1 "Splittings"):  */
/* the smallest s >= 0 whose hash gives every child exactly its part size.  */
/* ------------------------------------------------------------------------ */
static int split_search(const orc_shape *sh, const uint64_t *lo, uint32_t m, uint32_t depth,
                        uint64_t max_value, uint64_t *out, orc_stats *st) {
    uint32_t parts[ORC_MAX_PARTS], count[ORC_MAX_PARTS];
    uint32_t np = parts_of(sh, m, parts);
    uint64_t salt = orc_salt(level_of(sh, m, depth));
    int sk = kind_of(sh, m) == KIND_LOWER1 ? ST_LOWER1
           : kind_of(sh, m) == KIND_LOWER2 ? ST_LOWER2 : ST_UPPER;
    for (uint64_t s = 0;; s++) {
        memset(count, 0, sizeof(count));
        for (uint32_t i = 0; i < m; i++) {
            uint64_t pos = orc_mix64(lo[i] + salt + s) % m;
            count[child_of(sh, m, parts, pos)]++;
        }
        st->trials[sk]++;
        st->evals[sk] += m;
        int ok = 1;
        for (uint32_t c = 0; c < np; c++) ok &= count[c] == parts[c];
        if (ok) {
            *out = s;
            return ORC_OK;
        }
        if (s == max_value) return ORC_ESEARCH_LIMIT;
    }
}

/* ------------------------------------------------------------------------ */
/* Leaf bijection, plain brute force (Section 2.2 "Bijections"): smallest s */
/* whose hash mod m sets all m bits of the OR of 2^pos.                     */
/* ------------------------------------------------------------------------ */
static int leaf_plain(const uint64_t *lo, uint32_t m, uint64_t max_value, uint64_t *out,
                      orc_stats *st) {
    uint64_t salt = orc_salt(0);
    uint32_t full = (m == 32) ? 0xFFFFFFFFu : ((1u << m) - 1);
    for (uint64_t s = 0;; s++) {
        uint32_t mask = 0;
        for (uint32_t i = 0; i < m; i++) mask |= 1u << (orc_mix64(lo[i] + salt + s) % m);
        st->trials[ST_LEAF]++;
        st->evals[ST_LEAF] += m;
        if (mask == full) {
            *out = s;
            return ORC_OK;
        }
        if (s == max_value) return ORC_ESEARCH_LIMIT;
    }
}

/* rot_m^r(x): rotate the m low bits of x left by r (Section 2.1). */
static uint32_t rotl_m(uint32_t x, uint32_t r, uint32_t m) {
    uint32_t full = (1u << m) - 1;
    if (r == 0) return x & full;
    return ((x << r) | (x >> (m - r))) & full;
}

/* ------------------------------------------------------------------------ */
/* Leaf bijection with rotation fitting (Section 4).  Only seeds k*m are    */
/* hashed; the keys of A set bits of a, the keys of B bits of b.  The first */
/* k for which some rotation r makes a | rot(b, r) full is taken, with the  */
/* smallest such r, and k*m + r is stored (the smallest stored number, as   */
/* Section 5.1 requires).                                                   */
/* ------------------------------------------------------------------------ */
static int leaf_rotation(const uint64_t *lo, const uint64_t *hi, uint32_t m, uint64_t max_value,
                         uint64_t *out, orc_stats *st) {
    uint64_t salt = orc_salt(0);
    uint32_t full = (1u << m) - 1;
    for (uint64_t k = 0;; k++) {
        uint64_t s = k * m;
        if (s > max_value) return ORC_ESEARCH_LIMIT;
        uint32_t a = 0, b = 0;
        for (uint32_t i = 0; i < m; i++) {
            uint32_t bit = 1u << (orc_mix64(lo[i] + salt + s) % m);
            if (hi[i] & 1)
                b |= bit;
            else
                a |= bit;
        }
        st->trials[ST_LEAF]++;
        st->evals[ST_LEAF] += m;
        for (uint32_t r = 0; r < m; r++) {
            if ((a | rotl_m(b, r, m)) == full) {
                if (s + r > max_value) return ORC_ESEARCH_LIMIT;
                *out = s + r;
                return ORC_OK;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* R7: ShockHash leaves (Appendix C).  A trial is a pair of hash functions; */
/* the m keys are the edges of a multigraph on the m cells (a loop when     */
/* both cells agree).  A bijection picking one cell per key exists iff no   */
/* component has more keys than cells (with m keys on m cells: iff every    */
/* component has exactly one cycle).                                        */
/* ------------------------------------------------------------------------ */
static double binom(uint32_t n, uint32_t k);

/* The two cells of a key under seed s (Appendix C's two hash functions of
 * a trial; reading R14: the two halves of one 64-bit hash). */
static void sh_cells(uint64_t lo, uint64_t s, uint32_t m, uint32_t *c0, uint32_t *c1) {
    uint64_t h = orc_mix64(lo + orc_salt(0) + s);
    *c0 = (uint32_t)(h & 0xFFFFFFFFu) % m;
    *c1 = (uint32_t)(h >> 32) % m;
}

/* Union-find over the cells; orientable iff edges == cells in every
 * component (Appendix C: the graph must be a pseudo-forest). */
static int sh_orientable(const uint32_t *c0, const uint32_t *c1, uint32_t m) {
    uint32_t comp[ORC_MAX_LEAF], cells[ORC_MAX_LEAF], edges[ORC_MAX_LEAF];
    for (uint32_t v = 0; v < m; v++) {
        comp[v] = v;
        cells[v] = 1;
        edges[v] = 0;
    }
    for (uint32_t i = 0; i < m; i++) {
        uint32_t a = comp[c0[i]], b = comp[c1[i]];
        if (a != b) { /* merge component b into a */
            for (uint32_t v = 0; v < m; v++)
                if (comp[v] == b) comp[v] = a;
            cells[a] += cells[b];
            edges[a] += edges[b];
        }
        edges[a] += 1;
    }
    for (uint32_t v = 0; v < m; v++)
        if (comp[v] == v && edges[v] != cells[v]) return 0;
    return 1;
}

/* The canonical bijection of an orientable trial: beta[i] = 0 if key i takes
 * cell c0[i], 1 if c1[i].  First every cell of degree one takes its only
 * remaining key (the trees hanging off the cycles), then each remaining
 * cycle is walked from its key with the smallest lo word, which takes its
 * first cell. */
static void sh_orientation(const uint64_t *lo, const uint32_t *c0, const uint32_t *c1, uint32_t m,
                           uint8_t *beta) {
    uint32_t deg[ORC_MAX_LEAF];
    uint8_t alive[ORC_MAX_LEAF];
    memset(deg, 0, sizeof(deg));
    for (uint32_t i = 0; i < m; i++) {
        deg[c0[i]]++;
        deg[c1[i]]++;
        alive[i] = 1;
        beta[i] = 0;
    }
    for (;;) { /* peel cells of degree one */
        uint32_t c = m;
        for (uint32_t v = 0; v < m && c == m; v++)
            if (deg[v] == 1) c = v;
        if (c == m) break;
        uint32_t e = m;
        for (uint32_t i = 0; i < m && e == m; i++)
            if (alive[i] && (c0[i] == c || c1[i] == c)) e = i;
        beta[e] = c0[e] == c ? 0 : 1;
        alive[e] = 0;
        uint32_t other = c0[e] == c ? c1[e] : c0[e];
        deg[c] = 0;
        deg[other]--;
    }
    for (;;) { /* the cycles */
        uint32_t e0 = m;
        for (uint32_t i = 0; i < m; i++)
            if (alive[i] && (e0 == m || lo[i] < lo[e0])) e0 = i;
        if (e0 == m) break;
        beta[e0] = 0;
        alive[e0] = 0;
        uint32_t start = c0[e0], cur = c1[e0];
        while (cur != start) {
            uint32_t e = m;
            for (uint32_t i = 0; i < m && e == m; i++)
                if (alive[i] && (c0[i] == cur || c1[i] == cur)) e = i;
            beta[e] = c0[e] == cur ? 0 : 1;
            alive[e] = 0;
            cur = c0[e] == cur ? c1[e] : c0[e];
        }
    }
}

/* Retrieval of one bit per key (Appendix C; reading R16): solve row_i . Z = rhs_i over GF(2) by
 * Gauss-Jordan elimination, columns in increasing order, pivot row of a
 * column = the first remaining row with that bit.  Returns 1 and the
 * solution with zero non-pivot coordinates, or 0 if inconsistent. */
static int sh_solve(const uint32_t *row_in, const uint8_t *rhs_in, uint32_t m, uint32_t *z) {
    uint32_t row[ORC_MAX_LEAF];
    uint8_t rhs[ORC_MAX_LEAF], piv[ORC_MAX_LEAF];
    int32_t col_row[32];
    for (uint32_t i = 0; i < m; i++) {
        row[i] = row_in[i];
        rhs[i] = rhs_in[i];
        piv[i] = 0;
    }
    for (uint32_t j = 0; j < m; j++) {
        col_row[j] = -1;
        uint32_t p = m;
        for (uint32_t i = 0; i < m && p == m; i++)
            if (!piv[i] && ((row[i] >> j) & 1)) p = i;
        if (p == m) continue;
        piv[p] = 1;
        col_row[j] = (int32_t)p;
        for (uint32_t i = 0; i < m; i++)
            if (i != p && ((row[i] >> j) & 1)) {
                row[i] ^= row[p];
                rhs[i] ^= rhs[p];
            }
    }
    for (uint32_t i = 0; i < m; i++)
        if (!piv[i] && rhs[i]) return 0; /* a zero row with value one */
    uint32_t out = 0;
    for (uint32_t j = 0; j < m; j++)
        if (col_row[j] >= 0 && rhs[col_row[j]]) out |= 1u << j;
    *z = out;
    return 1;
}

/* A key's row of the retrieval system under seed s (reading R16, Appendix C). */
static uint32_t sh_row(uint64_t lo, uint64_t s, uint32_t m) {
    uint64_t h = orc_mix64(lo + orc_salt(ORC_SH_RETRIEVAL_LEVEL) + s);
    return (uint32_t)(h & ((1ull << m) - 1));
}

static int leaf_shockhash(const uint64_t *lo, uint32_t m, uint64_t max_value, uint64_t *out,
                          orc_stats *st) {
    uint32_t c0[ORC_MAX_LEAF], c1[ORC_MAX_LEAF], rows[ORC_MAX_LEAF];
    uint8_t beta[ORC_MAX_LEAF];
    if (max_value > ORC_SH_SEED_MASK) max_value = ORC_SH_SEED_MASK;
    for (uint64_t s = 0;; s++) {
        for (uint32_t i = 0; i < m; i++) sh_cells(lo[i], s, m, &c0[i], &c1[i]);
        st->trials[ST_LEAF]++;
        st->evals[ST_LEAF] += m;
        if (sh_orientable(c0, c1, m)) {
            sh_orientation(lo, c0, c1, m, beta);
            for (uint32_t i = 0; i < m; i++) rows[i] = sh_row(lo[i], s, m);
            uint32_t z;
            if (sh_solve(rows, beta, m, &z)) {
                *out = s | ((uint64_t)z << ORC_SH_SEED_BITS);
                return ORC_OK;
            }
        }
        if (s == max_value) return ORC_ESEARCH_LIMIT;
    }
}

/* Probability that m keys with two uniform cells each (out of m) admit a
 * bijection (Appendix C's success condition; used for tau, reading R17).  Counting labelled edge lists with ordered cell pairs: the
 * pairs (list, valid choice vector) number m! 2^m m^m (pick the bijection,
 * the bits, the free cell), and a list whose components are all unicyclic
 * has 2 choices per component.  With W(k) = k! 2^k k^k, the connected
 * unicyclic lists U(k) follow from W(k) = sum_j C(k-1,j-1) C(k,j) 2U(j)
 * W(k-j) (the component of cell 0 has j cells and j keys), and the
 * orientable lists O(k) = sum_j C(k-1,j-1) C(k,j) U(j) O(k-j). */
double orc_shockhash_orient_prob(uint32_t m) {
    double W[ORC_MAX_LEAF + 1], U[ORC_MAX_LEAF + 1], O[ORC_MAX_LEAF + 1];
    if (m == 0 || m > ORC_MAX_LEAF) return 0.0;
    W[0] = 1.0;
    O[0] = 1.0;
    for (uint32_t k = 1; k <= m; k++) {
        double w = 1.0;
        for (uint32_t i = 1; i <= k; i++) w *= (double)i * 2.0 * (double)k;
        W[k] = w;
        double rest = 0.0;
        for (uint32_t j = 1; j < k; j++) rest += binom(k - 1, j - 1) * binom(k, j) * 2.0 * U[j] * W[k - j];
        U[k] = (W[k] - rest) / 2.0;
        double o = 0.0;
        for (uint32_t j = 1; j <= k; j++) o += binom(k - 1, j - 1) * binom(k, j) * U[j] * O[k - j];
        O[k] = o;
    }
    return O[m] / pow((double)m, 2.0 * (double)m);
}

/* Probability that m uniform random GF(2) rows of m bits give a solvable
 * system for a fixed nonzero right-hand side (retrieval, reading R17): sum over the rank r of
 * P(rank r) * (2^r - 1)/(2^m - 1), the column space being a uniform
 * r-dimensional subspace; P(rank r) = 2^-(m-r)^2 prod_{i<r}
 * (1 - 2^(i-m))^2 / (1 - 2^(i-r)). */
double orc_retrieval_solvable_prob(uint32_t m) {
    double total = 0.0;
    for (uint32_t r = 0; r <= m; r++) {
        double p = ldexp(1.0, -(int)((m - r) * (m - r)));
        for (uint32_t i = 0; i < r; i++) {
            double a = 1.0 - ldexp(1.0, (int)i - (int)m);
            p *= a * a / (1.0 - ldexp(1.0, (int)i - (int)r));
        }
        total += p * (ldexp(1.0, (int)r) - 1.0) / (ldexp(1.0, (int)m) - 1.0);
    }
    return total;
}

/* ------------------------------------------------------------------------ */
/* R6: Golomb-Rice parameter per node (Section 2.2 "Representation": the    */
/* optimal parameter depends on the layer and is precomputed).              */
/* ------------------------------------------------------------------------ */

/* Probability that j keys hashed uniformly into m cells all differ. */
static double prob_distinct(uint32_t j, uint32_t m) {
    double p = 1.0;
    for (uint32_t i = 0; i < j; i++) p *= (double)(m - i) / (double)m;
    return p;
}

static double binom(uint32_t n, uint32_t k) {
    if (k > n) return 0.0;
    double c = 1.0;
    for (uint32_t i = 1; i <= k; i++) c = c * (double)(n - k + i) / (double)i;
    return c;
}

static uint32_t gcd_u32(uint32_t a, uint32_t b) {
    while (b) {
        uint32_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

static uint32_t euler_phi(uint32_t d) {
    uint32_t c = 0;
    for (uint32_t j = 1; j <= d; j++) c += gcd_u32(d, j) == 1;
    return c;
}

/* Appendix A lemma: lower bound of the probability that one hash function
 * (one k) gives a rotation-fitting bijection on a leaf of m keys of which a
 * are in A and b = m - a in B:
 *   P(A distinct) * P(B distinct) * m / sum_{d | gcd(a,b)} phi(d) C(m/d, b/d),
 * the last factor being one over the number of rotation classes of b-subsets. */
double orc_rotation_bound_given_a(uint32_t m, uint32_t a) {
    uint32_t b = m - a;
    uint32_t g = gcd_u32(a, b);
    double classes = 0.0;
    for (uint32_t d = 1; d <= g; d++)
        if (g % d == 0) classes += (double)euler_phi(d) * binom(m / d, b / d);
    double p_fit = (double)m / classes;
    if (p_fit > 1.0) p_fit = 1.0;
    return prob_distinct(a, m) * prob_distinct(b, m) * p_fit;
}

/* The same bound averaged over the fixed 1-bit split, |A| ~ Binomial(m, 1/2). */
double orc_rotation_success_bound(uint32_t m) {
    double total = 0.0;
    for (uint32_t a = 0; a <= m; a++)
        total += binom(m, a) * ldexp(1.0, -(int)m) * orc_rotation_bound_given_a(m, a);
    return total;
}

/* Success probability of one brute-force leaf trial: m!/m^m. */
double orc_plain_success(uint32_t m) { return prob_distinct(m, m); }

/* Success probability of one split trial (Section 2.2, "Splitting Trees"):
 * multinomial m!/prod p_i! prod (p_i/m)^p_i. */
static double split_success(const orc_shape *sh, uint32_t m) {
    uint32_t parts[ORC_MAX_PARTS];
    uint32_t np = parts_of(sh, m, parts);
    double lp = lgamma((double)m + 1.0);
    for (uint32_t i = 0; i < np; i++)
        lp += -lgamma((double)parts[i] + 1.0) + (double)parts[i] * log((double)parts[i] / (double)m);
    return exp(lp);
}

double orc_split_success(uint32_t leaf, uint32_t m) {
    orc_shape sh = shape_of(leaf);
    return split_success(&sh, m);
}

/* Kiely's rule for the Rice parameter of a geometric source with success
 * probability p per stored unit: max(0, 1 + floor(log2(ln(phi-1)/ln(1-p)))). */
uint32_t orc_kiely_tau(double p) {
    double golden = (1.0 + sqrt(5.0)) / 2.0;
    double t = 1.0 + floor(log2(log(golden - 1.0) / log1p(-p)));
    return t < 0.0 ? 0u : (uint32_t)t;
}

/* Success probability per stored unit of the node of m keys, the p of the
 * Golomb-Rice parameter (Section 2.2, "Representation"; reading R7; Appendix
 * A's bound for rotation leaves).  A ShockHash
 * trial succeeds when the graph admits a bijection and the retrieval system
 * of its chosen bits is solvable (taken as independent events). */
static double unit_success(const orc_shape *sh, int bij, uint32_t m) {
    if (kind_of(sh, m) == KIND_LEAF) {
        if (bij == ORC_BIJ_ROTATION) return orc_rotation_success_bound(m) / (double)m;
        if (bij == ORC_BIJ_SHOCKHASH)
            return orc_shockhash_orient_prob(m) * orc_retrieval_solvable_prob(m);
        return orc_plain_success(m);
    }
    return split_success(sh, m);
}

/* tau[m] for every node size m in [0, max_m]; m < 2 gives 0. */
void orc_tau_table(uint32_t leaf, int bij, uint32_t max_m, uint8_t *tau) {
    orc_shape sh = shape_of(leaf);
    for (uint32_t m = 0; m <= max_m; m++)
        tau[m] = m < 2 ? 0 : (uint8_t)orc_kiely_tau(unit_success(&sh, bij, m));
}

/* Fixed-part width of a node (Section 2.2, "Representation"): tau bits of
 * the value, plus the m retrieval bits of a ShockHash leaf (reading R16). */
static uint32_t fixed_width(const orc_shape *sh, int bij, const uint8_t *tau, uint32_t m) {
    uint32_t w = tau[m];
    if (bij == ORC_BIJ_SHOCKHASH && kind_of(sh, m) == KIND_LEAF) w += m;
    return w;
}

/* ------------------------------------------------------------------------ */
/* Elias-Fano (Section 2.1): low L bits of value i at bits [iL, iL+L) of    */
/* the low array; a 1 at position (v_i >> L) + i of the high array.         */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint32_t L;
    uint64_t low_words, high_words;
} ef_dims;

static uint32_t floor_log2_u64(uint64_t x) {
    uint32_t r = 0;
    while (x >>= 1) r++;
    return r;
}

/* Elias-Fano sizes of k values ending at `last` (Section 2.1, "Elias-Fano";
 * the two bucket sequences of Section 2.2, "Representation"; reading R9):
 * L = floor(log2(last / k)) low bits each. */
static ef_dims ef_dims_of(uint64_t k, uint64_t last) {
    ef_dims d;
    d.L = last >= k ? floor_log2_u64(last / k) : 0;
    d.low_words = (k * d.L + 63) / 64;
    d.high_words = ((last >> d.L) + k + 63) / 64;
    return d;
}

static void set_bit(uint64_t *w, uint64_t i) { w[i >> 6] |= 1ull << (i & 63); }
static int get_bit(const uint64_t *w, uint64_t i) { return (int)((w[i >> 6] >> (i & 63)) & 1); }

/* Elias-Fano encoding of v[0..k) (Section 2.1, "Elias-Fano"): the low L
 * bits of v[i] at i*L, a one at position (v[i] >> L) + i of the high part. */
static void ef_encode(const uint64_t *v, uint64_t k, ef_dims d, uint64_t *low, uint64_t *high) {
    for (uint64_t i = 0; i < k; i++) {
        for (uint32_t j = 0; j < d.L; j++)
            if ((v[i] >> j) & 1) set_bit(low, i * d.L + j);
        set_bit(high, (v[i] >> d.L) + i);
    }
}

static uint64_t ef_get(const uint64_t *low, const uint64_t *high, uint64_t high_words, ef_dims d,
                       uint64_t i) {
    /* select_1(i) on the high bits by scanning */
    uint64_t seen = 0, pos = 0;
    for (uint64_t w = 0; w < high_words; w++) {
        uint64_t word = high[w];
        uint32_t c = (uint32_t)__builtin_popcountll(word);
        if (seen + c > i) {
            for (uint32_t b = 0; b < 64; b++) {
                if ((word >> b) & 1) {
                    if (seen == i) {
                        pos = w * 64 + b;
                        goto found;
                    }
                    seen++;
                }
            }
        }
        seen += c;
    }
found:;
    uint64_t lowv = 0;
    for (uint32_t j = 0; j < d.L; j++) lowv |= (uint64_t)get_bit(low, i * d.L + j) << j;
    return ((pos - i) << d.L) | lowv;
}

/* ------------------------------------------------------------------------ */
/* The built function.                                                      */
/* ------------------------------------------------------------------------ */
typedef struct orc_mphf {
    uint64_t n, nb;
    uint32_t leaf, bucket_size, bij, key_bytes; /* bij: ORC_BIJ_* leaf method */
    uint64_t *cum_keys; /* nb+1: keys in buckets before i              */
    uint64_t *node_off; /* nb+1: first stored node of bucket i          */
    uint64_t *values;   /* node_off[nb] values, preorder in each bucket */
    uint64_t *bit_pos;  /* nb+1: first Golomb-Rice bit of bucket i      */
    uint64_t *gr;
    uint64_t gr_words, gr_bits;
    ef_dims ef_cum, ef_pos;
    uint64_t *ef; /* low(cum) | high(cum) | low(pos) | high(pos)   */
    uint64_t ef_words;
    uint8_t *tau;   /* tau[m], m in [0, ORC_MAX_BUCKET]           */
    uint64_t *nodes_tab, *fixed_tab; /* per m: stored nodes, fixed bits of the subtree */
    orc_stats stats;
} orc_mphf;

static void fill_subtree_tables(const orc_shape *sh, int bij, const uint8_t *tau, uint32_t max_m,
                                uint64_t *nodes_tab, uint64_t *fixed_tab) {
    for (uint32_t m = 0; m <= max_m; m++) {
        if (m <= 1) {
            nodes_tab[m] = 0;
            fixed_tab[m] = 0;
            continue;
        }
        uint32_t parts[ORC_MAX_PARTS];
        uint32_t np = parts_of(sh, m, parts);
        uint64_t c = 1, f = fixed_width(sh, bij, tau, m);
        for (uint32_t i = 0; i < np; i++) {
            c += nodes_tab[parts[i]];
            f += fixed_tab[parts[i]];
        }
        nodes_tab[m] = c;
        fixed_tab[m] = f;
    }
}

/* Per-bucket work: keys of one bucket, its search results in preorder. */
typedef struct {
    const orc_shape *sh;
    int bij;
    uint64_t max_value;
    uint64_t *values; /* where this bucket's nodes go */
    uint64_t count;   /* nodes written so far          */
    orc_stats *st;
} bucket_ctx;

/* Recursive preorder construction of one node (Section 2.2: the identifiers
 * are stored in preorder).  lo/hi hold the node's keys, tlo/thi a scratch
 * area of the same length used to regroup the keys by child. */
static int build_node(bucket_ctx *cx, uint64_t *lo, uint64_t *hi, uint64_t *tlo, uint64_t *thi,
                      uint32_t m, uint32_t depth) {
    const orc_shape *sh = cx->sh;
    int kind = kind_of(sh, m);
    if (kind == KIND_NONE) return ORC_OK;
    uint64_t x;
    int rc;
    if (kind == KIND_LEAF) {
        if (cx->bij == ORC_BIJ_ROTATION)
            rc = leaf_rotation(lo, hi, m, cx->max_value, &x, cx->st);
        else if (cx->bij == ORC_BIJ_SHOCKHASH)
            rc = leaf_shockhash(lo, m, cx->max_value, &x, cx->st);
        else
            rc = leaf_plain(lo, m, cx->max_value, &x, cx->st);
        if (rc) return rc;
        cx->values[cx->count++] = x;
        return ORC_OK;
    }
    rc = split_search(sh, lo, m, depth, cx->max_value, &x, cx->st);
    if (rc) return rc;
    cx->values[cx->count++] = x;
    /* regroup the keys by child with the seed found (Section 5.1, end of
     * "Splittings"): counting sort by child index */
    uint32_t parts[ORC_MAX_PARTS], start[ORC_MAX_PARTS];
    uint32_t np = parts_of(sh, m, parts);
    uint64_t salt = orc_salt(level_of(sh, m, depth));
    start[0] = 0;
    for (uint32_t c = 1; c < np; c++) start[c] = start[c - 1] + parts[c - 1];
    for (uint32_t i = 0; i < m; i++) {
        uint64_t pos = orc_mix64(lo[i] + salt + x) % m;
        uint32_t c = child_of(sh, m, parts, pos);
        tlo[start[c]] = lo[i];
        thi[start[c]] = hi[i];
        start[c]++;
    }
    memcpy(lo, tlo, (size_t)m * sizeof(uint64_t));
    memcpy(hi, thi, (size_t)m * sizeof(uint64_t));
    uint32_t off = 0;
    for (uint32_t c = 0; c < np; c++) {
        rc = build_node(cx, lo + off, hi + off, tlo + off, thi + off, parts[c], depth + 1);
        if (rc) return rc;
        off += parts[c];
    }
    return ORC_OK;
}

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : x > y;
}

/* Two keys of one bucket with the same lo word meet at every split and can
 * never be told apart by a leaf hash: the build refuses them (reading R12;
 * the paper assumes distinct keys, Section 1). */
static int has_duplicate(const uint64_t *lo, uint32_t m, uint64_t *scratch) {
    memcpy(scratch, lo, (size_t)m * sizeof(uint64_t));
    qsort(scratch, m, sizeof(uint64_t), cmp_u64);
    for (uint32_t i = 1; i < m; i++)
        if (scratch[i] == scratch[i - 1]) return 1;
    return 0;
}

/* Keys grouped by bucket (stable counting sort by bucket index). */
typedef struct {
    uint64_t n, nb;
    uint64_t *hi, *lo; /* in bucket order */
    uint64_t *cum;     /* nb+1            */
} grouped;

static int group_keys(const uint8_t *keys, uint64_t n, uint32_t key_bytes, uint64_t nb,
                      grouped *g) {
    g->n = n;
    g->nb = nb;
    uint64_t *hi = malloc((n ? n : 1) * sizeof(uint64_t));
    uint64_t *lo = malloc((n ? n : 1) * sizeof(uint64_t));
    g->hi = malloc((n ? n : 1) * sizeof(uint64_t));
    g->lo = malloc((n ? n : 1) * sizeof(uint64_t));
    g->cum = calloc(nb + 2, sizeof(uint64_t));
    uint64_t *cursor = calloc(nb + 1, sizeof(uint64_t));
    if (!hi || !lo || !g->hi || !g->lo || !g->cum || !cursor) {
        free(hi); free(lo); free(cursor);
        return ORC_ENOMEM;
    }
    orc_fingerprint(keys, n, key_bytes, hi, lo);
    for (uint64_t i = 0; i < n; i++) g->cum[orc_bucket_of(hi[i], nb) + 1]++;
    for (uint64_t b = 0; b < nb; b++) g->cum[b + 1] += g->cum[b];
    for (uint64_t b = 0; b < nb; b++) cursor[b] = g->cum[b];
    for (uint64_t i = 0; i < n; i++) {
        uint64_t b = orc_bucket_of(hi[i], nb);
        g->hi[cursor[b]] = hi[i];
        g->lo[cursor[b]] = lo[i];
        cursor[b]++;
    }
    free(hi);
    free(lo);
    free(cursor);
    return ORC_OK;
}

static void free_grouped(grouped *g) {
    free(g->hi);
    free(g->lo);
    free(g->cum);
}

/* Section 5.2: every thread takes a consecutive range of buckets. */
typedef struct {
    const grouped *g;
    const orc_shape *sh;
    int bij;
    uint64_t max_value;
    const uint64_t *bucket_list; /* buckets to build, in output order */
    const uint64_t *out_off;     /* first output node per list entry  */
    uint64_t first, last;        /* list range of this thread          */
    uint64_t *values;
    int phase; /* 0 = duplicate check, 1 = search */
    int rc;
    orc_stats st;
} worker;

static void *worker_run(void *arg) {
    worker *w = arg;
    uint64_t *lo = malloc(ORC_MAX_BUCKET * sizeof(uint64_t));
    uint64_t *hi = malloc(ORC_MAX_BUCKET * sizeof(uint64_t));
    uint64_t *tlo = malloc(ORC_MAX_BUCKET * sizeof(uint64_t));
    uint64_t *thi = malloc(ORC_MAX_BUCKET * sizeof(uint64_t));
    w->rc = ORC_OK;
    memset(&w->st, 0, sizeof(w->st));
    if (!lo || !hi || !tlo || !thi) {
        w->rc = ORC_ENOMEM;
        goto done;
    }
    for (uint64_t j = w->first; j < w->last; j++) {
        uint64_t b = w->bucket_list[j];
        uint64_t start = w->g->cum[b];
        uint32_t m = (uint32_t)(w->g->cum[b + 1] - start);
        memcpy(lo, w->g->lo + start, (size_t)m * sizeof(uint64_t));
        memcpy(hi, w->g->hi + start, (size_t)m * sizeof(uint64_t));
        if (w->phase == 0) {
            if (has_duplicate(lo, m, tlo)) {
                w->rc = ORC_EDUPLICATE;
                break;
            }
            continue;
        }
        bucket_ctx cx = {w->sh, w->bij, w->max_value, w->values + w->out_off[j], 0, &w->st};
        int rc = build_node(&cx, lo, hi, tlo, thi, m, 0);
        if (rc) {
            w->rc = rc;
            break;
        }
    }
done:
    free(lo);
    free(hi);
    free(tlo);
    free(thi);
    return NULL;
}

/* Runs the duplicate check over all listed buckets, then the searches. */
static int run_buckets(const grouped *g, const orc_shape *sh, int bij, uint64_t max_value,
                       const uint64_t *list, const uint64_t *out_off, uint64_t count,
                       uint64_t *values, int threads, orc_stats *st) {
    if (threads < 1) threads = 1;
    if ((uint64_t)threads > count) threads = count ? (int)count : 1;
    worker *ws = calloc((size_t)threads, sizeof(worker));
    pthread_t *tid = calloc((size_t)threads, sizeof(pthread_t));
    if (!ws || !tid) {
        free(ws); free(tid);
        return ORC_ENOMEM;
    }
    int rc = ORC_OK;
    for (int phase = 0; phase < 2 && rc == ORC_OK; phase++) {
        for (int t = 0; t < threads; t++) {
            worker *w = &ws[t];
            w->g = g; w->sh = sh; w->bij = bij; w->max_value = max_value;
            w->bucket_list = list; w->out_off = out_off; w->values = values;
            w->first = count * (uint64_t)t / (uint64_t)threads;
            w->last = count * (uint64_t)(t + 1) / (uint64_t)threads;
            w->phase = phase;
            if (threads == 1)
                worker_run(w);
            else
                pthread_create(&tid[t], NULL, worker_run, w);
        }
        if (threads > 1)
            for (int t = 0; t < threads; t++) pthread_join(tid[t], NULL);
        /* precedence: out of memory, then duplicates, then the search cap */
        for (int t = 0; t < threads; t++)
            if (ws[t].rc == ORC_ENOMEM) rc = ORC_ENOMEM;
        for (int t = 0; t < threads && rc == ORC_OK; t++)
            if (ws[t].rc) rc = ws[t].rc;
        if (phase == 1)
            for (int t = 0; t < threads; t++)
                for (int k = 0; k < ST_N; k++) {
                    st->trials[k] += ws[t].st.trials[k];
                    st->evals[k] += ws[t].st.evals[k];
                }
    }
    free(ws);
    free(tid);
    return rc;
}

static int check_params(uint64_t n, uint32_t key_bytes, uint32_t leaf, uint32_t bucket_size,
                        int bij) {
    if (bij < ORC_BIJ_PLAIN || bij > ORC_BIJ_SHOCKHASH) return ORC_EINVAL;
    if (key_bytes != 8 && key_bytes != 16) return ORC_EINVAL;
    if (leaf & ~(ORC_TREE_FANOUT2 | 0xFFu)) return ORC_EINVAL;
    leaf &= 0xFFu;
    if (leaf < 2 || leaf > ORC_MAX_LEAF) return ORC_EINVAL;
    if (bucket_size < 1 || bucket_size > 3000) return ORC_EINVAL;
    if (n >= (1ull << 32)) return ORC_EINVAL;
    return ORC_OK;
}

void orc_free(orc_mphf *h) {
    if (!h) return;
    free(h->cum_keys); free(h->node_off); free(h->values); free(h->bit_pos);
    free(h->gr); free(h->ef); free(h->tau); free(h->nodes_tab); free(h->fixed_tab);
    free(h);
}

/* Golomb-Rice writer (Section 2.1; Section 2.2 "Representation": per tree,
 * all fixed parts in preorder, then all unary parts in preorder). */
static int is_shock_leaf(const orc_mphf *h, const orc_shape *sh, uint32_t m) {
    return h->bij == ORC_BIJ_SHOCKHASH && kind_of(sh, m) == KIND_LEAF;
}

/* The Golomb-Rice coded number of a stored word (Section 2.2,
 * "Representation"): the seed of a ShockHash leaf (its retrieval vector goes
 * to the fixed part verbatim, reading R16), else the word. */
static uint64_t coded_value(const orc_mphf *h, const orc_shape *sh, uint32_t m, uint64_t v) {
    return is_shock_leaf(h, sh, m) ? (v & ORC_SH_SEED_MASK) : v;
}

static uint64_t bucket_bits(const orc_mphf *h, const orc_shape *sh, const uint64_t *vals,
                            const uint32_t *sizes, uint64_t count) {
    uint64_t bits = 0;
    for (uint64_t j = 0; j < count; j++) {
        uint32_t t = h->tau[sizes[j]];
        bits += fixed_width(sh, (int)h->bij, h->tau, sizes[j]) + 1 +
                (coded_value(h, sh, sizes[j], vals[j]) >> t);
    }
    return bits;
}

/* Node sizes of a bucket's tree in preorder (Section 2.2: the values are
 * stored in preorder). */
static void preorder_sizes(const orc_shape *sh, uint32_t m, uint32_t *out, uint64_t *count) {
    if (m <= 1) return;
    out[(*count)++] = m;
    if (m <= sh->leaf) return;
    uint32_t parts[ORC_MAX_PARTS];
    uint32_t np = parts_of(sh, m, parts);
    for (uint32_t i = 0; i < np; i++) preorder_sizes(sh, parts[i], out, count);
}

/* Builds buckets [b_lo, b_hi) of the function over n_total keys from the n
 * keys that fall into exactly those buckets (Section 5.2: a thread that
 * takes a consecutive range of buckets produces that range's node values,
 * a local Golomb-Rice sequence and local bucket offsets; the ranges'
 * sequences concatenated in bucket order are the function's).  The arrays
 * of the result are local to the range: cum_keys, node_off and bit_pos
 * start at 0.  A key whose bucket lies outside the range gives ORC_EINVAL.
 * A full build is the range [0, nb) of its own keys. */
static int build_range(const uint8_t *keys, uint64_t n, uint32_t key_bytes, uint64_t n_total,
                       uint32_t leaf, uint32_t bucket_size, int bij, uint64_t max_value,
                       int threads, uint64_t b_lo, uint64_t b_hi, orc_mphf **out) {
    *out = NULL;
    int rc = check_params(n_total, key_bytes, leaf, bucket_size, bij);
    if (rc) return rc;
    const uint64_t nb_total = (n_total + bucket_size - 1) / bucket_size;
    if (n > n_total || b_lo > b_hi || b_hi > nb_total) return ORC_EINVAL;
    orc_shape sh = shape_of(leaf);
    const uint64_t nb = b_hi - b_lo;
    grouped g;
    rc = group_keys(keys, n, key_bytes, nb_total, &g);
    if (rc) return rc;
    if (g.cum[b_lo] != 0 || g.cum[b_hi] != n) { /* some key belongs to another range */
        free_grouped(&g);
        return ORC_EINVAL;
    }
    orc_mphf *h = calloc(1, sizeof(orc_mphf));
    if (!h) { free_grouped(&g); return ORC_ENOMEM; }
    h->n = n; h->nb = nb; h->leaf = leaf; h->bucket_size = bucket_size;
    h->bij = (uint32_t)bij; h->key_bytes = key_bytes;
    h->tau = malloc(ORC_MAX_BUCKET + 1);
    h->nodes_tab = malloc((ORC_MAX_BUCKET + 1) * sizeof(uint64_t));
    h->fixed_tab = malloc((ORC_MAX_BUCKET + 1) * sizeof(uint64_t));
    h->cum_keys = malloc((nb + 1) * sizeof(uint64_t));
    h->node_off = malloc((nb + 1) * sizeof(uint64_t));
    h->bit_pos = malloc((nb + 1) * sizeof(uint64_t));
    uint64_t *list = malloc((nb ? nb : 1) * sizeof(uint64_t));
    if (!h->tau || !h->nodes_tab || !h->fixed_tab || !h->cum_keys || !h->node_off ||
        !h->bit_pos || !list) {
        rc = ORC_ENOMEM;
        goto fail;
    }
    orc_tau_table(leaf, bij, ORC_MAX_BUCKET, h->tau);
    fill_subtree_tables(&sh, bij, h->tau, ORC_MAX_BUCKET, h->nodes_tab, h->fixed_tab);
    memcpy(h->cum_keys, g.cum + b_lo, (nb + 1) * sizeof(uint64_t));
    h->node_off[0] = 0;
    for (uint64_t b = 0; b < nb; b++) {
        uint64_t m = h->cum_keys[b + 1] - h->cum_keys[b];
        if (m > ORC_MAX_BUCKET) { rc = ORC_EBUCKET; goto fail; }
        h->node_off[b + 1] = h->node_off[b] + count_nodes(&sh, (uint32_t)m);
        list[b] = b_lo + b;
    }
    h->values = calloc(h->node_off[nb] ? h->node_off[nb] : 1, sizeof(uint64_t));
    if (!h->values) { rc = ORC_ENOMEM; goto fail; }
    rc = run_buckets(&g, &sh, bij, max_value, list, h->node_off, nb, h->values, threads,
                     &h->stats);
    if (rc) goto fail;

    /* Golomb-Rice: bucket lengths, prefix sums, then the bits. */
    {
        uint32_t *sizes = malloc(ORC_MAX_BUCKET * sizeof(uint32_t));
        if (!sizes) { rc = ORC_ENOMEM; goto fail; }
        h->bit_pos[0] = 0;
        for (uint64_t b = 0; b < nb; b++) {
            uint32_t m = (uint32_t)(h->cum_keys[b + 1] - h->cum_keys[b]);
            uint64_t cnt = 0;
            preorder_sizes(&sh, m, sizes, &cnt);
            h->bit_pos[b + 1] = h->bit_pos[b] + bucket_bits(h, &sh, h->values + h->node_off[b], sizes, cnt);
        }
        h->gr_bits = h->bit_pos[nb];
        h->gr_words = (h->gr_bits + 63) / 64;
        h->gr = calloc(h->gr_words ? h->gr_words : 1, sizeof(uint64_t));
        if (!h->gr) { free(sizes); rc = ORC_ENOMEM; goto fail; }
        for (uint64_t b = 0; b < nb; b++) {
            uint32_t m = (uint32_t)(h->cum_keys[b + 1] - h->cum_keys[b]);
            uint64_t cnt = 0;
            preorder_sizes(&sh, m, sizes, &cnt);
            const uint64_t *vals = h->values + h->node_off[b];
            uint64_t pos = h->bit_pos[b];
            for (uint64_t j = 0; j < cnt; j++) { /* fixed parts */
                uint32_t t = h->tau[sizes[j]];
                uint64_t x = coded_value(h, &sh, sizes[j], vals[j]);
                for (uint32_t i = 0; i < t; i++)
                    if ((x >> i) & 1) set_bit(h->gr, pos + i);
                pos += t;
                if (is_shock_leaf(h, &sh, sizes[j])) { /* the retrieval vector */
                    uint64_t z = vals[j] >> ORC_SH_SEED_BITS;
                    for (uint32_t i = 0; i < sizes[j]; i++)
                        if ((z >> i) & 1) set_bit(h->gr, pos + i);
                    pos += sizes[j];
                }
            }
            for (uint64_t j = 0; j < cnt; j++) { /* unary parts */
                pos += coded_value(h, &sh, sizes[j], vals[j]) >> h->tau[sizes[j]];
                set_bit(h->gr, pos);
                pos++;
            }
        }
        free(sizes);
    }

    /* Elias-Fano over the bucket prefix sums and the bucket bit positions
     * (Section 2.2 "Representation"). */
    h->ef_cum = ef_dims_of(nb + 1, h->cum_keys[nb]);
    h->ef_pos = ef_dims_of(nb + 1, h->bit_pos[nb]);
    h->ef_words = h->ef_cum.low_words + h->ef_cum.high_words + h->ef_pos.low_words +
                  h->ef_pos.high_words;
    h->ef = calloc(h->ef_words ? h->ef_words : 1, sizeof(uint64_t));
    if (!h->ef) { rc = ORC_ENOMEM; goto fail; }
    {
        uint64_t *p = h->ef;
        ef_encode(h->cum_keys, nb + 1, h->ef_cum, p, p + h->ef_cum.low_words);
        p += h->ef_cum.low_words + h->ef_cum.high_words;
        ef_encode(h->bit_pos, nb + 1, h->ef_pos, p, p + h->ef_pos.low_words);
    }
    free(list);
    free_grouped(&g);
    *out = h;
    return ORC_OK;
fail:
    free(list);
    free_grouped(&g);
    orc_free(h);
    return rc;
}

/* Full build.  Returns ORC_OK and a new function in *out, or an error. */
int orc_build(const uint8_t *keys, uint64_t n, uint32_t key_bytes, uint32_t leaf,
              uint32_t bucket_size, int bij, uint64_t max_value, int threads,
              orc_mphf **out) {
    *out = NULL;
    if (bucket_size < 1) return ORC_EINVAL;
    const uint64_t nb = (n + bucket_size - 1) / bucket_size;
    return build_range(keys, n, key_bytes, n, leaf, bucket_size, bij, max_value, threads, 0, nb,
                       out);
}

/* One consecutive bucket range of the function over n_total keys (see
 * build_range); the result's query is not defined. */
int orc_build_range(const uint8_t *keys, uint64_t n, uint32_t key_bytes, uint64_t n_total,
                    uint32_t leaf, uint32_t bucket_size, int bij, uint64_t max_value, int threads,
                    uint64_t b_lo, uint64_t b_hi, orc_mphf **out) {
    return build_range(keys, n, key_bytes, n_total, leaf, bucket_size, bij, max_value, threads,
                       b_lo, b_hi, out);
}

/* Builds only the listed buckets of the full key set and writes their node
 * values, bucket after bucket in list order, each in preorder.  Used to
 * check large builds on a sample of buckets. */
int orc_build_sample(const uint8_t *keys, uint64_t n, uint32_t key_bytes, uint32_t leaf,
                     uint32_t bucket_size, int bij, uint64_t max_value, int threads,
                     const uint64_t *buckets, uint64_t count, uint64_t *values_out,
                     uint64_t *node_counts, uint64_t *stats_out) {
    int rc = check_params(n, key_bytes, leaf, bucket_size, bij);
    if (rc) return rc;
    orc_shape sh = shape_of(leaf);
    uint64_t nb = (n + bucket_size - 1) / bucket_size;
    grouped g;
    rc = group_keys(keys, n, key_bytes, nb, &g);
    if (rc) return rc;
    uint64_t *off = malloc((count + 1) * sizeof(uint64_t));
    if (!off) { free_grouped(&g); return ORC_ENOMEM; }
    off[0] = 0;
    for (uint64_t j = 0; j < count; j++) {
        if (buckets[j] >= nb) { free(off); free_grouped(&g); return ORC_EINVAL; }
        uint64_t m = g.cum[buckets[j] + 1] - g.cum[buckets[j]];
        if (m > ORC_MAX_BUCKET) { free(off); free_grouped(&g); return ORC_EBUCKET; }
        node_counts[j] = count_nodes(&sh, (uint32_t)m);
        off[j + 1] = off[j] + node_counts[j];
    }
    orc_stats st;
    memset(&st, 0, sizeof(st));
    rc = run_buckets(&g, &sh, bij, max_value, buckets, off, count, values_out, threads, &st);
    if (stats_out)
        for (int k = 0; k < ST_N; k++) {
            stats_out[2 * k] = st.trials[k];
            stats_out[2 * k + 1] = st.evals[k];
        }
    free(off);
    free_grouped(&g);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Query (Section 2.2 "Query"; Section 4: a rotation is an addition mod m   */
/* for the keys of B).                                                      */
/* ------------------------------------------------------------------------ */

/* select_1 in the unary region of a bucket: position of the j-th one. */
static uint64_t unary_select(const uint64_t *gr, uint64_t start, uint64_t j) {
    uint64_t seen = 0;
    for (uint64_t p = start;; p++) {
        if (get_bit(gr, p)) {
            if (seen == j) return p;
            seen++;
        }
    }
}

static uint64_t node_value(const orc_mphf *h, uint64_t fixed_pos, uint32_t tau,
                           uint64_t unary_start, uint64_t idx) {
    uint64_t fixed = 0;
    for (uint32_t i = 0; i < tau; i++) fixed |= (uint64_t)get_bit(h->gr, fixed_pos + i) << i;
    uint64_t end = unary_select(h->gr, unary_start, idx);
    uint64_t begin = idx == 0 ? unary_start : unary_select(h->gr, unary_start, idx - 1) + 1;
    return ((end - begin) << tau) | fixed;
}

/* The value of one key (Section 2.2, "Query"): its bucket, the bucket's key
 * offset and code start from the Elias-Fano sequences, then from the root
 * one decoded value and child per level, adding the sizes of the children to
 * the left, down to the leaf: the key's position under the leaf's seed, plus
 * r mod m for keys of B (Section 4), or the retrieved one of its two cells
 * (Appendix C). */
static uint64_t query_one(const orc_mphf *h, const orc_shape *sh, uint64_t hi, uint64_t lo) {
    uint64_t b = orc_bucket_of(hi, h->nb);
    const uint64_t *e = h->ef;
    uint64_t cum = ef_get(e, e + h->ef_cum.low_words, h->ef_cum.high_words, h->ef_cum, b);
    uint64_t next = ef_get(e, e + h->ef_cum.low_words, h->ef_cum.high_words, h->ef_cum, b + 1);
    const uint64_t *pe = e + h->ef_cum.low_words + h->ef_cum.high_words;
    uint64_t start = ef_get(pe, pe + h->ef_pos.low_words, h->ef_pos.high_words, h->ef_pos, b);
    uint32_t m = (uint32_t)(next - cum);
    uint64_t unary_start = start + h->fixed_tab[m];
    uint64_t fixed_pos = start, idx = 0, rank = 0;
    uint32_t depth = 0;
    while (m > sh->leaf) {
        uint64_t x = node_value(h, fixed_pos, h->tau[m], unary_start, idx);
        uint32_t parts[ORC_MAX_PARTS];
        parts_of(sh, m, parts);
        uint64_t pos = orc_mix64(lo + orc_salt(level_of(sh, m, depth)) + x) % m;
        uint32_t c = child_of(sh, m, parts, pos);
        fixed_pos += h->tau[m];
        idx += 1;
        for (uint32_t j = 0; j < c; j++) {
            rank += parts[j];
            fixed_pos += h->fixed_tab[parts[j]];
            idx += h->nodes_tab[parts[j]];
        }
        m = parts[c];
        depth++;
    }
    if (m <= 1) return cum + rank;
    uint64_t x = node_value(h, fixed_pos, h->tau[m], unary_start, idx);
    if (h->bij == ORC_BIJ_PLAIN) return cum + rank + orc_mix64(lo + orc_salt(0) + x) % m;
    if (h->bij == ORC_BIJ_SHOCKHASH) {
        /* the retrieval vector follows the seed's tau bits in the fixed part;
         * the key's bit selects which of its two cells it occupies */
        uint64_t z = 0;
        for (uint32_t i = 0; i < m; i++)
            z |= (uint64_t)get_bit(h->gr, fixed_pos + h->tau[m] + i) << i;
        uint32_t c0, c1;
        sh_cells(lo, x, m, &c0, &c1);
        uint32_t bit = (uint32_t)__builtin_popcountll(sh_row(lo, x, m) & z) & 1;
        return cum + rank + (bit ? c1 : c0);
    }
    uint64_t r = x % m;
    uint64_t pos = orc_mix64(lo + orc_salt(0) + (x - r)) % m;
    if (hi & 1) pos = (pos + r) % m;
    return cum + rank + pos;
}

void orc_query(const orc_mphf *h, const uint8_t *keys, uint64_t n, uint64_t *out) {
    orc_shape sh = shape_of(h->leaf);
    for (uint64_t i = 0; i < n; i++) {
        uint64_t hi, lo;
        orc_fingerprint(keys + i * h->key_bytes, 1, h->key_bytes, &hi, &lo);
        out[i] = query_one(h, &sh, hi, lo);
    }
}

/* ------------------------------------------------------------------------ */
/* Accessors for the test suite.                                            */
/* ------------------------------------------------------------------------ */
void orc_sizes(const orc_mphf *h, uint64_t *out) {
    out[0] = h->n;
    out[1] = h->nb;
    out[2] = h->node_off[h->nb];
    out[3] = h->gr_bits;
    out[4] = h->gr_words;
    out[5] = h->ef_words;
    out[6] = h->ef_cum.L;
    out[7] = h->ef_pos.L;
}

void orc_copy_out(const orc_mphf *h, uint64_t *cum_keys, uint64_t *node_off, uint64_t *values,
                  uint64_t *bit_pos, uint64_t *gr, uint64_t *ef, uint64_t *stats) {
    uint64_t nb = h->nb;
    if (cum_keys) memcpy(cum_keys, h->cum_keys, (nb + 1) * sizeof(uint64_t));
    if (node_off) memcpy(node_off, h->node_off, (nb + 1) * sizeof(uint64_t));
    if (values) memcpy(values, h->values, h->node_off[nb] * sizeof(uint64_t));
    if (bit_pos) memcpy(bit_pos, h->bit_pos, (nb + 1) * sizeof(uint64_t));
    if (gr) memcpy(gr, h->gr, h->gr_words * sizeof(uint64_t));
    if (ef) memcpy(ef, h->ef, h->ef_words * sizeof(uint64_t));
    if (stats)
        for (int k = 0; k < ST_N; k++) {
            stats[2 * k] = h->stats.trials[k];
            stats[2 * k + 1] = h->stats.evals[k];
        }
}

/* Single-node searches, for brute-force checks and per-node statistics.
 * kind: the node's own keys, its depth in the bucket tree (salt level of
 * fanout-2 nodes), and the values found / trials / hash evaluations. */
int orc_node_search(uint32_t leaf, int bij, const uint64_t *lo, const uint64_t *hi,
                    uint32_t m, uint32_t depth, uint64_t max_value, uint64_t *x, uint64_t *stats) {
    orc_shape sh = shape_of(leaf);
    orc_stats st;
    memset(&st, 0, sizeof(st));
    int rc;
    int kind = kind_of(&sh, m);
    if (kind == KIND_NONE) return ORC_EINVAL;
    if (kind == KIND_LEAF)
        rc = bij == ORC_BIJ_ROTATION    ? leaf_rotation(lo, hi, m, max_value, x, &st)
           : bij == ORC_BIJ_SHOCKHASH ? leaf_shockhash(lo, m, max_value, x, &st)
                                      : leaf_plain(lo, m, max_value, x, &st);
    else
        rc = split_search(&sh, lo, m, depth, max_value, x, &st);
    if (stats) {
        uint64_t t = 0, e = 0;
        for (int k = 0; k < ST_N; k++) { t += st.trials[k]; e += st.evals[k]; }
        stats[0] = t;
        stats[1] = e;
    }
    return rc;
}

/* Brute-force leaf search that stops hashing a trial at the first
 * collision; returns the seed found and the number of key hashes spent.
 * Used only to compare hash-evaluation counts (Appendix C figure on hash
 * function evaluations). */
uint64_t orc_leaf_plain_early_exit(const uint64_t *lo, uint32_t m, uint64_t *evals) {
    uint64_t salt = orc_salt(0);
    uint32_t full = (1u << m) - 1;
    uint64_t e = 0;
    for (uint64_t s = 0;; s++) {
        uint32_t mask = 0;
        uint32_t i;
        for (i = 0; i < m; i++) {
            uint32_t bit = 1u << (orc_mix64(lo[i] + salt + s) % m);
            e++;
            if (mask & bit) break;
            mask |= bit;
        }
        if (mask == full) {
            *evals = e;
            return s;
        }
    }
}
