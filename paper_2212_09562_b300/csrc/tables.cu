// tables.cu -- Golomb-Rice parameters and subtree sizes per node size.
//
// Section 2.2 ("Representation") stores the node values with Golomb-Rice
// codes whose parameter depends on the layer and is precomputed.  The
// parameter here follows Kiely's rule for a geometric source (A. Kiely,
// "Selecting the Golomb parameter in Rice coding", IPN Progress Report
// 42-159, 2004): tau = max(0, 1 + floor(log2(ln(phi - 1) / ln(1 - p)))),
// with p the success probability of one stored unit:
//   split of m keys into parts p_i: multinomial m! / prod p_i! * prod (p_i/m)^p_i
//   plain leaf of m keys:            m! / m^m
//   rotation-fitting leaf:           (Appendix A lemma bound, averaged over
//                                     |A| ~ Binomial(m, 1/2)) / m, since one
//                                     seed k*m covers m stored values.
//   ShockHash leaf (Appendix C):     P(the two cells of the m keys admit a
//                                     bijection) * P(the m x m GF(2)
//                                     retrieval system is solvable).
// A ShockHash leaf's fixed part also holds its m retrieval bits.
#include "tables.h"

#include <math.h>
#include <stdlib.h>

#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "mphf.h"

#include "common.cuh"

namespace rs {
namespace {

double all_distinct(uint32_t j, uint32_t m) {
    // probability that j uniform hashes into m cells are pairwise different
    double p = 1.0;
    for (uint32_t i = 1; i < j; i++) p *= 1.0 - (double)i / (double)m;
    return p;
}

double choose(uint32_t n, uint32_t k) {
    double r = 1.0;
    for (uint32_t i = 0; i < k; i++) r *= (double)(n - i) / (double)(i + 1);
    return r;
}

uint32_t gcd(uint32_t a, uint32_t b) { return b ? gcd(b, a % b) : a; }

uint32_t totient(uint32_t d) {
    uint32_t r = 0;
    for (uint32_t j = 1; j <= d; j++)
        if (gcd(j, d) == 1) r++;
    return r;
}

// Lemma of Appendix A: P(some rotation of b fills the holes of a | |A| = a)
// >= P(A distinct) P(B distinct) / (number of rotation classes of b-subsets),
// the number of classes being (1/m) sum_{d | gcd(a, b)} phi(d) C(m/d, b/d).
double rotation_leaf_success(uint32_t m) {
    double sum = 0.0;
    double half_pow = pow(0.5, (double)m);
    for (uint32_t a = 0; a <= m; a++) {
        uint32_t b = m - a;
        uint32_t g = gcd(a, b);
        double cls = 0.0;
        for (uint32_t d = 1; d <= g; d++)
            if (g % d == 0) cls += (double)totient(d) * choose(m / d, b / d);
        double fit = (double)m / cls;
        if (fit > 1.0) fit = 1.0;
        sum += choose(m, a) * half_pow * all_distinct(a, m) * all_distinct(b, m) * fit;
    }
    return sum;
}

double split_success(const Shape &s, uint32_t m) {
    double lg = lgamma((double)m + 1.0);
    uint32_t np = num_parts(s, m);
    for (uint32_t c = 0; c < np; c++) {
        double p = (double)part_size(s, m, c);
        lg += p * log(p / (double)m) - lgamma(p + 1.0);
    }
    return exp(lg);
}

// Cuckoo graph of m keys on m cells, each key an edge between its two cells
// (chosen uniformly, a loop when they agree).  A bijection exists iff every
// component carries exactly one cycle.  Counting over labelled cells and
// keys: pairs (edge list, bijective choice of one cell per key) number
// k! 2^k k^k on k cells; a connected one-cycle list has two choices.  Split
// off the component of the first cell (j cells of k, j keys of k):
//   pairs(k)  = sum_j C(k-1, j-1) C(k, j) * 2 conn(j) * pairs(k - j)
//   cycles(k) = sum_j C(k-1, j-1) C(k, j) * conn(j) * cycles(k - j)
// and P = cycles(m) / m^(2m).
double shock_bijection_prob(uint32_t m) {
    std::vector<double> pairs(m + 1), conn(m + 1), cycles(m + 1);
    pairs[0] = 1.0;
    cycles[0] = 1.0;
    for (uint32_t k = 1; k <= m; k++) {
        double w = 1.0;
        for (uint32_t i = 1; i <= k; i++) w *= 2.0 * (double)i * (double)k;
        pairs[k] = w;
        double other = 0.0, acc = 0.0;
        for (uint32_t j = 1; j < k; j++) {
            const double ways = choose(k - 1, j - 1) * choose(k, j);
            other += ways * 2.0 * conn[j] * pairs[k - j];
            acc += ways * conn[j] * cycles[k - j];
        }
        conn[k] = (pairs[k] - other) / 2.0;
        cycles[k] = acc + conn[k];
    }
    return cycles[m] / pow((double)m, 2.0 * (double)m);
}

// A fixed nonzero right-hand side against m uniform random rows of m bits:
// solvable with probability sum_r P(rank r) (2^r - 1) / (2^m - 1), where
// P(rank r) = 2^-((m-r)^2) prod_{i<r} (1 - 2^(i-m))^2 / (1 - 2^(i-r)).
double gf2_solvable_prob(uint32_t m) {
    double sum = 0.0;
    for (uint32_t r = 0; r <= m; r++) {
        const int d = (int)(m - r);
        double pr = ldexp(1.0, -d * d);
        for (uint32_t i = 0; i < r; i++) {
            const double q = 1.0 - ldexp(1.0, (int)i - (int)m);
            pr *= q * q / (1.0 - ldexp(1.0, (int)i - (int)r));
        }
        sum += pr * (ldexp(1.0, (int)r) - 1.0) / (ldexp(1.0, (int)m) - 1.0);
    }
    return sum;
}

uint8_t kiely(double p) {
    const double phi = (1.0 + sqrt(5.0)) / 2.0;
    double k = 1.0 + floor(log2(log(phi - 1.0) / log1p(-p)));
    return k < 0.0 ? 0 : (uint8_t)k;
}

}  // namespace

uint8_t node_tau(uint32_t leaf, uint32_t bij, uint32_t tree, uint32_t m) {
    if (m < 2) return 0;
    Shape s = make_shape(leaf, tree);
    double p;
    if (m > leaf)
        p = split_success(s, m);
    else if (bij == MPHF_BIJECTION_ROTATION)
        p = rotation_leaf_success(m) / (double)m;
    else if (bij == MPHF_BIJECTION_SHOCKHASH)
        p = shock_bijection_prob(m) * gf2_solvable_prob(m);
    else
        p = all_distinct(m, m);
    return kiely(p);
}

const SizeTables &size_tables(uint32_t leaf, uint32_t bij, uint32_t tree) {
    static std::mutex mu;
    static std::map<uint32_t, std::unique_ptr<SizeTables>> cache;
    std::lock_guard<std::mutex> g(mu);
    uint32_t key = (leaf * 4 + bij) * 2 + (tree ? 1 : 0);
    auto it = cache.find(key);
    if (it != cache.end()) return *it->second;
    auto t = std::make_unique<SizeTables>();
    t->leaf = leaf;
    t->bij = bij;
    t->tree = tree ? 1 : 0;
    Shape s = make_shape(leaf, t->tree);
    for (uint32_t m = 0; m <= 4096; m++) {
        t->tau[m] = node_tau(leaf, bij, t->tree, m);
        t->left[m] = node_kind(s, m) == NODE_UPPER ? (uint16_t)upper_left(s, m) : 0;
        if (m < 2) {
            t->nodes[m] = 0;
            t->fixed[m] = 0;
        } else if (m <= leaf) {
            t->nodes[m] = 1;
            t->fixed[m] = t->tau[m] + (bij == MPHF_BIJECTION_SHOCKHASH ? m : 0);
        } else {
            uint32_t nodes = 1, fixed = t->tau[m];
            for (uint32_t c = 0, np = num_parts(s, m); c < np; c++) {
                uint32_t q = part_size(s, m, c);  // q < m: already filled
                nodes += t->nodes[q];
                fixed += t->fixed[q];
            }
            t->nodes[m] = nodes;
            t->fixed[m] = fixed;
        }
    }
    const SizeTables &ref = *t;
    cache[key] = std::move(t);
    return ref;
}

const ModTables &mod_tables() {
    static std::once_flag once;
    static ModTables t;
    std::call_once(once, [] {
        t.c[0] = 0;
        t.M[0] = 0;
        for (uint32_t m = 1; m <= 4096; m++) {
            const ModRT r = make_mod(m);
            t.c[m] = r.c;
            t.M[m] = r.M;
        }
    });
    return t;
}

}  // namespace rs
