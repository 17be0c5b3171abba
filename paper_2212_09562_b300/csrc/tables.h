// tables.h -- host-side per-node-size tables of libmphf (internal).
#pragma once
#include <stdint.h>

namespace rs {

// Tables indexed by node size m in [0, MPHF_MAX_BUCKET] for one (l, leaf method, tree shape):
//   tau[m]    Golomb-Rice parameter of a node of m keys,
//   nodes[m]  stored nodes in the subtree of m keys,
//   fixed[m]  fixed-part bits of that subtree (sum of tau over its nodes, plus
//             m retrieval bits per ShockHash leaf of m keys).
struct SizeTables {
    uint32_t leaf;
    uint32_t bij;   // MPHF_BIJECTION_*
    uint32_t tree;  // MPHF_TREE_*
    uint8_t tau[4097];
    uint32_t nodes[4097];
    uint32_t fixed[4097];
    uint16_t left[4097];  // left part of a fanout-2 node of m keys (0 for other sizes)
};

// Exact remainder constants per node size m in [1, 4096] (the reduction of
// ModRT): c[m] = 2^32 mod m, M[m] = floor((2^64 - 1) / m) + 1; index 0 unused.
struct ModTables {
    uint32_t c[4097];
    uint64_t M[4097];
};
const ModTables &mod_tables();

// Computes (or returns the cached) tables for one leaf size / leaf method.
const SizeTables &size_tables(uint32_t leaf, uint32_t bij, uint32_t tree);

// Golomb-Rice parameter for a node of m keys.
uint8_t node_tau(uint32_t leaf, uint32_t bij, uint32_t tree, uint32_t m);

}  // namespace rs
