/*
 * c_abi_example.c -- the library used from C alone (no Python, no torch).
 *
 * Builds a function over n random 64-bit keys three ways (device keys with
 * rotation fitting, host keys, ShockHash leaves under the fanout-2 tree),
 * queries every key, checks that the values form a bijection onto [0, n),
 * serialises the function and loads the bytes back into a function that
 * must answer every key the same way.  Prints one line per build and exits
 * 0 when every check passes.
 *
 *   usage: c_abi_example [n]
 */
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "mphf.h"

#define CHECK(call)                                                                   \
    do {                                                                              \
        int rc_ = (call);                                                             \
        if (rc_ != MPHF_OK) {                                                         \
            fprintf(stderr, "%s failed: %s (%d)\n", #call, mphf_strerror(rc_), rc_);  \
            return 1;                                                                 \
        }                                                                             \
    } while (0)

static uint64_t splitmix(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* values must be a permutation of [0, n) */
static int is_bijection(const uint64_t *v, uint64_t n) {
    uint8_t *seen = (uint8_t *)calloc(n ? n : 1, 1);
    int ok = seen != NULL;
    for (uint64_t i = 0; ok && i < n; i++) {
        if (v[i] >= n || seen[v[i]]) ok = 0;
        else seen[v[i]] = 1;
    }
    free(seen);
    return ok;
}

static int check(const char *what, mphf_t *h, const uint64_t *d_keys, uint64_t n) {
    uint64_t *d_out = NULL, *out = (uint64_t *)malloc(n * sizeof(uint64_t));
    if (!out || cudaMalloc((void **)&d_out, n * sizeof(uint64_t)) != cudaSuccess) return 1;
    CHECK(mphf_query(h, d_keys, n, d_out, NULL));
    if (cudaMemcpy(out, d_out, n * sizeof(uint64_t), cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
    uint64_t bad = 1;
    CHECK(mphf_verify(h, d_keys, n, &bad, NULL));
    mphf_info info;
    CHECK(mphf_get_info(h, &info));
    size_t len = 0;
    CHECK(mphf_serialize(h, NULL, &len, NULL));
    void *blob = malloc(len);
    if (!blob) return 1;
    CHECK(mphf_serialize(h, blob, &len, NULL));
    /* load the bytes back: the loaded function must answer every key the same way */
    mphf_info info2;
    CHECK(mphf_load_info(blob, len, &info2));
    mphf_t *h2 = NULL;
    CHECK(mphf_load(blob, len, NULL, NULL, &h2));
    uint64_t *out2 = (uint64_t *)malloc(n * sizeof(uint64_t));
    if (!out2) return 1;
    CHECK(mphf_query(h2, d_keys, n, d_out, NULL));
    if (cudaMemcpy(out2, d_out, n * sizeof(uint64_t), cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
    CHECK(mphf_free(h2));
    const int same = info2.n_nodes == info.n_nodes && memcmp(out, out2, n * sizeof(uint64_t)) == 0;
    const int ok = bad == 0 && is_bijection(out, n) && info.n == n && same;
    printf("%s: n=%llu nb=%llu nodes=%llu bits/key=%.3f serialised=%zu bytes loaded=%s bijection=%s\n",
           what, (unsigned long long)info.n, (unsigned long long)info.nb,
           (unsigned long long)info.n_nodes, (double)info.gr_bits / (double)n, len,
           same ? "same" : "DIFFERENT", ok ? "yes" : "NO");
    free(out2);
    free(blob);
    free(out);
    cudaFree(d_out);
    return ok ? 0 : 1;
}

int main(int argc, char **argv) {
    const uint64_t n = argc > 1 ? strtoull(argv[1], NULL, 10) : 200000;
    uint64_t *keys = (uint64_t *)malloc(n * sizeof(uint64_t));
    if (!keys) return 1;
    uint64_t state = 2212;
    for (uint64_t i = 0; i < n; i++) keys[i] = splitmix(&state);  /* a bijection of i: distinct */
    uint64_t *d_keys = NULL;
    if (cudaMalloc((void **)&d_keys, n * sizeof(uint64_t)) != cudaSuccess ||
        cudaMemcpy(d_keys, keys, n * sizeof(uint64_t), cudaMemcpyHostToDevice) != cudaSuccess) {
        fprintf(stderr, "device memory\n");
        return 1;
    }
    int fails = 0;
    mphf_t *h = NULL;

    CHECK(mphf_build(d_keys, n, 12, 1000, NULL, &h));  /* device keys, rotation fitting */
    fails += check("device keys, l=12, rotation fitting", h, d_keys, n);
    CHECK(mphf_free(h));

    mphf_build_params p;
    mphf_default_params(&p);
    p.leaf_size = 8;
    p.bucket_size = 100;
    CHECK(mphf_build_host(keys, n, &p, NULL, &h));     /* host keys */
    fails += check("host keys, l=8, rotation fitting", h, d_keys, n);
    CHECK(mphf_free(h));

    mphf_default_params(&p);
    p.leaf_size = 24;
    p.bucket_size = 2000;
    p.leaf_bijection = MPHF_BIJECTION_SHOCKHASH;
    p.tree_shape = MPHF_TREE_FANOUT2;
    CHECK(mphf_build_ex(d_keys, n, &p, NULL, &h));     /* Appendix C configuration */
    fails += check("device keys, l=24, ShockHash, fanout-2 tree", h, d_keys, n);
    CHECK(mphf_free(h));

    cudaFree(d_keys);
    free(keys);
    printf("%s\n", fails ? "FAILED" : "ok");
    return fails ? 1 : 0;
}
