/*
 * Calls liblrcc through its C header alone (no Python, no PyTorch): ranks a
 * list and labels a graph in device memory and checks both against closed
 * forms computed here, then checks the error paths of the boundary.
 *
 *   abi_check [n]     exit status 0 when every check passes
 *
 * List: a random layout, succ[perm[k]] = perm[k + 1], so rank[perm[k]] must be
 * n - 1 - k. Graph: the same permutation cut into paths of 1000 vertices, each
 * path's label the smallest id on it.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "lrcc.h"

static uint64_t rng_state = 0x9E3779B97F4A7C15ull;
static uint64_t next_u64(void) {   /* xorshift64* (Vigna) */
    rng_state ^= rng_state >> 12;
    rng_state ^= rng_state << 25;
    rng_state ^= rng_state >> 27;
    return rng_state * 2685821657736338717ull;
}

static int fail(const char* what) {
    fprintf(stderr, "FAIL: %s\n", what);
    return 1;
}

int main(int argc, char** argv) {
    const int32_t n = argc > 1 ? atoi(argv[1]) : 300007;
    const int32_t seg = 1000;
    if (n < 2) return fail("n must be at least 2");
    int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* succ = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* out = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* src = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* dst = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* want = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!perm || !succ || !out || !src || !dst || !want) return fail("host allocation");
    for (int32_t i = 0; i < n; ++i) perm[i] = i;
    for (int32_t i = n - 1; i > 0; --i) {   /* Fisher-Yates */
        const int32_t j = (int32_t)(next_u64() % (uint64_t)(i + 1));
        const int32_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
    for (int32_t k = 0; k + 1 < n; ++k) succ[perm[k]] = perm[k + 1];
    succ[perm[n - 1]] = -1;

    int32_t *d_succ = NULL, *d_out = NULL, *d_src = NULL, *d_dst = NULL;
    const size_t bytes = sizeof(int32_t) * (size_t)n;
    if (cudaMalloc((void**)&d_succ, bytes) != cudaSuccess || cudaMalloc((void**)&d_out, bytes) != cudaSuccess ||
        cudaMalloc((void**)&d_src, bytes) != cudaSuccess || cudaMalloc((void**)&d_dst, bytes) != cudaSuccess)
        return fail("device allocation");
    cudaStream_t s;
    if (cudaStreamCreate(&s) != cudaSuccess) return fail("stream");

    /* list ranking, both methods */
    if (cudaMemcpy(d_succ, succ, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return fail("copy in");
    for (int method = 0; method < 2; ++method) {
        const lrcc_status st = method == 0 ? lr_rank(d_succ, n, perm[0], d_out, s)
                                           : lr_rank_wyllie(d_succ, n, perm[0], d_out, s);
        if (st != LRCC_OK) return fail(lrcc_status_str(st));
        if (lrcc_last_status(s) != LRCC_OK) return fail("device status after a valid list");
        if (cudaMemcpy(out, d_out, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return fail("copy out");
        for (int32_t k = 0; k < n; ++k)
            if (out[perm[k]] != n - 1 - k) return fail(method == 0 ? "lr_rank value" : "lr_rank_wyllie value");
    }

    /* components: paths of `seg` vertices along the permutation */
    int32_t m = 0;
    for (int32_t k = 0; k + 1 < n; ++k)
        if ((k + 1) % seg != 0) {
            src[m] = perm[k];
            dst[m] = perm[k + 1];
            ++m;
        }
    for (int32_t k0 = 0; k0 < n; k0 += seg) {
        const int32_t k1 = k0 + seg < n ? k0 + seg : n;
        int32_t lo = perm[k0];
        for (int32_t k = k0; k < k1; ++k) lo = perm[k] < lo ? perm[k] : lo;
        for (int32_t k = k0; k < k1; ++k) want[perm[k]] = lo;
    }
    if (cudaMemcpy(d_src, src, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_dst, dst, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail("copy edges");
    {
        const lrcc_status st = cc_label(d_src, d_dst, m, n, d_out, s);
        if (st != LRCC_OK) return fail(lrcc_status_str(st));
        if (lrcc_last_status(s) != LRCC_OK) return fail("device status after a valid graph");
        if (cudaMemcpy(out, d_out, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return fail("copy labels");
        for (int32_t v = 0; v < n; ++v)
            if (out[v] != want[v]) return fail("cc_label value");
    }

    /* host-buffer form: the same list from host memory */
    if (lr_rank_host(succ, n, perm[0], out, s) != LRCC_OK) return fail("lr_rank_host");
    if (cudaStreamSynchronize(s) != cudaSuccess || lrcc_last_status(s) != LRCC_OK) return fail("lr_rank_host status");
    for (int32_t k = 0; k < n; ++k)
        if (out[perm[k]] != n - 1 - k) return fail("lr_rank_host value");

    /* a context: reserve a second stream's workspace up front, rank on it, free it */
    {
        lrcc_ctx* ctx = NULL;
        cudaStream_t s2;
        if (cudaStreamCreate(&s2) != cudaSuccess) return fail("second stream");
        if (lrcc_ctx_create(&ctx, -1) != LRCC_ERR_ARG || ctx != NULL) return fail("bad device accepted");
        if (lrcc_ctx_create(&ctx, 0) != LRCC_OK || ctx == NULL) return fail("lrcc_ctx_create");
        if (lrcc_ctx_bytes(ctx) != 0) return fail("a new context holds bytes");
        const int64_t need = lrcc_workspace_query(1, n, 0);
        if (need < 0) return fail("lrcc_workspace_query");
        if (lrcc_ctx_reserve(ctx, s2, need) != LRCC_OK) return fail("lrcc_ctx_reserve");
        const int64_t held = lrcc_ctx_bytes(ctx);
        if (held < need) return fail("reserved bytes not counted");
        if (lr_rank(d_succ, n, perm[0], d_out, s2) != LRCC_OK) return fail("lr_rank on the reserved stream");
        if (lrcc_ctx_last_status(ctx, s2) != LRCC_OK) return fail("context status after a valid list");
        if (lrcc_ctx_bytes(ctx) != held) return fail("a call within the reservation grew the workspace");
        if (cudaMemcpy(out, d_out, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return fail("copy out (ctx)");
        for (int32_t k = 0; k < n; ++k)
            if (out[perm[k]] != n - 1 - k) return fail("lr_rank value on the reserved stream");
        if (lrcc_ctx_reserve(ctx, s2, -1) != LRCC_ERR_ARG) return fail("negative reservation accepted");
        lrcc_ctx_destroy(ctx);
        lrcc_ctx_destroy(NULL);
        cudaStreamDestroy(s2);
    }

    /* errors: argument errors return at once, input errors reach the status word */
    if (lr_rank(d_succ, n, n, d_out, s) != LRCC_ERR_ARG) return fail("head out of range accepted");
    if (lr_rank(NULL, n, 0, d_out, s) != LRCC_ERR_ARG) return fail("NULL input accepted");
    if (cc_label(d_src, d_dst, -1, n, d_out, s) != LRCC_ERR_ARG) return fail("negative edge count accepted");
    succ[perm[n - 1]] = perm[0];   /* the tail points back to the head: a cycle */
    if (cudaMemcpy(d_succ, succ, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return fail("copy cycle");
    if (lr_rank(d_succ, n, perm[0], d_out, s) != LRCC_OK) return fail("enqueue on a cycle");
    if (lrcc_last_status(s) != LRCC_ERR_INVALID_INPUT) return fail("cycle not reported");
    if (lrcc_last_status(s) != LRCC_OK) return fail("status not cleared");

    lrcc_release(s);
    cudaStreamDestroy(s);
    cudaFree(d_succ);
    cudaFree(d_out);
    cudaFree(d_src);
    cudaFree(d_dst);
    free(perm);
    free(succ);
    free(out);
    free(src);
    free(dst);
    free(want);
    printf("abi_check ok: n=%d, m=%d, version %d\n", n, m, lrcc_version());
    return 0;
}
