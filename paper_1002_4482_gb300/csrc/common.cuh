// Device-side helpers shared by the list-ranking and component kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lrcc.h"

namespace lrcc {

// ---------------------------------------------------------------- control --

// Per-workspace control block in device memory. Zeroed before every call
// except where noted.
struct DevCtl {
    int status;          // first device-detected error (lrcc_status), 0 = none
    int flag;            // component loop: some edge joined two roots this pass
    int rounds;          // component loop: hook passes so far
    int jump_rounds;     // pointer-jumping rounds (stats)
    int work[8];         // ruling set: next splitter to walk at each level
    int err_where;       // index that raised the error (debugging aid)
    int batch_next;      // batched kernels: next instance to take
    int ovf_next;        // read-only walk: overflow chunks claimed
    int pairs;           // read-only walk: (element, rank) pairs produced
    int place_next;      // read-only walk: next pair slice to place
    int cc_src;          // component loop: edges of the next pass (0 = input, 1/2 = active buffer)
    int cc_count[3];     // component loop: edges appended to active buffer 1 / 2
    int cc_overflow;     // component loop: an active buffer was too small
    int cc_stop;         // component loop: the last pass joined nothing
    int seg_next;        // batched union path: next edge slice of the current pass
    int seg_next_v;      // batched union path: next vertex slice of the current shortcut
    int scan_bad;        // weighted ranks: the values are outside the supported range; skip the work
    int ff_extra;        // forest ranks: list heads that became extra first-level splitters
    int pad[1];
    unsigned long long scan_total;   // weighted ranks: sum of the values
    unsigned long long edges_read;   // component loop: edges read by all hook passes
};

__device__ __forceinline__ void record_error(DevCtl* c, int code, int where = -1) {
    if (atomicCAS(&c->status, 0, code) == 0) c->err_where = where;
}

// ------------------------------------------------------------ packed words --

// List ranking moves (value, pointer) pairs as one 8-byte word so that a jump
// or a sublist step is a single gather (Sec. 3.1: the 64-bit "union").
constexpr uint32_t NIL = 0x7FFFFFFFu;   // no successor
constexpr uint32_t SPL = 0x80000000u;   // low word: this element is a splitter
constexpr uint32_t VIS = 0x80000000u;   // high word: visited by a sublist walk

__device__ __forceinline__ uint64_t pack(uint32_t lo, uint32_t hi) {
    return (static_cast<uint64_t>(hi) << 32) | lo;
}
__device__ __forceinline__ uint32_t lo32(uint64_t w) { return static_cast<uint32_t>(w); }
__device__ __forceinline__ uint32_t hi32(uint64_t w) { return static_cast<uint32_t>(w >> 32); }

// ------------------------------------------------------------ cache hints --

// L2 policy for data touched once per pass (edge streams, the input list):
// evict it first so that the parent / word arrays stay resident.
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// 16-byte streaming load, read-only path, no L1 allocation, L2 hint.
__device__ __forceinline__ int4 ld_stream_v4(const int32_t* p, uint64_t pol) {
    int4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ int32_t ld_stream(const int32_t* p, uint64_t pol) {
    int32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;"
                 : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

// Load through L1 with an L2 eviction-priority hint (for arrays that should
// stay resident in L2 while other data streams past).
__device__ __forceinline__ int32_t ld_hint(const int32_t* p, uint64_t pol) {
    int32_t v;
    asm volatile("ld.global.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
// Read-only path with an L2 eviction-priority hint.
__device__ __forceinline__ int32_t ld_nc_hint(const int32_t* p, uint64_t pol) {
    int32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
// One 32-byte streaming store (a whole sector) of 8 ints; p 32-byte aligned.
__device__ __forceinline__ void st_cs_v8(int32_t* p, const int32_t (&v)[8]) {
    asm volatile("st.global.cs.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 :: "l"(p), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}
// 8-byte store with an L2 eviction-priority hint.
__device__ __forceinline__ void st_hint_u64(uint64_t* p, uint64_t v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.u64 [%0], %1, %2;" :: "l"(p), "l"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ int32_t ld_cg_hint(const int32_t* p, uint64_t pol) {
    int32_t v;
    asm volatile("ld.global.cg.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

// Load that bypasses L1 (sees other SMs' atomics sooner than an L1 hit would).
__device__ __forceinline__ int32_t ld_cg(const int32_t* p) {
    int32_t v;
    asm volatile("ld.global.cg.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint64_t ld_cg_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.global.cg.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}

// ------------------------------------------- bulk copies (TMA) + mbarriers --

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// One arrival that also announces `bytes` of asynchronous transfers.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the phase with the given parity to complete; gives up after
// `limit` polls and returns false (callers report a timeout, never spin on).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int limit) {
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// Orders this thread's earlier generic-proxy accesses to shared memory before
// later asynchronous-proxy (bulk copy) writes into it.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Global -> shared bulk copy (no tensor map): both addresses 16-byte aligned,
// `bytes` a multiple of 16; completion is counted on `bar` in bytes.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

// ------------------------------------------------------------------ hash --

// 32-bit mixer: the finaliser of MurmurHash3 (Appleby, public domain). Used
// to place splitters; results never depend on where they fall.
__host__ __device__ __forceinline__ uint32_t mix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// Offset in [0, size) of the splitter of block b (stratified splitter choice).
__device__ __forceinline__ uint32_t block_offset(uint32_t b, uint32_t size, uint32_t seed) {
    return static_cast<uint32_t>((static_cast<uint64_t>(mix32(b * 0x9E3779B1u + seed)) * size) >> 32);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace lrcc
