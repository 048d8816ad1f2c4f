// List ranking kernels: Wyllie pointer jumping (Sec. 3.1, Algorithm 1) and the
// sparse ruling set / random splitter method (Sec. 3.2, Algorithms 2 and 3).
//
// Ruling set, as built here for sm_103a:
//   select   (RS1+RS2) one streaming pass packs succ into 8-byte words
//            W[i] = (next | splitter flag, splitter index or weight 1); one
//            random splitter per block of D indices, the head is splitter 0;
//   walk     (RS3) every splitter's sublist is walked once; each visited
//            word is overwritten IN PLACE with (prefix weight, owner | VIS),
//            so a step costs one random sector read plus its write-back;
//   recurse  (RS4) the list of splitters, weighted by sublist size, is again
//            cut by splitters until it fits one thread block, where Wyllie
//            runs in shared memory (Sec. 3.1, single-block variant);
//   expand   (RS5) streaming passes turn (prefix, owner) into ranks.
// Every level stores the inclusive suffix weight S (elements from a node to
// the tail, itself included); the final rank is S - 1.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "block_wyllie.cuh"
#include "common.cuh"
#include "internal.h"

namespace lrcc {

namespace {

constexpr int BLOCK = 256;
constexpr int FINAL_THREADS = 1024;

// ------------------------------------------------------- shared-memory Wyllie

template <int PER>
__device__ __forceinline__ void cta_wyllie(int* val, int* nxt, int r, DevCtl* ctl) {
    block_wyllie<PER, FINAL_THREADS>(val, nxt, r, ctl);
}

// One block ranks a whole list of n <= PER * FINAL_THREADS elements. With
// weights (w != nullptr) it writes the inclusive suffix sums of w instead of
// the ranks, after a first pass with unit weights that checks the list.
template <int PER>
__global__ void __launch_bounds__(FINAL_THREADS, 1)
    lr_small_kernel(const int32_t* __restrict__ succ, const int32_t* __restrict__ w, int n, int head,
                    int32_t* __restrict__ rank, DevCtl* ctl) {
    extern __shared__ int sm[];
    int* val = sm;
    int* nxt = sm + PER * FINAL_THREADS;
    auto load = [&](bool weighted) {
        for (int i = threadIdx.x; i < n; i += FINAL_THREADS) {
            const int s = succ[i];
            const bool tail = (s == -1) | (s == i);
            const bool bad = !tail && (s < 0 || s >= n);
            if (bad && !weighted) record_error(ctl, LRCC_ERR_INVALID_INPUT, i);
            nxt[i] = (tail || bad) ? (int)NIL : s;
            val[i] = weighted ? w[i] : 1;
        }
        __syncthreads();
    };
    load(false);
    cta_wyllie<PER>(val, nxt, n, ctl);
    if (threadIdx.x == 0 && val[head] != n) record_error(ctl, LRCC_ERR_INVALID_INPUT, head);
    if (w) {
        __syncthreads();
        load(true);
        cta_wyllie<PER>(val, nxt, n, ctl);
    }
    const int bias = w ? 0 : 1;
    for (int i = threadIdx.x; i < n; i += FINAL_THREADS) rank[i] = val[i] - bias;
}

// Last ruling-set level: one block ranks the weighted list of splitters held
// in packed words R[j] = (next index or NIL, weight) and writes the inclusive
// suffix weights S. The head splitter (index 0) must see the whole list.
template <int PER>
__global__ void __launch_bounds__(FINAL_THREADS, 1)
    rs_final_kernel(const uint64_t* __restrict__ R, int r, int32_t* __restrict__ S, int64_t expect,
                    DevCtl* ctl) {
    if (ctl->scan_bad) return;
    extern __shared__ int sm[];
    int* val = sm;
    int* nxt = sm + PER * FINAL_THREADS;
    // the splitters must form one list headed by splitter 0: every other
    // splitter has exactly one predecessor, splitter 0 none (this also covers
    // weighted sums, where the head's total says nothing about the count)
    for (int j = threadIdx.x; j < r; j += FINAL_THREADS) val[j] = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < r; j += FINAL_THREADS) {
        const uint32_t nx = lo32(R[j]);
        if (nx < (uint32_t)r) atomicAdd(&val[nx], 1);
        else if (nx != NIL) record_error(ctl, LRCC_ERR_INVALID_INPUT, -3);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < r; j += FINAL_THREADS)
        if (val[j] != (j == 0 ? 0 : 1)) record_error(ctl, LRCC_ERR_INVALID_INPUT, -3);
    __syncthreads();
    for (int j = threadIdx.x; j < r; j += FINAL_THREADS) {
        const uint64_t w = R[j];
        nxt[j] = (int)lo32(w);
        val[j] = (int)hi32(w);
    }
    __syncthreads();
    cta_wyllie<PER>(val, nxt, r, ctl);
    for (int j = threadIdx.x; j < r; j += FINAL_THREADS) S[j] = val[j];
    if (threadIdx.x == 0 && expect >= 0 && val[0] != expect)
        record_error(ctl, LRCC_ERR_INVALID_INPUT, -3);
}

// ------------------------------------------------------------ ruling set

// Splitter choice (Sec. 3.2, RS2), stratified: the elements are cut into
// blocks of D = 2^logD consecutive indices and each block contributes exactly
// one splitter at a hashed offset, so a splitter's index is its block number
// and no compaction is needed. The head's block takes the head as its
// splitter, and block numbers are rotated so that the head is splitter 0.
// Offsets come from the MurmurHash3 finaliser of (block, seed).

// Level-0 select: one streaming pass packs succ into walk words
// W[i] = (next | SPL, splitter index) for splitters, (next, weight) for the
// rest (weight 1, or the element's value for weighted sums), and records each
// splitter's successor and weight. Warps stride over
// groups of 4 elements (Sec. 2.5), with 16-byte loads and stores.
template <bool VEC>
__global__ void __launch_bounds__(BLOCK)
    rs_select0(const int32_t* __restrict__ succ, const int32_t* __restrict__ val, int64_t n, int32_t head,
               uint64_t* __restrict__ W, int32_t* __restrict__ snext, int32_t* __restrict__ sw, int logD,
               int64_t nb, uint32_t seed, DevCtl* ctl, bool mark = true) {
    if (ctl->scan_bad) return;
    const uint64_t pol = policy_evict_first();
    const int64_t D = int64_t(1) << logD;
    const int64_t bh = head >> logD;
    const int64_t ngroups = (n + 3) >> 2;
    for (int64_t g = static_cast<int64_t>(blockIdx.x) * BLOCK + threadIdx.x; g < ngroups;
         g += static_cast<int64_t>(gridDim.x) * BLOCK) {
        const int64_t i0 = g * 4;
        int s[4], wt[4] = {1, 1, 1, 1};
        if (VEC && i0 + 3 < n) {
            const int4 v = ld_stream_v4(succ + i0, pol);
            s[0] = v.x; s[1] = v.y; s[2] = v.z; s[3] = v.w;
            if (val) {
                const int4 x = ld_stream_v4(val + i0, pol);
                wt[0] = x.x; wt[1] = x.y; wt[2] = x.z; wt[3] = x.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                s[q] = (i0 + q < n) ? ld_stream(succ + i0 + q, pol) : -1;
                if (val && i0 + q < n) wt[q] = ld_stream(val + i0 + q, pol);
            }
        }
        // D >= 4 and i0 % 4 == 0, so the 4 elements share one block
        const int64_t b = i0 >> logD;
        const uint32_t size = (uint32_t)min(D, n - (b << logD));
        const uint32_t off = b == bh ? (uint32_t)(head - (b << logD)) : block_offset((uint32_t)b, size, seed);
        const int64_t j = b >= bh ? b - bh : b - bh + nb;
        uint64_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t i = i0 + q;
            const int v = s[q];
            const bool tail = (v == -1) | (v == i);
            const bool bad = !tail && (v < 0 || v >= n);
            if (i < n && bad) record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)i);
            const uint32_t nx = (tail || bad) ? NIL : (uint32_t)v;
            if (mark && i < n && (uint32_t)(i - (b << logD)) == off) {
                w[q] = pack(nx | SPL, (uint32_t)j);
                snext[j] = (int32_t)nx;
                sw[j] = wt[q];
            } else {
                w[q] = pack(nx, (uint32_t)wt[q]);
            }
        }
        if (i0 + 3 < n) {
            ulonglong2* d = reinterpret_cast<ulonglong2*>(W + i0);
            d[0] = make_ulonglong2(w[0], w[1]);
            d[1] = make_ulonglong2(w[2], w[3]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (i0 + q < n) W[i0 + q] = w[q];
        }
    }
}

// First-level splitters given by the caller (the even-splitter experiment of
// Sec. 3.2): spl[j] becomes splitter j of the words rs_select0 packed without
// splitters. spl[0] must be the head; an element out of range or given twice
// is reported (the first mark wins; the second finds SPL already set).
__global__ void __launch_bounds__(BLOCK)
    rs_mark_given(uint64_t* __restrict__ W, int64_t n, int32_t head, const int32_t* __restrict__ spl, int64_t r,
                  int32_t* __restrict__ snext, int32_t* __restrict__ sw, DevCtl* ctl) {
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * BLOCK + threadIdx.x; j < r;
         j += static_cast<int64_t>(gridDim.x) * BLOCK) {
        const int32_t x = spl[j];
        if (x < 0 || x >= n || (j == 0 && x != head)) {
            record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)j);
            snext[j] = (int32_t)NIL;
            sw[j] = 0;
            continue;
        }
        unsigned int* lo = reinterpret_cast<unsigned int*>(W + x);   // low word of the element's packed word
        const unsigned int old = atomicOr(lo, SPL);
        if (old & SPL) {
            record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)j);
            snext[j] = (int32_t)NIL;
            sw[j] = 0;
            continue;
        }
        const unsigned int weight = reinterpret_cast<const unsigned int*>(W + x)[1];
        reinterpret_cast<unsigned int*>(W + x)[1] = (unsigned int)j;
        snext[j] = (int32_t)old;
        sw[j] = (int32_t)weight;
    }
}

// Select at level >= 1: the elements are the previous level's splitters,
// whose packed words R[j] = (next, weight) are already walk words; the head
// is element 0. One thread per block rewrites its splitter's word as
// (next | SPL, block) and records its successor and weight.
__global__ void __launch_bounds__(BLOCK)
    rs_select(uint64_t* __restrict__ R, int64_t nl, int32_t* __restrict__ snext, int32_t* __restrict__ sw,
              int logD, int64_t nb, uint32_t seed, const DevCtl* ctl) {
    if (ctl->scan_bad) return;
    const int64_t D = int64_t(1) << logD;
    for (int64_t b = static_cast<int64_t>(blockIdx.x) * BLOCK + threadIdx.x; b < nb;
         b += static_cast<int64_t>(gridDim.x) * BLOCK) {
        const uint32_t size = (uint32_t)min(D, nl - (b << logD));
        const uint32_t off = b == 0 ? 0u : block_offset((uint32_t)b, size, seed);
        const int64_t sidx = (b << logD) + off;
        const uint64_t w = R[sidx];
        R[sidx] = pack(lo32(w) | SPL, (uint32_t)b);
        snext[b] = (int32_t)lo32(w);
        sw[b] = (int32_t)hi32(w);
    }
}

// Sublist walk (RS3). Each thread keeps K walks in flight so that K
// independent gathers are outstanding; a warp claims splitters in chunks of
// 64 with one atomic and hands them to lanes as their walks end, which
// balances the geometric spread of sublist lengths.
template <int K>
__global__ void __launch_bounds__(BLOCK)
    rs_walk(uint64_t* __restrict__ W, const int32_t* __restrict__ snext, const int32_t* __restrict__ sw,
            uint64_t* __restrict__ Rout, int r, int* work, int64_t nlevel, DevCtl* ctl,
            const int* r_extra = nullptr) {
    if (ctl->scan_bad) return;
    if (r_extra) r += *r_extra;   // splitters added on the device (forest heads)
    constexpr int CHUNK = 64;
    const int lane = threadIdx.x & 31;
    int pool = 0, pool_end = 0;
    bool exhausted = false;
    int j[K];
    uint32_t cur[K], pre[K];
    int64_t steps[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        j[q] = -1;
        cur[q] = NIL;
        pre[q] = 0;
        steps[q] = 0;
    }
    for (;;) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            bool need = j[q] < 0;
            unsigned m = __ballot_sync(0xffffffffu, need);
            while (m && !exhausted) {
                if (pool >= pool_end) {
                    int b = 0;
                    if (lane == 0) b = atomicAdd(work, CHUNK);
                    b = __shfl_sync(0xffffffffu, b, 0);
                    if (b >= r) {
                        exhausted = true;
                        break;
                    }
                    pool = b;
                    pool_end = min(b + CHUNK, r);
                }
                const int avail = pool_end - pool;
                const int rk = __popc(m & lanemask_lt());
                if (need && rk < avail) {
                    const int jj = pool + rk;
                    j[q] = jj;
                    cur[q] = (uint32_t)snext[jj];
                    pre[q] = (uint32_t)sw[jj];
                    steps[q] = 0;
                    need = false;
                }
                pool += min(avail, __popc(m));
                m = __ballot_sync(0xffffffffu, need);
            }
        }
        bool act = false;
#pragma unroll
        for (int q = 0; q < K; ++q) act |= j[q] >= 0;
        if (!__any_sync(0xffffffffu, act)) break;
        uint64_t w[K];
#pragma unroll
        for (int q = 0; q < K; ++q)
            w[q] = (j[q] >= 0 && cur[q] < (uint32_t)nlevel) ? W[cur[q]] : 0ull;
#pragma unroll
        for (int q = 0; q < K; ++q) {
            if (j[q] < 0) continue;
            if (cur[q] == NIL) {
                Rout[j[q]] = pack(NIL, pre[q]);
                j[q] = -1;
                continue;
            }
            const uint32_t lo = lo32(w[q]), hi = hi32(w[q]);
            if (cur[q] >= (uint32_t)nlevel || (!(lo & SPL) && ((hi & VIS) || ++steps[q] > nlevel))) {
                record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)cur[q]);
                Rout[j[q]] = pack(NIL, pre[q]);
                j[q] = -1;
            } else if (lo & SPL) {
                Rout[j[q]] = pack(hi, pre[q]);
                j[q] = -1;
            } else {
                W[cur[q]] = pack(pre[q], (uint32_t)j[q] | VIS);
                pre[q] += hi;
                cur[q] = lo;
            }
        }
    }
}

// Ceiling of the first-level walk's access pattern: dependent 4-byte reads of
// succ, with the walk's load form and none of its bookkeeping (no chunk
// writes, no splitter test). Chain c of `chains` starts at element
// floor(c * n / chains) and takes `steps` steps; a chain that reaches a tail
// (or an id outside [0, n)) continues from a hashed element, which costs no
// read. Each thread advances PROBE_K chains together, as the walk does; the
// wrapped sum of the elements reached goes to *out, so no load is dropped.
constexpr int PROBE_K = 4;
__global__ void __launch_bounds__(BLOCK)
    rs_chase_probe(const int32_t* __restrict__ succ, int64_t n, int64_t chains, int64_t steps,
                   unsigned long long* out) {
    const int64_t c0 = ((int64_t)blockIdx.x * BLOCK + threadIdx.x) * PROBE_K;
    int64_t cur[PROBE_K];
    bool live[PROBE_K];
#pragma unroll
    for (int q = 0; q < PROBE_K; ++q) {
        live[q] = c0 + q < chains;
        cur[q] = live[q] ? (c0 + q) * n / chains : 0;   // c < 2^31 and n <= 2^31: no overflow
    }
    unsigned long long acc = 0;
    for (int64_t k = 0; k < steps; ++k) {
        int32_t nx[PROBE_K];
#pragma unroll
        for (int q = 0; q < PROBE_K; ++q) nx[q] = live[q] ? __ldg(succ + cur[q]) : 0;
#pragma unroll
        for (int q = 0; q < PROBE_K; ++q) {
            if (!live[q]) continue;
            int64_t x = nx[q];
            if (x < 0 || x >= n || x == cur[q])
                x = (int64_t)(((uint64_t)mix32((uint32_t)cur[q] ^ (uint32_t)k * 0x9E3779B9u) * (uint64_t)n) >> 32);
            acc += (unsigned long long)x;
            cur[q] = x;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// ------------------------------------------------ level 0, read-only walk
//
// Random HBM accesses are limited by row activations, not bytes: a random
// read costs one activation, a random read-modify-write two. This level-0
// path therefore walks succ READ-ONLY (one activation per element) and never
// writes a per-element word at a random place:
//   walk     each walk buffers the elements it visits in registers and
//            writes them 8 at a time as one 32-byte chunk (ids in visiting
//            order, plus (first position k0, owner j)) into its block's
//            region; the block also counts its elements per coarse id
//            bucket (NBK buckets of consecutive ids);
//   scan     the per-(bucket, block) counts become output offsets;
//   scatter  each block turns its chunks into (element, rank) pairs with one
//            gather of the owner's suffix weight per chunk, written grouped
//            by bucket;
//   place    the pairs, in bucket order, write rank[element]; the writes of
//            one bucket fall in a window of a few MB that stays in L2, so
//            lines are complete before they are written back.
// A walk that runs longer than `careful` steps marks the elements it visits
// in a bitmap and stops with an error on a repeat, so a cycle without a
// splitter cannot trap it; valid lists never repeat an element.

constexpr int CIDS = 8;        // element ids per chunk (one 32-byte sector)
// Coarse id buckets of the scatter (a bucket's rank writes stay in L2 while
// rs_place works through it). More buckets make each round's runs shorter:
// with 1024 buckets at 2^28 elements the scatter took 2.67 ms instead of 1.41.
constexpr int NBK_LOG = 8;
constexpr int NBK = 1 << NBK_LOG;
constexpr int NSEG = 4;        // scatter work units per walk block region

struct Level0 {
    int64_t n, nb, bh;   // elements, splitters (blocks), the head's block
    int logD;
    uint32_t head_off;   // offset of the head inside its block
    uint32_t seed;
    // batched lists ranked as one list (see lr_enqueue_rs): the first list's
    // head, read on the device (bh and head_off are derived from it), and the
    // heads of the other lists that are extra splitters nb, nb + 1, ...
    const int64_t* head_dev = nullptr;
    const int32_t* extra = nullptr;
    const int* extra_count = nullptr;
};

struct Chunks {
    int32_t* ids;        // chunk c: ids[8c .. 8c+8), unused slots -1
    uint64_t* meta;      // meta[c] = k0 << 32 | j
    int* fill;           // chunks written into each block's own region
    int* counts;         // [NBK][units] elements per (bucket, scatter unit); then row offsets
    int* totals;         // [NBK] elements per bucket
    uint32_t* vis;       // careful-mode marks, one bit per element
    int64_t cap;         // chunks per block region (NSEG segments of segcap)
    int segcap;          // chunks per segment (even); a segment is one scatter work unit
    int units;           // scatter units: NSEG per block region, then the overflow pool's segments
    int64_t ovf_cap;     // overflow chunks
    int64_t ovf_base;    // index of the first overflow chunk (= grid * cap)
    int shift;           // coarse bucket of element x = x >> shift
    int64_t careful;     // steps after which a walk marks what it visits
};

// Index of x among the level-0 splitters, or -1 if x is not one.
__device__ __forceinline__ int64_t splitter_index0(int64_t x, const Level0& L0) {
    const int64_t D = int64_t(1) << L0.logD;
    const int64_t b = x >> L0.logD;
    const uint32_t size = (uint32_t)min(D, L0.n - (b << L0.logD));
    const uint32_t off = b == L0.bh ? L0.head_off : block_offset((uint32_t)b, size, L0.seed);
    if ((uint32_t)(x - (b << L0.logD)) != off) return -1;
    return b >= L0.bh ? b - L0.bh : b - L0.bh + L0.nb;
}

// Element of splitter j.
__device__ __forceinline__ int64_t splitter_node0(int64_t j, const Level0& L0) {
    if (j >= L0.nb) return L0.extra[j - L0.nb];
    const int64_t D = int64_t(1) << L0.logD;
    int64_t b = j + L0.bh;
    if (b >= L0.nb) b -= L0.nb;
    const uint32_t size = (uint32_t)min(D, L0.n - (b << L0.logD));
    const uint32_t off = b == L0.bh ? L0.head_off : block_offset((uint32_t)b, size, L0.seed);
    return (b << L0.logD) + off;
}

// 32-bit level-0 geometry (element ids are int32, so n < 2^31).
struct Geo32 {
    uint32_t n, nb, bh, head_off, seed, D;
    int logD;
};
__device__ __forceinline__ Geo32 geo32(const Level0& L0) {
    Geo32 g;
    g.n = (uint32_t)L0.n;
    g.nb = (uint32_t)L0.nb;
    g.bh = (uint32_t)L0.bh;
    g.head_off = L0.head_off;
    g.seed = L0.seed;
    g.logD = L0.logD;
    g.D = 1u << L0.logD;
    return g;
}
// offset of the splitter inside block b (the same value block_offset gives)
__device__ __forceinline__ uint32_t block_off32(uint32_t b, const Geo32& g) {
    if (b == g.bh) return g.head_off;
    const uint32_t base = b << g.logD;
    const uint32_t size = min(g.D, g.n - base);
    return __umulhi(mix32(b * 0x9E3779B1u + g.seed), size);
}
// index of x among the level-0 splitters, or -1
__device__ __forceinline__ int splitter_index32(uint32_t x, const Geo32& g) {
    const uint32_t b = x >> g.logD;
    if ((x & (g.D - 1)) != block_off32(b, g)) return -1;
    return (int)(b >= g.bh ? b - g.bh : b - g.bh + g.nb);
}
__device__ __forceinline__ uint32_t splitter_node32(uint32_t j, const Geo32& g, const int32_t* extra) {
    if (j >= g.nb) return (uint32_t)extra[j - g.nb];
    uint32_t b = j + g.bh;
    if (b >= g.nb) b -= g.nb;
    return (b << g.logD) + block_off32(b, g);
}

// Read-only sublist walk (RS3). Warps claim splitters in chunks of 64 and
// hand them to lanes as their walks end (the hardware scheduler then
// balances the uneven sublists, Sec. 3.2). Element arithmetic is 32-bit (ids
// are int32) and the ids a walk collects for its next chunk wait in shared
// memory: against 64-bit indices and an 8-entry register buffer, 7 % faster at
// 2^25 elements, 0.6 % at 2^28, where the random reads of succ bound it.
template <int K>
__global__ void __launch_bounds__(BLOCK)
    rs_walk0c(const int32_t* __restrict__ succ, Level0 L0, Chunks C, uint64_t* __restrict__ R1, int* work,
              DevCtl* ctl) {
    if (L0.head_dev) {
        const int64_t gh = *L0.head_dev;
        L0.bh = gh >> L0.logD;
        L0.head_off = (uint32_t)(gh - (L0.bh << L0.logD));
    }
    const Geo32 g = geo32(L0);
    constexpr int WCHUNK = 64;   // splitters a warp claims at once (32 and 128: no faster)
    __shared__ int s_fill;
    __shared__ int s_cnt[NSEG][NBK];
    // the ids a walk has visited since its last flush: slot t of chain q of thread i at
    // s_ids[(q * CIDS + t) * BLOCK + i] (one bank per thread)
    __shared__ int32_t s_ids[K * CIDS * BLOCK];
    for (int t = threadIdx.x; t < NSEG * NBK; t += BLOCK) (&s_cnt[0][0])[t] = 0;
    if (threadIdx.x == 0) s_fill = 0;
    __syncthreads();
    const uint32_t r = g.nb + (L0.extra_count ? (uint32_t)*L0.extra_count : 0u);
    const int lane = threadIdx.x & 31;
    int pool = 0, pool_end = 0;
    bool exhausted = false;
    int j[K];
    uint32_t cur[K], k[K], k0[K];
    int bn[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        j[q] = -1;
        cur[q] = 0;
        k[q] = k0[q] = 0;
        bn[q] = 0;
    }
    for (;;) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            bool need = j[q] < 0;
            unsigned m = __ballot_sync(0xffffffffu, need);
            while (m && !exhausted) {
                if (pool >= pool_end) {
                    int b = 0;
                    if (lane == 0) b = atomicAdd(work, WCHUNK);
                    b = __shfl_sync(0xffffffffu, b, 0);
                    if ((uint32_t)b >= r) {
                        exhausted = true;
                        break;
                    }
                    pool = b;
                    pool_end = (int)min((uint32_t)b + WCHUNK, r);
                }
                const int avail = pool_end - pool;
                const int rk = __popc(m & lanemask_lt());
                if (need && rk < avail) {
                    j[q] = pool + rk;
                    cur[q] = splitter_node32((uint32_t)j[q], g, L0.extra);
                    k[q] = k0[q] = 0;
                    bn[q] = 0;
                    need = false;
                }
                pool += min(avail, __popc(m));
                m = __ballot_sync(0xffffffffu, need);
            }
        }
        bool act = false;
#pragma unroll
        for (int q = 0; q < K; ++q) act |= j[q] >= 0;
        if (!__any_sync(0xffffffffu, act)) break;
        int32_t nx[K];
        // read-only loads at normal L2 priority: the part of succ that L2 holds (an
        // eighth at 2^28) then serves repeat visits; evict-first loads gave those
        // hits up and made the walk 5 % slower
#pragma unroll
        for (int q = 0; q < K; ++q) nx[q] = j[q] >= 0 ? __ldg(succ + cur[q]) : -1;
#pragma unroll
        for (int q = 0; q < K; ++q) {
            if (j[q] < 0) continue;
            bool end = false, bad = false;
            if (k[q] >= C.careful) {
                const uint32_t bit = 1u << (cur[q] & 31);
                if (atomicOr(C.vis + (cur[q] >> 5), bit) & bit) bad = true;   // element reached twice
            }
            s_ids[(q * CIDS + bn[q]) * BLOCK + threadIdx.x] = (int32_t)cur[q];
            ++bn[q];
            const int32_t x = nx[q];
            uint64_t rw = 0;
            if (bad) {
                end = true;
            } else if (x == -1 || (uint32_t)x == cur[q]) {
                rw = pack(NIL, k[q] + 1);
                end = true;
            } else if (x < 0 || (uint32_t)x >= g.n) {
                bad = end = true;
            } else {
                const int sj = splitter_index32((uint32_t)x, g);
                if (sj >= 0) {
                    rw = pack((uint32_t)sj, k[q] + 1);
                    end = true;
                }
            }
            if (bad) {
                record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)cur[q]);
                rw = pack(NIL, k[q] + 1);
            }
            if (bn[q] == CIDS || end) {
                // flush one chunk: own region first, then the shared overflow pool
                const int slot = atomicAdd(&s_fill, 1);
                int64_t c = -1;
                int ovf_unit = -1;   // scatter unit of an overflow chunk (counted in global memory)
                if (slot < C.cap) {
                    c = (int64_t)blockIdx.x * C.cap + slot;
                } else {
                    const int o = atomicAdd(&ctl->ovf_next, 1);
                    if (o < C.ovf_cap) {
                        c = C.ovf_base + o;
                        ovf_unit = (int)gridDim.x * NSEG + o / C.segcap;
                    } else {
                        record_error(ctl, LRCC_ERR_INVALID_INPUT, -4);
                    }
                }
                if (c >= 0) {
                    const int seg = slot / C.segcap;
                    int32_t v[CIDS];
#pragma unroll
                    for (int t = 0; t < CIDS; ++t)
                        v[t] = t < bn[q] ? s_ids[(q * CIDS + t) * BLOCK + threadIdx.x] : -1;
                    // streaming stores: the chunks are read once, by the scatter, and
                    // should not push succ out of L2; one 32-byte store per chunk (chunks
                    // are 32-byte aligned) moves a whole sector in one request instead of
                    // two 16-byte halves (5.55 -> 5.51 ms at 2^28)
                    st_cs_v8(C.ids + c * CIDS, v);
                    __stcs(reinterpret_cast<unsigned long long*>(C.meta + c),
                           (unsigned long long)((static_cast<uint64_t>(k0[q]) << 32) | static_cast<uint32_t>(j[q])));
#pragma unroll
                    for (int t = 0; t < CIDS; ++t)
                        if (t < bn[q]) {
                            if (ovf_unit < 0) atomicAdd(&s_cnt[seg][v[t] >> C.shift], 1);
                            else atomicAdd(&C.counts[(int64_t)(v[t] >> C.shift) * C.units + ovf_unit], 1);
                        }
                }
                k0[q] = k[q] + 1;
                bn[q] = 0;
            }
            if (end) {
                R1[j[q]] = rw;
                j[q] = -1;
            } else {
                cur[q] = (uint32_t)x;
                ++k[q];
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) C.fill[blockIdx.x] = min(s_fill, (int)C.cap);
    for (int t = threadIdx.x; t < NSEG * NBK; t += BLOCK) {
        const int bk = t % NBK, seg = t / NBK;
        C.counts[(int64_t)bk * C.units + (int64_t)blockIdx.x * NSEG + seg] = s_cnt[seg][bk];
    }
}

// Exclusive scan of each bucket's row of per-block counts, in place, one
// block per bucket; the row total goes to totals[bucket]. The start of each
// bucket (a scan over NBK totals) is formed by the scatter blocks themselves.
constexpr int SCAN_THREADS = 256;
__global__ void __launch_bounds__(SCAN_THREADS) rs_scan_counts(int* counts, int G, int* totals) {
    __shared__ int s_warp[SCAN_THREADS / 32];
    int* row = counts + (int64_t)blockIdx.x * G;
    const int per = (G + SCAN_THREADS - 1) / SCAN_THREADS;
    const int b = threadIdx.x * per, e = min(G, b + per);
    int sum = 0;
    for (int i = b; i < e; ++i) sum += row[i];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int v = lane < SCAN_THREADS / 32 ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane < SCAN_THREADS / 32) s_warp[lane] = v;
    }
    __syncthreads();
    int run = (wid ? s_warp[wid - 1] : 0) + incl - sum;
    for (int i = b; i < e; ++i) {
        const int c = row[i];
        row[i] = run;
        run += c;
    }
    if (threadIdx.x == SCAN_THREADS - 1) totals[blockIdx.x] = run;
}

// Chunks of walk block g -> (element, rank) pairs at block g's offsets of
// each bucket. Radix-partition style, in rounds of SC_CHUNKS chunks: the
// round's chunk ids and headers arrive in shared memory by bulk copy, the
// round's elements are ranked by bucket with shared atomics, their
// (element, rank) pairs laid out sorted by bucket in a tile, and every
// bucket's run is written with coalesced stores at the block's next offset
// for that bucket. The phases of a round are separated by block barriers and
// the kernel is bound by their latency, not by shared-memory bandwidth, so
// blocks per SM count most: at 2^28 elements a 16-bit slot-index tile with 4
// blocks per SM took 1.44 ms, the pair tile with two staging buffers (2 blocks
// per SM) 1.38 ms, rounds of 3 chunks per thread 1.47 ms, and the pair tile
// with one staging buffer (3 blocks per SM) 1.22 ms. Blocks
// are persistent and take work units u = blockIdx.x, + gridDim.x, ...: the
// NSEG segments of every walk block's region, then the segments of the shared
// overflow pool (each unit's per-bucket counts come from the walk).
// Compile-time shape of a round: chunks per thread (SC_U), staging buffers
// (SC_BUF) and the blocks per SM the launch bounds ask for. Rounds of one chunk
// per thread with two or three buffers and 4-6 blocks per SM took 1.54-1.78 ms
// at 2^28 against 1.21 ms for the default: a round's fixed cost (barriers, the
// scan, the owners' gathers) is paid per round, so fewer, larger rounds win.
#ifndef LRCC_SC_U
#define LRCC_SC_U 2
#endif
#ifndef LRCC_SC_BUF
#define LRCC_SC_BUF 1
#endif
#ifndef LRCC_SC_MINB
#define LRCC_SC_MINB 3
#endif

constexpr int SC_U = LRCC_SC_U;                 // chunks per thread and round
// One staging buffer: a round's ids and headers move into registers in its
// first phase, and the next round's bulk copy lands in the same buffer while
// this round is scanned and written out (0.35 against 0.40 ms at 2^26). With
// more buffers, the copy issued after round k's first phase is round k + SC_BUF.
constexpr int SC_BUF = LRCC_SC_BUF;
constexpr int SC_CHUNKS = SC_U * BLOCK;         // chunks per round
constexpr int SC_ITEMS = SC_CHUNKS * CIDS;      // element slots per round
// Polls of a bulk-copy barrier before giving up. A poll that finds the phase
// open suspends the thread for a few microseconds (about 4.3 us measured on
// GB300), so the limit is about one second.
constexpr int SC_WAIT_LIMIT = 1 << 18;
struct ScatterSmem {
    int32_t ids[SC_BUF][SC_ITEMS];      // chunk ids of the round in each buffer
    uint64_t meta[SC_BUF][SC_CHUNKS];   // chunk headers (k0 << 32 | owner)
    uint64_t tile[SC_ITEMS];       // the round's (element, rank) pairs sorted by bucket
    int cnt[NBK];                  // elements per bucket in the round
    int delta[NBK];                // pair position minus tile slot, per bucket, in the round
    int tstart[NBK];               // start of each bucket's run in the tile
    int warp[BLOCK / 32];
    uint64_t bar[SC_BUF];
};
constexpr size_t SC_SMEM = sizeof(ScatterSmem);

// The 8 ids of one chunk from shared memory. Lanes 4-7 of every 8 read the
// two 16-byte halves in the other order, so that each quarter-warp phase of
// the 16-byte loads touches all 32 banks once.
__device__ __forceinline__ void load_chunk(const int32_t* p, int32_t (&id)[CIDS]) {
    const int sw = (threadIdx.x >> 2) & 1;
    const int4* src = reinterpret_cast<const int4*>(p);
    const int4 a = src[sw], d = src[sw ^ 1];
    const int4 lo = sw ? d : a, hi = sw ? a : d;
    id[0] = lo.x; id[1] = lo.y; id[2] = lo.z; id[3] = lo.w;
    id[4] = hi.x; id[5] = hi.y; id[6] = hi.z; id[7] = hi.w;
}

__global__ void __launch_bounds__(BLOCK, LRCC_SC_MINB)
    rs_scatter(Chunks C, int G, const int32_t* __restrict__ S1, uint64_t* __restrict__ pairs, int64_t n,
               DevCtl* ctl) {
    extern __shared__ __align__(128) unsigned char sc_raw[];
    ScatterSmem& s = *reinterpret_cast<ScatterSmem*>(sc_raw);
    static_assert(NBK == BLOCK, "one thread per bucket");
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    // block-wide exclusive scan of one value per thread (uses s.warp; one sync).
    // Every caller passes another block barrier before the next scan rewrites
    // s.warp, so the scan needs no barrier after reading it.
    auto block_scan = [&](int v, int* total) {
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += x;
        }
        if (lane == 31) s.warp[wid] = incl;
        __syncthreads();
        int off = 0, all = 0;
#pragma unroll
        for (int w = 0; w < BLOCK / 32; ++w) {
            const int x = s.warp[w];
            off += w < wid ? x : 0;
            all += x;
        }
        *total = all;
        return off + incl - v;
    };
    int bstart;                     // start of bucket t in the pair array
    {
        int all = 0;
        bstart = block_scan(C.totals[t], &all);
        if (blockIdx.x == 0 && t == 0) ctl->pairs = all;
    }
    s.cnt[t] = 0;
    if (t == 0) {
        for (int b = 0; b < SC_BUF; ++b) mbar_init(&s.bar[b], 1);
        fence_proxy_async_smem();   // the initialised barriers are visible to the bulk copies
    }
    __syncthreads();
    // L2 hints: the chunks are read and the pairs written once (evict first),
    // while the owners' suffix ranks S1 (4 bytes per splitter) are gathered
    // once per chunk and should stay (evict last): 1.17 against 1.20 ms at 2^28
    const uint64_t pol = policy_evict_first();
    const uint64_t keep = policy_evict_last();
    uint32_t phase = 0;             // bit b: parity of the next completion of buffer b's barrier
    uint32_t in_flight = 0;         // bit b: a copy into buffer b is not yet waited for (thread 0)
    bool failed = false;
    int my_base = 0;                // next free pair of bucket t (this thread's) in the current unit

    // issue the bulk copy of round k of region g (chunks own0 + k*SC_CHUNKS ..) into buffer b
    auto issue = [&](int64_t first, int nf, int k, int b) {
        const int64_t c0 = first + (int64_t)k * SC_CHUNKS;
        const int cnt = min(SC_CHUNKS, nf - k * SC_CHUNKS);
        const int cm = (cnt + 1) & ~1;   // headers in pairs: 16-byte multiple (segments are even)
        const uint32_t bi = (uint32_t)cnt * CIDS * 4u, bm = (uint32_t)cm * 8u;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&s.bar[b], bi + bm);
        bulk_g2s(s.ids[b], C.ids + c0 * CIDS, bi, &s.bar[b], pol);
        bulk_g2s(s.meta[b], C.meta + c0, bm, &s.bar[b], pol);
        in_flight |= 1u << b;
    };

    // one round over buffer b, whose chunks [0, cnt) are valid (a chunk whose
    // first id is -1 is empty)
    auto process = [&](int b, int cnt, int64_t uc0, int unf, int knext) {
        // the owners' suffix ranks (L2 gathers) are issued first, so their latency
        // overlaps the counting and the scan
        int32_t top[SC_U];
#pragma unroll
        for (int u = 0; u < SC_U; ++u) {
            const int c = u * BLOCK + t;
            const uint64_t mt = s.meta[b][c];
            top[u] = (c < cnt && s.ids[b][c * CIDS] >= 0) ? ld_nc_hint(S1 + lo32(mt), keep) - 1 - (int32_t)hi32(mt) : 0;
        }
        int32_t id[SC_U][CIDS];
        int loc[SC_U][CIDS];
#pragma unroll
        for (int u = 0; u < SC_U; ++u) {
            const int c = u * BLOCK + t;
            load_chunk(&s.ids[b][c * CIDS], id[u]);
#pragma unroll
            for (int q = 0; q < CIDS; ++q) {
                if (c >= cnt) id[u][q] = -1;
                loc[u][q] = id[u][q] >= 0 ? atomicAdd(&s.cnt[id[u][q] >> C.shift], 1) : 0;
            }
        }
        fence_proxy_async_smem();   // this thread's reads of the buffer come before the next copy into it
        __syncthreads();
        // the round's ids and headers now sit in registers: the copy of round
        // k + SC_BUF goes into this buffer while this round is scanned and written out
        if (t == 0 && knext >= 0) issue(uc0, unf, knext, b);
        const int h = s.cnt[t];
        s.cnt[t] = 0;               // counts of the next round
        int items = 0;
        const int ts = block_scan(h, &items);
        s.tstart[t] = ts;
        s.delta[t] = my_base - ts;     // pair position of tile slot i of bucket t: delta[t] + i
        my_base += h;
        __syncthreads();
#pragma unroll
        for (int u = 0; u < SC_U; ++u)
#pragma unroll
            for (int q = 0; q < CIDS; ++q)
                if (id[u][q] >= 0)
                    s.tile[s.tstart[id[u][q] >> C.shift] + loc[u][q]] =
                        pack((uint32_t)id[u][q], (uint32_t)(top[u] - q));
        __syncthreads();
        for (int i = t; i < items; i += BLOCK) {
            const uint64_t pr = s.tile[i];
            const int64_t pos = (int64_t)s.delta[lo32(pr) >> C.shift] + i;
            if (pos < n) st_hint_u64(pairs + pos, pr, pol);
        }
        // no barrier here: the next round rebuilds the tile only after its own
        // barriers (the bounded wait's __syncthreads_or comes first, and a new
        // unit starts with one)
    };

    const int64_t no_all = min((int64_t)ctl->ovf_next, C.ovf_cap);
    const int own_units = G * NSEG;
    for (int unit = blockIdx.x; unit < C.units && !failed; unit += gridDim.x) {
        int nf;
        int64_t c0;
        if (unit < own_units) {
            // segment seg of walk block g's own region
            const int g = unit / NSEG, seg = unit % NSEG;
            nf = max(0, min(C.segcap, C.fill[g] - seg * C.segcap));
            c0 = (int64_t)g * C.cap + (int64_t)seg * C.segcap;
        } else {
            // a segment of the shared overflow pool
            const int64_t v0 = (int64_t)(unit - own_units) * C.segcap;
            nf = (int)max((int64_t)0, min((int64_t)C.segcap, no_all - v0));
            c0 = C.ovf_base + v0;
        }
        if (nf == 0) continue;
        my_base = bstart + C.counts[(int64_t)t * C.units + unit];
        const int nr = (nf + SC_CHUNKS - 1) / SC_CHUNKS;
        if (t == 0)
            for (int k = 0; k < SC_BUF && k < nr; ++k) issue(c0, nf, k, k);
        __syncthreads();
        for (int k = 0; k < nr; ++k) {
            const int b = k % SC_BUF;
            const bool ok = mbar_wait_bounded(&s.bar[b], (phase >> b) & 1u, SC_WAIT_LIMIT);
            if (ok) {
                phase ^= 1u << b;
                in_flight &= ~(1u << b);
            }
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            process(b, min(SC_CHUNKS, nf - k * SC_CHUNKS), c0, nf, k + SC_BUF < nr ? k + SC_BUF : -1);
        }
    }
    if (failed) {
        if (t == 0) {
            record_error(ctl, LRCC_ERR_TIMEOUT, -5);
            // let copies still in flight land before the block's shared memory goes away
            for (int b = 0; b < SC_BUF; ++b)
                if (in_flight & (1u << b)) mbar_wait_bounded(&s.bar[b], (phase >> b) & 1u, SC_WAIT_LIMIT);
        }
        __syncthreads();
    }
}

// Exercises the scatter's bounded wait on a barrier that no copy will ever
// complete: one arrival announces 16 bytes of transfer and no copy is issued,
// so the wait gives up after `polls` polls and records LRCC_ERR_TIMEOUT the
// way the scatter does. Nothing is in flight when the block exits.
__global__ void wait_check_kernel(DevCtl* ctl, int polls) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bar, 16);
    if (!mbar_wait_bounded(&bar, 0, polls)) record_error(ctl, LRCC_ERR_TIMEOUT, -6);
}

}  // namespace

cudaError_t wait_check_enqueue(DevCtl* ctl, int polls, cudaStream_t s) {
    wait_check_kernel<<<1, 32, 0, s>>>(ctl, polls);
    return cudaGetLastError();
}

namespace {

// rank[element] from the pairs. Blocks take slices of PLACE_SLICE pairs from
// one counter in order, so at any moment the pairs in flight cover a few
// buckets and their rank writes stay in a window that L2 holds until every
// line is complete (a grid-stride loop would let blocks drift apart and
// spread the writes over far more memory than L2 holds).
// One block per SM and slices of 8192 pairs: the fewer pairs in flight, the
// narrower the window of rank lines the writes keep open in L2 (at 2^28:
// 1.37 ms, against 1.47 with two blocks per SM and 1.82 with 16384-pair slices).
#ifndef LRCC_PLACE_BLOCKS_PER_SM
#define LRCC_PLACE_BLOCKS_PER_SM 1
#endif
#ifndef LRCC_PLACE_SLICE_WARPS
#define LRCC_PLACE_SLICE_WARPS 32
#endif
constexpr int PLACE_SLICE = BLOCK * LRCC_PLACE_SLICE_WARPS;
__global__ void __launch_bounds__(BLOCK)
    rs_place(const uint64_t* __restrict__ pairs, int64_t n, int32_t* __restrict__ rank, DevCtl* ctl) {
    __shared__ int s_start;
    const int64_t m = min((int64_t)ctl->pairs, n);
    for (;;) {
        if (threadIdx.x == 0) s_start = atomicAdd(&ctl->place_next, PLACE_SLICE);
        __syncthreads();
        const int64_t start = s_start;
        __syncthreads();
        if (start >= m) break;
        const int64_t end = min(start + PLACE_SLICE, m);
        if (end - start == PLACE_SLICE) {
            // full slice: 2 U pairs per thread in flight
            constexpr int U = PLACE_SLICE / (2 * BLOCK) / 4;
            static_assert(U >= 1, "a slice holds at least 8 pairs per thread");
            for (int w = 0; w < 4; ++w) {
                ulonglong2 p[U];
#pragma unroll
                for (int u = 0; u < U; ++u)
                    p[u] = __ldcs(reinterpret_cast<const ulonglong2*>(pairs + start) + (w * U + u) * BLOCK + threadIdx.x);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    // ids come from the scatter and are < n; the checks only keep
                    // a corrupted pair from writing outside rank
                    if (lo32(p[u].x) < (uint64_t)n) rank[lo32(p[u].x)] = (int32_t)hi32(p[u].x);
                    if (lo32(p[u].y) < (uint64_t)n) rank[lo32(p[u].y)] = (int32_t)hi32(p[u].y);
                }
            }
        } else {
            for (int64_t i = start + threadIdx.x; i < end; i += BLOCK) {
                const uint64_t p = pairs[i];
                if (lo32(p) < (uint64_t)n) rank[lo32(p)] = (int32_t)hi32(p);
            }
        }
    }
}

// Expand at level >= 1: S[c] = S_next[owner] - prefix (RS5).
__global__ void __launch_bounds__(BLOCK)
    rs_expand(const uint64_t* __restrict__ W, int r, const int32_t* __restrict__ Snext, int rnext,
              int32_t* __restrict__ S, DevCtl* ctl) {
    if (ctl->scan_bad) return;
    for (int c = blockIdx.x * BLOCK + threadIdx.x; c < r; c += gridDim.x * BLOCK) {
        const uint64_t w = W[c];
        const uint32_t lo = lo32(w), hi = hi32(w);
        // indices are checked so that a malformed input can only give wrong
        // values (with an error recorded), never an access outside Snext
        if ((lo & SPL) && hi < (uint32_t)rnext) {
            S[c] = Snext[hi];
        } else if (!(lo & SPL) && (hi & VIS) && (hi & ~VIS) < (uint32_t)rnext) {
            S[c] = (int32_t)((uint32_t)Snext[hi & ~VIS] - lo);
        } else {
            record_error(ctl, LRCC_ERR_INVALID_INPUT, c);
            S[c] = 0;
        }
    }
}

// Expand at level 0 into the caller's array: rank = S1[owner] - prefix - 1
// (bias 1); for weighted sums the inclusive suffix S1[owner] - prefix (bias 0).
template <bool VEC>
__global__ void __launch_bounds__(BLOCK)
    rs_expand0(const uint64_t* __restrict__ W, int64_t n, const int32_t* __restrict__ S1, int64_t r1,
               int32_t* __restrict__ rank, int bias, DevCtl* ctl) {
    if (ctl->scan_bad) return;
    const int64_t ngroups = (n + 3) >> 2;
    for (int64_t g = static_cast<int64_t>(blockIdx.x) * BLOCK + threadIdx.x; g < ngroups;
         g += static_cast<int64_t>(gridDim.x) * BLOCK) {
        const int64_t i0 = g * 4;
        uint64_t w[4];
        if (i0 + 3 < n) {
            const ulonglong2* s = reinterpret_cast<const ulonglong2*>(W + i0);
            const ulonglong2 a = __ldcs(s), b = __ldcs(s + 1);
            w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) w[q] = (i0 + q < n) ? W[i0 + q] : pack(SPL, 0);
        }
        int out[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t lo = lo32(w[q]), hi = hi32(w[q]);
            if ((lo & SPL) && hi < (uint64_t)r1) {
                out[q] = S1[hi] - bias;
            } else if (!(lo & SPL) && (hi & VIS) && (hi & ~VIS) < (uint64_t)r1) {
                out[q] = (int32_t)((uint32_t)S1[hi & ~VIS] - lo - (uint32_t)bias);
            } else {
                record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)(i0 + q));
                out[q] = -1;
            }
        }
        if (VEC && i0 + 3 < n) {
            __stcs(reinterpret_cast<int4*>(rank + i0), make_int4(out[0], out[1], out[2], out[3]));
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (i0 + q < n) rank[i0 + q] = out[q];
        }
    }
}

// ------------------------------------------------ level 0, split arrays
//
// The paper's other first-level layout (Sec. 3.2, the "48 bit" version): the
// walk reads succ itself and keeps each element's ownership mark and local
// rank in two arrays, so a step reads succ[x] and mark[x] and writes mark[x]
// and lrank[x] (two random reads and two random writes, where the packed
// in-place word takes one of each). The mark is 16 bits while the level has
// fewer than 65,535 splitters (the paper's 2 + 4 bytes per element), 32 bits
// otherwise. A mark of all ones means "not visited"; a splitter's mark is its
// own index and its local rank 0.

template <typename MT>
__global__ void __launch_bounds__(BLOCK)
    rs_select0s(const int32_t* __restrict__ succ, MT* __restrict__ mark, int32_t* __restrict__ lrank,
                int32_t* __restrict__ snext, int32_t* __restrict__ sw, Level0 L0, DevCtl* ctl) {
    constexpr MT UNSEEN = MT(~MT(0));
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * BLOCK + threadIdx.x; i < L0.n;
         i += static_cast<int64_t>(gridDim.x) * BLOCK) {
        const int64_t j = splitter_index0(i, L0);
        mark[i] = j >= 0 ? (MT)j : UNSEEN;
        if (j >= 0) {
            const int v = succ[i];
            const bool tail = (v == -1) | (v == i);
            const bool bad = !tail && (v < 0 || v >= L0.n);
            if (bad) record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)i);
            snext[j] = (tail || bad) ? (int32_t)NIL : v;
            sw[j] = 1;
            lrank[i] = 0;
        }
    }
}

// Sublist walk over the split arrays; the hand-out of splitters to lanes is
// the same as rs_walk's. Output per splitter j: R1[j] = (next splitter,
// elements from j up to it), the packed words of level 1.
template <typename MT, int K>
__global__ void __launch_bounds__(BLOCK)
    rs_walk0s(const int32_t* __restrict__ succ, MT* __restrict__ mark, int32_t* __restrict__ lrank,
              const int32_t* __restrict__ snext, uint64_t* __restrict__ R1, int* work, Level0 L0, DevCtl* ctl) {
    constexpr MT UNSEEN = MT(~MT(0));
    constexpr int CHUNK = 64;
    const int r = (int)L0.nb;
    const int64_t n = L0.n;
    const int lane = threadIdx.x & 31;
    int pool = 0, pool_end = 0;
    bool exhausted = false;
    int j[K];
    uint32_t cur[K], pre[K];
    int64_t steps[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        j[q] = -1;
        cur[q] = NIL;
        pre[q] = 0;
        steps[q] = 0;
    }
    for (;;) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            bool need = j[q] < 0;
            unsigned m = __ballot_sync(0xffffffffu, need);
            while (m && !exhausted) {
                if (pool >= pool_end) {
                    int b = 0;
                    if (lane == 0) b = atomicAdd(work, CHUNK);
                    b = __shfl_sync(0xffffffffu, b, 0);
                    if (b >= r) {
                        exhausted = true;
                        break;
                    }
                    pool = b;
                    pool_end = min(b + CHUNK, r);
                }
                const int avail = pool_end - pool;
                const int rk = __popc(m & lanemask_lt());
                if (need && rk < avail) {
                    const int jj = pool + rk;
                    j[q] = jj;
                    cur[q] = (uint32_t)snext[jj];
                    pre[q] = 1;
                    steps[q] = 0;
                    need = false;
                }
                pool += min(avail, __popc(m));
                m = __ballot_sync(0xffffffffu, need);
            }
        }
        bool act = false;
#pragma unroll
        for (int q = 0; q < K; ++q) act |= j[q] >= 0;
        if (!__any_sync(0xffffffffu, act)) break;
        MT mk[K];
        int sx[K];
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const bool live = j[q] >= 0 && cur[q] < (uint32_t)n;
            mk[q] = live ? mark[cur[q]] : UNSEEN;
            sx[q] = live ? succ[cur[q]] : -1;
        }
#pragma unroll
        for (int q = 0; q < K; ++q) {
            if (j[q] < 0) continue;
            if (cur[q] == NIL) {
                R1[j[q]] = pack(NIL, pre[q]);
                j[q] = -1;
                continue;
            }
            if (cur[q] >= (uint32_t)n || ++steps[q] > n) {
                record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)cur[q]);
                R1[j[q]] = pack(NIL, pre[q]);
                j[q] = -1;
                continue;
            }
            if (mk[q] != UNSEEN) {
                // a splitter ends the sublist; any other marked element was
                // reached twice, so the input is not one list
                if (splitter_index0(cur[q], L0) == (int64_t)mk[q]) {
                    R1[j[q]] = pack((uint32_t)mk[q], pre[q]);
                } else {
                    record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)cur[q]);
                    R1[j[q]] = pack(NIL, pre[q]);
                }
                j[q] = -1;
                continue;
            }
            mark[cur[q]] = (MT)j[q];
            lrank[cur[q]] = (int32_t)pre[q];
            pre[q] += 1;
            const int v = sx[q];
            const bool tail = (v == -1) | ((uint32_t)v == cur[q]);
            const bool bad = !tail && (v < 0 || v >= n);
            if (bad) record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)cur[q]);
            cur[q] = (tail || bad) ? NIL : (uint32_t)v;
        }
    }
}

// rank = S1[mark] - lrank - 1 (RS5 over the split arrays).
template <typename MT>
__global__ void __launch_bounds__(BLOCK)
    rs_expand0s(const MT* __restrict__ mark, const int32_t* __restrict__ lrank, int64_t n,
                const int32_t* __restrict__ S1, int64_t r1, int32_t* __restrict__ rank, DevCtl* ctl) {
    constexpr MT UNSEEN = MT(~MT(0));
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * BLOCK + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * BLOCK) {
        const MT m = __ldcs(mark + i);
        if (m == UNSEEN || (int64_t)m >= r1) {
            // never visited: not reachable from the head
            record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)i);
            __stcs(rank + i, -1);
        } else {
            __stcs(rank + i, (int32_t)((uint32_t)S1[m] - (uint32_t)__ldcs(lrank + i) - 1u));
        }
    }
}

// ---------------------------------------------------------------- Wyllie

template <bool VEC>
__global__ void __launch_bounds__(BLOCK)
    wy_pack(const int32_t* __restrict__ succ, int64_t n, uint64_t* __restrict__ W, DevCtl* ctl) {
    const uint64_t pol = policy_evict_first();
    const int64_t ngroups = (n + 3) >> 2;
    for (int64_t g = static_cast<int64_t>(blockIdx.x) * BLOCK + threadIdx.x; g < ngroups;
         g += static_cast<int64_t>(gridDim.x) * BLOCK) {
        const int64_t i0 = g * 4;
        int s[4];
        if (VEC && i0 + 3 < n) {
            const int4 v = ld_stream_v4(succ + i0, pol);
            s[0] = v.x; s[1] = v.y; s[2] = v.z; s[3] = v.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) s[q] = (i0 + q < n) ? succ[i0 + q] : -1;
        }
        uint64_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t i = i0 + q;
            const int v = s[q];
            const bool tail = (v == -1) | (v == i);
            const bool bad = !tail && (v < 0 || v >= n);
            if (i < n && bad) record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)i);
            // the tail points to itself with value 0, so jumps past it add nothing
            w[q] = (tail || bad) ? pack(0, (uint32_t)i) : pack(1, (uint32_t)v);
        }
        if (i0 + 3 < n) {
            ulonglong2* d = reinterpret_cast<ulonglong2*>(W + i0);
            d[0] = make_ulonglong2(w[0], w[1]);
            d[1] = make_ulonglong2(w[2], w[3]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (i0 + q < n) W[i0 + q] = w[q];
        }
    }
}

// One pointer-jumping round: (r, s) <- (r + r[s], s[s]) from one 8-byte gather.
__global__ void __launch_bounds__(BLOCK)
    wy_jump(const uint64_t* __restrict__ Win, uint64_t* __restrict__ Wout, int64_t n) {
    const int64_t ngroups = (n + 3) >> 2;
    for (int64_t g = static_cast<int64_t>(blockIdx.x) * BLOCK + threadIdx.x; g < ngroups;
         g += static_cast<int64_t>(gridDim.x) * BLOCK) {
        const int64_t i0 = g * 4;
        uint64_t w[4], x[4];
        if (i0 + 3 < n) {
            const ulonglong2* s = reinterpret_cast<const ulonglong2*>(Win + i0);
            const ulonglong2 a = s[0], b = s[1];
            w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) w[q] = (i0 + q < n) ? Win[i0 + q] : 0ull;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = (i0 + q < n) ? Win[hi32(w[q])] : 0ull;
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = pack(lo32(w[q]) + lo32(x[q]), hi32(x[q]));
        if (i0 + 3 < n) {
            ulonglong2* d = reinterpret_cast<ulonglong2*>(Wout + i0);
            d[0] = make_ulonglong2(w[0], w[1]);
            d[1] = make_ulonglong2(w[2], w[3]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (i0 + q < n) Wout[i0 + q] = w[q];
        }
    }
}

// Last round writes the ranks; the head must reach the tail in n - 1 links.
template <bool VEC>
__global__ void __launch_bounds__(BLOCK)
    wy_final(const uint64_t* __restrict__ Win, int64_t n, int32_t head, int32_t* __restrict__ rank,
             DevCtl* ctl) {
    const int64_t ngroups = (n + 3) >> 2;
    for (int64_t g = static_cast<int64_t>(blockIdx.x) * BLOCK + threadIdx.x; g < ngroups;
         g += static_cast<int64_t>(gridDim.x) * BLOCK) {
        const int64_t i0 = g * 4;
        int out[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            out[q] = 0;
            if (i0 + q < n) {
                const uint64_t w = Win[i0 + q];
                const uint64_t x = Win[hi32(w)];
                out[q] = (int)(lo32(w) + lo32(x));
                if (i0 + q == head && out[q] != n - 1) record_error(ctl, LRCC_ERR_INVALID_INPUT, head);
            }
        }
        if (VEC && i0 + 3 < n) {
            *reinterpret_cast<int4*>(rank + i0) = make_int4(out[0], out[1], out[2], out[3]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (i0 + q < n) rank[i0 + q] = out[q];
        }
    }
}

// ------------------------------------------------ batched lists as one list
//
// Lists k = 0..K-1 own elements [off[k], off[k+1]) with local ids. They are
// ranked as one list by the read-only first level: every element gets a
// global successor (off[k] + local, or -1 at a tail); the first non-empty
// list's head is the head; the head of every other list is a first-level
// splitter (its block's stratified splitter, or an extra splitter nb + e when
// that is another element); after the walk, the splitter that ends list k is
// linked to the head splitter of the next non-empty list, and the unused extra
// slots become a tail of empty splitters. Ranks along that one list are the
// local ranks plus the number of elements of the later lists, which are taken
// off the first-level splitters' suffix sums before the scatter. A walk never
// steps onto a head (nothing names it), so the walk recognises splitters by
// their hash as for one list.

// The list that holds element i (for empty lists, the last list starting at i).
__device__ __forceinline__ int64_t find_list(const int64_t* __restrict__ off, int64_t K, int64_t i) {
    int64_t lo = 0, hi = K - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

constexpr int BL_TILE = BLOCK * 16;

// Global successors; one binary search per tile of elements. Each thread
// loads its 16 elements of the tile first, so that 16 streaming reads are in
// flight, then converts them.
__global__ void __launch_bounds__(BLOCK)
    bl_gsucc(const int32_t* __restrict__ succ, const int64_t* __restrict__ off, int64_t K, int64_t n,
             int32_t* __restrict__ gsucc, DevCtl* ctl) {
    constexpr int PER = BL_TILE / BLOCK;
    __shared__ int64_t s_k;
    const uint64_t pol = policy_evict_first();
    for (int64_t t0 = (int64_t)blockIdx.x * BL_TILE; t0 < n; t0 += (int64_t)gridDim.x * BL_TILE) {
        if (threadIdx.x == 0) s_k = find_list(off, K, t0);
        __syncthreads();
        int64_t k = s_k;
        __syncthreads();
        const int64_t tend = min(t0 + BL_TILE, n);
        int32_t sx[PER];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int64_t i = t0 + threadIdx.x + (int64_t)q * BLOCK;
            sx[q] = i < tend ? ld_stream(succ + i, pol) : -1;
        }
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int64_t i = t0 + threadIdx.x + (int64_t)q * BLOCK;
            if (i >= tend) break;
            while (k + 1 < K && off[k + 1] <= i) ++k;
            const int64_t base = off[k], len = off[k + 1] - base;
            int32_t g = -1;
            if (sx[q] != -1 && sx[q] != i - base) {
                if (sx[q] < 0 || sx[q] >= len) record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)i);
                else g = (int32_t)(base + sx[q]);
            }
            gsucc[i] = g;
        }
    }
}

// One block: the first list's head, and the head splitter of every list.
__global__ void __launch_bounds__(1024)
    bl_heads(const int64_t* __restrict__ off, const int32_t* __restrict__ heads, int64_t K, int64_t n, int logD,
             int64_t nb, uint32_t seed, int32_t* __restrict__ head_spl, int32_t* __restrict__ extra_elem,
             int64_t* head_dev, DevCtl* ctl) {
    __shared__ int64_t s_first;
    __shared__ int s_warp[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    if (t == 0) {
        int64_t k0 = 0;
        while (k0 < K && off[k0 + 1] == off[k0]) ++k0;
        s_first = k0;
        int64_t gh = 0;
        if (k0 < K) {
            const int64_t len = off[k0 + 1] - off[k0];
            if (heads[k0] < 0 || heads[k0] >= len) record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)k0);
            else gh = off[k0] + heads[k0];
        }
        *head_dev = gh;
    }
    __syncthreads();
    const int64_t k0 = s_first;
    const int64_t gh0 = *head_dev;
    const int64_t D = int64_t(1) << logD;
    const int64_t bh = gh0 >> logD;
    const int64_t per = (K + 1023) / 1024;
    const int64_t kb = min(K, (int64_t)t * per), ke = min(K, kb + per);
    // a list's head and whether it is its block's stratified splitter
    auto head_of = [&](int64_t k, int64_t* gh, bool* strat) {
        const int64_t len = off[k + 1] - off[k];
        int64_t h = off[k];
        if (heads[k] < 0 || heads[k] >= len) record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)k);
        else h = off[k] + heads[k];
        const int64_t b = h >> logD;
        const uint32_t size = (uint32_t)min(D, n - (b << logD));
        *gh = h;
        *strat = b != bh && (uint32_t)(h - (b << logD)) == block_offset((uint32_t)b, size, seed);
    };
    int cnt = 0;
    for (int64_t k = kb; k < ke; ++k) {
        if (k == k0 || off[k + 1] == off[k]) continue;
        int64_t gh;
        bool strat;
        head_of(k, &gh, &strat);
        cnt += !strat;
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < 32; ++w) {
        before += w < wid ? s_warp[w] : 0;
        total += s_warp[w];
    }
    int e = before + incl - cnt;
    for (int64_t k = kb; k < ke; ++k) {
        if (off[k + 1] == off[k]) {
            head_spl[k] = -1;
            continue;
        }
        if (k == k0) {
            head_spl[k] = 0;
            continue;
        }
        int64_t gh;
        bool strat;
        head_of(k, &gh, &strat);
        if (strat) {
            const int64_t b = gh >> logD;
            head_spl[k] = (int32_t)(b >= bh ? b - bh : b - bh + nb);
        } else {
            head_spl[k] = (int32_t)(nb + e);
            extra_elem[e] = (int32_t)gh;
            ++e;
        }
    }
    if (t == 0) ctl->ff_extra = total;
}

// After the first-level walk: the splitter that ends list k (its word names no
// next splitter) is linked to the next non-empty list's head splitter; the
// unused extra slots become a chain of empty splitters after the last list.
__global__ void __launch_bounds__(BLOCK)
    bl_link(uint64_t* __restrict__ R1, int64_t r1_max, const int64_t* __restrict__ off, int64_t K,
            const int32_t* __restrict__ head_spl, Level0 L0, DevCtl* ctl) {
    const int64_t gh = *L0.head_dev;
    L0.bh = gh >> L0.logD;
    L0.head_off = (uint32_t)(gh - (L0.bh << L0.logD));
    const int64_t r_real = L0.nb + *L0.extra_count;
    for (int64_t j = (int64_t)blockIdx.x * BLOCK + threadIdx.x; j < r1_max; j += (int64_t)gridDim.x * BLOCK) {
        if (j >= r_real) {
            R1[j] = pack(j + 1 < r1_max ? (uint32_t)(j + 1) : NIL, 0);
            continue;
        }
        const uint64_t w = R1[j];
        if (lo32(w) != NIL) continue;
        const int64_t e = splitter_node0(j, L0);
        int64_t k = find_list(off, K, e) + 1;
        while (k < K && off[k + 1] == off[k]) ++k;
        uint32_t nx = NIL;
        if (k < K) nx = (uint32_t)head_spl[k];
        else if (r_real < r1_max) nx = (uint32_t)r_real;
        R1[j] = pack(nx, hi32(w));
    }
}

// Global ranks -> local ranks: every element of list k is ahead of the
// n - off[k + 1] elements of the later lists, which its local rank does not
// count. A sublist never leaves its list (each list ends in a tail), so the
// correction is taken once per first-level splitter, from its suffix sum,
// before the scatter turns suffix sums into ranks.
__global__ void __launch_bounds__(BLOCK)
    bl_adjust(int32_t* __restrict__ S1, const int64_t* __restrict__ off, int64_t K, int64_t n, Level0 L0) {
    const int64_t gh = *L0.head_dev;
    L0.bh = gh >> L0.logD;
    L0.head_off = (uint32_t)(gh - (L0.bh << L0.logD));
    const int64_t r_real = L0.nb + *L0.extra_count;   // the empty tail splitters own nothing
    for (int64_t j = (int64_t)blockIdx.x * BLOCK + threadIdx.x; j < r_real; j += (int64_t)gridDim.x * BLOCK) {
        const int64_t e = splitter_node0(j, L0);
        if (e < 0 || e >= n) continue;
        const int64_t k = find_list(off, K, e);
        S1[j] = (int32_t)((uint32_t)S1[j] - (uint32_t)(n - off[k + 1]));
    }
}

// ------------------------------------------- range check of the values

// Weighted ranks by the ruling set keep every partial sum in the 31-bit
// fields of the packed words, whose top bits are the splitter and visited
// flags: the values must be non-negative and their total below 2^31. This pass
// (one streaming read of val) checks both; when they do not hold, the later
// kernels of the call return at once and the call reports invalid input.
__global__ void __launch_bounds__(BLOCK)
    rs_scan_check(const int32_t* __restrict__ val, int64_t n, DevCtl* ctl) {
    const uint64_t pol = policy_evict_first();
    unsigned long long sum = 0;
    bool neg = false;
    for (int64_t i = (int64_t)blockIdx.x * BLOCK + threadIdx.x; i < n; i += (int64_t)gridDim.x * BLOCK) {
        const int32_t v = ld_stream(val + i, pol);
        neg |= v < 0;
        sum += (unsigned long long)(uint32_t)v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (__any_sync(0xffffffffu, neg) && (threadIdx.x & 31) == 0) ctl->scan_bad = 1;
    if ((threadIdx.x & 31) == 0 && sum) atomicAdd(&ctl->scan_total, sum);
}

__global__ void rs_scan_verdict(DevCtl* ctl) {
    if (ctl->scan_bad || ctl->scan_total >= (1ull << 31)) {
        ctl->scan_bad = 1;
        record_error(ctl, LRCC_ERR_INVALID_INPUT, -6);
    }
}

// ------------------------------------------- weighted ranks of a forest

// A forest of lists has no single head. Its weighted ranks take the ruling
// set with every list head as an extra first-level splitter (the heads are the
// elements no successor names, found with one bit per element in a bitmap L2
// holds, which also catches an element named twice); the first level walks
// as for one list, and the splitters, a much smaller forest, are summed by
// pointer jumping (Sec. 3.1): words (next or NIL, value), rounds of (next,
// value) <- (next[next], value + value[next]); a splitter still linked after
// the last round lies on a cycle. When the values rule out the 31-bit fields
// of the first level (a negative value, or a total of 2^31 or more), the
// whole forest is summed by pointer jumping instead (fs_pack).
__global__ void __launch_bounds__(BLOCK)
    ff_indeg(const int32_t* __restrict__ succ, int64_t n, uint32_t* has_pred, DevCtl* ctl) {
    const uint64_t pol = policy_evict_first();
    for (int64_t i = (int64_t)blockIdx.x * BLOCK + threadIdx.x; i < n; i += (int64_t)gridDim.x * BLOCK) {
        const int32_t sx = ld_stream(succ + i, pol);
        const bool tail = (sx == -1) | (sx == i);
        if (tail) continue;
        if (sx < 0 || sx >= n) {
            record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)i);
            continue;
        }
        const uint32_t bit = 1u << (sx & 31);
        if (atomicOr(has_pred + (sx >> 5), bit) & bit) record_error(ctl, LRCC_ERR_INVALID_INPUT, sx);
    }
}

// Forest first level: the stratified splitter of every block of D ids keeps
// its block number as index; every other head takes an index from nb on (one
// counter atomic per warp). Walk words as in rs_select0, with the value as
// weight.
__global__ void __launch_bounds__(BLOCK)
    ff_select0(const int32_t* __restrict__ succ, const int32_t* __restrict__ val, int64_t n,
               const uint32_t* __restrict__ has_pred, uint64_t* __restrict__ W, int32_t* __restrict__ snext,
               int32_t* __restrict__ sw, int logD, int64_t nb, int64_t r1_max, uint32_t seed, DevCtl* ctl) {
    if (ctl->scan_bad) return;
    const uint64_t pol = policy_evict_first();
    const int64_t D = int64_t(1) << logD;
    const int lane = threadIdx.x & 31;
    // warp-uniform trip count for the ballot
    for (int64_t base = (int64_t)blockIdx.x * BLOCK + (threadIdx.x & ~31); base < n; base += (int64_t)gridDim.x * BLOCK) {
        const int64_t i = base + lane;
        const bool in = i < n;
        int32_t sx = -1, v = 0;
        if (in) {
            sx = ld_stream(succ + i, pol);
            v = ld_stream(val + i, pol);
        }
        const bool tail = (sx == -1) | (sx == i);
        const uint32_t nx = (tail || sx < 0 || sx >= n) ? NIL : (uint32_t)sx;
        const int64_t b = i >> logD;
        const uint32_t size = in ? (uint32_t)min(D, n - (b << logD)) : 1u;
        const bool strat = in && (uint32_t)(i - (b << logD)) == block_offset((uint32_t)b, size, seed);
        const bool head = in && !((has_pred[i >> 5] >> (i & 31)) & 1u);
        const bool extra = head && !strat;
        const unsigned m = __ballot_sync(0xffffffffu, extra);
        int first = 0;
        if (lane == 0 && m) first = atomicAdd(&ctl->ff_extra, __popc(m));
        first = __shfl_sync(0xffffffffu, first, 0);
        if (!in) continue;
        int64_t j = -1;
        if (strat) j = b;
        else if (extra) j = nb + first + __popc(m & lanemask_lt());
        if (j >= r1_max) {
            record_error(ctl, LRCC_ERR_INVALID_INPUT, -7);
            j = -1;
        }
        if (j >= 0) {
            W[i] = pack(nx | SPL, (uint32_t)j);
            snext[j] = (int32_t)nx;
            sw[j] = v;
        } else {
            W[i] = pack(nx, (uint32_t)v);
        }
    }
}

// Verdict for the forest: values outside the first level's range select the
// pointer-jumping form (no error; that form takes any values).
__global__ void ff_verdict(DevCtl* ctl) {
    if (ctl->scan_bad || ctl->scan_total >= (1ull << 31)) ctl->scan_bad = 1;
}

__global__ void __launch_bounds__(BLOCK)
    fs_pack(const int32_t* __restrict__ succ, const int32_t* __restrict__ val, int64_t n, uint64_t* __restrict__ W,
            uint32_t* named, DevCtl* ctl) {
    if (!ctl->scan_bad) return;   // only when the ruling-set form cannot take the values
    const uint64_t pol = policy_evict_first();
    for (int64_t i = (int64_t)blockIdx.x * BLOCK + threadIdx.x; i < n; i += (int64_t)gridDim.x * BLOCK) {
        const int32_t sx = ld_stream(succ + i, pol);
        const bool tail = (sx == -1) | (sx == i);
        const bool bad = !tail && (sx < 0 || sx >= n);
        W[i] = pack((tail || bad) ? NIL : (uint32_t)sx, (uint32_t)ld_stream(val + i, pol));
    }
}

__global__ void __launch_bounds__(BLOCK)
    fs_jump(const uint64_t* __restrict__ Win, uint64_t* __restrict__ Wout, int64_t n, const int* extra,
            const DevCtl* ctl) {
    // two uses: the whole forest when the values rule out the ruling set
    // (extra == nullptr), or the forest of first-level splitters (n + *extra of them)
    if (extra ? ctl->scan_bad : !ctl->scan_bad) return;
    if (extra) n += *extra;
    for (int64_t i = (int64_t)blockIdx.x * BLOCK + threadIdx.x; i < n; i += (int64_t)gridDim.x * BLOCK) {
        uint64_t w = Win[i];
        const uint32_t nx = lo32(w);
        if (nx != NIL) {
            const uint64_t x = Win[nx];
            w = pack(lo32(x), hi32(w) + hi32(x));
        }
        Wout[i] = w;
    }
}

__global__ void __launch_bounds__(BLOCK)
    fs_final(const uint64_t* __restrict__ W, int64_t n, int32_t* __restrict__ out, const int* extra, DevCtl* ctl) {
    if (extra ? ctl->scan_bad : !ctl->scan_bad) return;
    if (extra) n += *extra;
    for (int64_t i = (int64_t)blockIdx.x * BLOCK + threadIdx.x; i < n; i += (int64_t)gridDim.x * BLOCK) {
        const uint64_t w = W[i];
        if (lo32(w) != NIL) record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)i);
        out[i] = (int32_t)hi32(w);
    }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

int small_per(int n) { return n <= 4096 ? 4 : (n <= 8192 ? 8 : 16); }

lrcc_status launch_small(Ctx* c, cudaStream_t s, const int32_t* succ, int n, int head, int32_t* rank,
                         const int32_t* val = nullptr) {
    const int per = small_per(n);
    const size_t smem = 2 * sizeof(int) * per * FINAL_THREADS;
    const void* k = per == 4 ? (const void*)lr_small_kernel<4>
                  : per == 8 ? (const void*)lr_small_kernel<8> : (const void*)lr_small_kernel<16>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    phase_begin(c, s);
    if (per == 4) lr_small_kernel<4><<<1, FINAL_THREADS, smem, s>>>(succ, val, n, head, rank, c->ctl);
    else if (per == 8) lr_small_kernel<8><<<1, FINAL_THREADS, smem, s>>>(succ, val, n, head, rank, c->ctl);
    else lr_small_kernel<16><<<1, FINAL_THREADS, smem, s>>>(succ, val, n, head, rank, c->ctl);
    phase_end(c, s, PH_SMALL);
    return cuda_status(cudaGetLastError());
}

int stream_grid(Ctx* c, int64_t groups, const void* kernel) {
    const int pg = persistent_grid(c, kernel, BLOCK);
    const int64_t need = (groups + BLOCK - 1) / BLOCK;
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, pg));
}

}  // namespace

// --------------------------------------------------------------- planning

lrcc_status rs_chase_probe_run(Ctx* c, const int32_t* succ, int64_t n, int64_t chains, int64_t steps,
                               int64_t* out) {
    cudaMemsetAsync(out, 0, sizeof(int64_t), c->stream);
    const int64_t threads = (chains + PROBE_K - 1) / PROBE_K;
    const int64_t g = (threads + BLOCK - 1) / BLOCK;
    rs_chase_probe<<<(unsigned)g, BLOCK, 0, c->stream>>>(succ, n, chains, steps,
                                                         reinterpret_cast<unsigned long long*>(out));
    return cuda_status(cudaGetLastError());
}

int rs_walk_grid(Ctx* c, const Plan& p) {
    const void* k = p.rs_chains >= 4 ? (const void*)rs_walk0c<4>
                  : p.rs_chains == 2 ? (const void*)rs_walk0c<2> : (const void*)rs_walk0c<1>;
    return persistent_grid(c, k, BLOCK);
}

int rs_walk_grid_current(const Plan& p) {
    int dev = 0, sms = 0, per_sm = 0;
    const void* k = p.rs_chains >= 4 ? (const void*)rs_walk0c<4>
                  : p.rs_chains == 2 ? (const void*)rs_walk0c<2> : (const void*)rs_walk0c<1>;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, BLOCK, 0) != cudaSuccess || per_sm < 1 ||
        sms < 1) {
        cudaGetLastError();
        return 152 * 8;
    }
    return per_sm * sms;
}

RsLayout rs_layout(int64_t n, const Plan& p, int walk_grid, int64_t extra1, int64_t given1) {
    RsLayout L;
    L.size[0] = n;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    // in-place walk words, the (element, rank) pairs of the read-only walk, or
    // the split mark and local-rank arrays (each 256-byte aligned)
    L.off_W0 = take(sizeof(uint64_t) * (size_t)n + 256);
    int64_t cur = n;
    int lvl = 0;
    while (cur > p.rs_small && lvl < MAX_LEVELS) {
        // spacing: a power of two, at least 4 (one block holds whole 4-element groups)
        int64_t spacing = lvl == 0 ? p.rs_spacing0 : p.rs_spacing;
        int logD = 2;
        while (logD < 20 && (int64_t(1) << (logD + 1)) <= spacing) ++logD;
        if (lvl == MAX_LEVELS - 1)  // last allowed level must fit one block
            while (logD < 30 && ((cur + (int64_t(1) << logD) - 1) >> logD) > p.rs_small) ++logD;
        // level 1 may hold extra splitters (the heads of batched lists ranked as one list)
        int64_t nb = ((cur + (int64_t(1) << logD) - 1) >> logD) + (lvl == 0 ? extra1 : 0);
        if (lvl == 0 && given1 > 0) nb = given1;   // first-level splitters chosen by the caller
        L.logD[lvl] = logD;
        ++lvl;
        L.size[lvl] = nb;
        L.off_R[lvl] = take(sizeof(uint64_t) * (size_t)nb);
        L.off_snext[lvl] = take(sizeof(int32_t) * (size_t)nb);
        L.off_sw[lvl] = take(sizeof(int32_t) * (size_t)nb);
        L.off_S[lvl] = take(sizeof(int32_t) * (size_t)nb);
        cur = nb;
    }
    L.levels = lvl;
    L.readonly = p.rs_level0 == 2 && lvl > 0 && walk_grid > 0;
    L.split = p.rs_level0 == 3 && lvl > 0;
    if (L.readonly) {
        const int64_t G = walk_grid;
        L.grid = G;
        // own region per block: its share of the elements in chunks of 8, plus
        // the padding of its share of the sublists, with 30 % slack
        L.cap = (int64_t)(1.1 * (double)n / (double)G / CIDS + 0.6 * (double)L.size[1] / (double)G) + 16;
        // NSEG segments of an even number of chunks, so every segment's headers
        // start 16-byte aligned (bulk copies)
        L.segcap = (int)((L.cap + 2 * NSEG - 1) / (2 * NSEG)) * 2;
        L.cap = (int64_t)L.segcap * NSEG;
        // the shared pool alone can hold every chunk of a valid list (at most
        // n/8 full chunks plus one partial chunk per sublist), however unevenly
        // the sublists fall on the blocks
        L.ovf_cap = n / CIDS + L.size[1] + 1024;
        L.ovf_cap += L.ovf_cap & 1;
        L.units = (int)(G * NSEG + (L.ovf_cap + L.segcap - 1) / L.segcap);
        const int64_t chunks = G * L.cap + L.ovf_cap;
        L.off_ids = take(sizeof(int32_t) * CIDS * (size_t)chunks);
        L.off_meta = take(sizeof(uint64_t) * (size_t)chunks);
        L.off_fill = take(sizeof(int) * (size_t)G);
        L.off_counts = take(sizeof(int) * (size_t)NBK * (size_t)L.units);
        L.off_totals = take(sizeof(int) * (size_t)NBK);
        L.off_vis = take(sizeof(uint32_t) * (size_t)((n + 31) / 32));
    }
    L.bytes = off;
    return L;
}

// Batched lists as one list: the plan, the layout and the workspace.
constexpr int64_t BATCH_UNION_MIN = int64_t(1) << 22;

bool batch_union_applies(int64_t total, const Plan& batch_plan) {
    return total >= BATCH_UNION_MIN && batch_plan.rs_level0 == 2;
}

struct UnionPlan {
    Plan p;
    RsLayout L;
    size_t off_gsucc, off_head_spl, off_extra, off_head_dev, bytes;
};

UnionPlan union_plan(Ctx* c, int64_t total, int64_t K) {
    UnionPlan U;
    U.p = plan_for(KIND_LR, total);
    U.p.rs_level0 = 2;
    U.L = rs_layout(total, U.p, rs_walk_grid(c, U.p), K);
    size_t off = align_up(U.L.bytes, 256);
    U.off_gsucc = off;
    off = align_up(off + sizeof(int32_t) * (size_t)total, 256);
    U.off_head_spl = off;
    off = align_up(off + sizeof(int32_t) * (size_t)K, 256);
    U.off_extra = off;
    off = align_up(off + sizeof(int32_t) * (size_t)K, 256);
    U.off_head_dev = off;
    U.bytes = off + 256;
    return U;
}

size_t lr_batched_union_ws(Ctx* c, int64_t total, int64_t K) { return union_plan(c, total, K).bytes; }

lrcc_status lr_batched_union(Ctx* c, cudaStream_t s, const int32_t* succ, const int64_t* off, const int32_t* heads,
                             int64_t K, int64_t total, int32_t* rank) {
    const UnionPlan P = union_plan(c, total, K);
    if (!P.L.readonly || P.L.levels == 0 || c->ws_bytes < P.bytes) return LRCC_ERR_ARG;
    char* base = static_cast<char*>(c->ws);
    BatchUnion U;
    U.off = off;
    U.heads = heads;
    U.K = K;
    U.gsucc = reinterpret_cast<int32_t*>(base + P.off_gsucc);
    U.head_spl = reinterpret_cast<int32_t*>(base + P.off_head_spl);
    U.extra_elem = reinterpret_cast<int32_t*>(base + P.off_extra);
    U.head_dev = reinterpret_cast<int64_t*>(base + P.off_head_dev);
    return lr_enqueue_rs(c, s, succ, total, 0, rank, P.p, P.L, nullptr, &U);
}

size_t lr_wyllie_ws(int64_t n, const Plan&) { return 2 * align_up(sizeof(uint64_t) * (size_t)n, 256); }

// ------------------------------------------------------------ enqueueing

lrcc_status lr_enqueue_rs(Ctx* c, cudaStream_t s, const int32_t* succ, int64_t n, int32_t head,
                          int32_t* rank, const Plan& p, const RsLayout& L, const int32_t* val,
                          const BatchUnion* U, const int32_t* given, int64_t given_r) {
    // caller-chosen first-level splitters need the in-place first level
    if (given && (L.readonly || L.split || U)) return LRCC_ERR_ARG;
    // batched lists ranked as one list need the read-only first level
    if (U && (!L.readonly || val)) return LRCC_ERR_ARG;
    // weighted sums use the in-place first level (the others count positions)
    if (val && (L.readonly || L.split)) return LRCC_ERR_ARG;
    if (val) {
        phase_begin(c, s);
        rs_scan_check<<<stream_grid(c, n, (const void*)rs_scan_check), BLOCK, 0, s>>>(val, n, c->ctl);
        rs_scan_verdict<<<1, 1, 0, s>>>(c->ctl);
        phase_end(c, s, PH_SELECT0);
    }
    if (n <= p.rs_small || L.levels == 0) return launch_small(c, s, succ, (int)n, head, rank, val);
    char* base = static_cast<char*>(c->ws);
    auto R = [&](int l) { return reinterpret_cast<uint64_t*>(base + L.off_R[l]); };
    auto SN = [&](int l) { return reinterpret_cast<int32_t*>(base + L.off_snext[l]); };
    auto SW = [&](int l) { return reinterpret_cast<int32_t*>(base + L.off_sw[l]); };
    auto S = [&](int l) { return reinterpret_cast<int32_t*>(base + L.off_S[l]); };
    uint64_t* W0 = reinterpret_cast<uint64_t*>(base + L.off_W0);
    DevCtl* ctl = c->ctl;
    const uint32_t seed0 = (uint32_t)(p.seed ^ (p.seed >> 32));

    // level 0
    const bool vec = aligned16(succ) && (!val || aligned16(val));
    const int64_t groups = (n + 3) / 4;
    if (!L.readonly && !L.split) {
        const void* k = vec ? (const void*)rs_select0<true> : (const void*)rs_select0<false>;
        const int g = stream_grid(c, groups, k);
        phase_begin(c, s);
        if (vec)
            rs_select0<true><<<g, BLOCK, 0, s>>>(succ, val, n, head, W0, SN(1), SW(1), L.logD[0], L.size[1],
                                                 seed0, ctl, given == nullptr);
        else
            rs_select0<false><<<g, BLOCK, 0, s>>>(succ, val, n, head, W0, SN(1), SW(1), L.logD[0], L.size[1],
                                                  seed0, ctl, given == nullptr);
        if (given) {
            const int gm = stream_grid(c, given_r, (const void*)rs_mark_given);
            rs_mark_given<<<gm, BLOCK, 0, s>>>(W0, n, head, given, given_r, SN(1), SW(1), ctl);
        }
        phase_end(c, s, PH_SELECT0);
    }
    Level0 L0;
    L0.n = n;
    L0.logD = L.logD[0];
    L0.nb = (n + (int64_t(1) << L0.logD) - 1) >> L0.logD;   // stratified splitters (level 1 may hold more)
    L0.bh = (int64_t)head >> L0.logD;
    L0.head_off = (uint32_t)(head - (L0.bh << L0.logD));
    L0.seed = seed0;
    if (U) {
        const int g = stream_grid(c, (n + BL_TILE - 1) / BL_TILE * BLOCK, (const void*)bl_gsucc);
        phase_begin(c, s);
        bl_gsucc<<<g, BLOCK, 0, s>>>(succ, U->off, U->K, n, U->gsucc, ctl);
        bl_heads<<<1, 1024, 0, s>>>(U->off, U->heads, U->K, n, L0.logD, L0.nb, seed0, U->head_spl, U->extra_elem,
                                    U->head_dev, ctl);
        phase_end(c, s, PH_BATCH_PREP);
        succ = U->gsucc;
        L0.head_dev = U->head_dev;
        L0.extra = U->extra_elem;
        L0.extra_count = &ctl->ff_extra;
    }
    // split arrays: 16-bit marks while every splitter index fits below the
    // all-ones "not visited" value
    const bool mark16 = L.size[1] < 0xFFFF;
    void* mark = base + L.off_W0;
    int32_t* lrank = reinterpret_cast<int32_t*>(
        base + L.off_W0 + align_up((mark16 ? sizeof(uint16_t) : sizeof(uint32_t)) * (size_t)n, 256));
    if (L.split) {
        phase_begin(c, s);
        if (mark16) {
            const int g = stream_grid(c, n, (const void*)rs_select0s<uint16_t>);
            rs_select0s<uint16_t><<<g, BLOCK, 0, s>>>(succ, (uint16_t*)mark, lrank, SN(1), SW(1), L0, ctl);
        } else {
            const int g = stream_grid(c, n, (const void*)rs_select0s<uint32_t>);
            rs_select0s<uint32_t><<<g, BLOCK, 0, s>>>(succ, (uint32_t*)mark, lrank, SN(1), SW(1), L0, ctl);
        }
        phase_end(c, s, PH_SELECT0);
    }
    Chunks C;
    C.ids = reinterpret_cast<int32_t*>(base + L.off_ids);
    C.meta = reinterpret_cast<uint64_t*>(base + L.off_meta);
    C.fill = reinterpret_cast<int*>(base + L.off_fill);
    C.counts = reinterpret_cast<int*>(base + L.off_counts);
    C.totals = reinterpret_cast<int*>(base + L.off_totals);
    C.vis = reinterpret_cast<uint32_t*>(base + L.off_vis);
    C.cap = L.cap;
    C.segcap = L.segcap;
    C.units = L.units;
    C.ovf_cap = L.ovf_cap;
    C.ovf_base = L.grid * L.cap;
    int lg = 0;
    while ((int64_t(1) << lg) < n) ++lg;
    C.shift = std::max(0, lg - NBK_LOG);
    C.careful = int64_t(32) << L.logD[0];
    auto walk = [&](int l, uint64_t* Wl, int64_t nl) {
        const int r = (int)L.size[l + 1];
        int* work = &ctl->work[l];
        phase_begin(c, s);
        if (p.rs_chains >= 4) {
            const int g = persistent_grid(c, (const void*)rs_walk<4>, BLOCK);
            rs_walk<4><<<g, BLOCK, 0, s>>>(Wl, SN(l + 1), SW(l + 1), R(l + 1), r, work, nl, ctl);
        } else if (p.rs_chains == 2) {
            const int g = persistent_grid(c, (const void*)rs_walk<2>, BLOCK);
            rs_walk<2><<<g, BLOCK, 0, s>>>(Wl, SN(l + 1), SW(l + 1), R(l + 1), r, work, nl, ctl);
        } else {
            const int g = persistent_grid(c, (const void*)rs_walk<1>, BLOCK);
            rs_walk<1><<<g, BLOCK, 0, s>>>(Wl, SN(l + 1), SW(l + 1), R(l + 1), r, work, nl, ctl);
        }
        phase_end(c, s, l == 0 ? PH_WALK0 : PH_WALK);
    };
    if (L.readonly) {
        cudaMemsetAsync(C.vis, 0, sizeof(uint32_t) * (size_t)((n + 31) / 32), s);
        // overflow units' counts are accumulated with atomics (own units are stored whole)
        cudaMemsetAsync(C.counts, 0, sizeof(int) * (size_t)NBK * (size_t)L.units, s);
        const int G = (int)L.grid;
        phase_begin(c, s);
        if (p.rs_chains >= 4) rs_walk0c<4><<<G, BLOCK, 0, s>>>(succ, L0, C, R(1), &ctl->work[0], ctl);
        else if (p.rs_chains == 2) rs_walk0c<2><<<G, BLOCK, 0, s>>>(succ, L0, C, R(1), &ctl->work[0], ctl);
        else rs_walk0c<1><<<G, BLOCK, 0, s>>>(succ, L0, C, R(1), &ctl->work[0], ctl);
        phase_end(c, s, PH_WALK0);
        phase_begin(c, s);
        rs_scan_counts<<<NBK, SCAN_THREADS, 0, s>>>(C.counts, L.units, C.totals);
        phase_end(c, s, PH_SCAN);
        if (U) {
            phase_begin(c, s);
            bl_link<<<stream_grid(c, L.size[1], (const void*)bl_link), BLOCK, 0, s>>>(R(1), L.size[1], U->off, U->K,
                                                                                    U->head_spl, L0, ctl);
            phase_end(c, s, PH_BATCH_PREP);
        }
    } else if (L.split) {
        auto walk0s = [&](auto mt, auto k) {
            using MT = decltype(mt);
            constexpr int K = decltype(k)::value;
            const int g = persistent_grid(c, (const void*)rs_walk0s<MT, K>, BLOCK);
            rs_walk0s<MT, K><<<g, BLOCK, 0, s>>>(succ, (MT*)mark, lrank, SN(1), R(1), &ctl->work[0], L0, ctl);
        };
        phase_begin(c, s);
        if (mark16) {
            if (p.rs_chains >= 4) walk0s(uint16_t(), std::integral_constant<int, 4>());
            else if (p.rs_chains == 2) walk0s(uint16_t(), std::integral_constant<int, 2>());
            else walk0s(uint16_t(), std::integral_constant<int, 1>());
        } else {
            if (p.rs_chains >= 4) walk0s(uint32_t(), std::integral_constant<int, 4>());
            else if (p.rs_chains == 2) walk0s(uint32_t(), std::integral_constant<int, 2>());
            else walk0s(uint32_t(), std::integral_constant<int, 1>());
        }
        phase_end(c, s, PH_WALK0);
    } else {
        walk(0, W0, n);
    }
    for (int l = 1; l < L.levels; ++l) {
        const uint32_t seed = mix32(seed0 + 0x9E3779B9u * (uint32_t)l);
        const int g = stream_grid(c, L.size[l + 1], (const void*)rs_select);
        phase_begin(c, s);
        rs_select<<<g, BLOCK, 0, s>>>(R(l), L.size[l], SN(l + 1), SW(l + 1), L.logD[l], L.size[l + 1], seed, ctl);
        phase_end(c, s, PH_SELECT);
        walk(l, R(l), L.size[l]);
    }
    {
        const int lf = L.levels;
        const int r = (int)L.size[lf];
        const int per = small_per(r);
        const size_t smem = 2 * sizeof(int) * per * FINAL_THREADS;
        phase_begin(c, s);
        if (per == 4) {
            cudaFuncSetAttribute((const void*)rs_final_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            rs_final_kernel<4><<<1, FINAL_THREADS, smem, s>>>(R(lf), r, S(lf), val ? -1 : n, ctl);
        } else if (per == 8) {
            cudaFuncSetAttribute((const void*)rs_final_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            rs_final_kernel<8><<<1, FINAL_THREADS, smem, s>>>(R(lf), r, S(lf), val ? -1 : n, ctl);
        } else {
            cudaFuncSetAttribute((const void*)rs_final_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            rs_final_kernel<16><<<1, FINAL_THREADS, smem, s>>>(R(lf), r, S(lf), val ? -1 : n, ctl);
        }
        phase_end(c, s, PH_FINAL);
    }
    for (int l = L.levels - 1; l >= 1; --l) {
        const int g = stream_grid(c, L.size[l], (const void*)rs_expand);
        phase_begin(c, s);
        rs_expand<<<g, BLOCK, 0, s>>>(R(l), (int)L.size[l], S(l + 1), (int)L.size[l + 1], S(l), ctl);
        phase_end(c, s, PH_EXPAND);
    }
    if (U) {
        phase_begin(c, s);
        bl_adjust<<<stream_grid(c, L.size[1], (const void*)bl_adjust), BLOCK, 0, s>>>(S(1), U->off, U->K, n, L0);
        phase_end(c, s, PH_BATCH_PREP);
    }
    if (L.readonly) {
        phase_begin(c, s);
        cudaFuncSetAttribute((const void*)rs_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SC_SMEM);
        const int gs = std::min((int)L.grid, persistent_grid(c, (const void*)rs_scatter, BLOCK, SC_SMEM));
        rs_scatter<<<gs, BLOCK, SC_SMEM, s>>>(C, (int)L.grid, S(1), W0, n, ctl);
        phase_end(c, s, PH_SCATTER);
        phase_begin(c, s);
        rs_place<<<LRCC_PLACE_BLOCKS_PER_SM * c->sms, BLOCK, 0, s>>>(W0, n, rank, ctl);
        phase_end(c, s, PH_EXPAND0);
    } else if (L.split) {
        phase_begin(c, s);
        if (mark16) {
            const int g = stream_grid(c, n, (const void*)rs_expand0s<uint16_t>);
            rs_expand0s<uint16_t><<<g, BLOCK, 0, s>>>((const uint16_t*)mark, lrank, n, S(1), L.size[1], rank, ctl);
        } else {
            const int g = stream_grid(c, n, (const void*)rs_expand0s<uint32_t>);
            rs_expand0s<uint32_t><<<g, BLOCK, 0, s>>>((const uint32_t*)mark, lrank, n, S(1), L.size[1], rank, ctl);
        }
        phase_end(c, s, PH_EXPAND0);
    } else {
        const bool v = vec && aligned16(rank);
        const void* k = v ? (const void*)rs_expand0<true> : (const void*)rs_expand0<false>;
        const int g = stream_grid(c, groups, k);
        phase_begin(c, s);
        const int bias = val ? 0 : 1;
        if (v) rs_expand0<true><<<g, BLOCK, 0, s>>>(W0, n, S(1), L.size[1], rank, bias, ctl);
        else rs_expand0<false><<<g, BLOCK, 0, s>>>(W0, n, S(1), L.size[1], rank, bias, ctl);
        phase_end(c, s, PH_EXPAND0);
    }
    return cuda_status(cudaGetLastError());
}

// Forest layout: walk words W0 (8 B per element), the has-predecessor bitmap,
// then for r1_max = nb + n first-level splitters (every element could be a
// head) their successor and weight, two word buffers and the sums. The
// pointer-jumping form reuses W0 and the first word buffer.
struct ForestLayout {
    int logD;
    int64_t nb, r1_max;
    size_t off_W0, off_pred, off_snext, off_sw, off_R1, off_R1b, off_S1, bytes;
};

ForestLayout forest_layout(int64_t n, int spacing0) {
    ForestLayout F;
    F.logD = 2;
    while (F.logD < 20 && (int64_t(1) << (F.logD + 1)) <= spacing0) ++F.logD;
    F.nb = (n + (int64_t(1) << F.logD) - 1) >> F.logD;
    F.r1_max = F.nb + n;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    F.off_W0 = take(sizeof(uint64_t) * (size_t)n);
    F.off_pred = take(sizeof(uint32_t) * (size_t)((n + 31) / 32));
    F.off_snext = take(sizeof(int32_t) * (size_t)F.r1_max);
    F.off_sw = take(sizeof(int32_t) * (size_t)F.r1_max);
    F.off_R1 = take(sizeof(uint64_t) * (size_t)F.r1_max);
    F.off_R1b = take(sizeof(uint64_t) * (size_t)F.r1_max);
    F.off_S1 = take(sizeof(int32_t) * (size_t)F.r1_max);
    F.bytes = off;
    return F;
}

size_t lr_scan_forest_ws(int64_t n, const Plan& p) { return forest_layout(n, p.rs_spacing0).bytes; }

lrcc_status lr_enqueue_scan_forest(Ctx* c, cudaStream_t s, const int32_t* succ, const int32_t* val, int64_t n,
                                   int32_t* out, const Plan& p) {
    const ForestLayout F = forest_layout(n, p.rs_spacing0);
    char* base = static_cast<char*>(c->ws);
    uint64_t* W0 = reinterpret_cast<uint64_t*>(base + F.off_W0);
    uint32_t* pred = reinterpret_cast<uint32_t*>(base + F.off_pred);
    int32_t* snext = reinterpret_cast<int32_t*>(base + F.off_snext);
    int32_t* sw = reinterpret_cast<int32_t*>(base + F.off_sw);
    uint64_t* R1 = reinterpret_cast<uint64_t*>(base + F.off_R1);
    uint64_t* R1b = reinterpret_cast<uint64_t*>(base + F.off_R1b);
    int32_t* S1 = reinterpret_cast<int32_t*>(base + F.off_S1);
    DevCtl* ctl = c->ctl;
    const int g = stream_grid(c, n, (const void*)ff_indeg);
    const uint32_t seed = (uint32_t)(p.seed ^ (p.seed >> 32));
    cudaMemsetAsync(pred, 0, sizeof(uint32_t) * (size_t)((n + 31) / 32), s);
    phase_begin(c, s);
    ff_indeg<<<g, BLOCK, 0, s>>>(succ, n, pred, ctl);
    rs_scan_check<<<g, BLOCK, 0, s>>>(val, n, ctl);
    ff_verdict<<<1, 1, 0, s>>>(ctl);
    ff_select0<<<g, BLOCK, 0, s>>>(succ, val, n, pred, W0, snext, sw, F.logD, F.nb, F.r1_max, seed, ctl);
    phase_end(c, s, PH_SELECT0);
    phase_begin(c, s);
    {
        const int gw = persistent_grid(c, (const void*)rs_walk<1>, BLOCK);
        rs_walk<1><<<gw, BLOCK, 0, s>>>(W0, snext, sw, R1, (int)F.nb, &ctl->work[0], n, ctl, &ctl->ff_extra);
    }
    phase_end(c, s, PH_WALK0);
    // the splitter forest by pointer jumping; rounds for the largest possible count
    int rounds = 0;
    while ((int64_t(1) << rounds) < F.r1_max) ++rounds;
    const int g1 = stream_grid(c, F.nb, (const void*)fs_jump);
    uint64_t* a = R1;
    uint64_t* b = R1b;
    for (int r = 0; r < rounds; ++r) {
        phase_begin(c, s);
        fs_jump<<<g1, BLOCK, 0, s>>>(a, b, F.nb, &ctl->ff_extra, ctl);
        phase_end(c, s, PH_WY_JUMP);
        std::swap(a, b);
    }
    phase_begin(c, s);
    fs_final<<<g1, BLOCK, 0, s>>>(a, F.nb, S1, &ctl->ff_extra, ctl);
    phase_end(c, s, PH_FINAL);
    {
        const bool v = aligned16(out);
        const void* k = v ? (const void*)rs_expand0<true> : (const void*)rs_expand0<false>;
        const int ge = stream_grid(c, (n + 3) / 4, k);
        phase_begin(c, s);
        if (v) rs_expand0<true><<<ge, BLOCK, 0, s>>>(W0, n, S1, F.r1_max, out, 0, ctl);
        else rs_expand0<false><<<ge, BLOCK, 0, s>>>(W0, n, S1, F.r1_max, out, 0, ctl);
        phase_end(c, s, PH_EXPAND0);
    }
    // values out of the first level's range: the whole forest by pointer jumping
    // (these kernels return at once otherwise)
    {
        uint64_t* x = W0;
        uint64_t* y = R1;   // r1_max >= n words
        phase_begin(c, s);
        fs_pack<<<g, BLOCK, 0, s>>>(succ, val, n, x, pred, ctl);
        phase_end(c, s, PH_WY_PACK);
        int rr = 0;
        while ((int64_t(1) << rr) < n) ++rr;
        for (int r = 0; r < rr; ++r) {
            phase_begin(c, s);
            fs_jump<<<g, BLOCK, 0, s>>>(x, y, n, nullptr, ctl);
            phase_end(c, s, PH_WY_JUMP);
            std::swap(x, y);
        }
        phase_begin(c, s);
        fs_final<<<g, BLOCK, 0, s>>>(x, n, out, nullptr, ctl);
        phase_end(c, s, PH_WY_FINAL);
    }
    return cuda_status(cudaGetLastError());
}

lrcc_status lr_enqueue_wyllie(Ctx* c, cudaStream_t s, const int32_t* succ, int64_t n, int32_t head,
                              int32_t* rank, const Plan& p) {
    if (n <= p.rs_small) return launch_small(c, s, succ, (int)n, head, rank);
    uint64_t* W0 = static_cast<uint64_t*>(c->ws);
    uint64_t* W1 = reinterpret_cast<uint64_t*>(static_cast<char*>(c->ws) +
                                               align_up(sizeof(uint64_t) * (size_t)n, 256));
    const int64_t groups = (n + 3) / 4;
    const bool vec = aligned16(succ) && aligned16(rank);
    {
        const void* k = vec ? (const void*)wy_pack<true> : (const void*)wy_pack<false>;
        const int g = stream_grid(c, groups, k);
        phase_begin(c, s);
        if (vec) wy_pack<true><<<g, BLOCK, 0, s>>>(succ, n, W0, c->ctl);
        else wy_pack<false><<<g, BLOCK, 0, s>>>(succ, n, W0, c->ctl);
        phase_end(c, s, PH_WY_PACK);
    }
    int rounds = 0;
    while ((int64_t(1) << rounds) < n) ++rounds;
    const int gj = stream_grid(c, groups, (const void*)wy_jump);
    uint64_t* a = W0;
    uint64_t* b = W1;
    for (int r = 0; r + 1 < rounds; ++r) {
        phase_begin(c, s);
        wy_jump<<<gj, BLOCK, 0, s>>>(a, b, n);
        phase_end(c, s, PH_WY_JUMP);
        std::swap(a, b);
    }
    {
        const void* k = vec ? (const void*)wy_final<true> : (const void*)wy_final<false>;
        const int g = stream_grid(c, groups, k);
        phase_begin(c, s);
        if (vec) wy_final<true><<<g, BLOCK, 0, s>>>(a, n, head, rank, c->ctl);
        else wy_final<false><<<g, BLOCK, 0, s>>>(a, n, head, rank, c->ctl);
        phase_end(c, s, PH_WY_FINAL);
    }
    return cuda_status(cudaGetLastError());
}

}  // namespace lrcc
