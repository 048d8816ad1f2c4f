// Batched list ranking and connected components: many independent instances
// in one persistent launch with a work queue over instances.
//
// A preparation kernel orders the instances by size, largest first (longest
// processing time first). Each block of the persistent kernel then takes the
// next instance from a device counter and solves it alone, synchronising
// with __syncthreads only (no block ever waits on another block):
//   lists   up to SMEM_ELEMS elements: loaded into shared memory and ranked by
//           Wyllie's pointer jumping there (Sec. 3.1, single-block variant);
//           larger: a ruling set inside the block (Sec. 3.2): stratified
//           splitters, in-place 8-byte walk words in global workspace, the
//           splitter list held and ranked in shared memory, then the expand.
//   graphs  up to SMEM_ELEMS * 2 vertices: the parent array lives in shared
//           memory, hooks follow both ends to their roots and re-link until
//           joined; up to CC_LARGE vertices: the parent array is the
//           instance's label slice in global memory and hooks are single
//           atomicMin links. Rounds of hooking and shortcutting repeat until
//           __syncthreads_or sees no edge between two trees (Sec. 4,
//           Algorithm 4, step 5).
// Graphs above CC_LARGE vertices would keep one block busy far longer than
// the rest of the batch, so they are labelled together instead, as one
// disjoint union in global ids (voff[k] + local id), by grid-wide hook and
// shortcut kernels looped on the device; components never cross instances,
// so the union's min-id labels minus voff[k] are each instance's labels.
#include <algorithm>

#include "block_wyllie.cuh"
#include "cc_device.cuh"
#include "common.cuh"
#include "internal.h"

namespace lrcc {

namespace {

constexpr int BT = 512;                   // threads per batched block
constexpr int SMEM_ELEMS = 8192;          // list elements / splitters held in shared memory
constexpr int PER = SMEM_ELEMS / BT;      // per-thread share in block_wyllie
constexpr int CC_SMEM_VERTS = 2 * SMEM_ELEMS;
constexpr size_t SMEM_BYTES = 2 * sizeof(int) * SMEM_ELEMS;   // 64 KB, both kinds
constexpr int NCLASS = 33;
constexpr int64_t CC_LARGE = int64_t(1) << 15;   // graphs above this many vertices go to the union path
constexpr int SEG_BLOCK = 256;

// Order instances by size class (floor(log2 size)), largest first.
__global__ void __launch_bounds__(1024)
    batch_order(const int64_t* __restrict__ off_a, const int64_t* __restrict__ off_b, const int32_t* heads,
                int64_t count, int32_t* __restrict__ order, DevCtl* ctl) {
    __shared__ int s_hist[NCLASS];
    __shared__ int s_start[NCLASS];
    for (int t = threadIdx.x; t < NCLASS; t += blockDim.x) s_hist[t] = 0;
    __syncthreads();
    // size class of instance k, -> class 0 when its offsets or head are invalid
    auto klass = [&](int64_t k) -> int {
        const int64_t na = off_a[k + 1] - off_a[k];
        bool bad = na < 0 || na > 0x7FFFFFFELL || (k == 0 && off_a[0] != 0);
        int64_t size = na;
        if (off_b) {
            const int64_t nbv = off_b[k + 1] - off_b[k];
            bad |= nbv < 0 || nbv > 0x7FFFFFFELL || (k == 0 && off_b[0] != 0);
            size += nbv;
        }
        if (heads && na > 0) bad |= heads[k] < 0 || heads[k] >= na;
        if (bad) {
            record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)k);
            return 0;
        }
        return size <= 1 ? 0 : min(63 - __clzll((unsigned long long)size), NCLASS - 1);
    };
    for (int64_t k = threadIdx.x; k < count; k += blockDim.x) atomicAdd(&s_hist[klass(k)], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int c = NCLASS - 1; c >= 0; --c) {
            s_start[c] = run;
            run += s_hist[c];
        }
    }
    __syncthreads();
    for (int64_t k = threadIdx.x; k < count; k += blockDim.x) order[atomicAdd(&s_start[klass(k)], 1)] = (int32_t)k;
}

__device__ __forceinline__ int64_t take_instance(int* s_k, int64_t count, DevCtl* ctl) {
    __syncthreads();
    if (threadIdx.x == 0) *s_k = atomicAdd(&ctl->batch_next, 1);
    __syncthreads();
    return *s_k < count ? *s_k : -1;
}

// ----------------------------------------------------------------- lists

// Rank one list of n <= SMEM_ELEMS elements in shared memory.
__device__ void list_in_smem(const int32_t* succ, int n, int head, int32_t* rank, int* val, int* nxt,
                             DevCtl* ctl) {
    for (int i = threadIdx.x; i < n; i += BT) {
        const int s = succ[i];
        const bool tail = (s == -1) | (s == i);
        const bool bad = !tail && (s < 0 || s >= n);
        if (bad) record_error(ctl, LRCC_ERR_INVALID_INPUT, i);
        nxt[i] = (tail || bad) ? (int)NIL : s;
        val[i] = 1;
    }
    __syncthreads();
    block_wyllie<PER, BT>(val, nxt, n, ctl);
    for (int i = threadIdx.x; i < n; i += BT) rank[i] = val[i] - 1;
    if (threadIdx.x == 0 && val[head] != n) record_error(ctl, LRCC_ERR_INVALID_INPUT, head);
}

// Rank one larger list with a ruling set inside the block; W is the list's
// slice of the 8-byte word workspace.
__device__ void list_ruling_set(const int32_t* succ, int64_t n, int head, int32_t* rank, uint64_t* W,
                                int* val, int* nxt, int* s_work, uint32_t seed, int min_logD, DevCtl* ctl) {
    // spacing: a power of two, at least 2^min_logD, with at most SMEM_ELEMS splitters
    int logD = max(2, min_logD);
    while (((n + (int64_t(1) << logD) - 1) >> logD) > SMEM_ELEMS) ++logD;
    const int64_t D = int64_t(1) << logD;
    const int r = (int)((n + D - 1) >> logD);
    const int64_t bh = head >> logD;
    const uint32_t head_off = (uint32_t)(head - (bh << logD));
    // select (RS1+RS2): walk words, and each splitter's successor in nxt[j]
    for (int64_t i = threadIdx.x; i < n; i += BT) {
        const int s = succ[i];
        const bool tail = (s == -1) | (s == i);
        const bool bad = !tail && (s < 0 || s >= n);
        if (bad) record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)i);
        const uint32_t nx = (tail || bad) ? NIL : (uint32_t)s;
        const int64_t b = i >> logD;
        const uint32_t size = (uint32_t)min(D, n - (b << logD));
        const uint32_t off = b == bh ? head_off : block_offset((uint32_t)b, size, seed);
        if ((uint32_t)(i - (b << logD)) == off) {
            const int j = (int)(b >= bh ? b - bh : b - bh + r);
            W[i] = pack(nx | SPL, (uint32_t)j);
            nxt[j] = (int)nx;
        } else {
            W[i] = pack(nx, 1);
        }
    }
    if (threadIdx.x == 0) *s_work = 0;
    __syncthreads();
    // walk (RS3): one sublist per thread at a time, claimed from a shared counter
    for (;;) {
        const int j = atomicAdd(s_work, 1);
        if (j >= r) break;
        uint32_t cur = (uint32_t)nxt[j];
        uint32_t pre = 1;
        uint32_t next = NIL;
        int64_t steps = 0;
        while (cur != NIL) {
            if (cur >= n) {
                record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)cur);
                break;
            }
            const uint64_t w = W[cur];
            const uint32_t lo = lo32(w), hi = hi32(w);
            if (lo & SPL) {
                next = hi;
                break;
            }
            if ((hi & VIS) || ++steps > n) {
                record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)cur);
                break;
            }
            W[cur] = pack(pre, (uint32_t)j | VIS);
            pre += hi;
            cur = lo;
        }
        nxt[j] = (int)next;
        val[j] = (int)pre;
    }
    __syncthreads();
    // rank the splitters (RS4) in shared memory
    block_wyllie<PER, BT>(val, nxt, r, ctl);
    if (threadIdx.x == 0 && val[0] != n) record_error(ctl, LRCC_ERR_INVALID_INPUT, -3);
    // expand (RS5)
    for (int64_t i = threadIdx.x; i < n; i += BT) {
        const uint64_t w = W[i];
        const uint32_t lo = lo32(w), hi = hi32(w);
        int out;
        if (lo & SPL) {
            out = val[hi] - 1;
        } else if (hi & VIS) {
            out = val[hi & ~VIS] - (int)lo - 1;
        } else {
            record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)i);
            out = -1;
        }
        rank[i] = out;
    }
}

__global__ void __launch_bounds__(BT)
    lr_batch_kernel(const int32_t* __restrict__ succ, const int64_t* __restrict__ off, const int32_t* __restrict__ heads,
                    int64_t count, const int32_t* __restrict__ order, int32_t* __restrict__ rank, uint64_t* W,
                    uint32_t seed, int min_logD, DevCtl* ctl) {
    extern __shared__ int sm[];
    int* val = sm;
    int* nxt = sm + SMEM_ELEMS;
    __shared__ int s_k, s_work;
    for (;;) {
        const int64_t q = take_instance(&s_k, count, ctl);
        if (q < 0) break;
        const int64_t k = order[q];
        const int64_t b = off[k], n = off[k + 1] - b;
        if (n <= 0 || n > 0x7FFFFFFELL) continue;
        const int head = heads[k];
        if (head < 0 || head >= n) continue;
        if (n <= SMEM_ELEMS)
            list_in_smem(succ + b, (int)n, head, rank + b, val, nxt, ctl);
        else
            list_ruling_set(succ + b, n, head, rank + b, W + b, val, nxt, &s_work, seed ^ (uint32_t)k, min_logD, ctl);
    }
}

// ---------------------------------------------------------------- graphs

// Root of x in a shared-memory forest, with path halving.
__device__ __forceinline__ int smem_root(int* p, int x) {
    int px = p[x];
    while (px != x) {
        const int g = p[px];
        p[x] = g;
        x = px;
        px = g;
    }
    return x;
}

__device__ void graph_in_smem(const int32_t* src, const int32_t* dst, int64_t m, int n, int32_t* label,
                              int* p, int cap, DevCtl* ctl) {
    for (int v = threadIdx.x; v < n; v += BT) p[v] = v;
    __syncthreads();
    for (int round = 0;; ++round) {
        bool changed = false;
        for (int64_t e = threadIdx.x; e < m; e += BT) {
            int u = src[e], v = dst[e];
            if (u < 0 || u >= n || v < 0 || v >= n) {
                record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)e);
                continue;
            }
            // re-link until joined: every edge is joined by the end of the pass
            for (;;) {
                u = smem_root(p, u);
                v = smem_root(p, v);
                if (u == v) break;
                const int hi = max(u, v), lo = min(u, v);
                const int old = atomicMin(p + hi, lo);
                changed = true;
                if (old == hi) break;
                u = old;
                v = lo;
            }
        }
        __syncthreads();
        // chases longer than CHASE_QUIET steps store their progress in their own
        // entry, so chases through it jump ahead (see chase_step)
        for (int v = threadIdx.x; v < n; v += BT) {
            int x = p[v];
            for (int step = 0; p[x] != x; ++step) {
                x = p[x];
                if (step >= CHASE_QUIET) p[v] = x;
            }
            p[v] = x;
        }
        if (!__syncthreads_or(changed)) break;
        if (round + 1 >= cap) {
            if (threadIdx.x == 0) record_error(ctl, LRCC_ERR_NOT_CONVERGED, round);
            break;
        }
    }
    for (int v = threadIdx.x; v < n; v += BT) label[v] = p[v];
}

__device__ void graph_in_global(const int32_t* src, const int32_t* dst, int64_t m, int64_t n, int32_t* p,
                                int cap, DevCtl* ctl) {
    for (int64_t v = threadIdx.x; v < n; v += BT) p[v] = (int32_t)v;
    __syncthreads();
    for (int round = 0;; ++round) {
        bool changed = false;
        for (int64_t e = threadIdx.x; e < m; e += BT) {
            const int u = src[e], v = dst[e];
            if (u < 0 || u >= n || v < 0 || v >= n) {
                record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)e);
                continue;
            }
            const int a = ld_cg(p + u), b = ld_cg(p + v);
            if (a != b) {
                const int hi = max(a, b), lo = min(a, b);
                if (ld_cg(p + hi) > lo) atomicMin(p + hi, lo);
                changed = true;
            }
        }
        __syncthreads();
        for (int64_t v = threadIdx.x; v < n; v += BT) {
            int x = ld_cg(p + v);
            if (x == v) continue;
            for (int step = 0;; ++step) {
                const int y = ld_cg(p + x);
                if (y == x) break;
                x = y;
                if (step >= CHASE_QUIET) p[v] = x;   // progress for chases through v (see chase_step)
            }
            p[v] = x;
        }
        if (!__syncthreads_or(changed)) break;
        if (round + 1 >= cap) {
            if (threadIdx.x == 0) record_error(ctl, LRCC_ERR_NOT_CONVERGED, round);
            break;
        }
    }
}

__global__ void __launch_bounds__(BT)
    cc_batch_kernel(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, const int64_t* __restrict__ eoff,
                    const int64_t* __restrict__ voff, int64_t count, const int32_t* __restrict__ order,
                    int32_t* label, int max_rounds, DevCtl* ctl) {
    extern __shared__ int sm[];
    __shared__ int s_k;
    for (;;) {
        const int64_t q = take_instance(&s_k, count, ctl);
        if (q < 0) break;
        const int64_t k = order[q];
        const int64_t eb = eoff[k], m = eoff[k + 1] - eb;
        const int64_t vb = voff[k], n = voff[k + 1] - vb;
        if (n <= 0 || m < 0 || n > 0x7FFFFFFELL || n > CC_LARGE) continue;
        int lg = 0;
        while ((int64_t(1) << lg) < n) ++lg;
        const int cap = max_rounds > 0 ? max_rounds : 64 + 4 * lg;
        if (n <= CC_SMEM_VERTS)
            graph_in_smem(src + eb, dst + eb, m, (int)n, label + vb, sm, cap, ctl);
        else
            graph_in_global(src + eb, dst + eb, m, n, label + vb, cap, ctl);
    }
}

// ---------------------------------------------------- graphs: the union path

// The large instances, in instance order, with prefix sums of their edge and
// vertex counts; nlarge = their number. One block.
struct LargeSet {
    int32_t* ids;
    int64_t* lep;   // [nlarge + 1] edge prefix
    int64_t* lvp;   // [nlarge + 1] vertex prefix
    int* nlarge;
};

__device__ __forceinline__ int64_t block_exclusive_scan64(int64_t v, int64_t* s_tmp, int64_t* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_tmp[wid] = incl;
    __syncthreads();
    int64_t off = 0, all = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        off += w < wid ? s_tmp[w] : 0;
        all += s_tmp[w];
    }
    __syncthreads();
    *total = all;
    return off + incl - v;
}

__global__ void __launch_bounds__(1024)
    large_prep(const int64_t* __restrict__ eoff, const int64_t* __restrict__ voff, int64_t count, LargeSet L) {
    __shared__ int64_t s_tmp[32];
    const int64_t per = (count + blockDim.x - 1) / blockDim.x;
    const int64_t b = threadIdx.x * per, e = min(count, b + per);
    auto large = [&](int64_t k) {
        const int64_t n = voff[k + 1] - voff[k], m = eoff[k + 1] - eoff[k];
        return n > CC_LARGE && n <= 0x7FFFFFFELL && m >= 0;
    };
    int64_t c = 0, me = 0, mv = 0;
    for (int64_t k = b; k < e; ++k)
        if (large(k)) {
            ++c;
            me += eoff[k + 1] - eoff[k];
            mv += voff[k + 1] - voff[k];
        }
    int64_t tc, te, tv;
    int64_t at = block_exclusive_scan64(c, s_tmp, &tc);
    int64_t ae = block_exclusive_scan64(me, s_tmp, &te);
    int64_t av = block_exclusive_scan64(mv, s_tmp, &tv);
    for (int64_t k = b; k < e; ++k)
        if (large(k)) {
            L.ids[at] = (int32_t)k;
            L.lep[at] = ae;
            L.lvp[at] = av;
            ++at;
            ae += eoff[k + 1] - eoff[k];
            av += voff[k + 1] - voff[k];
        }
    if (threadIdx.x == 0) {
        *L.nlarge = (int)tc;
        L.lep[tc] = te;
        L.lvp[tc] = tv;
    }
}

// Largest i with pre[i] <= x, over pre[0..nl] (pre[0] = 0, x < pre[nl]).
__device__ __forceinline__ int seg_find(const int64_t* pre, int nl, int64_t x) {
    int lo = 0, hi = nl;   // invariant: pre[lo] <= x < pre[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(pre + mid) <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

constexpr int SEG_RUN = 8;   // consecutive vertices or edges per thread

// Vertex passes over the large instances take tiles of SEG_TILE union
// positions x (one binary search per tile); thread t handles x = t0 + t +
// q * SEG_BLOCK, so consecutive threads touch consecutive vertices.
constexpr int SEG_PER = 16;
constexpr int64_t SEG_TILE = (int64_t)SEG_BLOCK * SEG_PER;

// label[g] = g for every vertex g of a large instance (g = voff[k] + local).
__global__ void __launch_bounds__(SEG_BLOCK) seg_init(LargeSet L, const int64_t* __restrict__ voff, int32_t* label) {
    __shared__ int s_i;
    const int nl = *L.nlarge;
    const int64_t V = L.lvp[nl];
    for (int64_t t0 = (int64_t)blockIdx.x * SEG_TILE; t0 < V; t0 += (int64_t)gridDim.x * SEG_TILE) {
        if (threadIdx.x == 0) s_i = seg_find(L.lvp, nl, t0);
        __syncthreads();
        int i = s_i;
        __syncthreads();
        const int64_t tend = min(t0 + SEG_TILE, V);
#pragma unroll
        for (int q = 0; q < SEG_PER; ++q) {
            const int64_t x = t0 + threadIdx.x + (int64_t)q * SEG_BLOCK;
            if (x >= tend) break;
            while (x >= L.lvp[i + 1]) ++i;
            const int64_t g = voff[L.ids[i]] + (x - L.lvp[i]);
            label[g] = (int32_t)g;
        }
    }
}

// Global labels -> local labels (label[g] - voff[k]); the tile's labels are
// loaded first, so that SEG_PER reads are in flight.
__global__ void __launch_bounds__(SEG_BLOCK) seg_finalize(LargeSet L, const int64_t* __restrict__ voff, int32_t* label) {
    __shared__ int s_i;
    const int nl = *L.nlarge;
    const int64_t V = L.lvp[nl];
    for (int64_t t0 = (int64_t)blockIdx.x * SEG_TILE; t0 < V; t0 += (int64_t)gridDim.x * SEG_TILE) {
        if (threadIdx.x == 0) s_i = seg_find(L.lvp, nl, t0);
        __syncthreads();
        int i = s_i;
        __syncthreads();
        const int64_t tend = min(t0 + SEG_TILE, V);
        int64_t g[SEG_PER], base[SEG_PER];
        int32_t v[SEG_PER];
#pragma unroll
        for (int q = 0; q < SEG_PER; ++q) {
            const int64_t x = t0 + threadIdx.x + (int64_t)q * SEG_BLOCK;
            g[q] = -1;
            if (x >= tend) continue;
            while (x >= L.lvp[i + 1]) ++i;
            base[q] = voff[L.ids[i]];
            g[q] = base[q] + (x - L.lvp[i]);
        }
#pragma unroll
        for (int q = 0; q < SEG_PER; ++q) v[q] = g[q] >= 0 ? label[g[q]] : 0;
#pragma unroll
        for (int q = 0; q < SEG_PER; ++q)
            if (g[q] >= 0) label[g[q]] = (int32_t)(v[q] - base[q]);
    }
}

// One hook pass over the large instances (single atomicMin hooks with a read
// before the atomic, as in the single-instance path). The first two passes
// read the instances' edges (local ids, instance found by binary search);
// from the second pass on, edges still joining two trees are appended as
// global (u, v) pairs to the active buffer that the next pass reads instead.
struct SegActive {
    int2* buf[2];
    int64_t cap;
};

// Blocks take slices of the pass's edges from a counter, in order, so the
// edges in flight belong to a few consecutive graphs and their parent
// entries stay in L2 (a grid-stride loop would let blocks drift across many
// graphs, whose parent arrays together are far larger than L2).
constexpr int SEG_SLICE = SEG_BLOCK * 64;
constexpr int SEG_STAGE = 32 * SEG_RUN;   // active edges a warp stages before appending

__global__ void __launch_bounds__(SEG_BLOCK)
    seg_hook(LargeSet L, const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
             const int64_t* __restrict__ eoff, const int64_t* __restrict__ voff, int32_t* label, SegActive act,
             int mode, DevCtl* ctl) {
    __shared__ int s_slice, s_i;
    const bool relink = mode == 2 || (mode == 3 && ctl->rounds > 0);
    const bool direct = mode == 5 && ctl->rounds == 0;   // rule 5's first pass (see cc.cu)
    const uint64_t keep = policy_evict_last();
    const uint64_t stream_pol = policy_evict_first();
    const int nl = *L.nlarge;
    const int sel = ctl->cc_src;
    const int out_sel = sel == 1 ? 2 : 1;
    const bool compact = ctl->rounds > 0 && act.cap > 0;
    const int64_t E = sel == 0 ? L.lep[nl] : min((int64_t)ctl->cc_count[sel], act.cap);
    const int lane = threadIdx.x & 31;
    bool changed = false;
    // active edges are staged per warp and appended in batches (one counter
    // atomic per batch instead of one per warp iteration)
    __shared__ int2 s_stage[SEG_BLOCK / 32][SEG_STAGE];
    int2* stage = s_stage[threadIdx.x >> 5];
    int2* out = act.buf[out_sel - 1];
    int staged = 0;   // warp-uniform
    auto flush = [&]() {
        __syncwarp();
        int base = 0;
        if (lane == 0) base = atomicAdd(&ctl->cc_count[out_sel], staged);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (lane == 0 && (int64_t)base + staged > act.cap) ctl->cc_overflow = 1;
        for (int j = lane; j < staged; j += 32)
            if ((int64_t)base + j < act.cap) out[base + j] = stage[j];
        __syncwarp();
        staged = 0;
    };
    for (;;) {
        if (threadIdx.x == 0) {
            s_slice = atomicAdd(&ctl->seg_next, 1);
            const int64_t st = (int64_t)s_slice * SEG_SLICE;
            s_i = sel == 0 && st < E ? seg_find(L.lep, nl, st) : 0;
        }
        __syncthreads();
        const int64_t start = (int64_t)s_slice * SEG_SLICE;
        int i = s_i;   // the slice's first graph; each thread advances from it
        __syncthreads();
        if (start >= E) break;
        // the graph of the thread's current edge: instance, end of its edges in
        // the union, edge offset, vertex base and count
        int g_k = 0;
        int64_t g_hi = -1, g_at = 0, g_base = 0, g_n = 0;
        const int64_t end = min(start + SEG_SLICE, E);
        for (int64_t c0 = start; c0 < end; c0 += (int64_t)SEG_BLOCK * SEG_RUN) {
            int32_t u[SEG_RUN], v[SEG_RUN];
#pragma unroll
            for (int q = 0; q < SEG_RUN; ++q) {
                u[q] = v[q] = -1;
                const int64_t e = c0 + (int64_t)q * SEG_BLOCK + threadIdx.x;   // coalesced across the block
                if (e >= end) continue;
                if (sel != 0) {
                    const int2 x = __ldcs(act.buf[sel - 1] + e);
                    u[q] = x.x;
                    v[q] = x.y;
                } else {
                    // the graph's offsets are loaded once per graph, not once per edge
                    // (24.8 -> 24.2 ms for the 4096-instance mix's graphs)
                    if (e >= g_hi) {   // e grows within a slice: refresh on leaving the graph
                        while (e >= L.lep[i + 1]) ++i;
                        g_k = L.ids[i];
                        g_hi = L.lep[i + 1];
                        g_at = eoff[g_k] - L.lep[i];
                        g_base = voff[g_k];
                        g_n = voff[g_k + 1] - g_base;
                    }
                    const int k = g_k;
                    const int64_t at = e + g_at, base = g_base, n = g_n;
                    const int a = ld_stream(src + at, stream_pol), b = ld_stream(dst + at, stream_pol);
                    if (a < 0 || a >= n || b < 0 || b >= n) {
                        record_error(ctl, LRCC_ERR_INVALID_INPUT, k);
                        continue;
                    }
                    u[q] = (int32_t)(base + a);
                    v[q] = (int32_t)(base + b);
                }
            }
            if (direct) {   // first pass: nothing is kept, so no compaction either
#pragma unroll
                for (int q = 0; q < SEG_RUN; ++q)
                    if (u[q] >= 0) changed |= link_direct(label, u[q], v[q], keep);
                continue;
            }
            int32_t pa[SEG_RUN], pb[SEG_RUN];
#pragma unroll
            for (int q = 0; q < SEG_RUN; ++q) {
                pa[q] = u[q] >= 0 ? ld_hint(label + u[q], keep) : 0;
                pb[q] = u[q] >= 0 ? ld_hint(label + v[q], keep) : 0;
            }
            int nkeep = 0;
#pragma unroll
            for (int q = 0; q < SEG_RUN; ++q) {
                const bool active = u[q] >= 0 && pa[q] != pb[q];
                if (active) changed |= hook_pair(label, pa[q], pb[q], relink, keep);
                if (!active) u[q] = -1;
                nkeep += active;
            }
            if (compact) {
                int total = 0;
                const int excl = warp_prefix_small(nkeep, &total);
                if (total > 0) {   // warp-uniform
                    if (staged + total > SEG_STAGE) flush();
                    int at = staged + excl;
#pragma unroll
                    for (int q = 0; q < SEG_RUN; ++q)
                        if (u[q] >= 0) stage[at++] = make_int2(u[q], v[q]);
                    staged += total;
                }
            }
        }
    }
    if (compact && staged > 0) flush();
    if (__any_sync(0xffffffffu, changed) && lane == 0) ctl->flag = 1;
}

__global__ void seg_control(DevCtl* ctl, cudaGraphConditionalHandle h, int cap, bool compacting) {
    const int r = ++ctl->rounds;
    const int f = ctl->flag;
    ctl->flag = 0;
    unsigned cont = f != 0;
    if (cont && r >= cap) {
        record_error(ctl, LRCC_ERR_NOT_CONVERGED, r);
        cont = 0;
    }
    if (ctl->status) cont = 0;
    ctl->cc_stop = !cont;
    // next pass: the active buffer this pass filled (from the second pass on)
    const int sel = ctl->cc_src;
    const int out_sel = sel == 1 ? 2 : 1;
    int next = 0;
    if (compacting && r > 1 && !ctl->cc_overflow) next = out_sel;
    ctl->cc_overflow = 0;
    ctl->cc_src = next;
    ctl->cc_count[next == 1 ? 2 : 1] = 0;
    ctl->seg_next = 0;
    ctl->seg_next_v = 0;
    cudaGraphSetConditional(h, cont);
}

// The same decision for a host-driven loop (plain launches): answer in ctl->pad[0].
__global__ void seg_control_host(DevCtl* ctl, int cap, bool compacting) {
    const int r = ++ctl->rounds;
    const int f = ctl->flag;
    ctl->flag = 0;
    int cont = f != 0;
    if (cont && r >= cap) {
        record_error(ctl, LRCC_ERR_NOT_CONVERGED, r);
        cont = 0;
    }
    if (ctl->status) cont = 0;
    ctl->cc_stop = !cont;
    const int sel = ctl->cc_src;
    const int out_sel = sel == 1 ? 2 : 1;
    int next = 0;
    if (compacting && r > 1 && !ctl->cc_overflow) next = out_sel;
    ctl->cc_overflow = 0;
    ctl->cc_src = next;
    ctl->cc_count[next == 1 ? 2 : 1] = 0;
    ctl->seg_next = 0;
    ctl->seg_next_v = 0;
    ctl->pad[0] = cont;
}

// Pointer jumping to stars over the large instances' vertices (skipped after
// the pass that joined nothing). Blocks take slices in order, so the chases in
// flight stay within a few graphs whose parent entries L2 holds.
__global__ void __launch_bounds__(SEG_BLOCK)
    seg_shortcut(LargeSet L, const int64_t* __restrict__ voff, int32_t* label, DevCtl* ctl) {
    __shared__ int s_slice, s_i;
    if (ctl->cc_stop) return;
    const uint64_t keep = policy_evict_last();
    const int nl = *L.nlarge;
    const int64_t V = L.lvp[nl];
    for (;;) {
        if (threadIdx.x == 0) {
            s_slice = atomicAdd(&ctl->seg_next_v, 1);
            const int64_t st = (int64_t)s_slice * SEG_SLICE;
            s_i = st < V ? seg_find(L.lvp, nl, st) : 0;
        }
        __syncthreads();
        const int64_t start = (int64_t)s_slice * SEG_SLICE;
        int i = s_i;
        __syncthreads();
        if (start >= V) break;
        const int64_t end = min(start + SEG_SLICE, V);
        for (int64_t x = start + threadIdx.x; x < end; x += SEG_BLOCK) {
            while (x >= L.lvp[i + 1]) ++i;
            const int64_t g = voff[L.ids[i]] + (x - L.lvp[i]);
            const int p = label[g];
            if (p != g) {
                const int r = chase_root(label, (int32_t)g, p, keep);
                if (r != p) label[g] = r;
            }
        }
    }
}

lrcc_status set_smem(const void* k) {
    return cuda_status(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
}

}  // namespace

size_t lr_batched_ws(int64_t total_nodes, int64_t count) {
    return align_up(sizeof(uint64_t) * (size_t)std::max<int64_t>(total_nodes, 1), 256) +
           align_up(sizeof(int32_t) * (size_t)std::max<int64_t>(count, 1), 256);
}

// Active-edge buffers of the union path: a quarter of all edges each. On the
// 4096-instance mix (ER, 4 edges per vertex) the second pass keeps more than
// an eighth of the edges, so with buffers of m/8 the third pass read every
// edge again (24.2 ms against 23.8 with m/4 and 23.9 with m/2).
int64_t cc_batched_active_cap(int64_t total_edges) {
    return total_edges >= (int64_t(1) << 16) ? total_edges / 4 : 0;
}

size_t cc_batched_ws(int64_t count, int64_t total_edges) {
    const size_t c = (size_t)std::max<int64_t>(count, 1);
    const int64_t acap = cc_batched_active_cap(total_edges);
    return 2 * align_up(sizeof(int32_t) * c, 256) + 2 * align_up(sizeof(int64_t) * (c + 1), 256) + 256 +
           (acap > 0 ? 2 * align_up(sizeof(int2) * (size_t)acap, 256) : 0);
}

lrcc_status lr_batched_run(Ctx* c, const int32_t* succ, const int64_t* off, const int32_t* heads, int64_t count,
                           int32_t* rank, int64_t total_nodes, const Plan& p) {
    cudaStream_t s = c->stream;
    uint64_t* W = static_cast<uint64_t*>(c->ws);
    int32_t* order = reinterpret_cast<int32_t*>(static_cast<char*>(c->ws) +
                                                align_up(sizeof(uint64_t) * (size_t)std::max<int64_t>(total_nodes, 1), 256));
    phase_begin(c, s);
    batch_order<<<1, 1024, 0, s>>>(off, nullptr, heads, count, order, c->ctl);
    phase_end(c, s, PH_BATCH_PREP);
    lrcc_status st = set_smem((const void*)lr_batch_kernel);
    if (st != LRCC_OK) return st;
    const int g = (int)std::min<int64_t>(count, persistent_grid(c, (const void*)lr_batch_kernel, BT, SMEM_BYTES));
    phase_begin(c, s);
    int min_logD = 2;
    while (min_logD < 20 && (1 << (min_logD + 1)) <= p.rs_spacing0) ++min_logD;
    lr_batch_kernel<<<g, BT, SMEM_BYTES, s>>>(succ, off, heads, count, order, rank, W,
                                              (uint32_t)(p.seed ^ (p.seed >> 32)), min_logD, c->ctl);
    phase_end(c, s, PH_LR_BATCH);
    return cuda_status(cudaGetLastError());
}

lrcc_status cc_batched_run(Ctx* c, const int32_t* src, const int32_t* dst, const int64_t* eoff, const int64_t* voff,
                           int64_t count, int64_t total_edges, int32_t* label, const Plan& p) {
    cudaStream_t s = c->stream;
    const size_t cnt = (size_t)std::max<int64_t>(count, 1);
    char* w = static_cast<char*>(c->ws);
    int32_t* order = reinterpret_cast<int32_t*>(w);
    w += align_up(sizeof(int32_t) * cnt, 256);
    LargeSet L;
    L.ids = reinterpret_cast<int32_t*>(w);
    w += align_up(sizeof(int32_t) * cnt, 256);
    L.lep = reinterpret_cast<int64_t*>(w);
    w += align_up(sizeof(int64_t) * (cnt + 1), 256);
    L.lvp = reinterpret_cast<int64_t*>(w);
    w += align_up(sizeof(int64_t) * (cnt + 1), 256);
    L.nlarge = reinterpret_cast<int*>(w);
    w += 256;
    SegActive act{{nullptr, nullptr}, cc_batched_active_cap(total_edges)};
    if (act.cap > 0) {
        act.buf[0] = reinterpret_cast<int2*>(w);
        act.buf[1] = reinterpret_cast<int2*>(w + align_up(sizeof(int2) * (size_t)act.cap, 256));
    }

    phase_begin(c, s);
    batch_order<<<1, 1024, 0, s>>>(voff, eoff, nullptr, count, order, c->ctl);
    large_prep<<<1, 1024, 0, s>>>(eoff, voff, count, L);
    phase_end(c, s, PH_BATCH_PREP);

    // the union of the large graphs: init, device-side loop, finalize
    const int gs = persistent_grid(c, (const void*)seg_hook, SEG_BLOCK);
    const int gv = persistent_grid(c, (const void*)seg_shortcut, SEG_BLOCK);
    const int cap = 64 + 4 * 31;
    phase_begin(c, s);
    seg_init<<<gv, SEG_BLOCK, 0, s>>>(L, voff, label);
    if (p.use_graphs == 2) {
        // host-driven loop, one flag read per pass (so profilers see every kernel)
        int* host_flag = nullptr;
        if (cudaMallocHost(&host_flag, sizeof(int)) != cudaSuccess) return LRCC_ERR_NOMEM;
        lrcc_status st = LRCC_OK;
        for (int r = 0; r <= cap; ++r) {
            seg_hook<<<gs, SEG_BLOCK, 0, s>>>(L, src, dst, eoff, voff, label, act, p.cc_hook, c->ctl);
            seg_control_host<<<1, 1, 0, s>>>(c->ctl, cap, act.cap > 0);
            seg_shortcut<<<gv, SEG_BLOCK, 0, s>>>(L, voff, label, c->ctl);
            cudaMemcpyAsync(host_flag, &c->ctl->pad[0], sizeof(int), cudaMemcpyDeviceToHost, s);
            if (cudaStreamSynchronize(s) != cudaSuccess) {
                st = LRCC_ERR_CUDA;
                break;
            }
            if (!*host_flag) break;
        }
        cudaFreeHost(host_flag);
        if (st != LRCC_OK) return st;
    } else {
    const std::vector<uint64_t> key = {(uint64_t)KIND_CC_BATCH, (uint64_t)src, (uint64_t)dst, (uint64_t)eoff,
                                       (uint64_t)voff, (uint64_t)count, (uint64_t)label, (uint64_t)c->ws,
                                       (uint64_t)act.cap, (uint64_t)p.cc_hook};
    GraphEntry* e = nullptr;
    for (auto& ge : c->graphs)
        if (ge.key == key) e = &ge;
    if (!e) {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ex = nullptr;
        lrcc_status st = LRCC_OK;
        cudaGraphConditionalHandle h;
        cudaGraphNode_t node;
        cudaGraphNodeParams cp = {};
        if (cudaGraphCreate(&g, 0) != cudaSuccess) return LRCC_ERR_CUDA;
        if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) st = LRCC_ERR_CUDA;
        if (st == LRCC_OK) {
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) != cudaSuccess) st = LRCC_ERR_CUDA;
        }
        if (st == LRCC_OK) {
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            if (cudaStreamBeginCaptureToGraph(c->capture, body, nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                st = LRCC_ERR_CUDA;
            } else {
                seg_hook<<<gs, SEG_BLOCK, 0, c->capture>>>(L, src, dst, eoff, voff, label, act, p.cc_hook, c->ctl);
                seg_control<<<1, 1, 0, c->capture>>>(c->ctl, h, cap, act.cap > 0);
                seg_shortcut<<<gv, SEG_BLOCK, 0, c->capture>>>(L, voff, label, c->ctl);
                cudaGraph_t captured = nullptr;
                if (cudaStreamEndCapture(c->capture, &captured) != cudaSuccess) st = LRCC_ERR_CUDA;
            }
        }
        if (st == LRCC_OK && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) st = LRCC_ERR_CUDA;
        cudaGraphDestroy(g);
        if (st != LRCC_OK) {
            cudaGetLastError();
            return st;
        }
        if (c->graphs.size() >= 16) {
            auto it = std::min_element(c->graphs.begin(), c->graphs.end(),
                                       [](const GraphEntry& x, const GraphEntry& y) { return x.last_use < y.last_use; });
            cudaGraphExecDestroy(it->exec);
            c->graphs.erase(it);
        }
        c->graphs.push_back(GraphEntry{key, ex, 0});
        e = &c->graphs.back();
    }
    e->last_use = ++c->tick;
    if (cudaGraphLaunch(e->exec, s) != cudaSuccess) return LRCC_ERR_CUDA;
    }
    seg_finalize<<<gv, SEG_BLOCK, 0, s>>>(L, voff, label);
    phase_end(c, s, PH_CC_LOOP);

    // every other graph: one block each, largest first
    lrcc_status st = set_smem((const void*)cc_batch_kernel);
    if (st != LRCC_OK) return st;
    const int g = (int)std::min<int64_t>(count, persistent_grid(c, (const void*)cc_batch_kernel, BT, SMEM_BYTES));
    phase_begin(c, s);
    cc_batch_kernel<<<g, BT, SMEM_BYTES, s>>>(src, dst, eoff, voff, count, order, label, p.cc_max_rounds, c->ctl);
    phase_end(c, s, PH_CC_BATCH);
    return cuda_status(cudaGetLastError());
}

}  // namespace lrcc
