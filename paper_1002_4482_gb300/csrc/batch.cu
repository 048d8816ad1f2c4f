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
//           joined; larger: the parent array is the instance's label slice in
//           global memory and hooks are single atomicMin links. Rounds of
//           hooking and shortcutting repeat until __syncthreads_or sees no
//           edge between two trees (Sec. 4, Algorithm 4, step 5).
#include <algorithm>

#include "block_wyllie.cuh"
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
                                int* val, int* nxt, int* s_work, uint32_t seed, DevCtl* ctl) {
    // spacing: a power of two with at most SMEM_ELEMS splitters
    int logD = 2;
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
                    uint32_t seed, DevCtl* ctl) {
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
            list_ruling_set(succ + b, n, head, rank + b, W + b, val, nxt, &s_work, seed ^ (uint32_t)k, ctl);
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
        for (int v = threadIdx.x; v < n; v += BT) {
            int x = p[v];
            while (p[x] != x) x = p[x];
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
            for (;;) {
                const int y = ld_cg(p + x);
                if (y == x) break;
                x = y;
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
        if (n <= 0 || m < 0 || n > 0x7FFFFFFELL) continue;
        int lg = 0;
        while ((int64_t(1) << lg) < n) ++lg;
        const int cap = max_rounds > 0 ? max_rounds : 64 + 4 * lg;
        if (n <= CC_SMEM_VERTS)
            graph_in_smem(src + eb, dst + eb, m, (int)n, label + vb, sm, cap, ctl);
        else
            graph_in_global(src + eb, dst + eb, m, n, label + vb, cap, ctl);
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

size_t cc_batched_ws(int64_t count) { return align_up(sizeof(int32_t) * (size_t)std::max<int64_t>(count, 1), 256); }

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
    lr_batch_kernel<<<g, BT, SMEM_BYTES, s>>>(succ, off, heads, count, order, rank, W,
                                              (uint32_t)(p.seed ^ (p.seed >> 32)), c->ctl);
    phase_end(c, s, PH_LR_BATCH);
    return cuda_status(cudaGetLastError());
}

lrcc_status cc_batched_run(Ctx* c, const int32_t* src, const int32_t* dst, const int64_t* eoff, const int64_t* voff,
                           int64_t count, int32_t* label, const Plan& p) {
    cudaStream_t s = c->stream;
    int32_t* order = static_cast<int32_t*>(c->ws);
    phase_begin(c, s);
    batch_order<<<1, 1024, 0, s>>>(voff, eoff, nullptr, count, order, c->ctl);
    phase_end(c, s, PH_BATCH_PREP);
    lrcc_status st = set_smem((const void*)cc_batch_kernel);
    if (st != LRCC_OK) return st;
    const int g = (int)std::min<int64_t>(count, persistent_grid(c, (const void*)cc_batch_kernel, BT, SMEM_BYTES));
    phase_begin(c, s);
    cc_batch_kernel<<<g, BT, SMEM_BYTES, s>>>(src, dst, eoff, voff, count, order, label, p.cc_max_rounds, c->ctl);
    phase_end(c, s, PH_CC_BATCH);
    return cuda_status(cudaGetLastError());
}

}  // namespace lrcc
