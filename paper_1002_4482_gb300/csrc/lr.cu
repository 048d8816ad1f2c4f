// List ranking kernels: Wyllie pointer jumping (Sec. 3.1, Algorithm 1) and the
// sparse ruling set / random splitter method (Sec. 3.2, Algorithms 2 and 3).
//
// Ruling set, as built here for sm_103a:
//   select   (RS1+RS2) one streaming pass packs succ into 8-byte words
//            W[i] = (next | splitter flag, splitter index or weight 1) and
//            compacts the randomly chosen splitters (the head is always
//            splitter 0);
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

#include "common.cuh"
#include "internal.h"

namespace lrcc {

namespace {

constexpr int BLOCK = 256;
constexpr int FINAL_THREADS = 1024;

// ------------------------------------------------------- shared-memory Wyllie

// Wyllie's pointer jumping on val/nxt arrays held in shared memory by one
// block of FINAL_THREADS threads (Sec. 3.1: the single-kernel variant using
// __syncthreads). On return val[j] = sum of val over j and every element
// after it. Rounds are capped at ceil(log2 r) + 2; a list that still has
// links then must contain a cycle, which is recorded as invalid input.
template <int PER>
__device__ void cta_wyllie(int* val, int* nxt, int r, DevCtl* ctl) {
    const int tid = threadIdx.x;
    int cap = 2;
    while ((1 << (cap - 2)) < r) ++cap;
    for (int round = 0;; ++round) {
        int nv[PER], nn[PER];
        bool any = false;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int j = tid + q * FINAL_THREADS;
            nv[q] = 0;
            nn[q] = (int)NIL;
            if (j < r) {
                const int x = nxt[j];
                nv[q] = val[j];
                if (x != (int)NIL) {
                    nv[q] += val[x];
                    nn[q] = nxt[x];
                    any = true;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int j = tid + q * FINAL_THREADS;
            if (j < r) {
                val[j] = nv[q];
                nxt[j] = nn[q];
            }
        }
        if (!__syncthreads_or(any)) break;
        if (round >= cap) {
            if (tid == 0) record_error(ctl, LRCC_ERR_INVALID_INPUT, -2);
            break;
        }
    }
}

// One block ranks a whole list of n <= PER * FINAL_THREADS elements.
template <int PER>
__global__ void __launch_bounds__(FINAL_THREADS, 1)
    lr_small_kernel(const int32_t* __restrict__ succ, int n, int head, int32_t* __restrict__ rank,
                    DevCtl* ctl) {
    extern __shared__ int sm[];
    int* val = sm;
    int* nxt = sm + PER * FINAL_THREADS;
    for (int i = threadIdx.x; i < n; i += FINAL_THREADS) {
        const int s = succ[i];
        const bool tail = (s == -1) | (s == i);
        const bool bad = !tail && (s < 0 || s >= n);
        if (bad) record_error(ctl, LRCC_ERR_INVALID_INPUT, i);
        nxt[i] = (tail || bad) ? (int)NIL : s;
        val[i] = 1;
    }
    __syncthreads();
    cta_wyllie<PER>(val, nxt, n, ctl);
    for (int i = threadIdx.x; i < n; i += FINAL_THREADS) rank[i] = val[i] - 1;
    if (threadIdx.x == 0 && val[head] != n) record_error(ctl, LRCC_ERR_INVALID_INPUT, head);
}

// Last ruling-set level: one block ranks the weighted list of splitters held
// in packed words R[j] = (next index or NIL, weight) and writes the inclusive
// suffix weights S. The head splitter (index 0) must see the whole list.
template <int PER>
__global__ void __launch_bounds__(FINAL_THREADS, 1)
    rs_final_kernel(const uint64_t* __restrict__ R, const int* cnt, int cap, int32_t* __restrict__ S,
                    int64_t expect, DevCtl* ctl) {
    extern __shared__ int sm[];
    int* val = sm;
    int* nxt = sm + PER * FINAL_THREADS;
    const int r = min(1 + *cnt, cap);
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

// Level-0 select: pack succ into walk words and compact the splitters.
// Warps stride over groups of 4 elements (Sec. 2.5 striding), so loads and
// stores are 16-byte and coalesced.
template <bool VEC>
__global__ void __launch_bounds__(BLOCK)
    rs_select0(const int32_t* __restrict__ succ, int64_t n, int32_t head, uint64_t* __restrict__ W,
               int32_t* __restrict__ snext, int32_t* __restrict__ sw, int cap, uint32_t thr,
               uint32_t seed, DevCtl* ctl) {
    const uint64_t pol = policy_evict_first();
    const int lane = threadIdx.x & 31;
    const int64_t ngroups = (n + 3) >> 2;
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * BLOCK + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * BLOCK) >> 5;
    for (int64_t gb = warp * 32; gb < ngroups; gb += nwarps * 32) {
        const int64_t i0 = (gb + lane) * 4;
        int s[4];
        if (VEC && i0 + 3 < n) {
            const int4 v = ld_stream_v4(succ + i0, pol);
            s[0] = v.x; s[1] = v.y; s[2] = v.z; s[3] = v.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) s[q] = (i0 + q < n) ? ld_stream(succ + i0 + q, pol) : -1;
        }
        uint32_t nx[4];
        bool sp[4];
        int cnt = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t i = i0 + q;
            const bool valid = i < n;
            const int v = s[q];
            const bool tail = (v == -1) | (v == i);
            const bool bad = !tail && (v < 0 || v >= n);
            if (valid && bad) record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)i);
            nx[q] = (tail || bad) ? NIL : (uint32_t)v;
            sp[q] = valid && i != head && pick((uint32_t)i, seed, thr);
            cnt += sp[q];
        }
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        int base = 0;
        if (lane == 31 && total) base = atomicAdd(&ctl->spl_count[0], total);
        base = __shfl_sync(0xffffffffu, base, 31);
        int j = 1 + base + incl - cnt;
        uint64_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t i = i0 + q;
            if (i == head) {
                w[q] = pack(nx[q] | SPL, 0);
                snext[0] = (int32_t)nx[q];
                sw[0] = 1;
            } else if (sp[q]) {
                if (j < cap) {
                    w[q] = pack(nx[q] | SPL, (uint32_t)j);
                    snext[j] = (int32_t)nx[q];
                    sw[j] = 1;
                } else {
                    w[q] = pack(nx[q], 1);
                }
                ++j;
            } else {
                w[q] = pack(nx[q], 1);
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

// Select at level >= 1: the elements are the previous level's splitters,
// whose packed words R[j] = (next, weight) are already walk words. Only the
// chosen splitters are read and rewritten as (next | SPL, new index).
__global__ void __launch_bounds__(BLOCK)
    rs_select(uint64_t* __restrict__ R, const int* cnt_in, int cap_in, int32_t* __restrict__ snext,
              int32_t* __restrict__ sw, int cap, uint32_t thr, uint32_t seed, int* cnt_out) {
    const int r = min(1 + *cnt_in, cap_in);
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * BLOCK + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * BLOCK) >> 5;
    for (int jb = warp * 32; jb < r; jb += nwarps * 32) {
        const int j = jb + lane;
        const bool sp = j < r && j != 0 && pick((uint32_t)j, seed, thr);
        const unsigned m = __ballot_sync(0xffffffffu, sp);
        int base = 0;
        if (lane == 0 && m) base = atomicAdd(cnt_out, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        const int jj = 1 + base + __popc(m & lanemask_lt());
        if (j == 0) {
            const uint64_t w = R[0];
            R[0] = pack(lo32(w) | SPL, 0);
            snext[0] = (int32_t)lo32(w);
            sw[0] = (int32_t)hi32(w);
        } else if (sp && jj < cap) {
            const uint64_t w = R[j];
            R[j] = pack(lo32(w) | SPL, (uint32_t)jj);
            snext[jj] = (int32_t)lo32(w);
            sw[jj] = (int32_t)hi32(w);
        }
    }
}

// Sublist walk (RS3). Each thread keeps K walks in flight so that K
// independent gathers are outstanding; a warp claims splitters in chunks of
// 64 with one atomic and hands them to lanes as their walks end, which
// balances the geometric spread of sublist lengths.
template <int K>
__global__ void __launch_bounds__(BLOCK)
    rs_walk(uint64_t* __restrict__ W, const int32_t* __restrict__ snext, const int32_t* __restrict__ sw,
            uint64_t* __restrict__ Rout, const int* cnt, int cap, int* work, int64_t nlevel,
            DevCtl* ctl) {
    constexpr int CHUNK = 64;
    const int r = min(1 + *cnt, cap);
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

// Expand at level >= 1: S[c] = S_next[owner] - prefix (RS5).
__global__ void __launch_bounds__(BLOCK)
    rs_expand(const uint64_t* __restrict__ W, const int* cnt, int cap, const int32_t* __restrict__ Snext,
              int32_t* __restrict__ S, DevCtl* ctl) {
    const int r = min(1 + *cnt, cap);
    for (int c = blockIdx.x * BLOCK + threadIdx.x; c < r; c += gridDim.x * BLOCK) {
        const uint64_t w = W[c];
        const uint32_t lo = lo32(w), hi = hi32(w);
        if (lo & SPL) {
            S[c] = Snext[hi];
        } else if (hi & VIS) {
            S[c] = Snext[hi & ~VIS] - (int32_t)lo;
        } else {
            record_error(ctl, LRCC_ERR_INVALID_INPUT, c);
            S[c] = 0;
        }
    }
}

// Expand at level 0 into the caller's rank array: rank = S1[owner] - prefix - 1.
template <bool VEC>
__global__ void __launch_bounds__(BLOCK)
    rs_expand0(const uint64_t* __restrict__ W, int64_t n, const int32_t* __restrict__ S1,
               int32_t* __restrict__ rank, DevCtl* ctl) {
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
            if (lo & SPL) {
                out[q] = S1[hi] - 1;
            } else if (hi & VIS) {
                out[q] = S1[hi & ~VIS] - (int32_t)lo - 1;
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

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

int small_per(int n) { return n <= 4096 ? 4 : (n <= 8192 ? 8 : 16); }

lrcc_status launch_small(Ctx* c, cudaStream_t s, const int32_t* succ, int n, int head, int32_t* rank) {
    const int per = small_per(n);
    const size_t smem = 2 * sizeof(int) * per * FINAL_THREADS;
    const void* k = per == 4 ? (const void*)lr_small_kernel<4>
                  : per == 8 ? (const void*)lr_small_kernel<8> : (const void*)lr_small_kernel<16>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    phase_begin(c, s);
    if (per == 4) lr_small_kernel<4><<<1, FINAL_THREADS, smem, s>>>(succ, n, head, rank, c->ctl);
    else if (per == 8) lr_small_kernel<8><<<1, FINAL_THREADS, smem, s>>>(succ, n, head, rank, c->ctl);
    else lr_small_kernel<16><<<1, FINAL_THREADS, smem, s>>>(succ, n, head, rank, c->ctl);
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

RsLayout rs_layout(int64_t n, const Plan& p) {
    RsLayout L;
    L.size[0] = n;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    L.off_W0 = take(sizeof(uint64_t) * (size_t)n);
    int64_t cur = n;
    int lvl = 0;
    while (cur > p.rs_small && lvl < MAX_LEVELS) {
        int64_t spacing = lvl == 0 ? p.rs_spacing0 : p.rs_spacing;
        spacing = std::max<int64_t>(2, spacing);
        const double expect = std::ceil((double)cur / (double)spacing);
        int64_t cap = (int64_t)(expect + 4.0 * std::sqrt(expect) + 32.0);
        cap = std::min<int64_t>(cap, cur);
        if (lvl == MAX_LEVELS - 1) cap = std::min<int64_t>(cap, p.rs_small);
        L.thr[lvl] = (uint32_t)std::min<double>(4294967295.0, 4294967296.0 / (double)spacing);
        ++lvl;
        L.size[lvl] = cap;
        L.off_R[lvl] = take(sizeof(uint64_t) * (size_t)cap);
        L.off_snext[lvl] = take(sizeof(int32_t) * (size_t)cap);
        L.off_sw[lvl] = take(sizeof(int32_t) * (size_t)cap);
        L.off_S[lvl] = take(sizeof(int32_t) * (size_t)cap);
        cur = cap;
    }
    L.levels = lvl;
    L.bytes = off;
    return L;
}

size_t lr_wyllie_ws(int64_t n, const Plan&) { return 2 * align_up(sizeof(uint64_t) * (size_t)n, 256); }

// ------------------------------------------------------------ enqueueing

lrcc_status lr_enqueue_rs(Ctx* c, cudaStream_t s, const int32_t* succ, int64_t n, int32_t head,
                          int32_t* rank, const Plan& p, const RsLayout& L) {
    if (n <= p.rs_small || L.levels == 0) return launch_small(c, s, succ, (int)n, head, rank);
    char* base = static_cast<char*>(c->ws);
    auto R = [&](int l) { return reinterpret_cast<uint64_t*>(base + L.off_R[l]); };
    auto SN = [&](int l) { return reinterpret_cast<int32_t*>(base + L.off_snext[l]); };
    auto SW = [&](int l) { return reinterpret_cast<int32_t*>(base + L.off_sw[l]); };
    auto S = [&](int l) { return reinterpret_cast<int32_t*>(base + L.off_S[l]); };
    uint64_t* W0 = reinterpret_cast<uint64_t*>(base + L.off_W0);
    DevCtl* ctl = c->ctl;
    const uint32_t seed0 = (uint32_t)(p.seed ^ (p.seed >> 32));

    // level 0
    const bool vec = aligned16(succ);
    const int64_t groups = (n + 3) / 4;
    {
        const void* k = vec ? (const void*)rs_select0<true> : (const void*)rs_select0<false>;
        const int g = stream_grid(c, groups, k);
        phase_begin(c, s);
        if (vec)
            rs_select0<true><<<g, BLOCK, 0, s>>>(succ, n, head, W0, SN(1), SW(1), (int)L.size[1], L.thr[0],
                                                 seed0, ctl);
        else
            rs_select0<false><<<g, BLOCK, 0, s>>>(succ, n, head, W0, SN(1), SW(1), (int)L.size[1], L.thr[0],
                                                  seed0, ctl);
        phase_end(c, s, PH_SELECT0);
    }
    auto walk = [&](int l, uint64_t* Wl, int64_t nl) {
        const int* cnt = &ctl->spl_count[l];
        const int cap = (int)L.size[l + 1];
        int* work = &ctl->work[l];
        phase_begin(c, s);
        if (p.rs_chains >= 4) {
            const int g = persistent_grid(c, (const void*)rs_walk<4>, BLOCK);
            rs_walk<4><<<g, BLOCK, 0, s>>>(Wl, SN(l + 1), SW(l + 1), R(l + 1), cnt, cap, work, nl, ctl);
        } else if (p.rs_chains == 2) {
            const int g = persistent_grid(c, (const void*)rs_walk<2>, BLOCK);
            rs_walk<2><<<g, BLOCK, 0, s>>>(Wl, SN(l + 1), SW(l + 1), R(l + 1), cnt, cap, work, nl, ctl);
        } else {
            const int g = persistent_grid(c, (const void*)rs_walk<1>, BLOCK);
            rs_walk<1><<<g, BLOCK, 0, s>>>(Wl, SN(l + 1), SW(l + 1), R(l + 1), cnt, cap, work, nl, ctl);
        }
        phase_end(c, s, l == 0 ? PH_WALK0 : PH_WALK);
    };
    walk(0, W0, n);
    for (int l = 1; l < L.levels; ++l) {
        const uint32_t seed = mix32(seed0 + 0x9E3779B9u * (uint32_t)l);
        const int g = stream_grid(c, (L.size[l] + 3) / 4, (const void*)rs_select);
        phase_begin(c, s);
        rs_select<<<g, BLOCK, 0, s>>>(R(l), &ctl->spl_count[l - 1], (int)L.size[l], SN(l + 1), SW(l + 1),
                                      (int)L.size[l + 1], L.thr[l], seed, &ctl->spl_count[l]);
        phase_end(c, s, PH_SELECT);
        walk(l, R(l), L.size[l]);
    }
    {
        const int lf = L.levels;
        const int per = small_per((int)L.size[lf]);
        const size_t smem = 2 * sizeof(int) * per * FINAL_THREADS;
        const int* cnt = &ctl->spl_count[lf - 1];
        const int cap = (int)L.size[lf];
        phase_begin(c, s);
        if (per == 4) {
            cudaFuncSetAttribute((const void*)rs_final_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            rs_final_kernel<4><<<1, FINAL_THREADS, smem, s>>>(R(lf), cnt, cap, S(lf), n, ctl);
        } else if (per == 8) {
            cudaFuncSetAttribute((const void*)rs_final_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            rs_final_kernel<8><<<1, FINAL_THREADS, smem, s>>>(R(lf), cnt, cap, S(lf), n, ctl);
        } else {
            cudaFuncSetAttribute((const void*)rs_final_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            rs_final_kernel<16><<<1, FINAL_THREADS, smem, s>>>(R(lf), cnt, cap, S(lf), n, ctl);
        }
        phase_end(c, s, PH_FINAL);
    }
    for (int l = L.levels - 1; l >= 1; --l) {
        const int g = stream_grid(c, L.size[l], (const void*)rs_expand);
        phase_begin(c, s);
        rs_expand<<<g, BLOCK, 0, s>>>(R(l), &ctl->spl_count[l - 1], (int)L.size[l], S(l + 1), S(l), ctl);
        phase_end(c, s, PH_EXPAND);
    }
    {
        const bool v = vec && aligned16(rank);
        const void* k = v ? (const void*)rs_expand0<true> : (const void*)rs_expand0<false>;
        const int g = stream_grid(c, groups, k);
        phase_begin(c, s);
        if (v) rs_expand0<true><<<g, BLOCK, 0, s>>>(W0, n, S(1), rank, ctl);
        else rs_expand0<false><<<g, BLOCK, 0, s>>>(W0, n, S(1), rank, ctl);
        phase_end(c, s, PH_EXPAND0);
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
