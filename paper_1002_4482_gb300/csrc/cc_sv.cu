// Connected components by the Shiloach-Vishkin round structure itself
// (Sec. 4, Algorithm 4, Table 4): plan.cc_hook = 4.
//
// Per round s (step names as in the paper's kernels SV0-SV5):
//   SV1a  shortcut: D(i) = D(D(i))
//   SV1b  mark the trees that are not stars: Q(D(D(i))) = s when D(i) != D(D(i))
//         (every tree of depth >= 2 has a vertex of depth 2, whose grandparent is
//         the root, so the root of every such tree is marked)
//   SV2   conditional hooking, for both orientations (i, j) of every edge: when
//         D(i) is a root and D(j) < D(i), D(D(i)) = D(j) and Q(D(j)) = s
//   SV3   unconditional hooking of stagnant stars: when D(i) is a root not marked
//         in this round and D(i) != D(j), D(D(i)) = D(j)
//   SV4   shortcut again
//   SV5   continue while some Q(i) = s (a warp ballot per warp, one write of the
//         round flag per warp that saw a mark: the parallel OR through a
//         concurrent write)
// The PRAM "arbitrary" concurrent writes of SV2/SV3 are plain stores here: any
// of the racing writes may win, as in that model. Two adjacent trees cannot both
// be stagnant stars in SV3 (the one with the larger root would have hooked in
// SV2), so unconditional hooks close no cycle; SV2 links always point to smaller
// ids. When a round marks nothing, every tree is a star and no edge joins two
// trees. The roots are then not always the smallest ids of their trees (SV3
// links may point up), so a final pass takes each star's minimum vertex id as
// its label, which makes the labels the same as every other hook rule's.
#include <algorithm>
#include <climits>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace lrcc {

namespace {

constexpr int SVB = 256;

__global__ void __launch_bounds__(SVB) sv_init(int32_t* __restrict__ D, int32_t* __restrict__ Q, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * SVB + threadIdx.x; i < n; i += (int64_t)gridDim.x * SVB) {
        D[i] = (int32_t)i;
        Q[i] = 0;
    }
}

// SV1a / SV4: one pointer-jumping step. A value read while another thread
// rewrites it is still an ancestor, so the step only ever shortens paths.
__global__ void __launch_bounds__(SVB) sv_jump(int32_t* D, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * SVB + threadIdx.x; i < n; i += (int64_t)gridDim.x * SVB) {
        const int32_t p = D[i];
        const int32_t g = D[p];
        if (g != p) D[i] = g;
    }
}

// SV1b: D is not written here, so every vertex sees the state SV1a left.
__global__ void __launch_bounds__(SVB) sv_mark(const int32_t* __restrict__ D, int32_t* Q, int64_t n,
                                                const DevCtl* ctl) {
    const int32_t s = ctl->rounds + 1;
    for (int64_t i = (int64_t)blockIdx.x * SVB + threadIdx.x; i < n; i += (int64_t)gridDim.x * SVB) {
        const int32_t p = D[i];
        const int32_t g = D[p];
        if (p != g) Q[g] = s;
    }
}

__device__ __forceinline__ bool edge_ok(int32_t u, int32_t v, int64_t n) {
    return u >= 0 && u < n && v >= 0 && v < n;
}

// SV2 for one orientation (i, j).
__device__ __forceinline__ void sv_cond(int32_t* D, int32_t* Q, int32_t i, int32_t j, int32_t s) {
    const int32_t di = D[i], dj = D[j];
    if (dj < di && D[di] == di) {
        D[di] = dj;
        Q[dj] = s;
    }
}

// SV3 for one orientation (i, j).
__device__ __forceinline__ void sv_uncond(int32_t* D, const int32_t* Q, int32_t i, int32_t j, int32_t s) {
    const int32_t di = D[i];
    if (D[di] == di && Q[di] < s) {
        const int32_t dj = D[j];
        if (dj != di) D[di] = dj;
    }
}

template <bool UNCOND>
__global__ void __launch_bounds__(SVB)
    sv_hook(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m, int32_t* D, int32_t* Q,
            int64_t n, DevCtl* ctl) {
    const int32_t s = ctl->rounds + 1;
    const uint64_t stream_pol = policy_evict_first();
    for (int64_t e = (int64_t)blockIdx.x * SVB + threadIdx.x; e < m; e += (int64_t)gridDim.x * SVB) {
        const int32_t u = ld_stream(src + e, stream_pol), v = ld_stream(dst + e, stream_pol);
        if (!edge_ok(u, v, n)) {
            if (!UNCOND) record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)e);
            continue;
        }
        if (UNCOND) {
            sv_uncond(D, Q, u, v, s);
            sv_uncond(D, Q, v, u, s);
        } else {
            sv_cond(D, Q, u, v, s);
            sv_cond(D, Q, v, u, s);
        }
    }
}

// SV5 and the loop decision in one: OR of (Q(i) = s) by warp ballots, then the
// last block to finish decides whether another round runs.
__global__ void __launch_bounds__(SVB) sv_check(const int32_t* __restrict__ Q, int64_t n, DevCtl* ctl) {
    const int32_t s = ctl->rounds + 1;
    bool any = false;
    for (int64_t i = (int64_t)blockIdx.x * SVB + threadIdx.x; i < n; i += (int64_t)gridDim.x * SVB)
        any |= Q[i] == s;
    if (__any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) ctl->flag = 1;
}

__global__ void sv_control(DevCtl* ctl, cudaGraphConditionalHandle h, int cap) {
    const int r = ++ctl->rounds;
    unsigned cont = ctl->flag != 0;
    ctl->flag = 0;
    if (cont && r >= cap) {
        record_error(ctl, LRCC_ERR_NOT_CONVERGED, r);
        cont = 0;
    }
    if (ctl->status) cont = 0;
    cudaGraphSetConditional(h, cont);
}

__global__ void sv_control_host(DevCtl* ctl, int cap) {
    const int r = ++ctl->rounds;
    int cont = ctl->flag != 0;
    ctl->flag = 0;
    if (cont && r >= cap) {
        record_error(ctl, LRCC_ERR_NOT_CONVERGED, r);
        cont = 0;
    }
    if (ctl->status) cont = 0;
    ctl->pad[0] = cont;
}

// Canonical labels: every tree is a star now; each star's label is its
// minimum vertex id (Q is free for the minima).
__global__ void __launch_bounds__(SVB) sv_min_init(int32_t* Q, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * SVB + threadIdx.x; i < n; i += (int64_t)gridDim.x * SVB) Q[i] = INT_MAX;
}
__global__ void __launch_bounds__(SVB) sv_min(const int32_t* __restrict__ D, int32_t* Q, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * SVB + threadIdx.x; i < n; i += (int64_t)gridDim.x * SVB)
        atomicMin(Q + D[i], (int32_t)i);
}
__global__ void __launch_bounds__(SVB) sv_relabel(int32_t* D, const int32_t* __restrict__ Q, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * SVB + threadIdx.x; i < n; i += (int64_t)gridDim.x * SVB)
        D[i] = Q[D[i]];
}

struct SvArgs {
    const int32_t* src;
    const int32_t* dst;
    int64_t m, n;
    int32_t* D;
    int32_t* Q;
    int gv, ge;   // grids of the vertex and edge kernels
};

void enqueue_round_body(Ctx* c, cudaStream_t s, const SvArgs& a) {
    phase_begin(c, s);
    sv_jump<<<a.gv, SVB, 0, s>>>(a.D, a.n);
    sv_mark<<<a.gv, SVB, 0, s>>>(a.D, a.Q, a.n, c->ctl);
    phase_end(c, s, PH_CC_SHORTCUT);
    phase_begin(c, s);
    if (a.m > 0) {
        sv_hook<false><<<a.ge, SVB, 0, s>>>(a.src, a.dst, a.m, a.D, a.Q, a.n, c->ctl);
        sv_hook<true><<<a.ge, SVB, 0, s>>>(a.src, a.dst, a.m, a.D, a.Q, a.n, c->ctl);
    }
    phase_end(c, s, PH_CC_HOOK);
    phase_begin(c, s);
    sv_jump<<<a.gv, SVB, 0, s>>>(a.D, a.n);
    sv_check<<<a.gv, SVB, 0, s>>>(a.Q, a.n, c->ctl);
    phase_end(c, s, PH_CC_SHORTCUT);
}

lrcc_status build_sv_graph(Ctx* c, const SvArgs& a, int cap, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return LRCC_ERR_CUDA;
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
        cudaGraphDestroy(g);
        return LRCC_ERR_CUDA;
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) != cudaSuccess) {
        cudaGraphDestroy(g);
        return LRCC_ERR_CUDA;
    }
    if (cudaStreamBeginCaptureToGraph(c->capture, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGraphDestroy(g);
        return LRCC_ERR_CUDA;
    }
    enqueue_round_body(c, c->capture, a);
    sv_control<<<1, 1, 0, c->capture>>>(c->ctl, h, cap);
    cudaGraph_t captured = nullptr;
    lrcc_status st = cudaStreamEndCapture(c->capture, &captured) == cudaSuccess ? LRCC_OK : LRCC_ERR_CUDA;
    if (st == LRCC_OK && cudaGraphInstantiate(out, g, 0) != cudaSuccess) st = LRCC_ERR_CUDA;
    cudaGraphDestroy(g);
    cudaGetLastError();
    return st;
}

}  // namespace

// Round bound of the method, floor(log_{3/2} n) + 2 (Sec. 4); the loop's cap
// leaves room above it.
int sv_round_bound(int64_t n) {
    return n > 1 ? (int)std::floor(std::log((double)n) / std::log(1.5)) + 2 : 2;
}

size_t cc_sv_ws(int64_t n) { return align_up(sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1), 256); }

lrcc_status cc_run_sv(Ctx* c, const int32_t* src, const int32_t* dst, int64_t m, int64_t n, int32_t* label,
                      const Plan& p) {
    if (c->ws_bytes < cc_sv_ws(n)) return LRCC_ERR_NOMEM;
    SvArgs a{src, dst, m, n, label, static_cast<int32_t*>(c->ws), 1, 1};
    const int gmax = persistent_grid(c, (const void*)sv_hook<false>, SVB);
    a.gv = (int)std::max<int64_t>(1, std::min<int64_t>((n + SVB - 1) / SVB, gmax));
    a.ge = (int)std::max<int64_t>(1, std::min<int64_t>((m + SVB - 1) / SVB, gmax));
    const int cap = p.cc_max_rounds > 0 ? p.cc_max_rounds : 2 * sv_round_bound(n) + 8;
    cudaStream_t s = c->stream;
    phase_begin(c, s);
    sv_init<<<a.gv, SVB, 0, s>>>(a.D, a.Q, n);
    phase_end(c, s, PH_CC_INIT);
    lrcc_status st = LRCC_OK;
    if (p.use_graphs != 2) {
        const std::vector<uint64_t> key = {(uint64_t)KIND_CC, 4, (uint64_t)src, (uint64_t)dst, (uint64_t)m,
                                           (uint64_t)n, (uint64_t)label, (uint64_t)a.Q, (uint64_t)cap};
        GraphEntry* e = nullptr;
        for (auto& ge : c->graphs)
            if (ge.key == key) e = &ge;
        if (!e) {
            cudaGraphExec_t ex = nullptr;
            st = build_sv_graph(c, a, cap, &ex);
            if (st != LRCC_OK) return st;
            if (c->graphs.size() >= 16) {
                auto it = std::min_element(c->graphs.begin(), c->graphs.end(),
                                           [](const GraphEntry& x, const GraphEntry& y) {
                                               return x.last_use < y.last_use;
                                           });
                cudaGraphExecDestroy(it->exec);
                c->graphs.erase(it);
            }
            c->graphs.push_back(GraphEntry{key, ex, 0});
            e = &c->graphs.back();
        }
        e->last_use = ++c->tick;
        phase_begin(c, s);
        st = cuda_status(cudaGraphLaunch(e->exec, s));
        phase_end(c, s, PH_CC_LOOP);
        if (st != LRCC_OK) return st;
    } else {
        int* host_flag = nullptr;
        if (cudaMallocHost(&host_flag, sizeof(int)) != cudaSuccess) return LRCC_ERR_NOMEM;
        for (int r = 0; r <= cap; ++r) {
            enqueue_round_body(c, s, a);
            sv_control_host<<<1, 1, 0, s>>>(c->ctl, cap);
            cudaMemcpyAsync(host_flag, &c->ctl->pad[0], sizeof(int), cudaMemcpyDeviceToHost, s);
            if (cudaStreamSynchronize(s) != cudaSuccess) {
                st = LRCC_ERR_CUDA;
                break;
            }
            if (!*host_flag) break;
        }
        cudaFreeHost(host_flag);
        if (st != LRCC_OK) return st;
    }
    phase_begin(c, s);
    sv_min_init<<<a.gv, SVB, 0, s>>>(a.Q, n);
    sv_min<<<a.gv, SVB, 0, s>>>(a.D, a.Q, n);
    sv_relabel<<<a.gv, SVB, 0, s>>>(a.D, a.Q, n);
    phase_end(c, s, PH_CC_SHORTCUT);
    return cuda_status(cudaGetLastError());
}

}  // namespace lrcc
