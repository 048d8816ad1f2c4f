// Connected components (Sec. 4, Algorithm 4), restated for sm_103a.
//
// The parent array is the caller's label array. Each round is
//   hook      stream the edge list in 16-byte vectors (evict-first in L2 so
//             the parent array stays resident); for an edge whose endpoints
//             have different parents, atomicMin links the larger root below
//             the smaller one (priority write in place of the paper's
//             "arbitrary" concurrent write);
//   control   a one-thread kernel reads the change flag (SV step 5, raised by
//             one warp-ballot store per warp) and sets the condition of a
//             CUDA-graph while-node, so the loop runs without the host;
//   shortcut  pointer jumping until every tree is a star (SV steps 1a / 4),
//             skipped after the final pass that joined nothing.
// Links always point from a larger id to a smaller one, so no cycle can form
// and every root is the smallest id of its tree; when a pass finds no edge
// between two trees the trees are the components and the roots their
// minimum-id labels.
//
// Hook rules (plan.cc_hook): 1 = one atomicMin per edge and pass, as in the
// Shiloach-Vishkin round structure; 2 = when the atomicMin finds that the
// larger root was linked meanwhile, keep joining (old parent, smaller root)
// until one link lands, so each pass joins every edge and the next pass only
// confirms; 3 = rule 1 in the first pass, rule 2 after it; 5 = in the first
// pass (when every vertex is still its own root) no parent is gathered: each
// edge links its endpoints with atomicMin and carries every link the atomic
// displaces on to the next pair (link_direct), so that pass joins every edge
// it reads, and rule 1 after it. All give the same labels. Rule 4, the
// paper's own round structure, is in cc_sv.cu.
//
// Before the loop, an optional sample pass (plan.cc_sample) hooks and
// shortcuts a prefix of the edge list, which forms most of a large component
// for a fraction of a pass (see cc_run).
#include <algorithm>

#include "cc_device.cuh"
#include "common.cuh"
#include "internal.h"

namespace lrcc {

namespace {

constexpr int BLOCK = 256;
constexpr int CC_STAGE = 256;   // active edges a warp stages before appending (>= 32 lanes x 4)

template <bool VEC>
__global__ void __launch_bounds__(BLOCK) cc_init(int32_t* __restrict__ parent, int64_t n) {
    const int64_t ngroups = (n + 3) >> 2;
    for (int64_t g = static_cast<int64_t>(blockIdx.x) * BLOCK + threadIdx.x; g < ngroups;
         g += static_cast<int64_t>(gridDim.x) * BLOCK) {
        const int64_t i0 = g * 4;
        if (VEC && i0 + 3 < n) {
            *reinterpret_cast<int4*>(parent + i0) =
                make_int4((int)i0, (int)i0 + 1, (int)i0 + 2, (int)i0 + 3);
        } else {
            for (int q = 0; q < 4; ++q)
                if (i0 + q < n) parent[i0 + q] = (int)(i0 + q);
        }
    }
}

// Hook pass. mode 1: single hooks every pass; mode 2: relink every pass;
// mode 3: single hooks in the first pass (cheap while every tree is a
// singleton), relink afterwards.
//
// Edges of a pass come from the input or from an active-edge buffer: from
// the first pass after a shortcut on (the sample pass counts as a round), an
// edge whose endpoints already share a parent (after the shortcut, a root)
// can never join two trees again, because trees only merge; the others are
// staged per warp in shared memory and appended in batches to the buffer the
// next pass reads. The first pass of all (every parent still the vertex
// itself) appends nothing: every edge would be kept.
struct ActiveEdges {
    int2* buf[2];      // active buffers 1 and 2 (edge = (u, v))
    int64_t cap;       // edges each buffer holds; 0 = no compaction
};

template <bool VEC>
__global__ void __launch_bounds__(BLOCK, 6)
    cc_hook(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
            int32_t* parent, int64_t n, int mode, ActiveEdges act, DevCtl* ctl) {
    const uint64_t stream_pol = policy_evict_first();
    const uint64_t keep = policy_evict_last();
    const int pass = ctl->rounds;
    const bool first = pass == 0;
    const bool relink = mode == 2 || (mode == 3 && !first);
    const bool direct = mode == 5 && first;   // rule 5's first pass: link the endpoints themselves
    const int sel = ctl->cc_src;                       // 0 = input edges, 1/2 = active buffer
    const int out_sel = sel == 1 ? 2 : 1;
    const bool compact = !first && act.cap > 0;
    const int64_t me = sel == 0 ? m : min((int64_t)ctl->cc_count[sel], act.cap);
    const int2* in = sel == 0 ? nullptr : act.buf[sel - 1];
    int2* out = act.cap > 0 ? act.buf[out_sel - 1] : nullptr;
    const int lane = threadIdx.x & 31;
    const int64_t ngroups = (me + 3) >> 2;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&ctl->edges_read, (unsigned long long)me);
    bool changed = false;
    // each warp stages its active edges in shared memory and appends them in
    // batches (one counter atomic per batch, coalesced writes), so that a pass
    // with a few active edges in every warp does not queue one atomic per warp
    // iteration on the single counter
    __shared__ int2 s_stage[BLOCK / 32][CC_STAGE];
    int2* stage = s_stage[threadIdx.x >> 5];
    int staged = 0;   // warp-uniform
    auto flush = [&]() {
        __syncwarp();
        int base = 0;
        if (lane == 0) base = atomicAdd(&ctl->cc_count[out_sel], staged);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (lane == 0 && (int64_t)base + staged > act.cap) ctl->cc_overflow = 1;
        for (int i = lane; i < staged; i += 32)
            if ((int64_t)base + i < act.cap) out[base + i] = stage[i];
        __syncwarp();
        staged = 0;
    };
    // warp-uniform trip count so that the warp-wide append can use full masks
    const int64_t warp_base = (static_cast<int64_t>(blockIdx.x) * BLOCK + (threadIdx.x & ~31));
    const int64_t stride = static_cast<int64_t>(gridDim.x) * BLOCK;
    for (int64_t gb = warp_base; gb < ngroups; gb += stride) {
        const int64_t g = gb + lane;
        const int64_t e0 = g * 4;
        int u[4], v[4];
        bool ok[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) ok[q] = e0 + q < me;
        if (sel != 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int2 e = ok[q] ? __ldcs(in + e0 + q) : make_int2(0, 0);
                u[q] = e.x;
                v[q] = e.y;
            }
        } else if (VEC && e0 + 3 < me) {
            const int4 a = ld_stream_v4(src + e0, stream_pol);
            const int4 b = ld_stream_v4(dst + e0, stream_pol);
            u[0] = a.x; u[1] = a.y; u[2] = a.z; u[3] = a.w;
            v[0] = b.x; v[1] = b.y; v[2] = b.z; v[3] = b.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                u[q] = ok[q] ? ld_stream(src + e0 + q, stream_pol) : 0;
                v[q] = ok[q] ? ld_stream(dst + e0 + q, stream_pol) : 0;
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (ok[q] && (u[q] < 0 || u[q] >= n || v[q] < 0 || v[q] >= n)) {
                record_error(ctl, LRCC_ERR_INVALID_INPUT, (int)(e0 + q));
                u[q] = v[q] = 0;
            }
        }
        if (direct) {   // first pass: nothing is kept, so no compaction either
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (ok[q]) changed |= link_direct(parent, u[q], v[q], keep);
            continue;
        }
        int32_t a[4], b[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            a[q] = ld_hint(parent + u[q], keep);
            b[q] = ld_hint(parent + v[q], keep);
        }
        int keep_cnt = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const bool active = ok[q] && a[q] != b[q];
            if (active) {
                if (!relink && !first) {
                    // after the first pass a hook seldom finds its root already linked
                    // lower (that is the hubs of the first pass), so the atomic goes
                    // without the read hook_pair makes first (2.44 -> 2.42 ms, R-MAT 24)
                    atomicMin(parent + max(a[q], b[q]), min(a[q], b[q]));
                    changed = true;
                } else {
                    changed |= hook_pair(parent, a[q], b[q], relink, keep);
                }
            }
            keep_cnt += active;
            ok[q] = active;
        }
        if (compact && __any_sync(0xffffffffu, keep_cnt)) {   // most iterations keep nothing
            int total = 0;
            const int excl = warp_prefix_small(keep_cnt, &total);
            if (staged + total > CC_STAGE) flush();
            int at = staged + excl;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (ok[q]) stage[at++] = make_int2(u[q], v[q]);
            staged += total;
        }
    }
    if (compact && staged > 0) flush();
    if (__any_sync(0xffffffffu, changed) && lane == 0) ctl->flag = 1;
}

// Ceiling of a hook pass's memory traffic: the same edge stream (16-byte
// evict-first loads) and the same two gathers per edge (through L1, evict-last
// in L2) over a table the size of the parent array, with none of the hooking.
// The gathered values are summed (one atomic per block) so that no load is
// dropped.
template <bool VEC>
__global__ void __launch_bounds__(BLOCK, 6)
    cc_gather_probe(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                    const int32_t* table, int64_t n, unsigned long long* out) {
    const uint64_t stream_pol = policy_evict_first();
    const uint64_t keep = policy_evict_last();
    const int64_t ngroups = (m + 3) >> 2;
    unsigned long long acc = 0;
    for (int64_t g = static_cast<int64_t>(blockIdx.x) * BLOCK + threadIdx.x; g < ngroups;
         g += static_cast<int64_t>(gridDim.x) * BLOCK) {
        const int64_t e0 = g * 4;
        int u[4], v[4];
        if (VEC && e0 + 3 < m) {
            const int4 a = ld_stream_v4(src + e0, stream_pol);
            const int4 b = ld_stream_v4(dst + e0, stream_pol);
            u[0] = a.x; u[1] = a.y; u[2] = a.z; u[3] = a.w;
            v[0] = b.x; v[1] = b.y; v[2] = b.z; v[3] = b.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                u[q] = e0 + q < m ? ld_stream(src + e0 + q, stream_pol) : 0;
                v[q] = e0 + q < m ? ld_stream(dst + e0 + q, stream_pol) : 0;
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (e0 + q >= m) continue;
            // ids outside [0, n) read entry 0 instead (the probe never faults)
            const int uq = (u[q] >= 0 && u[q] < n) ? u[q] : 0;
            const int vq = (v[q] >= 0 && v[q] < n) ? v[q] : 0;
            acc += (unsigned)ld_hint(table + uq, keep) + (unsigned)ld_hint(table + vq, keep);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// Pointer jumping to stars: parent[v] <- root(v). Roots do not move during
// this pass and every value read is an ancestor, so one pass suffices.
template <bool VEC>
__global__ void __launch_bounds__(BLOCK) cc_shortcut(int32_t* parent, int64_t n, const DevCtl* ctl) {
    // runs after the loop control: a pass that joined nothing left every tree a star
    if (ctl->cc_stop) return;
    const uint64_t keep = policy_evict_last();
    const int64_t ngroups = (n + 3) >> 2;
    for (int64_t g = static_cast<int64_t>(blockIdx.x) * BLOCK + threadIdx.x; g < ngroups;
         g += static_cast<int64_t>(gridDim.x) * BLOCK) {
        const int64_t i0 = g * 4;
        if (VEC && i0 + 3 < n) {
            const int4 p = *reinterpret_cast<const int4*>(parent + i0);
            // the four chases advance together, so four loads are in flight at a time;
            // their first steps read through L1 and deep chases write their progress
            // (chase_step)
            int x[4] = {p.x, p.y, p.z, p.w};
            bool live[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) live[q] = x[q] != (int)(i0 + q);
            bool any = live[0] | live[1] | live[2] | live[3];
            bool ch = false;
            for (int step = 0; any; ++step) {
                int nx[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    nx[q] = live[q] ? chase_step(parent, (int32_t)(i0 + q), x[q], step, keep) : x[q];
                any = false;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (live[q] && nx[q] != x[q]) {
                        x[q] = nx[q];
                        ch = true;
                        any = true;
                    } else {
                        live[q] = false;
                    }
                }
            }
            if (ch) *reinterpret_cast<int4*>(parent + i0) = make_int4(x[0], x[1], x[2], x[3]);
        } else {
            for (int q = 0; q < 4; ++q) {
                const int64_t v = i0 + q;
                if (v < n) {
                    const int p = parent[v];
                    if (p != v) {
                        const int r = chase_root(parent, (int32_t)v, p, keep);
                        if (r != p) parent[v] = r;
                    }
                }
            }
        }
    }
}

// After a pass: choose the next pass's edges (the active buffer this pass
// filled, unless it overflowed or this was the first pass) and clear that
// buffer's successor for appends.
__device__ __forceinline__ void next_edges(DevCtl* ctl, bool compacting) {
    const int sel = ctl->cc_src;
    const int out_sel = sel == 1 ? 2 : 1;
    int next = 0;
    if (compacting && ctl->rounds > 1 && !ctl->cc_overflow) next = out_sel;
    ctl->cc_overflow = 0;
    ctl->cc_src = next;
    ctl->cc_count[next == 1 ? 2 : 1] = 0;
}

// Loop control on the device: continue while the last hook pass joined
// something, the round cap is not reached and no error was recorded.
__global__ void cc_control(DevCtl* ctl, cudaGraphConditionalHandle h, int cap, bool compacting) {
    const int r = ++ctl->rounds;
    const int f = ctl->flag;
    ctl->flag = 0;
    unsigned cont = f != 0;
    if (cont && r >= cap) {
        record_error(ctl, LRCC_ERR_NOT_CONVERGED, r);
        cont = 0;
    }
    if (ctl->status) cont = 0;
    next_edges(ctl, compacting);
    ctl->cc_stop = !cont;
    cudaGraphSetConditional(h, cont);
}

// Same decision for the host-driven loop: the answer is left in ctl->pad[0].
__global__ void cc_control_host(DevCtl* ctl, int cap, bool compacting) {
    const int r = ++ctl->rounds;
    const int f = ctl->flag;
    ctl->flag = 0;
    int cont = f != 0;
    if (cont && r >= cap) {
        record_error(ctl, LRCC_ERR_NOT_CONVERGED, r);
        cont = 0;
    }
    if (ctl->status) cont = 0;
    next_edges(ctl, compacting);
    ctl->cc_stop = !cont;
    ctl->pad[0] = cont;
}

// After the sample pass: it counts as the first round (parents are no longer
// the vertices themselves, so the next pass, over all edges, compacts), and
// its change flag is dropped (the loop's own passes decide convergence).
__global__ void cc_sample_done(DevCtl* ctl) {
    ctl->rounds = 1;
    ctl->flag = 0;
    ctl->cc_stop = 0;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

struct CcArgs {
    const int32_t* src;
    const int32_t* dst;
    int64_t m, n;
    int32_t* label;
    int mode;
    int cap;
    ActiveEdges act;
};

// Enqueues one round's hook pass, and (separately) its shortcut pass; the
// loop control runs between them. `phase` names the pass in timing mode.
lrcc_status enqueue_hook(Ctx* c, cudaStream_t s, const CcArgs& a, int phase = PH_CC_HOOK) {
    const bool ve = aligned16(a.src) && aligned16(a.dst);
    const bool vn = aligned16(a.label);
    const void* hk = ve ? (const void*)cc_hook<true> : (const void*)cc_hook<false>;
    const int64_t eg = (a.m + 3) / 4;
    if (eg > 0) {
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>((eg + BLOCK - 1) / BLOCK,
                                                                  persistent_grid(c, hk, BLOCK)));
        phase_begin(c, s);
        if (ve) cc_hook<true><<<g, BLOCK, 0, s>>>(a.src, a.dst, a.m, a.label, a.n, a.mode, a.act, c->ctl);
        else cc_hook<false><<<g, BLOCK, 0, s>>>(a.src, a.dst, a.m, a.label, a.n, a.mode, a.act, c->ctl);
        phase_end(c, s, phase);
    }
    return cuda_status(cudaGetLastError());
}

lrcc_status enqueue_shortcut(Ctx* c, cudaStream_t s, const CcArgs& a) {
    const bool vn = aligned16(a.label);
    const void* sk = vn ? (const void*)cc_shortcut<true> : (const void*)cc_shortcut<false>;
    const int64_t ng = (a.n + 3) / 4;
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((ng + BLOCK - 1) / BLOCK,
                                                              persistent_grid(c, sk, BLOCK)));
    phase_begin(c, s);
    if (vn) cc_shortcut<true><<<g, BLOCK, 0, s>>>(a.label, a.n, c->ctl);
    else cc_shortcut<false><<<g, BLOCK, 0, s>>>(a.label, a.n, c->ctl);
    phase_end(c, s, PH_CC_SHORTCUT);
    return cuda_status(cudaGetLastError());
}

lrcc_status build_loop_graph(Ctx* c, const CcArgs& a, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return LRCC_ERR_CUDA;
    cudaGraphConditionalHandle h;
    lrcc_status st = LRCC_OK;
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
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(c->capture, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGraphDestroy(g);
        return LRCC_ERR_CUDA;
    }
    st = enqueue_hook(c, c->capture, a);
    cc_control<<<1, 1, 0, c->capture>>>(c->ctl, h, a.cap, a.act.cap > 0);
    if (st == LRCC_OK) st = enqueue_shortcut(c, c->capture, a);
    cudaGraph_t captured = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(c->capture, &captured);
    if (st == LRCC_OK && ce != cudaSuccess) st = LRCC_ERR_CUDA;
    if (st == LRCC_OK && cudaGraphInstantiate(out, g, 0) != cudaSuccess) st = LRCC_ERR_CUDA;
    cudaGraphDestroy(g);
    cudaGetLastError();
    return st;
}

}  // namespace

lrcc_status cc_gather_probe_run(Ctx* c, const int32_t* src, const int32_t* dst, int64_t m, const int32_t* table,
                                int64_t n, int64_t* out) {
    const bool ve = aligned16(src) && aligned16(dst);
    const void* k = ve ? (const void*)cc_gather_probe<true> : (const void*)cc_gather_probe<false>;
    const int64_t eg = (m + 3) / 4;
    cudaMemsetAsync(out, 0, sizeof(int64_t), c->stream);
    if (eg == 0) return cuda_status(cudaGetLastError());
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((eg + BLOCK - 1) / BLOCK, persistent_grid(c, k, BLOCK)));
    unsigned long long* o = reinterpret_cast<unsigned long long*>(out);
    if (ve) cc_gather_probe<true><<<g, BLOCK, 0, c->stream>>>(src, dst, m, table, n, o);
    else cc_gather_probe<false><<<g, BLOCK, 0, c->stream>>>(src, dst, m, table, n, o);
    return cuda_status(cudaGetLastError());
}

// Active-edge buffers: each holds an eighth of the edges (a pass that keeps
// more falls back to the full edge list); none for small graphs.
int64_t cc_active_cap(int64_t m) { return m >= (int64_t(1) << 16) ? m / 8 : 0; }
size_t cc_ws(int64_t m) {
    const int64_t cap = cc_active_cap(m);
    return cap > 0 ? 2 * align_up(sizeof(int2) * (size_t)cap, 256) : 0;
}

lrcc_status cc_run(Ctx* c, const int32_t* src, const int32_t* dst, int64_t m, int64_t n,
                   int32_t* label, const Plan& p) {
    CcArgs a{src, dst, m, n, label, p.cc_hook == 5 ? 5 : std::min(std::max(p.cc_hook, 1), 3), 0, ActiveEdges{}};
    const int64_t acap = cc_active_cap(m);
    if (acap > 0 && c->ws_bytes >= cc_ws(m)) {
        a.act.buf[0] = static_cast<int2*>(c->ws);
        a.act.buf[1] = reinterpret_cast<int2*>(static_cast<char*>(c->ws) + align_up(sizeof(int2) * (size_t)acap, 256));
        a.act.cap = acap;
    }
    int lg = 0;
    while ((int64_t(1) << lg) < n) ++lg;
    a.cap = p.cc_max_rounds > 0 ? p.cc_max_rounds : 64 + 4 * lg;
    cudaStream_t s = c->stream;
    const void* ik = aligned16(label) ? (const void*)cc_init<true> : (const void*)cc_init<false>;
    const int64_t ng = (n + 3) / 4;
    const int gi = (int)std::max<int64_t>(1, std::min<int64_t>((ng + BLOCK - 1) / BLOCK,
                                                               persistent_grid(c, ik, BLOCK)));
    phase_begin(c, s);
    if (aligned16(label)) cc_init<true><<<gi, BLOCK, 0, s>>>(label, n);
    else cc_init<false><<<gi, BLOCK, 0, s>>>(label, n);
    phase_end(c, s, PH_CC_INIT);

    // Sample pass: hook and shortcut over a prefix of the edge list first. On
    // graphs with large components this forms most of them for a fraction of a
    // pass, and the first pass over all edges then finds most edges inside one
    // tree and drops them. Which edges are hooked first does not change the
    // labels; the loop below still runs until a pass over the remaining edges
    // joins nothing.
    int samp = p.cc_sample;
    if (samp < 0) {
        // automatic (measured on R-MAT and uniform random graphs on a GB300): a
        // sample of about one edge per vertex from 8 edges per vertex up, two
        // from 4 up, none below (sparse graphs have no large component to form)
        const int64_t per_vertex = n > 0 ? m / n : 0;
        samp = per_vertex >= 8 ? (int)std::min<int64_t>(per_vertex, 1024) : per_vertex >= 4 ? (int)(per_vertex / 2) : 1;
    }
    const int64_t ms = samp > 1 ? m / samp : 0;
    if (ms >= 4096 && a.act.cap > 0) {
        CcArgs sa = a;
        sa.m = ms;
        sa.act = ActiveEdges{};
        lrcc_status st = enqueue_hook(c, s, sa);
        if (st != LRCC_OK) return st;
        cc_sample_done<<<1, 1, 0, s>>>(c->ctl);
        st = enqueue_shortcut(c, s, sa);
        if (st != LRCC_OK) return st;
    }

    if (p.use_graphs != 2) {
        const std::vector<uint64_t> key = {(uint64_t)KIND_CC, (uint64_t)src, (uint64_t)dst, (uint64_t)m,
                                           (uint64_t)n, (uint64_t)label, (uint64_t)a.mode, (uint64_t)a.cap,
                                           (uint64_t)a.act.buf[0], (uint64_t)a.act.cap};
        GraphEntry* e = nullptr;
        for (auto& ge : c->graphs)
            if (ge.key == key) e = &ge;
        if (!e) {
            cudaGraphExec_t ex = nullptr;
            const lrcc_status st = build_loop_graph(c, a, &ex);
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
        const lrcc_status st = cuda_status(cudaGraphLaunch(e->exec, s));
        phase_end(c, s, PH_CC_LOOP);
        return st;
    }
    // host-driven loop: one flag read per round
    int* host_flag = nullptr;
    if (cudaMallocHost(&host_flag, sizeof(int)) != cudaSuccess) return LRCC_ERR_NOMEM;
    lrcc_status st = LRCC_OK;
    for (int r = 0; r < a.cap + 1; ++r) {
        // the first pass of the loop reads every edge (later ones the active edges)
        st = enqueue_hook(c, s, a, r == 0 ? PH_CC_HOOK_FULL : PH_CC_HOOK);
        if (st != LRCC_OK) break;
        cc_control_host<<<1, 1, 0, s>>>(c->ctl, a.cap, a.act.cap > 0);
        st = enqueue_shortcut(c, s, a);
        if (st != LRCC_OK) break;
        cudaMemcpyAsync(host_flag, &c->ctl->pad[0], sizeof(int), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            st = LRCC_ERR_CUDA;
            break;
        }
        if (!*host_flag) break;
    }
    cudaFreeHost(host_flag);
    return st;
}

}  // namespace lrcc
