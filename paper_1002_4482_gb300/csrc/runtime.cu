// Runtime of liblrcc.so: per-stream workspaces, the plan table, graph
// capture/caching and the extern "C" entry points declared in lrcc.h.
#include <algorithm>
#include <atomic>
#include <cstddef>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <utility>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "internal.h"

namespace lrcc {

namespace {

// A named range around each entry point for tracing tools (NVTX; a no-op
// unless a tool is attached).
struct ApiRange {
    explicit ApiRange(const char* name) { nvtxRangePushA(name); }
    ~ApiRange() { nvtxRangePop(); }
};

// Allocation failures injected on the host (lrcc_debug_fail_allocs): the next
// g_fail_allocs device allocations of the library fail as if cudaMalloc had.
std::atomic<int> g_fail_allocs{0};
bool inject_alloc_failure() {
    int k = g_fail_allocs.load();
    while (k > 0)
        if (g_fail_allocs.compare_exchange_weak(k, k - 1)) return true;
    return false;
}

std::mutex g_mu;
std::atomic<int> g_timing{0};
const char* const kPhaseNames[PH_COUNT] = {
    "rs_select0", "rs_walk0", "rs_select", "rs_walk", "rs_final", "rs_expand", "rs_expand0", "lr_small",
    "wy_pack", "wy_jump", "wy_final", "cc_init", "cc_loop", "cc_hook", "cc_shortcut",
    "lr_batch", "cc_batch", "batch_prep", "rs_scan", "rs_scatter", "cc_hook_full"};
std::map<std::pair<int, cudaStream_t>, Ctx*> g_ctx;
// per device: the streams that carry the host-buffer calls' uploads and downloads
std::map<int, std::pair<cudaStream_t, cudaStream_t>> g_copy;
std::mutex g_plan_mu;
bool g_plan_init = false;
Plan g_plan[PLAN_KINDS][33];

int log2_ceil(int64_t n) {
    int l = 0;
    while (l < 32 && (int64_t(1) << l) < n) ++l;
    return l;
}

// Built-in plans: the choices of an autotune run on a GB300
// (python -m paper_1002_4482_gb300.autotune), per size class of ceil(log2 n),
// with the first level of 2^23..2^28 from a sweep of every size in that range.
void init_plans_locked() {
    if (g_plan_init) return;
    for (int k = 0; k < PLAN_KINDS; ++k)
        for (int l = 0; l <= 32; ++l) {
            Plan& p = g_plan[k][l];
            p = Plan{};
            p.rs_small = 16384;
            if (l <= 22) {
                // deeper levels at spacing 4: their walks are latency-bound, and
                // shorter sublists beat fewer levels up to 2^22 (with L2 flushed
                // before each call: 2^18 0.116 ms against 0.145 at spacing 16, 2^20
                // 0.153 against 0.177 at spacing 8)
                p.rs_level0 = 1, p.rs_spacing0 = 8, p.rs_spacing = 4;
            } else if (l <= 24) {
                p.rs_level0 = 1, p.rs_spacing0 = 16, p.rs_spacing = 8;
            } else if (l <= 27) {
                // the read-only first level pays off once the list outgrows L2
                // (8-byte walk words of 2^25 elements are 256 MB)
                p.rs_level0 = 2, p.rs_spacing0 = 16, p.rs_spacing = 8;
            } else {
                p.rs_level0 = 2, p.rs_spacing0 = 32, p.rs_spacing = 8;
            }
            // batched lists: minimum spacing of the in-block ruling sets
            if (k == KIND_LR_BATCH) p.rs_spacing0 = 64;
            // sparse graphs whose parent array outgrows L2 (uniform random graphs of
            // 4 edges per vertex, 2^26 vertices: 13.6 ms against 15.6 with rule 1 and
            // no sample): a sample pass over an eighth of the edges, then re-linking
            if (k == KIND_CC_SPARSE && l >= 25) p.cc_hook = 3, p.cc_sample = 8;
        }
    g_plan_init = true;
}

// Zero every control field except the sticky status word.
void reset_ctl(Ctx* c, cudaStream_t s) {
    cudaMemsetAsync(reinterpret_cast<char*>(c->ctl) + offsetof(DevCtl, flag), 0,
                    sizeof(DevCtl) - offsetof(DevCtl, flag), s);
}

void drop_graphs(Ctx* c) {
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
}

// Launch the work `rec` records, through a cached graph unless disabled.
lrcc_status launch_recorded(Ctx* c, const Plan& p, std::vector<uint64_t> key,
                            const std::function<lrcc_status(cudaStream_t)>& rec) {
    if (p.use_graphs == 2 || timing_enabled()) return rec(c->stream);
    key.push_back(reinterpret_cast<uint64_t>(c->ws));
    GraphEntry* e = nullptr;
    for (auto& ge : c->graphs)
        if (ge.key == key) e = &ge;
    if (!e) {
        if (cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return LRCC_ERR_CUDA;
        lrcc_status st = rec(c->capture);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(c->capture, &g);
        if (st == LRCC_OK && ce != cudaSuccess) st = LRCC_ERR_CUDA;
        cudaGraphExec_t ex = nullptr;
        if (st == LRCC_OK && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) st = LRCC_ERR_CUDA;
        if (g) cudaGraphDestroy(g);
        if (st != LRCC_OK) {
            cudaGetLastError();
            return st;
        }
        if (c->graphs.size() >= 16) {
            auto it = std::min_element(c->graphs.begin(), c->graphs.end(),
                                       [](const GraphEntry& a, const GraphEntry& b) {
                                           return a.last_use < b.last_use;
                                       });
            cudaGraphExecDestroy(it->exec);
            c->graphs.erase(it);
        }
        c->graphs.push_back(GraphEntry{std::move(key), ex, 0});
        e = &c->graphs.back();
    }
    e->last_use = ++c->tick;
    return cuda_status(cudaGraphLaunch(e->exec, c->stream));
}

std::vector<uint64_t> plan_key(const Plan& p) {
    return {(uint64_t)p.rs_spacing0, (uint64_t)p.rs_spacing, (uint64_t)p.rs_small, (uint64_t)p.rs_chains,
            (uint64_t)p.rs_level0, (uint64_t)p.cc_hook, (uint64_t)p.cc_max_rounds, p.seed,
            (uint64_t)p.cc_sample};
}

}  // namespace

lrcc_status cuda_status(cudaError_t e) { return e == cudaSuccess ? LRCC_OK : LRCC_ERR_CUDA; }

bool timing_enabled() { return g_timing.load(std::memory_order_relaxed) != 0; }

namespace {
bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return st != cudaStreamCaptureStatusNone;
}
cudaEvent_t next_event(Ctx* c, size_t* idx) {
    if (c->events_used == c->events.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        c->events.push_back(e);
    }
    *idx = c->events_used++;
    return c->events[*idx];
}
}  // namespace

void phase_begin(Ctx* c, cudaStream_t s) {
    if (!timing_enabled() || capturing(s)) return;
    size_t i = 0;
    cudaEvent_t e = next_event(c, &i);
    if (e && cudaEventRecord(e, s) == cudaSuccess) c->cur_begin = i;
}

void phase_end(Ctx* c, cudaStream_t s, int phase) {
    if (!timing_enabled() || capturing(s)) return;
    size_t i = 0;
    cudaEvent_t e = next_event(c, &i);
    if (e && cudaEventRecord(e, s) == cudaSuccess) c->recs.push_back(Ctx::Rec{phase, c->cur_begin, i});
}

Plan plan_for(int kind, int64_t n) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    init_plans_locked();
    const int k = (kind == KIND_LR_WYLLIE) ? KIND_LR : kind;
    return g_plan[std::min(std::max(k, 0), PLAN_KINDS - 1)][log2_ceil(std::max<int64_t>(n, 1))];
}

int persistent_grid(Ctx* c, const void* kernel, int block, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(c->device, kernel);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int g = per_sm * c->sms;
    cache[key] = g;
    return g;
}

lrcc_status ctx_for(void* stream, Ctx** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LRCC_ERR_CUDA;
    return ctx_for_device(dev, stream, out);
}

lrcc_status ctx_for_device(int dev, void* stream, Ctx** out) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_pair(dev, s);
    auto it = g_ctx.find(key);
    if (it != g_ctx.end()) {
        *out = it->second;
        return LRCC_OK;
    }
    Ctx* c = new Ctx();
    c->device = dev;
    c->stream = s;
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return LRCC_ERR_CUDA;
    }
    if (cudaMalloc(&c->ctl, sizeof(DevCtl)) != cudaSuccess) {
        cudaStreamDestroy(c->capture);
        delete c;
        return LRCC_ERR_NOMEM;
    }
    if (cudaMemset(c->ctl, 0, sizeof(DevCtl)) != cudaSuccess) {
        cudaFree(c->ctl);
        cudaStreamDestroy(c->capture);
        delete c;
        return LRCC_ERR_CUDA;
    }
    g_ctx[key] = c;
    *out = c;
    return LRCC_OK;
}

lrcc_status ensure_ws(Ctx* c, size_t bytes) {
    if (bytes <= c->ws_bytes) return LRCC_OK;
    const size_t old = c->ws_bytes;
    // the old workspace may still be in use by queued work on this stream
    if (c->ws) {
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return LRCC_ERR_CUDA;
        drop_graphs(c);
        cudaFree(c->ws);
        c->ws = nullptr;
        c->ws_bytes = 0;
    }
    const size_t want = std::max(bytes, old + old / 4);
    if (inject_alloc_failure()) return LRCC_ERR_NOMEM;
    if (cudaMalloc(&c->ws, want) != cudaSuccess) {
        cudaGetLastError();
        if (cudaMalloc(&c->ws, bytes) != cudaSuccess) {
            cudaGetLastError();
            c->ws = nullptr;
            return LRCC_ERR_NOMEM;
        }
        c->ws_bytes = bytes;
        return LRCC_OK;
    }
    c->ws_bytes = want;
    return LRCC_OK;
}

// Device staging for the host-buffer entry points (kept apart from the
// workspace so that its address, and the graphs keyed on it, stay put).
lrcc_status ensure_io(Ctx* c, size_t bytes) {
    if (bytes <= c->io_bytes) return LRCC_OK;
    if (c->io) {
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return LRCC_ERR_CUDA;
        drop_graphs(c);
        cudaFree(c->io);
        c->io = nullptr;
        c->io_bytes = 0;
    }
    if (inject_alloc_failure() || cudaMalloc(&c->io, bytes) != cudaSuccess) {
        cudaGetLastError();
        c->io = nullptr;
        return LRCC_ERR_NOMEM;
    }
    c->io_bytes = bytes;
    return LRCC_OK;
}

// Runs a host-buffer call: `up` enqueues the uploads, `compute` the device
// method on the caller's stream, `down` the downloads. Uploads and downloads go
// through two copy streams shared by all calls on the device, so that the
// uploads of calls on different streams run one after another at full
// bandwidth (and overlap other calls' kernels) instead of splitting it.
// Order: the stream's earlier work (which may still read the staging) ->
// uploads -> compute -> downloads -> the stream's later work.
lrcc_status host_call(Ctx* c, const std::function<cudaError_t(cudaStream_t)>& up,
                      const std::function<lrcc_status()>& compute,
                      const std::function<cudaError_t(cudaStream_t)>& down) {
    cudaStream_t in = nullptr, out = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_copy.find(c->device);
        if (it == g_copy.end()) {
            if (cudaStreamCreateWithFlags(&in, cudaStreamNonBlocking) != cudaSuccess) return LRCC_ERR_CUDA;
            if (cudaStreamCreateWithFlags(&out, cudaStreamNonBlocking) != cudaSuccess) {
                cudaStreamDestroy(in);
                return LRCC_ERR_CUDA;
            }
            g_copy[c->device] = std::make_pair(in, out);
        } else {
            in = it->second.first;
            out = it->second.second;
        }
    }
    for (auto& e : c->io_ev)
        if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            e = nullptr;
            return LRCC_ERR_CUDA;
        }
    cudaEvent_t free_ev = c->io_ev[0], in_ev = c->io_ev[1], done_ev = c->io_ev[2], out_ev = c->io_ev[3];
    if (cudaEventRecord(free_ev, c->stream) != cudaSuccess || cudaStreamWaitEvent(in, free_ev, 0) != cudaSuccess ||
        up(in) != cudaSuccess || cudaEventRecord(in_ev, in) != cudaSuccess ||
        cudaStreamWaitEvent(c->stream, in_ev, 0) != cudaSuccess)
        return LRCC_ERR_CUDA;
    const lrcc_status st = compute();
    if (st != LRCC_OK) return st;
    if (cudaEventRecord(done_ev, c->stream) != cudaSuccess || cudaStreamWaitEvent(out, done_ev, 0) != cudaSuccess ||
        down(out) != cudaSuccess || cudaEventRecord(out_ev, out) != cudaSuccess ||
        cudaStreamWaitEvent(c->stream, out_ev, 0) != cudaSuccess)
        return LRCC_ERR_CUDA;
    return LRCC_OK;
}

}  // namespace lrcc

using namespace lrcc;

extern "C" {

const char* lrcc_status_str(lrcc_status status) {
    switch (status) {
        case LRCC_OK: return "ok";
        case LRCC_ERR_ARG: return "bad argument";
        case LRCC_ERR_NOMEM: return "out of device memory";
        case LRCC_ERR_CUDA: return "CUDA runtime error";
        case LRCC_ERR_INVALID_INPUT: return "invalid input (not a single list, or an id out of range)";
        case LRCC_ERR_NOT_CONVERGED: return "component loop reached its round cap";
        case LRCC_ERR_TIMEOUT: return "device-side wait timed out";
        default: return "unknown status";
    }
}

int lrcc_version(void) { return 101; }

namespace {

// lr_rank on device buffers, with the context's lock held.
lrcc_status lr_rank_locked(Ctx* c, const int32_t* succ, int64_t n, int32_t head, int32_t* rank,
                           const int32_t* val = nullptr) {
    lrcc_status st = LRCC_OK;
    Plan p = plan_for(KIND_LR, n);
    if (val) p.rs_level0 = 1;   // weighted sums: the in-place first level carries the values
    const RsLayout L = rs_layout(n, p, rs_walk_grid(c, p));
    if (n > p.rs_small) {
        st = ensure_ws(c, L.bytes);
        if (st != LRCC_OK) return st;
    }
    std::vector<uint64_t> key = {(uint64_t)KIND_LR, (uint64_t)succ, (uint64_t)n, (uint64_t)head, (uint64_t)rank,
                                 (uint64_t)val};
    const auto pk = plan_key(p);
    key.insert(key.end(), pk.begin(), pk.end());
    st = launch_recorded(c, p, key, [&](cudaStream_t s) {
        reset_ctl(c, s);
        return lr_enqueue_rs(c, s, succ, n, head, rank, p, L, val);
    });
    c->last_kind = val ? 6 : KIND_LR;
    c->last_levels = n > p.rs_small ? L.levels : 0;
    for (int l = 0; l < MAX_LEVELS; ++l) c->last_splitter_cap[l] = l < L.levels ? L.size[l + 1] : 0;
    return st;
}

// cc_label on device buffers, with the context's lock held.
lrcc_status cc_label_locked(Ctx* c, const int32_t* src, const int32_t* dst, int64_t m, int64_t n, int32_t* label) {
    const Plan p = plan_for(cc_plan_kind(m, n), n);
    const bool sv = p.cc_hook == 4;
    lrcc_status st = ensure_ws(c, sv ? cc_sv_ws(n) : cc_ws(m));
    if (st != LRCC_OK) return st;
    reset_ctl(c, c->stream);
    st = sv ? cc_run_sv(c, src, dst, m, n, label, p) : cc_run(c, src, dst, m, n, label, p);
    c->last_kind = KIND_CC;
    return st;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

lrcc_status lr_rank(const int32_t* succ, int64_t n, int32_t head, int32_t* rank, void* stream) {
    ApiRange range_("lr_rank");
    if (n < 0 || n > 0x7FFFFFFELL) return LRCC_ERR_ARG;
    if (n == 0) return LRCC_OK;
    if (!succ || !rank || head < 0 || head >= n) return LRCC_ERR_ARG;
    Ctx* c = nullptr;
    lrcc_status st = ctx_for(stream, &c);
    if (st != LRCC_OK) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    return lr_rank_locked(c, succ, n, head, rank);
}

lrcc_status lr_rank_splitters(const int32_t* succ, int64_t n, int32_t head, const int32_t* spl, int64_t r,
                              int32_t* rank, void* stream) {
    ApiRange range_("lr_rank_splitters");
    if (n < 0 || n > 0x7FFFFFFELL) return LRCC_ERR_ARG;
    if (n == 0) return LRCC_OK;
    if (!succ || !rank || !spl || head < 0 || head >= n || r < 1 || r > n) return LRCC_ERR_ARG;
    Ctx* c = nullptr;
    lrcc_status st = ctx_for(stream, &c);
    if (st != LRCC_OK) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    Plan p = plan_for(KIND_LR, n);
    p.rs_level0 = 1;   // the in-place first level carries the given splitters in its words
    const RsLayout L = rs_layout(n, p, rs_walk_grid(c, p), 0, r);
    if (n > p.rs_small) {
        st = ensure_ws(c, L.bytes);
        if (st != LRCC_OK) return st;
    }
    std::vector<uint64_t> key = {8, (uint64_t)succ, (uint64_t)n, (uint64_t)head, (uint64_t)rank, (uint64_t)spl,
                                 (uint64_t)r};
    const auto pk = plan_key(p);
    key.insert(key.end(), pk.begin(), pk.end());
    st = launch_recorded(c, p, key, [&](cudaStream_t s) {
        reset_ctl(c, s);
        return lr_enqueue_rs(c, s, succ, n, head, rank, p, L, nullptr, nullptr, spl, r);
    });
    c->last_kind = KIND_LR;
    c->last_levels = n > p.rs_small ? L.levels : 0;
    for (int l = 0; l < MAX_LEVELS; ++l) c->last_splitter_cap[l] = l < L.levels ? L.size[l + 1] : 0;
    return st;
}

lrcc_status lr_scan(const int32_t* succ, const int32_t* val, int64_t n, int32_t head, int32_t* out, void* stream) {
    ApiRange range_("lr_scan");
    if (n < 0 || n > 0x7FFFFFFELL) return LRCC_ERR_ARG;
    if (n == 0) return LRCC_OK;
    if (!succ || !val || !out || head < 0 || head >= n) return LRCC_ERR_ARG;
    Ctx* c = nullptr;
    lrcc_status st = ctx_for(stream, &c);
    if (st != LRCC_OK) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    return lr_rank_locked(c, succ, n, head, out, val);
}

lrcc_status lr_scan_forest(const int32_t* succ, const int32_t* val, int64_t n, int32_t* out, void* stream) {
    ApiRange range_("lr_scan_forest");
    if (n < 0 || n > 0x7FFFFFFELL) return LRCC_ERR_ARG;
    if (n == 0) return LRCC_OK;
    if (!succ || !val || !out) return LRCC_ERR_ARG;
    Ctx* c = nullptr;
    lrcc_status st = ctx_for(stream, &c);
    if (st != LRCC_OK) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    const Plan p = plan_for(KIND_LR, n);
    st = ensure_ws(c, lr_scan_forest_ws(n, p));
    if (st != LRCC_OK) return st;
    const std::vector<uint64_t> key = {7, (uint64_t)succ, (uint64_t)val, (uint64_t)n, (uint64_t)out};
    st = launch_recorded(c, p, key, [&](cudaStream_t s) {
        reset_ctl(c, s);
        return lr_enqueue_scan_forest(c, s, succ, val, n, out, p);
    });
    c->last_kind = 7;
    c->last_levels = 0;
    return st;
}

lrcc_status lr_rank_host(const int32_t* succ, int64_t n, int32_t head, int32_t* rank, void* stream) {
    ApiRange range_("lr_rank_host");
    if (n < 0 || n > 0x7FFFFFFELL) return LRCC_ERR_ARG;
    if (n == 0) return LRCC_OK;
    if (!succ || !rank || head < 0 || head >= n) return LRCC_ERR_ARG;
    Ctx* c = nullptr;
    lrcc_status st = ctx_for(stream, &c);
    if (st != LRCC_OK) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    const size_t bytes = sizeof(int32_t) * (size_t)n;
    st = ensure_io(c, 2 * align256(bytes));
    if (st != LRCC_OK) return st;
    int32_t* d_succ = static_cast<int32_t*>(c->io);
    int32_t* d_rank = reinterpret_cast<int32_t*>(static_cast<char*>(c->io) + align256(bytes));
    return host_call(
        c, [&](cudaStream_t s) { return cudaMemcpyAsync(d_succ, succ, bytes, cudaMemcpyHostToDevice, s); },
        [&] { return lr_rank_locked(c, d_succ, n, head, d_rank); },
        [&](cudaStream_t s) { return cudaMemcpyAsync(rank, d_rank, bytes, cudaMemcpyDeviceToHost, s); });
}

lrcc_status lr_rank_wyllie(const int32_t* succ, int64_t n, int32_t head, int32_t* rank, void* stream) {
    ApiRange range_("lr_rank_wyllie");
    if (n < 0 || n > 0x7FFFFFFELL) return LRCC_ERR_ARG;
    if (n == 0) return LRCC_OK;
    if (!succ || !rank || head < 0 || head >= n) return LRCC_ERR_ARG;
    Ctx* c = nullptr;
    lrcc_status st = ctx_for(stream, &c);
    if (st != LRCC_OK) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    const Plan p = plan_for(KIND_LR_WYLLIE, n);
    if (n > p.rs_small) {
        st = ensure_ws(c, lr_wyllie_ws(n, p));
        if (st != LRCC_OK) return st;
    }
    std::vector<uint64_t> key = {(uint64_t)KIND_LR_WYLLIE, (uint64_t)succ, (uint64_t)n, (uint64_t)head,
                                 (uint64_t)rank, (uint64_t)p.rs_small};
    st = launch_recorded(c, p, key, [&](cudaStream_t s) {
        reset_ctl(c, s);
        return lr_enqueue_wyllie(c, s, succ, n, head, rank, p);
    });
    c->last_kind = KIND_LR_WYLLIE;
    c->last_levels = 0;
    return st;
}

lrcc_status cc_label(const int32_t* src, const int32_t* dst, int64_t m, int64_t n, int32_t* label,
                     void* stream) {
    ApiRange range_("cc_label");
    if (n < 0 || m < 0 || n > 0x7FFFFFFELL) return LRCC_ERR_ARG;
    if (n == 0) return m == 0 ? LRCC_OK : LRCC_ERR_ARG;
    if (!label || (m > 0 && (!src || !dst))) return LRCC_ERR_ARG;
    Ctx* c = nullptr;
    lrcc_status st = ctx_for(stream, &c);
    if (st != LRCC_OK) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    return cc_label_locked(c, src, dst, m, n, label);
}

lrcc_status cc_label_host(const int32_t* src, const int32_t* dst, int64_t m, int64_t n, int32_t* label,
                          void* stream) {
    ApiRange range_("cc_label_host");
    if (n < 0 || m < 0 || n > 0x7FFFFFFELL) return LRCC_ERR_ARG;
    if (n == 0) return m == 0 ? LRCC_OK : LRCC_ERR_ARG;
    if (!label || (m > 0 && (!src || !dst))) return LRCC_ERR_ARG;
    Ctx* c = nullptr;
    lrcc_status st = ctx_for(stream, &c);
    if (st != LRCC_OK) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    const size_t eb = sizeof(int32_t) * (size_t)m, vb = sizeof(int32_t) * (size_t)n;
    st = ensure_io(c, 2 * align256(eb) + align256(vb));
    if (st != LRCC_OK) return st;
    char* io = static_cast<char*>(c->io);
    int32_t* d_src = reinterpret_cast<int32_t*>(io);
    int32_t* d_dst = reinterpret_cast<int32_t*>(io + align256(eb));
    int32_t* d_label = reinterpret_cast<int32_t*>(io + 2 * align256(eb));
    return host_call(
        c,
        [&](cudaStream_t s) {
            if (m == 0) return cudaSuccess;
            const cudaError_t e = cudaMemcpyAsync(d_src, src, eb, cudaMemcpyHostToDevice, s);
            return e != cudaSuccess ? e : cudaMemcpyAsync(d_dst, dst, eb, cudaMemcpyHostToDevice, s);
        },
        [&] { return cc_label_locked(c, d_src, d_dst, m, n, d_label); },
        [&](cudaStream_t s) { return cudaMemcpyAsync(label, d_label, vb, cudaMemcpyDeviceToHost, s); });
}

lrcc_status lr_rank_batched_sized(const int32_t* succ, const int64_t* node_off, const int32_t* heads,
                                  int64_t num_lists, int64_t total_nodes, int32_t* rank, void* stream) {
    ApiRange range_("lr_rank_batched_sized");
    if (num_lists < 0 || total_nodes < 0) return LRCC_ERR_ARG;
    if (num_lists == 0) return LRCC_OK;
    if (!node_off || !heads || (total_nodes > 0 && (!succ || !rank))) return LRCC_ERR_ARG;
    Ctx* c = nullptr;
    lrcc_status st = ctx_for(stream, &c);
    if (st != LRCC_OK) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    // the batched plan is looked up by the total element count: its first-level
    // mode decides between one block per list and the lists ranked as one list
    const Plan p = plan_for(KIND_LR_BATCH, total_nodes);
    if (batch_union_applies(total_nodes, p)) {
        // the lists ranked together as one list by the read-only first level
        st = ensure_ws(c, lr_batched_union_ws(c, total_nodes, num_lists));
        if (st != LRCC_OK) return st;
        reset_ctl(c, c->stream);
        st = lr_batched_union(c, c->stream, succ, node_off, heads, num_lists, total_nodes, rank);
    } else {
        st = ensure_ws(c, lr_batched_ws(total_nodes, num_lists));
        if (st != LRCC_OK) return st;
        reset_ctl(c, c->stream);
        st = lr_batched_run(c, succ, node_off, heads, num_lists, rank, total_nodes, p);
    }
    c->last_kind = KIND_LR_BATCH;
    return st;
}

lrcc_status lr_rank_batched(const int32_t* succ, const int64_t* node_off, const int32_t* heads,
                            int64_t num_lists, int32_t* rank, void* stream) {
    ApiRange range_("lr_rank_batched");
    if (num_lists < 0) return LRCC_ERR_ARG;
    if (num_lists == 0) return LRCC_OK;
    if (!node_off || !heads) return LRCC_ERR_ARG;
    // the workspace is sized from the total element count, node_off[num_lists]
    int64_t total = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&total, node_off + num_lists, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return LRCC_ERR_CUDA;
    if (total < 0) return LRCC_ERR_ARG;
    return lr_rank_batched_sized(succ, node_off, heads, num_lists, total, rank, stream);
}

lrcc_status cc_label_batched_sized(const int32_t* src, const int32_t* dst, const int64_t* edge_off,
                                   const int64_t* vert_off, int64_t num_graphs, int64_t total_edges,
                                   int32_t* label, void* stream) {
    ApiRange range_("cc_label_batched_sized");
    if (num_graphs < 0 || total_edges < 0) return LRCC_ERR_ARG;
    if (num_graphs == 0) return LRCC_OK;
    if (!edge_off || !vert_off || !label || (total_edges > 0 && (!src || !dst))) return LRCC_ERR_ARG;
    Ctx* c = nullptr;
    lrcc_status st = ctx_for(stream, &c);
    if (st != LRCC_OK) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    const Plan p = plan_for(KIND_CC_BATCH, 0);
    st = ensure_ws(c, cc_batched_ws(num_graphs, total_edges));
    if (st != LRCC_OK) return st;
    reset_ctl(c, c->stream);
    st = cc_batched_run(c, src, dst, edge_off, vert_off, num_graphs, total_edges, label, p);
    c->last_kind = KIND_CC_BATCH;
    return st;
}

lrcc_status cc_label_batched(const int32_t* src, const int32_t* dst, const int64_t* edge_off,
                             const int64_t* vert_off, int64_t num_graphs, int32_t* label, void* stream) {
    ApiRange range_("cc_label_batched");
    if (num_graphs < 0) return LRCC_ERR_ARG;
    if (num_graphs == 0) return LRCC_OK;
    if (!edge_off || !vert_off) return LRCC_ERR_ARG;
    // the active-edge buffers are sized from the total edge count, edge_off[num_graphs]
    int64_t total = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&total, edge_off + num_graphs, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return LRCC_ERR_CUDA;
    if (total < 0) return LRCC_ERR_ARG;
    return cc_label_batched_sized(src, dst, edge_off, vert_off, num_graphs, total, label, stream);
}

lrcc_status lrcc_gather_probe(const int32_t* src, const int32_t* dst, int64_t m, const int32_t* table, int64_t n,
                              int64_t* out, void* stream) {
    if (m < 0 || n < 1 || !out || !table || (m > 0 && (!src || !dst))) return LRCC_ERR_ARG;
    Ctx* c = nullptr;
    lrcc_status st = ctx_for(stream, &c);
    if (st != LRCC_OK) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    return cc_gather_probe_run(c, src, dst, m, table, n, out);
}

lrcc_status lrcc_chase_probe(const int32_t* succ, int64_t n, int64_t chains, int64_t steps, int64_t* out,
                             void* stream) {
    if (n < 1 || n > INT32_MAX || chains < 1 || chains > (int64_t(1) << 31) || steps < 0 || !succ || !out)
        return LRCC_ERR_ARG;
    Ctx* c = nullptr;
    lrcc_status st = ctx_for(stream, &c);
    if (st != LRCC_OK) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    return rs_chase_probe_run(c, succ, n, chains, steps, out);
}

int lrcc_debug_fail_allocs(int count) { return g_fail_allocs.exchange(count < 0 ? 0 : count); }

lrcc_status lrcc_wait_check(int polls, void* stream) {
    if (polls < 1 || polls > (1 << 20)) return LRCC_ERR_ARG;
    Ctx* c = nullptr;
    lrcc_status st = ctx_for(stream, &c);
    if (st != LRCC_OK) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    return cuda_status(wait_check_enqueue(c->ctl, polls, c->stream));
}

lrcc_status lrcc_last_status(void* stream) {
    Ctx* c = nullptr;
    lrcc_status st = ctx_for(stream, &c);
    if (st != LRCC_OK) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return LRCC_ERR_CUDA;
    int v = 0;
    if (cudaMemcpy(&v, &c->ctl->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return LRCC_ERR_CUDA;
    if (v != 0 && cudaMemset(&c->ctl->status, 0, sizeof(int)) != cudaSuccess) return LRCC_ERR_CUDA;
    return static_cast<lrcc_status>(v);
}

lrcc_status lrcc_last_stats(void* stream, lrcc_stats* out) {
    if (!out) return LRCC_ERR_ARG;
    Ctx* c = nullptr;
    lrcc_status st = ctx_for(stream, &c);
    if (st != LRCC_OK) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return LRCC_ERR_CUDA;
    DevCtl h;
    if (cudaMemcpy(&h, c->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost) != cudaSuccess) return LRCC_ERR_CUDA;
    std::memset(out, 0, sizeof(*out));
    out->kind = c->last_kind;
    out->levels = c->last_levels;
    for (int l = 0; l < c->last_levels && l < 8; ++l) out->splitters[l] = c->last_splitter_cap[l];
    out->rounds = h.rounds;
    out->jump_rounds = h.jump_rounds;
    out->overflow_chunks = h.ovf_next;
    out->edges_read = (int64_t)h.edges_read;
    return LRCC_OK;
}

lrcc_status lrcc_set_plan(int kind, int log2_lo, int log2_hi, const lrcc_plan* plan) {
    const bool known = (kind >= 1 && kind <= 5) || kind == KIND_CC_SPARSE;
    if (!plan || !known || log2_lo < 0 || log2_hi > 32 || log2_lo > log2_hi) return LRCC_ERR_ARG;
    if (plan->rs_small < 0 || plan->rs_small > 16384 || plan->rs_spacing0 < 0 || plan->rs_spacing < 0 ||
        (plan->rs_spacing0 > 0 && plan->rs_spacing0 < 2) || (plan->rs_spacing > 0 && plan->rs_spacing < 2) ||
        (plan->rs_small > 0 && plan->rs_small < 1024) || plan->rs_chains < 0 || plan->rs_chains > 4 ||
        plan->cc_hook < 0 || plan->cc_hook > 5 || plan->cc_max_rounds < -1 || plan->use_graphs < 0 ||
        plan->use_graphs > 2 || plan->rs_level0 < 0 || plan->rs_level0 > 3 || plan->cc_sample < -1 ||
        plan->cc_sample > 1024)
        return LRCC_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_plan_mu);
    init_plans_locked();
    for (int l = log2_lo; l <= log2_hi; ++l) {
        Plan& p = g_plan[kind][l];
        if (plan->rs_spacing0) p.rs_spacing0 = plan->rs_spacing0;
        if (plan->rs_spacing) p.rs_spacing = plan->rs_spacing;
        if (plan->rs_small) p.rs_small = plan->rs_small;
        if (plan->rs_chains) p.rs_chains = plan->rs_chains;
        if (plan->cc_hook) p.cc_hook = plan->cc_hook;
        if (plan->cc_max_rounds) p.cc_max_rounds = plan->cc_max_rounds < 0 ? 0 : plan->cc_max_rounds;
        if (plan->use_graphs) p.use_graphs = plan->use_graphs;
        if (plan->rs_level0) p.rs_level0 = plan->rs_level0;
        if (plan->seed) p.seed = plan->seed;
        if (plan->cc_sample) p.cc_sample = plan->cc_sample;
    }
    return LRCC_OK;
}

lrcc_status lrcc_reset_plans(void) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_plan_init = false;
    init_plans_locked();
    return LRCC_OK;
}

lrcc_status lrcc_get_plan(int kind, int64_t n, lrcc_plan* out) {
    if (!out || !((kind >= 1 && kind <= 5) || kind == KIND_CC_SPARSE)) return LRCC_ERR_ARG;
    const Plan p = plan_for(kind, n);
    std::memset(out, 0, sizeof(*out));
    out->rs_spacing0 = p.rs_spacing0;
    out->rs_spacing = p.rs_spacing;
    out->rs_small = p.rs_small;
    out->rs_chains = p.rs_chains;
    out->cc_hook = p.cc_hook;
    out->cc_max_rounds = p.cc_max_rounds;
    out->use_graphs = p.use_graphs;
    out->rs_level0 = p.rs_level0;
    out->seed = p.seed;
    out->cc_sample = p.cc_sample;
    return LRCC_OK;
}

lrcc_status lrcc_set_l2_fetch_granularity(int bytes) {
    if (bytes != 0 && bytes != 32 && bytes != 64 && bytes != 128) return LRCC_ERR_ARG;
    if (bytes == 0) return LRCC_OK;
    return cuda_status(cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)bytes));
}

int lrcc_get_l2_fetch_granularity(void) {
    size_t v = 0;
    if (cudaDeviceGetLimit(&v, cudaLimitMaxL2FetchGranularity) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return (int)v;
}

lrcc_status lrcc_set_timing(int enable) {
    g_timing.store(enable ? 1 : 0);
    return LRCC_OK;
}

int lrcc_phase_count(void) { return PH_COUNT; }

const char* lrcc_phase_name(int phase) {
    return (phase >= 0 && phase < PH_COUNT) ? kPhaseNames[phase] : "unknown";
}

lrcc_status lrcc_phase_times(void* stream, double* ms_total, int64_t* launches) {
    if (!ms_total || !launches) return LRCC_ERR_ARG;
    Ctx* c = nullptr;
    lrcc_status st = ctx_for(stream, &c);
    if (st != LRCC_OK) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return LRCC_ERR_CUDA;
    for (const auto& r : c->recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->events[r.a], c->events[r.b]) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        ms_total[r.phase] += ms;
        launches[r.phase] += 1;
    }
    c->recs.clear();
    c->events_used = 0;
    return LRCC_OK;
}

lrcc_status lrcc_release(void* stream) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LRCC_ERR_CUDA;
    release_device_stream(dev, stream);
    return LRCC_OK;
}

}  // extern "C"

namespace lrcc {

// Frees the workspace of (device, stream), if any, after waiting for the
// stream. The caller has that device current.
void release_device_stream(int dev, void* stream) {
    Ctx* c = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_ctx.find(std::make_pair(dev, static_cast<cudaStream_t>(stream)));
        if (it == g_ctx.end()) return;
        c = it->second;
        g_ctx.erase(it);
    }
    cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    for (auto e : c->events) cudaEventDestroy(e);
    if (c->ws) cudaFree(c->ws);
    if (c->io) cudaFree(c->io);
    for (auto e : c->io_ev)
        if (e) cudaEventDestroy(e);
    cudaFree(c->ctl);
    cudaStreamDestroy(c->capture);
    delete c;
}

int64_t ctx_bytes(const Ctx* c) { return (int64_t)(c->ws_bytes + c->io_bytes) + (int64_t)sizeof(DevCtl); }

}  // namespace lrcc

// A context: the streams of one device whose workspaces were reserved through
// it (the workspaces themselves stay in the per-(device, stream) table).
struct lrcc_ctx {
    int device = 0;
    std::mutex mu;
    std::vector<cudaStream_t> streams;
};

namespace {
// Makes `dev` current for the guard's lifetime and restores the caller's device.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        ok = cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};
}  // namespace

extern "C" {

lrcc_status lrcc_ctx_create(lrcc_ctx** ctx, int device) {
    if (!ctx) return LRCC_ERR_ARG;
    *ctx = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) {
        cudaGetLastError();
        return LRCC_ERR_CUDA;
    }
    if (device < 0 || device >= count) return LRCC_ERR_ARG;
    lrcc_ctx* c = new (std::nothrow) lrcc_ctx();
    if (!c) return LRCC_ERR_NOMEM;
    c->device = device;
    *ctx = c;
    return LRCC_OK;
}

void lrcc_ctx_destroy(lrcc_ctx* ctx) {
    if (!ctx) return;
    {
        DeviceGuard g(ctx->device);
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (g.ok)
            for (cudaStream_t s : ctx->streams) release_device_stream(ctx->device, s);
    }
    delete ctx;
}

lrcc_status lrcc_ctx_reserve(lrcc_ctx* ctx, void* stream, int64_t bytes) {
    if (!ctx || bytes < 0) return LRCC_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return LRCC_ERR_CUDA;
    Ctx* c = nullptr;
    lrcc_status st = ctx_for_device(ctx->device, stream, &c);
    if (st != LRCC_OK) return st;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        st = ensure_ws(c, (size_t)bytes);
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (std::find(ctx->streams.begin(), ctx->streams.end(), s) == ctx->streams.end()) ctx->streams.push_back(s);
    return st;
}

int64_t lrcc_ctx_bytes(lrcc_ctx* ctx) {
    if (!ctx) return -1;
    std::lock_guard<std::mutex> lk(ctx->mu);
    std::lock_guard<std::mutex> lk2(g_mu);
    int64_t t = 0;
    for (cudaStream_t s : ctx->streams) {
        auto it = g_ctx.find(std::make_pair(ctx->device, s));
        if (it != g_ctx.end()) t += ctx_bytes(it->second);
    }
    return t;
}

lrcc_status lrcc_ctx_last_status(lrcc_ctx* ctx, void* stream) {
    if (!ctx) return LRCC_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return LRCC_ERR_CUDA;
    return lrcc_last_status(stream);
}

int64_t lrcc_workspace_bytes(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    int64_t t = 0;
    for (auto& kv : g_ctx) t += ctx_bytes(kv.second);
    return t;
}

int64_t lrcc_workspace_query(int kind, int64_t n, int64_t m) {
    (void)m;
    if (n < 0) return -1;
    const Plan p = kind == KIND_CC ? plan_for(cc_plan_kind(m, n), n) : plan_for(kind > 5 ? KIND_LR : kind, n);
    switch (kind) {
        case 6: {   // lr_scan: the in-place first level
            Plan ps = p;
            ps.rs_level0 = 1;
            return n > ps.rs_small ? (int64_t)rs_layout(n, ps, rs_walk_grid_current(ps)).bytes : 0;
        }
        case 7: return (int64_t)lr_scan_forest_ws(n, p);   // lr_scan_forest
        case KIND_LR: {
            // the walk's block count on the current device (as on a GB300 when none can be queried)
            return n > p.rs_small ? (int64_t)rs_layout(n, p, rs_walk_grid_current(p)).bytes : 0;
        }
        case KIND_LR_WYLLIE: return n > p.rs_small ? (int64_t)lr_wyllie_ws(n, p) : 0;
        case KIND_CC: return (int64_t)(p.cc_hook == 4 ? cc_sv_ws(n) : cc_ws(m));
        case KIND_LR_BATCH: {   // n = total elements, m = lists
            const Plan pb = plan_for(KIND_LR_BATCH, n);
            if (!batch_union_applies(n, pb)) return (int64_t)lr_batched_ws(n, m);
            Plan pu = plan_for(KIND_LR, n);
            pu.rs_level0 = 2;
            // the lists ranked as one list: the one-list layout with m extra splitters,
            // global successors, two int32 per list
            return (int64_t)(rs_layout(n, pu, rs_walk_grid_current(pu), m).bytes + 4 * (size_t)n + 8 * (size_t)m + 1024);
        }
        case KIND_CC_BATCH: return (int64_t)cc_batched_ws(m, n);   // n = total edges, m = graphs
        default: return -1;
    }
}

}  // extern "C"
