// Host-side internals shared by the translation units of liblrcc.so.
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "lrcc.h"

namespace lrcc {

struct DevCtl;
struct Ctx;

constexpr int KIND_LR = 1;
constexpr int KIND_LR_WYLLIE = 2;
constexpr int KIND_CC = 3;
constexpr int KIND_LR_BATCH = 4;
constexpr int KIND_CC_BATCH = 5;
// Plan class of graphs with fewer than 4 edges per vertex (m < 4n); 6 and 7
// name the weighted-rank calls in statistics and workspace queries.
constexpr int KIND_CC_SPARSE = 8;
constexpr int PLAN_KINDS = 9;
// Plan class of a components call: sparse graphs are planned apart.
inline int cc_plan_kind(int64_t m, int64_t n) { return (n > 0 && m < 4 * n) ? KIND_CC_SPARSE : KIND_CC; }

// Resolved tuning knobs (every field set).
struct Plan {
    int rs_spacing0 = 32;
    int rs_spacing = 16;
    int rs_small = 8192;
    int rs_chains = 1;
    int rs_level0 = 2;      // 1 = in-place walk words, 2 = read-only walk + chunked records,
                            // 3 = split mark / local-rank arrays
    int cc_hook = 1;
    int cc_max_rounds = 0;
    int use_graphs = 1;
    int cc_sample = -1;     // 1 = no sample pass; k = a first pass over the first m / k edges; -1 = auto
    uint64_t seed = 0x5eedULL;
};
Plan plan_for(int kind, int64_t n);

// Ruling-set level layout for a list of n elements (host-side plan).
constexpr int MAX_LEVELS = 8;
struct RsLayout {
    int levels = 0;                 // L: levels with a walk; level L is ranked by one block
                                    // size[l+1] = ceil(size[l] / 2^logD[l]) splitters at level l
    int64_t size[MAX_LEVELS + 1];   // element bound of each level (size[0] = n)
    int logD[MAX_LEVELS];           // log2 of the splitter spacing of each walked level
    size_t off_R[MAX_LEVELS + 1], off_snext[MAX_LEVELS + 1], off_sw[MAX_LEVELS + 1],
        off_S[MAX_LEVELS + 1];
    size_t off_W0 = 0;
    bool readonly = false;          // level 0 by the read-only walk (chunks, scan, scatter, place)
    bool split = false;             // level 0 over split mark / local-rank arrays
    int64_t grid = 0, cap = 0, ovf_cap = 0;
    int segcap = 0, units = 0;
    size_t off_ids = 0, off_meta = 0, off_fill = 0, off_counts = 0, off_totals = 0,
        off_vis = 0;
    size_t bytes = 0;
};
// extra1: extra first-level splitters (the heads of batched lists ranked as one list)
// given1: the number of first-level splitters when the caller chooses them
RsLayout rs_layout(int64_t n, const Plan& p, int walk_grid, int64_t extra1 = 0, int64_t given1 = 0);

// Batched lists ranked as one list by the read-only first level: K lists own
// [off[k], off[k+1]) of succ with local ids; device scratch for the global
// successors, each list's head splitter, the extra splitters' elements and the
// first list's global head.
struct BatchUnion {
    const int64_t* off = nullptr;
    const int32_t* heads = nullptr;
    int64_t K = 0;
    int32_t* gsucc = nullptr;
    int32_t* head_spl = nullptr;
    int32_t* extra_elem = nullptr;
    int64_t* head_dev = nullptr;
};
int rs_walk_grid(Ctx* c, const Plan& p);
// The same grid for the current device without a workspace (152 x 8 when no
// device can be queried).
int rs_walk_grid_current(const Plan& p);

// Phase ids for timing mode (names in runtime.cu).
enum Phase {
    PH_SELECT0, PH_WALK0, PH_SELECT, PH_WALK, PH_FINAL, PH_EXPAND, PH_EXPAND0, PH_SMALL,
    PH_WY_PACK, PH_WY_JUMP, PH_WY_FINAL, PH_CC_INIT, PH_CC_LOOP, PH_CC_HOOK, PH_CC_SHORTCUT,
    PH_LR_BATCH, PH_CC_BATCH, PH_BATCH_PREP, PH_SCAN, PH_SCATTER, PH_CC_HOOK_FULL, PH_COUNT
};

struct GraphEntry {
    std::vector<uint64_t> key;
    cudaGraphExec_t exec = nullptr;
    uint64_t last_use = 0;
};

// One workspace per (device, stream).
struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;    // the caller's stream this workspace serves
    cudaStream_t capture = nullptr;   // private stream used to capture graphs
    DevCtl* ctl = nullptr;            // device control block
    void* ws = nullptr;
    size_t ws_bytes = 0;
    void* io = nullptr;               // device copies of host-buffer calls' inputs and outputs
    size_t io_bytes = 0;
    cudaEvent_t io_ev[4] = {};        // host-buffer calls: staging free, uploaded, computed, downloaded
    int sms = 0;
    std::vector<GraphEntry> graphs;
    uint64_t tick = 0;
    // host-side facts about the most recent call
    int last_kind = 0;
    int last_levels = 0;
    int64_t last_splitter_cap[MAX_LEVELS] = {};
    std::mutex mu;                    // serialises host calls that use this workspace
    // timing mode: events recorded around phases, read by lrcc_phase_times
    std::vector<cudaEvent_t> events;
    size_t events_used = 0;
    size_t cur_begin = 0;
    struct Rec { int phase; size_t a, b; };
    std::vector<Rec> recs;
};

// Timing mode. phase_begin/phase_end bracket one kernel (or loop) on stream s
// when timing is on and s is not capturing; they do nothing otherwise.
bool timing_enabled();
void phase_begin(Ctx* c, cudaStream_t s);
void phase_end(Ctx* c, cudaStream_t s, int phase);

// Returns the workspace of `stream` on the current device, creating it.
lrcc_status ctx_for(void* stream, Ctx** out);
// The same for an explicit device (which the caller has made current).
lrcc_status ctx_for_device(int dev, void* stream, Ctx** out);
// Frees the workspace of (dev, stream) after waiting for the stream (dev current).
void release_device_stream(int dev, void* stream);
// Device bytes held by one workspace: kernel workspace, host-call staging, control block.
int64_t ctx_bytes(const Ctx* c);
lrcc_status ensure_ws(Ctx* c, size_t bytes);
lrcc_status cuda_status(cudaError_t e);

// Persistent grid size for a kernel: SMs x resident blocks per SM.
int persistent_grid(Ctx* c, const void* kernel, int block, size_t smem = 0);

// --- list ranking (lr.cu)
// val != nullptr: inclusive weighted suffix sums (modulo 2^32) instead of ranks;
// needs the in-place first level (L.readonly false).
lrcc_status lr_enqueue_rs(Ctx* c, cudaStream_t s, const int32_t* succ, int64_t n, int32_t head,
                          int32_t* rank, const Plan& p, const RsLayout& L, const int32_t* val = nullptr,
                          const BatchUnion* U = nullptr, const int32_t* given = nullptr, int64_t given_r = 0);
// Weighted ranks of a forest of lists (ruling set with the heads as extra
// splitters; pointer jumping when the values rule that out).
size_t lr_scan_forest_ws(int64_t n, const Plan& p);
lrcc_status lr_enqueue_scan_forest(Ctx* c, cudaStream_t s, const int32_t* succ, const int32_t* val, int64_t n,
                                   int32_t* out, const Plan& p);
cudaError_t wait_check_enqueue(DevCtl* ctl, int polls, cudaStream_t s);
lrcc_status lr_enqueue_wyllie(Ctx* c, cudaStream_t s, const int32_t* succ, int64_t n, int32_t head,
                              int32_t* rank, const Plan& p);
size_t lr_wyllie_ws(int64_t n, const Plan& p);
// Dependent reads of succ without the walk's work (the walk's ceiling).
lrcc_status rs_chase_probe_run(Ctx* c, const int32_t* succ, int64_t n, int64_t chains, int64_t steps,
                               int64_t* out);

// --- connected components (cc.cu)
lrcc_status cc_run(Ctx* c, const int32_t* src, const int32_t* dst, int64_t m, int64_t n,
                   int32_t* label, const Plan& p);
int64_t cc_active_cap(int64_t m);
// The hook pass's edge stream and parent gathers without the hooking (a ceiling).
lrcc_status cc_gather_probe_run(Ctx* c, const int32_t* src, const int32_t* dst, int64_t m, const int32_t* table,
                                int64_t n, int64_t* out);
size_t cc_ws(int64_t m);
// The Shiloach-Vishkin round structure (plan.cc_hook = 4): workspace, run, round bound.
size_t cc_sv_ws(int64_t n);
lrcc_status cc_run_sv(Ctx* c, const int32_t* src, const int32_t* dst, int64_t m, int64_t n, int32_t* label,
                      const Plan& p);
int sv_round_bound(int64_t n);

// --- batched (batch.cu)
lrcc_status lr_batched_run(Ctx* c, const int32_t* succ, const int64_t* off, const int32_t* heads,
                           int64_t count, int32_t* rank, int64_t total_nodes, const Plan& p);
lrcc_status cc_batched_run(Ctx* c, const int32_t* src, const int32_t* dst, const int64_t* eoff,
                           const int64_t* voff, int64_t count, int64_t total_edges, int32_t* label, const Plan& p);
size_t lr_batched_ws(int64_t total_nodes, int64_t count);
// Batched lists of at least 2^22 elements in all whose batched plan (looked up
// by the total) has the read-only first level are ranked together as one list.
bool batch_union_applies(int64_t total, const Plan& batch_plan);
size_t lr_batched_union_ws(Ctx* c, int64_t total, int64_t K);
lrcc_status lr_batched_union(Ctx* c, cudaStream_t s, const int32_t* succ, const int64_t* off, const int32_t* heads,
                             int64_t K, int64_t total, int32_t* rank);
size_t cc_batched_ws(int64_t count, int64_t total_edges);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace lrcc
