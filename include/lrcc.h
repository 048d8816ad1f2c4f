/*
 * lrcc — list ranking and connected components on NVIDIA GB300 (sm_103a).
 *
 * C ABI of liblrcc.so. Every array argument is a DEVICE pointer owned by the
 * caller; inputs are read only and never modified; outputs are written in
 * full. Calls are asynchronous on `stream` (a cudaStream_t passed as void*,
 * NULL = the legacy default stream): a call returns once its work is
 * enqueued. Node and vertex ids are int32 (at most 2^31 - 2 of them); counts
 * are int64 so that batched totals may exceed 2^31.
 *
 * Errors. Argument errors that the host can see (a NULL pointer with a
 * non-zero size, a negative size, a head outside [0, n), a size above the
 * id range) return at once and enqueue nothing. Errors that only the device
 * can see (the input is not a single list, an id is out of range, the
 * component loop hit its round cap) are recorded in a status word that
 * belongs to the stream; lrcc_last_status() waits for the stream and returns
 * and clears it. After any error the outputs are undefined.
 *
 * Workspace. The library keeps one workspace per (device, stream): it is
 * allocated with cudaMalloc on the first call that needs it, grown when a
 * later call needs more, and freed by lrcc_release(stream). Calls on the same
 * stream share it safely because they are ordered; calls on different streams
 * use different workspaces. The first call on a stream therefore allocates
 * and must not be made during stream capture.
 */
#ifndef LRCC_H
#define LRCC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lrcc_status {
    LRCC_OK = 0,
    LRCC_ERR_ARG = 1,            /* bad argument, detected on the host */
    LRCC_ERR_NOMEM = 2,          /* workspace allocation failed */
    LRCC_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    LRCC_ERR_INVALID_INPUT = 4,  /* not a list / id out of range, detected on the device */
    LRCC_ERR_NOT_CONVERGED = 5,  /* the component loop reached its round cap */
    LRCC_ERR_TIMEOUT = 6         /* a bounded device-side wait gave up */
} lrcc_status;

/* Human-readable name of a status code. Never NULL. */
const char* lrcc_status_str(lrcc_status status);

/* ABI version of this header (major * 100 + minor). */
int lrcc_version(void);

/*
 * List ranking (Sec. 3 of Dehne & Yogaratnam, "Exploring the Limits of GPUs
 * With Parallel Graph Algorithms"): the list is stored as a successor array;
 * the rank of an element is its distance to the last element of the list.
 *
 *   succ  int32[n]  successor of each element; the tail has succ = -1 (the
 *                   paper's convention succ[j] = j is accepted as a tail too)
 *   n              number of elements; the input must be ONE list holding
 *                   all n elements, otherwise LRCC_ERR_INVALID_INPUT is
 *                   recorded on the stream
 *   head            index of the first element, in [0, n)
 *   rank  int32[n]  output: rank[i] = number of links from i to the tail
 *                   (head: n - 1, tail: 0)
 *
 * lr_rank uses the sparse ruling set / random splitter method (Sec. 3.2,
 * Algorithm 2 and Algorithm 3): random splitters cut the list into sublists,
 * each sublist is walked once, the list of splitters is ranked recursively
 * and the ranks are expanded back. Expected work O(n).
 */
lrcc_status lr_rank(const int32_t* succ, int64_t n, int32_t head, int32_t* rank, void* stream);

/*
 * Same contract, computed by Wyllie's pointer jumping (Sec. 3.1,
 * Algorithm 1): ceil(log2 n) rounds of rank[i] += rank[succ[i]],
 * succ[i] = succ[succ[i]] over packed 64-bit (rank, successor) words.
 * O(n log n) work; kept as the baseline the paper compares against.
 */
lrcc_status lr_rank_wyllie(const int32_t* succ, int64_t n, int32_t head, int32_t* rank, void* stream);

/*
 * List ranking with the first-level splitters chosen by the caller: the
 * paper's comparison of random splitters with a perfect set of even splitters
 * that cut the list into sublists of equal length (Sec. 3.2, Table 3).
 *
 *   succ, n, head, rank   as for lr_rank
 *   spl   int32[r]        device array of distinct element ids; spl[0] must be
 *                         head; spl[j] becomes splitter j
 *   r                     1 <= r <= n
 *
 * The first level is the in-place one (64-bit words, plan rs_level0 = 1),
 * whose packed words carry the splitter marks, so the given splitters cost
 * the walk nothing extra; the deeper levels choose their splitters as
 * lr_rank does. Lists of at most the plan's rs_small elements are ranked in
 * one block and do not use spl. An id out of range, an id given twice or
 * spl[0] != head records LRCC_ERR_INVALID_INPUT. The ranks do not depend on
 * the splitters.
 */
lrcc_status lr_rank_splitters(const int32_t* succ, int64_t n, int32_t head, const int32_t* spl, int64_t r,
                              int32_t* rank, void* stream);

/*
 * List ranking for callers that cannot allocate device memory: code whose
 * device memory is fixed up front (a framework that owns the allocator, a
 * service that only uses memory reserved at start-up, a loop where a
 * cudaMalloc could stall or fail). There is no counterpart in the paper; it
 * is lr_rank's method with its scratch in a fixed file-scope device array.
 *
 * Same arguments as lr_rank, with n <= 2^20 (larger n returns LRCC_ERR_ARG
 * at once). The call allocates nothing. Its scratch (about 10 MiB) is held by
 * a GPU until the process exits; the first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) and should be made before any
 * stream capture. Under CUDA's default lazy module loading that lookup is what
 * loads the library's device code onto the device, so the 10 MiB are committed
 * during the first call on each device (which can then fail for lack of
 * memory), not when the library is loaded: make one warm-up call per device
 * during set-up, or run with CUDA_MODULE_LOADING=EAGER. All calls on a device share
 * the array, so calls whose work overlaps on the GPU race: order them (one
 * stream). An input that is not a single list sets rank[head] = -1 (the
 * stream's status word is not used). Returns LRCC_ERR_ARG while phase timing
 * (lrcc_set_timing) is on, because timing creates CUDA events.
 */
lrcc_status lr_rank_noalloc(const int32_t* succ, int64_t n, int32_t head, int32_t* rank, void* stream);

/*
 * Weighted list ranking (Sec. 3.2 notes that the method generalises by
 * replacing each sublist's length with the sum of its values).
 *
 *   succ, head   one list, as for lr_rank
 *   val  int32[n]  a value per element
 *   out  int32[n]  output: out[i] = sum of val[j] over the elements j from i
 *                  to the tail, both included. With val = 1, out = rank + 1.
 *
 * Same method as lr_rank (the walk sums values instead of counting), always
 * with the in-place first level. The partial sums live in the 31-bit fields of
 * the packed walk words, so the values must be non-negative with a total
 * below 2^31; otherwise the call records LRCC_ERR_INVALID_INPUT (and leaves
 * out undefined). Other errors as for lr_rank.
 */
lrcc_status lr_scan(const int32_t* succ, const int32_t* val, int64_t n, int32_t head, int32_t* out,
                    void* stream);

/*
 * Weighted list ranking of a forest of lists: succ holds any number of
 * disjoint lists covering all n elements (tails -1 or self-loops; no head is
 * given), and out[i] is the sum of val from i to the tail of i's own list,
 * modulo 2^32. The heads (elements no successor names) become extra splitters
 * of the ruling set's first level, and the much smaller forest of splitters is
 * summed by pointer jumping (Sec. 3.1). When a value is negative or the values
 * total 2^31 or more, the whole forest is summed by pointer jumping instead
 * (O(n log n) work, any values). An element named by two successors, a cycle
 * or a successor out of range records LRCC_ERR_INVALID_INPUT. Workspace: 37 to
 * 40 bytes per element (the first level is sized for every element a head).
 */
lrcc_status lr_scan_forest(const int32_t* succ, const int32_t* val, int64_t n, int32_t* out, void* stream);

/*
 * Connected components (Sec. 4, Algorithm 4, after Shiloach and Vishkin) of
 * an undirected graph given as an edge list.
 *
 *   src, dst  int32[m]  edge e joins src[e] and dst[e]; ids in [0, n);
 *                       self-loops and repeated edges are allowed
 *   m, n                edge and vertex counts
 *   label     int32[n]  output: the smallest vertex id of the component of
 *                       each vertex. It is also the working parent array.
 *
 * Method: parent[v] = v; then rounds of hooking (for every edge whose
 * endpoints have different roots, atomicMin links the larger root below the
 * smaller) and shortcutting (pointer jumping until every tree is a star),
 * until a hook pass finds no edge joining two roots. The round count is
 * capped; reaching the cap records LRCC_ERR_NOT_CONVERGED.
 */
lrcc_status cc_label(const int32_t* src, const int32_t* dst, int64_t m, int64_t n,
                     int32_t* label, void* stream);

/*
 * Host-buffer forms of lr_rank and cc_label: the same arguments and results,
 * with every array (succ and rank; src, dst and label) in HOST memory. The
 * call copies the inputs into device staging owned by the stream's context,
 * runs the device method, and copies the result back, ordered after the
 * stream's earlier work and before its later work. The copies run on two
 * copy streams the library keeps per device (uploads, downloads), so calls
 * queued on different streams pipeline: one call's upload runs at full
 * bandwidth while another call's kernels run. The call returns once the work
 * is queued: the output is valid, and the inputs may be changed or freed,
 * only after `stream` has been synchronised. Not for use inside a stream
 * capture. Page-locked host buffers (cudaHostAlloc / pinned) make both
 * copies asynchronous; pageable buffers also work, with copies the driver
 * stages itself. The staging (8 bytes per list element; 8 bytes per edge plus
 * 4 per vertex) stays allocated until lrcc_release. Device-detected errors
 * are reported through lrcc_last_status as for the device forms.
 */
lrcc_status lr_rank_host(const int32_t* succ, int64_t n, int32_t head, int32_t* rank, void* stream);
lrcc_status cc_label_host(const int32_t* src, const int32_t* dst, int64_t m, int64_t n,
                          int32_t* label, void* stream);

/*
 * Batched list ranking: num_lists independent lists in one launch (a
 * persistent kernel takes the lists from a device work queue, largest first;
 * each list is ranked by one thread block).
 * List k owns elements [node_off[k], node_off[k+1]) of succ and rank;
 * succ values and heads[k] are LOCAL ids (0-based within list k), and the
 * ranks are local too. node_off is int64[num_lists + 1] on the device,
 * non-decreasing, node_off[0] = 0. Every list must be valid.
 */
lrcc_status lr_rank_batched(const int32_t* succ, const int64_t* node_off, const int32_t* heads,
                            int64_t num_lists, int32_t* rank, void* stream);

/*
 * lr_rank_batched sizes its workspace from node_off[num_lists], which it
 * reads back with a small copy that waits for `stream`. Callers that know
 * the total element count pass it here instead and the call stays
 * asynchronous (total_nodes must equal node_off[num_lists]).
 */
lrcc_status lr_rank_batched_sized(const int32_t* succ, const int64_t* node_off, const int32_t* heads,
                                  int64_t num_lists, int64_t total_nodes, int32_t* rank, void* stream);

/*
 * Batched connected components: num_graphs independent graphs in one launch
 * (a persistent kernel, one thread block per graph, largest first).
 * Graph k owns edges [edge_off[k], edge_off[k+1]) of src/dst and vertices
 * [vert_off[k], vert_off[k+1]) of label; edge endpoints and labels are LOCAL
 * ids. Offsets are int64[num_graphs + 1] on the device, non-decreasing, 0 first.
 */
lrcc_status cc_label_batched(const int32_t* src, const int32_t* dst, const int64_t* edge_off,
                             const int64_t* vert_off, int64_t num_graphs, int32_t* label,
                             void* stream);

/*
 * cc_label_batched reads edge_off[num_graphs] back (a small copy that waits
 * for `stream`) to size its buffers; with the total edge count given here
 * the call stays asynchronous (total_edges must equal edge_off[num_graphs]).
 */
lrcc_status cc_label_batched_sized(const int32_t* src, const int32_t* dst, const int64_t* edge_off,
                                   const int64_t* vert_off, int64_t num_graphs, int64_t total_edges,
                                   int32_t* label, void* stream);

/*
 * Waits for `stream`, then returns and clears the device status word of its
 * workspace (LRCC_OK if nothing was recorded since the last call).
 */
lrcc_status lrcc_last_status(void* stream);

/*
 * Check of the device-side timeout path: runs, on `stream`, the bounded wait
 * that guards the bulk copies of lr_rank's read-only first level, on a barrier
 * that no copy completes. After `polls` polls (1 to 2^20; others return
 * LRCC_ERR_ARG) the wait gives up and records LRCC_ERR_TIMEOUT on the stream,
 * as a copy that never lands would; the context stays usable. Allocates
 * nothing beyond the stream's status word.
 */
lrcc_status lrcc_wait_check(int polls, void* stream);

/*
 * Measurement aid: the memory traffic of one components hook pass without its
 * work. Streams the edge list (src, dst: int32[m], device) as the hook pass
 * does and gathers table[src[e]] and table[dst[e]] for every edge from a
 * device table of n int32 (the parent array's size and cache policy); the
 * wrapped sum of the gathered values goes to *out (a device int64), so no
 * load is dropped. Ids outside [0, n) gather entry 0. Asynchronous on
 * `stream`; allocates nothing beyond the stream's status word.
 */
lrcc_status lrcc_gather_probe(const int32_t* src, const int32_t* dst, int64_t m, const int32_t* table, int64_t n,
                              int64_t* out, void* stream);

/*
 * Measurement aid: the access pattern of the first-level sublist walk (Sec. 3.2,
 * RS3) without its work. `chains` chains of dependent reads over succ (int32[n],
 * device): chain c starts at element floor(c * n / chains) and reads `steps`
 * successors one after the other, with the walk's load form; a chain that
 * reaches a tail (-1 or a self-loop) or an id outside [0, n) continues from a
 * hashed element, which costs no read. The wrapped sum of the elements reached
 * goes to *out (a device int64), so no load is dropped. n in [1, 2^31 - 1],
 * chains in [1, 2^31], steps >= 0 (LRCC_ERR_ARG otherwise). Asynchronous on
 * `stream`; allocates nothing beyond the stream's status word.
 */
lrcc_status lrcc_chase_probe(const int32_t* succ, int64_t n, int64_t chains, int64_t steps, int64_t* out,
                             void* stream);

/*
 * Fault injection on the host, for testing a caller's out-of-memory handling:
 * the next `count` device allocations the library makes (workspaces, host-call
 * staging) fail as if cudaMalloc had, and the calls that needed them return
 * LRCC_ERR_NOMEM without enqueueing work. count <= 0 clears it. Returns the
 * count that was pending. Nothing is done on the device.
 */
int lrcc_debug_fail_allocs(int count);

/* Statistics of the most recent call on `stream` (waits for the stream). */
typedef struct lrcc_stats {
    int32_t kind;            /* 1 = lr_rank, 2 = lr_rank_wyllie, 3 = cc_label, 4/5 = batched,
                                6 = lr_scan, 7 = lr_scan_forest */
    int32_t levels;          /* lr_rank: ruling-set levels before the one-block rank */
    int64_t splitters[8];    /* lr_rank: splitters chosen at each level */
    int32_t rounds;          /* cc_label: hook passes (including the final, quiet one) */
    int32_t jump_rounds;     /* lr_rank_wyllie: pointer-jumping rounds */
    int64_t overflow_chunks; /* lr_rank, read-only first level: 8-element chunks that did not fit
                                their walk block's region and went to the shared overflow pool */
    int64_t edges_read;      /* cc_label (hook rules 1-3): edges read by all hook passes, the
                                sample pass and the compacted active edges included */
} lrcc_stats;
lrcc_status lrcc_last_stats(void* stream, lrcc_stats* out);

/*
 * Tuning knobs (a process-wide table indexed by ceil(log2 n)). Any field set
 * to 0 keeps the library's default for that field.
 */
typedef struct lrcc_plan {
    int32_t rs_spacing0;     /* mean sublist length at the first ruling-set level */
    int32_t rs_spacing;      /* mean sublist length at deeper levels */
    int32_t rs_small;        /* lists of at most this many elements are ranked by one block */
    int32_t rs_chains;       /* sublist walks interleaved per thread: 1, 2 or 4 */
    int32_t cc_hook;         /* 1 = one atomicMin per edge and pass, 2 = re-link until joined,
                                3 = rule 1 in the first pass, rule 2 after, 4 = the
                                Shiloach-Vishkin rounds themselves (shortcut, mark, conditional
                                and stagnant-tree hooking, shortcut, check; Sec. 4 SV0-SV5),
                                5 = rule 1 after a first pass that gathers no parents: each
                                edge links its endpoints by atomicMin and carries every link
                                the atomic displaces on, so that pass joins every edge it
                                reads; same labels; batched calls treat 4 as 1, and their
                                graphs of at most 2^15 vertices, labelled inside one block,
                                re-link until joined whatever the rule */
    int32_t cc_max_rounds;   /* cap on hook passes (-1 = back to the automatic cap) */
    int32_t use_graphs;      /* 1 = replay captured CUDA graphs, 2 = plain launches */
    int32_t rs_level0;       /* first ruling-set level: 1 = the walk rewrites 8-byte words in
                                place; 2 = the walk only reads succ and writes what it visits
                                as 32-byte chunks, which are turned into ranks by a scatter
                                into id-range buckets and a placement pass; 3 = the walk
                                reads succ and keeps an ownership mark (16 bits below 65,535
                                splitters, else 32) and a local rank in two arrays (the
                                paper's "48 bit" form, Sec. 3.2). lr_scan and lr_scan_forest
                                always use 1 */
    uint64_t seed;           /* splitter seed (results do not depend on it) */
    int32_t cc_sample;       /* components: before the first pass over all edges, one hook pass
                                and shortcut over the first m / cc_sample edges (a sample that
                                forms most of the large components cheaply); 1 = no sample pass,
                                -1 = automatic (about one sampled edge per vertex on graphs with
                                at least 8 edges per vertex, two with 4 to 7, no sample below) */
} lrcc_plan;

/* kind: 1 = list ranking, 2 = its Wyllie form, 3 = connected components of
 * graphs with at least 4 edges per vertex, 8 = connected components of graphs
 * with fewer (m < 4n), 4 / 5 = the batched calls; sizes with ceil(log2 n) in
 * [log2_lo, log2_hi] get `plan`. */
lrcc_status lrcc_set_plan(int kind, int log2_lo, int log2_hi, const lrcc_plan* plan);
lrcc_status lrcc_get_plan(int kind, int64_t n, lrcc_plan* out);
/* Restores the built-in plan table (undoing every lrcc_set_plan). */
lrcc_status lrcc_reset_plans(void);

/*
 * Phase timing. While enabled (process-wide), list-ranking calls launch their
 * kernels directly (no graph replay) and record a pair of CUDA events around
 * every kernel on the caller's stream; component calls record events around
 * the initialisation and around the whole device-side hook/shortcut loop.
 * lrcc_phase_times() waits for `stream`, adds the elapsed time and launch
 * count of every phase recorded since the previous query into ms_total[p]
 * and launches[p] (arrays of at least lrcc_phase_count() entries) and
 * forgets the recorded events.
 */
lrcc_status lrcc_set_timing(int enable);
int lrcc_phase_count(void);
const char* lrcc_phase_name(int phase);
lrcc_status lrcc_phase_times(void* stream, double* ms_total, int64_t* launches);

/*
 * L2 fetch granularity of the current device's context, in bytes (32, 64 or
 * 128; 0 = leave the driver's default). Random 4- and 8-byte gathers over
 * arrays larger than L2 (the sublist walk, the hook's parent reads) move a
 * whole fetch unit from HBM per access, so a 32-byte unit cuts their DRAM
 * traffic. It is a hint the driver may clamp, it applies to every kernel of
 * the process on that device (not only this library's), and it ends with the
 * process. lrcc_get_l2_fetch_granularity returns the current value or -1.
 */
lrcc_status lrcc_set_l2_fetch_granularity(int bytes);
int lrcc_get_l2_fetch_granularity(void);

/*
 * Contexts: an explicit handle on the library's workspaces of one device, for
 * callers that account for device memory themselves (a serving loop with a
 * memory budget). The compute calls above keep taking only a stream; the
 * state a call uses is the workspace of (current device, stream). A context
 * adopts the workspaces of the streams it reserves for, so that their bytes
 * can be counted and freed together.
 *
 * lrcc_ctx_create     a context for `device` (0 .. device count - 1); nothing is
 *                     allocated until a reservation. LRCC_ERR_ARG for a bad device.
 * lrcc_ctx_reserve    allocates the workspace of (ctx's device, stream) now, at
 *                     least `bytes` large (lrcc_workspace_query gives the bytes a
 *                     call needs), so that later calls on that stream of up to
 *                     that size allocate nothing; it waits for the stream when an
 *                     existing workspace has to grow. LRCC_ERR_NOMEM when the
 *                     allocation fails (the stream keeps no workspace then).
 * lrcc_ctx_bytes      device bytes held by the workspaces the context adopted
 *                     (kernel workspace, host-call staging and the status word of
 *                     each stream, including growth by later calls); -1 for NULL.
 * lrcc_ctx_last_status  lrcc_last_status for `stream` on the context's device.
 * lrcc_ctx_destroy    waits for each adopted stream and frees its workspace and
 *                     cached graphs, then the handle. NULL is ignored.
 * The device is made current only for the duration of each call.
 */
typedef struct lrcc_ctx lrcc_ctx;
lrcc_status lrcc_ctx_create(lrcc_ctx** ctx, int device);
lrcc_status lrcc_ctx_reserve(lrcc_ctx* ctx, void* stream, int64_t bytes);
int64_t lrcc_ctx_bytes(lrcc_ctx* ctx);
lrcc_status lrcc_ctx_last_status(lrcc_ctx* ctx, void* stream);
void lrcc_ctx_destroy(lrcc_ctx* ctx);

/* Frees the workspace and cached graphs of `stream` (waits for it first). */
lrcc_status lrcc_release(void* stream);

/* Bytes of device workspace (and host-call staging) currently held by the library (all streams). */
int64_t lrcc_workspace_bytes(void);

/* Device workspace a call of the given kind and size would need (kinds as
 * in lrcc_stats; batched lists: n = total elements, m = lists; batched graphs:
 * n = total edges, m = graphs; 6 = lr_scan, 7 = lr_scan_forest). */
int64_t lrcc_workspace_query(int kind, int64_t n, int64_t m);

#ifdef __cplusplus
}
#endif

#endif /* LRCC_H */
