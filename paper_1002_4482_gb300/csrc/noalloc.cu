// lr_rank_noalloc: list ranking for callers that cannot allocate device
// memory.
//
// Who needs it: code whose device memory is budgeted up front and must not
// grow afterwards (an embedding framework that owns the allocator, a long
// running service that only uses memory reserved at start-up, a real-time
// loop where a cudaMalloc could stall or fail), and callers that forbid a
// library to allocate behind their back. lr_rank allocates its workspace on
// the first call on each stream; this variant never does.
//
// How: its scratch (the 8-byte walk words, the deeper ruling-set levels and
// the control block) is one file-scope __device__ array of fixed size that a
// GPU holds, once it has it, until the process exits. Host code cannot use the
// array's name as a device address, so the first call on each device looks
// the address up with cudaGetSymbolAddress while that device is current, and
// passes it to the kernels. With CUDA's default lazy module loading the
// library's device code, this array included, is loaded onto a device at that
// first lookup: the array's memory is committed during the first call on
// each device, not when the library is loaded, and that first call can fail
// for lack of memory (LRCC_ERR_CUDA). A caller with a fixed budget makes one
// warm-up call per device while setting up (or runs with
// CUDA_MODULE_LOADING=EAGER, which loads the module when the context is
// created). That first call should also come before any stream capture. The
// call makes no cudaMalloc, cudaFree, cudaStreamCreate or cudaEventCreate call.
//
// Limits: at most NOALLOC_MAX_N elements. All calls on a device share the one
// array and it keeps the last call's contents: the control counters are
// cleared at the start of every call, everything else is written before it is
// read. Calls whose work overlaps on the GPU (different streams, or threads
// without ordering between them) race on the array and give undefined
// results; order them, e.g. by using one stream.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace lrcc {

namespace {

constexpr int64_t NOALLOC_MAX_N = int64_t(1) << 20;
// The walk words (8 bytes per element), the level-1 and level-2 arrays of the
// fixed plan below, the control block, and alignment slack.
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(10) << 20;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
int g_noalloc_sms[NOALLOC_MAX_DEVICES] = {};

// Fixed plan: in-place first level (no chunk buffers), spacing 16 at every
// level, lists of at most 8192 elements ranked by one block.
Plan noalloc_plan() {
    Plan p;
    p.rs_spacing0 = 16;
    p.rs_spacing = 16;
    p.rs_small = 8192;
    p.rs_chains = 1;
    p.rs_level0 = 1;
    p.use_graphs = 2;
    return p;
}

// Device address of the scratch array on the current device (set up once).
lrcc_status scratch_for(int dev, void** out, int* sms) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return LRCC_ERR_CUDA;
        }
        int n_sm = 0;
        if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LRCC_ERR_CUDA;
        g_noalloc_sms[dev] = n_sm;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    *sms = g_noalloc_sms[dev];
    return LRCC_OK;
}

// A device-detected error is reported through the output: rank[head] = -1
// (a valid list always gives the head rank n - 1).
__global__ void noalloc_report(const DevCtl* ctl, int32_t head, int32_t* rank) {
    if (ctl->status != 0) rank[head] = -1;
}

}  // namespace

}  // namespace lrcc

using namespace lrcc;

extern "C" lrcc_status lr_rank_noalloc(const int32_t* succ, int64_t n, int32_t head, int32_t* rank, void* stream) {
    if (n < 0 || n > NOALLOC_MAX_N) return LRCC_ERR_ARG;
    if (n == 0) return LRCC_OK;
    if (!succ || !rank || head < 0 || head >= n) return LRCC_ERR_ARG;
    // phase timing creates CUDA events on demand, so it cannot be combined
    if (timing_enabled()) return LRCC_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LRCC_ERR_CUDA;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return LRCC_ERR_ARG;
    void* scratch = nullptr;
    int sms = 0;
    lrcc_status st = scratch_for(dev, &scratch, &sms);
    if (st != LRCC_OK) return st;
    const Plan p = noalloc_plan();
    const RsLayout L = rs_layout(n, p, 0);
    const size_t ctl_off = align_up(L.bytes, 256);
    if (ctl_off + sizeof(DevCtl) > NOALLOC_SCRATCH_BYTES) return LRCC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Ctx c;
    c.device = dev;
    c.stream = s;
    c.ws = scratch;
    c.ws_bytes = ctl_off;
    c.sms = sms;
    c.ctl = reinterpret_cast<DevCtl*>(static_cast<char*>(scratch) + ctl_off);
    // counters and the status word must start at zero; the array keeps the
    // previous call's contents
    if (cudaMemsetAsync(c.ctl, 0, sizeof(DevCtl), s) != cudaSuccess) return LRCC_ERR_CUDA;
    st = lr_enqueue_rs(&c, s, succ, n, head, rank, p, L);
    if (st != LRCC_OK) return st;
    noalloc_report<<<1, 1, 0, s>>>(c.ctl, head, rank);
    return cuda_status(cudaGetLastError());
}
