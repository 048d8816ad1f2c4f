// Device functions of the component kernels (hooking and root finding),
// shared by the single-instance and batched paths.
#pragma once

#include "common.cuh"

namespace lrcc {

// Chases of the shortcut passes: steps taken through L1 without writing
// before a chase switches to its deep mode (see chase_step). 4, 16 and 64 all
// label the bench graphs in the same time; 16 is a little faster on a path of
// 2^24 consecutive ids (0.97 against 1.01 and 1.22 ms).
#ifndef LRCC_CHASE_QUIET
#define LRCC_CHASE_QUIET 16
#endif
constexpr int CHASE_QUIET = LRCC_CHASE_QUIET;

// One step of a shortcut chase of vertex v, now at ancestor x: returns x's
// parent. Roots do not move while a shortcut pass runs and every value read
// is an ancestor, so the first CHASE_QUIET steps read through L1 (the hot
// roots of large trees then hit L1 instead of queueing on one L2 slice) and
// write nothing: trees after a hook pass are mostly stars. Deeper chases read
// through L2 and store the ancestor reached in parent[v] (v's own entry, which
// no other thread writes during the pass), so that chases passing through v
// jump ahead. On a chain of n links, such as a path whose edges join
// consecutive ids (every vertex hooked below its predecessor), the chases of
// a pass then double their reach at every step, O(log n) steps each; chases
// that stored only the root they reached took about sqrt(2n) steps each when
// all advance together and more when they do not (a path of 2^24 consecutive
// ids: 487 ms against 0.97 ms with the progress stores).
__device__ __forceinline__ int32_t chase_step(int32_t* parent, int32_t v, int32_t x, int step, uint64_t keep) {
    if (step < CHASE_QUIET) return ld_hint(parent + x, keep);
    const int32_t nx = ld_cg_hint(parent + x, keep);
    if (nx != x) parent[v] = nx;
    return nx;
}

// Root of vertex v whose parent is p, by chase_step. Every link goes to a
// smaller id, so the chase ends within n steps on any state the kernels can
// produce.
__device__ __forceinline__ int32_t chase_root(int32_t* parent, int32_t v, int32_t p, uint64_t keep) {
    int32_t x = p;
    for (int step = 0;; ++step) {
        const int32_t nx = chase_step(parent, v, x, step, keep);
        if (nx == x) return x;
        x = nx;
    }
}

// Root of x with path halving: each visited element is re-pointed to its
// grandparent. The store may race with an atomicMin on the same element;
// either value is an ancestor, and a link that such a store replaces is
// re-made by the thread whose atomicMin saw it (it goes on to join the old
// parent with its smaller root), so no connection is lost.
__device__ __forceinline__ int32_t find_root_halving(int32_t* parent, int32_t x, uint64_t keep) {
    int32_t p = ld_cg_hint(parent + x, keep);
    while (p != x) {
        const int32_t g = ld_cg_hint(parent + p, keep);
        if (g == p) return p;
        parent[x] = g;
        x = g;
        p = ld_cg_hint(parent + x, keep);
    }
    return x;
}

// One edge whose endpoints currently have parents a and b.
//  relink = false: a single atomicMin links the larger parent below the
//                  smaller one (one Shiloach-Vishkin style hook);
//  relink = true:  both ends are followed to their roots; when the atomicMin
//                  finds the larger root already linked below `old` by
//                  another thread, the join continues with (old, smaller
//                  root), so the edge's endpoints share a tree when it returns.
// Returns whether a link was written.
__device__ __forceinline__ bool hook_pair(int32_t* parent, int32_t a, int32_t b, bool relink, uint64_t keep) {
    if (a == b) return false;
    if (!relink) {
        // Read before the atomic: on hubs most hooks find the parent already
        // at or below `lo`, and skipping those keeps same-address atomics
        // from serialising in L2.
        const int32_t hi = max(a, b), lo = min(a, b);
        if (ld_cg_hint(parent + hi, keep) > lo) atomicMin(parent + hi, lo);
        return true;
    }
    bool linked = false;
    for (;;) {
        a = find_root_halving(parent, a, keep);
        b = find_root_halving(parent, b, keep);
        if (a == b) return linked;
        const int32_t hi = max(a, b), lo = min(a, b);
        const int32_t old = atomicMin(parent + hi, lo);
        linked = true;
        if (old == hi) return true;
        // hi had been linked below `old` by another thread: join old and lo
        a = old;
        b = lo;
    }
}

// One edge (x, y) in a first pass, when no parent has been read: the
// endpoints themselves are linked. atomicMin(&parent[hi], lo) returns hi's
// parent before the call. If that was hi, hi was a root and now hangs below
// lo: the edge is joined. Otherwise hi hung below `old` and now hangs below
// min(old, lo), so the join goes on with (old, lo): the link the atomic may
// have replaced is made again further up, and no connection is lost. The
// larger id falls at every step, so the loop ends. A read before each atomic
// skips it when the parent is already at or below lo (on hubs most are),
// with the same continuation. Returns whether a parent was lowered.
__device__ __forceinline__ bool link_direct(int32_t* parent, int32_t x, int32_t y, uint64_t keep) {
    bool lowered = false;
    while (x != y) {
        const int32_t hi = max(x, y), lo = min(x, y);
        int32_t old = ld_cg_hint(parent + hi, keep);
        if (old > lo) {
            old = atomicMin(parent + hi, lo);
            if (old > lo) lowered = true;
            if (old == hi) break;
        }
        x = old;
        y = lo;
    }
    return lowered;
}

// Exclusive prefix over the warp of a per-lane count in [0, 15], and the warp
// total, from four ballots (one per bit) instead of a shuffle scan: ballots do
// not queue on the memory pipe that the gathers of a hook pass keep busy.
__device__ __forceinline__ int warp_prefix_small(int cnt, int* total) {
    const unsigned lt = lanemask_lt();
    int excl = 0, all = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const unsigned m = __ballot_sync(0xffffffffu, (cnt >> b) & 1);
        excl += __popc(m & lt) << b;
        all += __popc(m) << b;
    }
    *total = all;
    return excl;
}

}  // namespace lrcc
