// Wyllie's pointer jumping inside one thread block, on arrays in shared memory
// (Sec. 3.1: the single-kernel variant that synchronises with __syncthreads).
#pragma once

#include "common.cuh"

namespace lrcc {

// val[j] += val[nxt[j]], nxt[j] = nxt[nxt[j]] for every j < r until no link
// is left; on return val[j] is the sum of val over j and every element after
// it (modulo 2^32). THREADS threads each own PER elements (r <= PER * THREADS). Rounds are
// capped at ceil(log2 r) + 2; a list that still has links then contains a
// cycle, which is recorded as invalid input.
template <int PER, int THREADS>
__device__ void block_wyllie(int* val, int* nxt, int r, DevCtl* ctl) {
    const int tid = threadIdx.x;
    int cap = 2;
    while ((1 << (cap - 2)) < r) ++cap;
    for (int round = 0;; ++round) {
        int nv[PER], nn[PER];
        bool any = false;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int j = tid + q * THREADS;
            nv[q] = 0;
            nn[q] = (int)NIL;
            if (j < r) {
                const int x = nxt[j];
                nv[q] = val[j];
                if (x != (int)NIL) {
                    nv[q] = (int)((unsigned)nv[q] + (unsigned)val[x]);   // sums modulo 2^32
                    nn[q] = nxt[x];
                    any = true;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int j = tid + q * THREADS;
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

}  // namespace lrcc
