// Grid-wide barrier for cooperative launches (all CTAs co-resident).
#pragma once

#include <cuda_runtime.h>

namespace softsim {

constexpr int kGridWaitPolls = 1 << 22;  // polls (L2 round trips) of one grid-barrier wait before it gives up

// Barrier over all CTAs of a cooperative launch on one 32-bit word (zero
// before the launch): CTA 0 adds 2^31 - (n - 1), every other CTA adds 1, so
// the word's top bit flips exactly once per barrier, when the last CTA
// arrives; a CTA waits until the bit differs from the value it saw when it
// arrived (the next barrier cannot complete before this CTA reaches it).  One
// atomic per CTA; returns false in every thread of the CTA when the wait ran
// out (the caller raises an error flag and leaves; the other CTAs then give
// up at their next barrier).
__device__ __forceinline__ bool grid_barrier(unsigned int *word, unsigned int n_blocks)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int inc = blockIdx.x == 0 ? 0x80000000u - (n_blocks - 1u) : 1u;
        int ok = 1;
        __threadfence();  // this CTA's writes before its arrival
        const unsigned int old = atomicAdd(word, inc);
        volatile unsigned int *vw = word;
        int i = 0;
        while (((old ^ *vw) & 0x80000000u) == 0u) {
            if (++i > kGridWaitPolls) {
                ok = 0;
                break;
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

}  // namespace softsim
