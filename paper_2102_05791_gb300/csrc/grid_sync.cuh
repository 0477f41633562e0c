// Grid-wide barrier for cooperative launches (all CTAs co-resident), and the
// cluster barrier and distributed-shared-memory loads for one-cluster grids.
#pragma once

#include <cstdint>
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

// Thread-block cluster primitives (the whole grid is one cluster of at most
// 16 CTAs): a hardware barrier over every thread of the cluster with
// release/acquire semantics at cluster scope, and loads from another CTA's
// shared memory (distributed shared memory).
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address of the same shared-memory object in the CTA of the given cluster rank.
__device__ __forceinline__ uint32_t dsmem_addr(const void *local, uint32_t rank)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(local);
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

__device__ __forceinline__ float2 ld_dsmem_f2(const void *local, uint32_t rank)
{
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(dsmem_addr(local, rank))
                 : "memory");
    return v;
}

__device__ __forceinline__ double ld_dsmem_f64(const void *local, uint32_t rank)
{
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(dsmem_addr(local, rank)) : "memory");
    return v;
}

__device__ __forceinline__ int ld_dsmem_s32(const void *local, uint32_t rank)
{
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(dsmem_addr(local, rank)) : "memory");
    return v;
}

}  // namespace softsim
