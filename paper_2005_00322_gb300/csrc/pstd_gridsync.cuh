// pstd_gridsync.cuh -- software barrier of all CTAs of a cooperative launch.
//
// The CTAs of a cooperative launch are all resident, so they can meet at a
// barrier in global memory.  Every wait is bounded: after `spin_limit` polls
// the waiting CTA writes a non-zero status word and returns false, and every
// other CTA sees the status at its next poll and returns false too, so a
// stall ends the kernel with an error the host can read and leaves the
// context usable.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pstd {

// Member of batch work item `it` of one pass, whose members own the item
// ranges prefix[m] .. prefix[m + 1] - 1: the last m with prefix[m] <= it
// (members with no items are skipped over).
__host__ __device__ inline int member_of(const int64_t* prefix, int members, int64_t it) {
    int lo = 0, hi = members - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= it) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct GridSync {
    unsigned* count;         // arrivals at the current barrier
    unsigned* gen;           // barrier generation
    int* status;             // 0 ok, 1 a wait gave up
    unsigned expected;       // arrivals that release a barrier (gridDim.x, more to test a stall)
    long long spin_limit;    // polls before giving up
};

#ifdef __CUDA_ARCH__
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_acquire_i(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Barrier of all CTAs of the launch; false if a bounded wait gave up (here or
// in another CTA).  All threads of every CTA must call it.
__device__ bool grid_sync(const GridSync& g) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned my_gen = ld_acquire(g.gen);
        __threadfence();
        const unsigned arrived = atomicAdd(g.count, 1u) + 1u;
        if (arrived == g.expected) {
            atomicExch(g.count, 0u);
            __threadfence();
            atomicAdd(g.gen, 1u);
        } else {
            long long spins = 0;
            while (ld_acquire(g.gen) == my_gen) {
                if (ld_acquire_i(g.status) != 0 || ++spins > g.spin_limit) {
                    atomicExch(g.status, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}
#endif

}  // namespace pstd
