// pstd_persist.cuh -- one cooperative kernel for a whole run of leapfrog steps.
//
// The CTAs of a cooperative launch are all resident, so they can meet at a
// software grid barrier between axis passes instead of at kernel boundaries:
// each step runs the axis passes last axis first (as the per-axis kernels do),
// every CTA taking work items (line-pair groups or tiles) blockIdx.x,
// blockIdx.x + gridDim.x, ..., and all CTAs meeting at the barrier after each
// pass.  Every wait at the barrier is bounded: after `spin_limit` polls the
// waiting CTA writes a non-zero status word and returns, and every other CTA
// sees the status at its next poll and returns too, so a stall ends the kernel
// with an error the host can read (pstd_sync -> PSTD_ETIMEOUT) and leaves the
// context usable.
#pragma once

#include "pstd_wcta.cuh"

namespace pstd {

struct GridSync {
    unsigned* count;         // arrivals at the current barrier
    unsigned* gen;           // barrier generation
    int* status;             // 0 ok, 1 a wait gave up
    unsigned expected;       // arrivals that release a barrier (gridDim.x, more to test a stall)
    long long spin_limit;    // polls before giving up
};

struct PersistArgs {
    WStep ax[3];
    int strided[3];
    int64_t items[3];        // work items of each axis pass
    int ndim;
    int64_t nsteps;
    GridSync sync;
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

template <class S>
__device__ void persistent_run(const PersistArgs& a, float2* smem) {
#ifdef __CUDA_ARCH__
    for (int64_t s = 0; s < a.nsteps; ++s) {
        for (int ax = a.ndim - 1; ax >= 0; --ax) {
            for (int64_t it = blockIdx.x; it < a.items[ax]; it += gridDim.x) {
                if (a.strided[ax]) wk::step_strided<S>(a.ax[ax], it, smem, threadIdx.x, blockDim.x);
                else wk::step_contig<S>(a.ax[ax], it, smem, threadIdx.x, blockDim.x);
                __syncthreads();     // shared memory is reused by the next item
            }
            if (!grid_sync(a.sync)) return;
        }
    }
#endif
}

}  // namespace pstd
