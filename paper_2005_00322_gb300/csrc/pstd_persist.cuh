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

#include "pstd_gridsync.cuh"
#include "pstd_wcta.cuh"

namespace pstd {

// One plan (members == 0: the passes in ax / strided / items) or a batch of
// plans on one schedule (members > 0): pass k of a step (k = 0 the last axis)
// is, over all members, prefix[k][members] work items, member m owning items
// prefix[k][m] .. prefix[k][m + 1] - 1 with its pass mem[m * 3 + k].
struct PersistArgs {
    WStep ax[3];
    int strided[3];
    int64_t items[3];        // work items of each axis pass
    int ndim;                // axis passes per step (a batch: the most of any member)
    int64_t nsteps;
    GridSync sync;
    int members;
    const WStep* mem;        // [members][3], device memory
    const int64_t* prefix;   // [3][members + 1], device memory
};

template <class S>
__device__ void persistent_run(const PersistArgs& a, float2* smem) {
#ifdef __CUDA_ARCH__
    for (int64_t s = 0; s < a.nsteps; ++s) {
        for (int k = 0; k < a.ndim; ++k) {
            if (a.members == 0) {
                const int ax = a.ndim - 1 - k;
                for (int64_t it = blockIdx.x; it < a.items[ax]; it += gridDim.x) {
                    if (a.strided[ax]) wk::step_strided<S>(a.ax[ax], it, smem, threadIdx.x, blockDim.x);
                    else wk::step_contig<S>(a.ax[ax], it, smem, threadIdx.x, blockDim.x);
                    __syncthreads();     // shared memory is reused by the next item
                }
            } else {
                const int64_t* pre = a.prefix + (size_t)k * (a.members + 1);
                for (int64_t it = blockIdx.x; it < pre[a.members]; it += gridDim.x) {
                    const int m = member_of(pre, a.members, it);
                    const WStep& w = a.mem[(size_t)m * 3 + k];
                    if (w.ax.inner > 1) wk::step_strided<S>(w, it - pre[m], smem, threadIdx.x, blockDim.x);
                    else wk::step_contig<S>(w, it - pre[m], smem, threadIdx.x, blockDim.x);
                    __syncthreads();
                }
            }
            if (!grid_sync(a.sync)) return;
        }
    }
#endif
}

}  // namespace pstd
