// pstd_kernels.cu -- the device kernels (one CTA program per block) and
// their launchers.
#include "pstd_cta.cuh"
#include "pstd_gridsync.cuh"

namespace pstd {

constexpr int kThreads = 256;

// Fused per-axis leapfrog pass (see pstd_cta.cuh, cta_step).
__global__ void __launch_bounds__(kThreads) k_step(StepArgs a) {
    extern __shared__ float4 smem_f4[];
    cta_step(a, blockIdx.x, smem_f4, threadIdx.x, blockDim.x);
}

// Every member's passes of a whole run in one cooperative kernel: the CTAs
// take the work items of a pass over all members, then meet at the grid
// barrier (bounded waits, see pstd_gridsync.cuh) before the next pass.
__global__ void __launch_bounds__(kThreads) k_step_persist(StepPersistArgs a, GridSync sync) {
#ifdef __CUDA_ARCH__
    extern __shared__ float4 smem_f4[];
    for (int64_t s = 0; s < a.nsteps; ++s) {
        for (int k = 0; k < a.npass; ++k) {
            const int64_t* pre = a.prefix + (size_t)k * (a.members + 1);
            for (int64_t it = blockIdx.x; it < pre[a.members]; it += gridDim.x) {
                const int m = member_of(pre, a.members, it);
                cta_step(a.mem[(size_t)m * 3 + k], it - pre[m], smem_f4, threadIdx.x, blockDim.x);
                __syncthreads();     // shared memory is reused by the next item
            }
            if (!grid_sync(sync)) return;
        }
    }
#endif
}

// One staggered derivative, optionally accumulated (see cta_grad).
__global__ void __launch_bounds__(kThreads) k_grad(GradArgs a) {
    extern __shared__ float4 smem_f4[];
    cta_grad(a, blockIdx.x, smem_f4, threadIdx.x, blockDim.x);
}

// y <- alpha x + beta y (the second-order form's change of variables).
__global__ void __launch_bounds__(kThreads) k_axpby(int64_t n, float alpha, const float* x, float beta, float* y) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        y[i] = fmaf(alpha, x[i], beta * y[i]);
}

cudaError_t launch_k_axpby(int64_t n, float alpha, const float* x, float beta, float* y, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + kThreads - 1) / kThreads;
    if (blocks > 8 * 152) blocks = 8 * 152;
    k_axpby<<<(unsigned)blocks, kThreads, 0, st>>>(n, alpha, x, beta, y);
    return cudaGetLastError();
}

cudaError_t launch_k_step(unsigned grid, size_t smem, cudaStream_t st, const StepArgs& a) {
    k_step<<<grid, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_k_step_persist(unsigned grid, size_t smem, cudaStream_t st, const StepPersistArgs& a,
                                  const GridSync& sync) {
    void* args[] = {(void*)&a, (void*)&sync};
    return cudaLaunchCooperativeKernel((const void*)k_step_persist, dim3(grid), dim3(kThreads), args, smem, st);
}

cudaError_t k_step_persist_blocks(size_t smem, int* blocks) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_step_persist, kThreads, smem);
}

cudaError_t launch_k_grad(unsigned grid, size_t smem, cudaStream_t st, const GradArgs& a) {
    k_grad<<<grid, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

// Raise the kernels' dynamic shared-memory limit to the device's opt-in
// maximum (never lowered, so plans with different needs coexist).
cudaError_t set_max_smem(int bytes) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (bytes > optin) return cudaErrorInvalidValue;
    bytes = optin;
    e = cudaFuncSetAttribute(k_step, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    {
        // the cooperative kernel also holds the grid barrier's static word
        cudaFuncAttributes fa{};
        e = cudaFuncGetAttributes(&fa, k_step_persist);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_step_persist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 bytes - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
    }
    return cudaFuncSetAttribute(k_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace pstd
