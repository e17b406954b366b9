// pstd_kernels.cu -- the device kernels (one CTA program per block) and
// their launchers.
#include "pstd_cta.cuh"

namespace pstd {

constexpr int kThreads = 256;

// Fused per-axis leapfrog pass (see pstd_cta.cuh, cta_step).
__global__ void __launch_bounds__(kThreads) k_step(StepArgs a) {
    extern __shared__ float4 smem_f4[];
    cta_step(a, blockIdx.x, smem_f4, threadIdx.x, blockDim.x);
}

// One staggered derivative, optionally accumulated (see cta_grad).
__global__ void __launch_bounds__(kThreads) k_grad(GradArgs a) {
    extern __shared__ float4 smem_f4[];
    cta_grad(a, blockIdx.x, smem_f4, threadIdx.x, blockDim.x);
}

cudaError_t launch_k_step(unsigned grid, size_t smem, cudaStream_t st, const StepArgs& a) {
    k_step<<<grid, kThreads, smem, st>>>(a);
    return cudaGetLastError();
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
    return cudaFuncSetAttribute(k_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace pstd
