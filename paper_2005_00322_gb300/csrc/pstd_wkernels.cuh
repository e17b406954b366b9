// pstd_wkernels.cuh -- kernels of the register-FFT axis passes, templated on
// the FFT length L, and their launchers.  Each .cu file that includes this
// header instantiates one group of lengths (see pstd_wkernels_*.cu).
#pragma once

#include <vector>

#include "pstd_persist.cuh"
#include "pstd_wcta.cuh"

namespace pstd {

// Resident CTAs of 256 threads per SM that a pass kernel is compiled for:
// the latency passes of the 3-D sizes (L <= 768) run at 128 registers, their
// shared-table form (V = 4) at 80 (768: 128, 12 elements per lane) and their
// global-table form (V = 5) at 64.
template <int L, int V>
constexpr int wmin_blocks() {
    return V == 5 ? 4 : V == 4 ? (L == 768 ? 2 : 3) : (V == 1 && L <= 768) ? 2 : 1;
}

// The contiguous latency pass of the 3-D sizes (L <= 768, the lean form of
// step_contig) also runs at 128 registers.
template <int L, int V>
__global__ void __launch_bounds__(256, wmin_blocks<L, V>()) k_wstep_c(WStep a) {
    extern __shared__ float4 wsm4[];  // 16-byte aligned for cp.async
    float2* wsm = (float2*)wsm4;
    wk::step_contig<wf::Sched<L, V>>(a, blockIdx.x, wsm, threadIdx.x, blockDim.x);
}
// The strided latency pass of the 3-D sizes (L <= 768) runs at 128 registers,
// 4 CTAs of 128 threads per SM (a few bytes of spill), for occupancy.
template <int L, int V>
__global__ void __launch_bounds__(256, wmin_blocks<L, V>()) k_wstep_s(WStep a) {
    extern __shared__ float4 wsm4[];  // 16-byte aligned for cp.async
    float2* wsm = (float2*)wsm4;
    wk::step_strided<wf::Sched<L, V>>(a, blockIdx.x, wsm, threadIdx.x, blockDim.x);
}
template <int L, int V>
__global__ void __launch_bounds__(256) k_wgrad_c(WGrad a) {
    extern __shared__ float4 wsm4[];  // 16-byte aligned for cp.async
    float2* wsm = (float2*)wsm4;
    wk::grad_contig<wf::Sched<L, V>>(a, blockIdx.x, wsm, threadIdx.x, blockDim.x);
}
template <int L, int V>
__global__ void __launch_bounds__(256) k_wgrad_s(WGrad a) {
    extern __shared__ float4 wsm4[];  // 16-byte aligned for cp.async
    float2* wsm = (float2*)wsm4;
    wk::grad_strided<wf::Sched<L, V>>(a, blockIdx.x, wsm, threadIdx.x, blockDim.x);
}

// One cooperative launch for a whole run (pstd_persist.cuh).  It holds both
// pass kinds: the table-in-memory schedules (V = 4, 5) fit 3 CTAs per SM
// without spilling, the others keep their full register budget.
template <int L, int V>
__global__ void __launch_bounds__(256, V >= 4 ? (L == 768 ? 2 : 3) : 1) k_persist(PersistArgs a) {
    extern __shared__ float4 wsm4[];
    persistent_run<wf::Sched<L, V>>(a, (float2*)wsm4);
}

// Launch geometry shared by the host plan and the launchers.
struct WLaunch {
    unsigned grid;
    int threads;
    size_t smem;
};

// Launch with programmatic stream serialisation (the kernels wait with
// griddepcontrol.wait before reading fields), so that a pass's launch and
// table loads overlap the drain of the previous one.
template <class... Args>
cudaError_t launch_pdl(void (*kernel)(Args...), const WLaunch& g, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(g.grid);
    cfg.blockDim = dim3(g.threads);
    cfg.dynamicSmemBytes = g.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int L, int V>
cudaError_t wlaunch_step(bool strided, const WLaunch& g, cudaStream_t st, const WStep& a) {
    return launch_pdl(strided ? k_wstep_s<L, V> : k_wstep_c<L, V>, g, st, a);
}
template <int L, int V>
cudaError_t wlaunch_grad(bool strided, const WLaunch& g, cudaStream_t st, const WGrad& a) {
    // the second-order form's passes follow one another: overlap each launch
    // with the previous pass's drain, as the leapfrog passes do
    if (a.dir == 4) return launch_pdl(strided ? k_wgrad_s<L, V> : k_wgrad_c<L, V>, g, st, a);
    if (strided) k_wgrad_s<L, V><<<g.grid, g.threads, g.smem, st>>>(a);
    else k_wgrad_c<L, V><<<g.grid, g.threads, g.smem, st>>>(a);
    return cudaGetLastError();
}
template <int L, int V>
cudaError_t wlaunch_persist(const WLaunch& g, cudaStream_t st, const PersistArgs& a) {
    void* args[] = {(void*)&a};
    return cudaLaunchCooperativeKernel((const void*)k_persist<L, V>, dim3(g.grid), dim3(g.threads), args, g.smem,
                                       st);
}
template <int L, int V>
cudaError_t wpersist_blocks(int threads, size_t smem, int* blocks) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_persist<L, V>, threads, smem);
}
// Dynamic shared-memory limit of one kernel: `bytes` minus its static share.
template <class K>
cudaError_t wset_one(K* kernel, int bytes) {
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                bytes - (int)fa.sharedSizeBytes);
}
template <int L, int V>
cudaError_t wset_smem(int bytes) {
    cudaError_t e;
    if ((e = wset_one(k_persist<L, V>, bytes))) return e;
    if ((e = cudaFuncSetAttribute(k_wstep_s<L, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
    if ((e = cudaFuncSetAttribute(k_wstep_c<L, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
    if ((e = cudaFuncSetAttribute(k_wgrad_s<L, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
    return cudaFuncSetAttribute(k_wgrad_c<L, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}
// pass twiddles of Sched<L, V>, FP64 angles rounded once
template <int L, int V>
void wtwiddles(std::vector<float2>& out) {
    using S = wf::Sched<L, V>;
    // even length (16-byte copies), at least one pair
    const int n = (wf::tw_total<S>() + 1) & ~1;
    out.assign(n > 0 ? n : 2, make_float2(1.0f, 0.0f));
    wf::fill_pass_twiddles<S>([&](int idx, long m, long n) {
        const double ang = 2.0 * wf::kPi * (double)m / (double)n;
        out[idx] = make_float2((float)cos(ang), (float)-sin(ang));
    });
}

// Dispatch over the (length, variant) pairs one translation unit
// instantiates; the key is 8 L + V.
#define PSTD_WDISPATCH(NAME, LIST)                                                                        \
    cudaError_t NAME##_step(int L, int V, bool s, const WLaunch& g, cudaStream_t st, const WStep& a) {   \
        switch (8 * L + V) { LIST(PSTD_WCASE_STEP) default: return cudaErrorInvalidValue; }              \
    }                                                                                                    \
    cudaError_t NAME##_grad(int L, int V, bool s, const WLaunch& g, cudaStream_t st, const WGrad& a) {   \
        switch (8 * L + V) { LIST(PSTD_WCASE_GRAD) default: return cudaErrorInvalidValue; }              \
    }                                                                                                    \
    cudaError_t NAME##_smem(int L, int V, int bytes) {                                                   \
        switch (8 * L + V) { LIST(PSTD_WCASE_SMEM) default: return cudaErrorInvalidValue; }              \
    }                                                                                                    \
    bool NAME##_twiddles(int L, int V, std::vector<float2>& out) {                                       \
        switch (8 * L + V) { LIST(PSTD_WCASE_TW) default: return false; }                                \
    }                                                                                                    \
    cudaError_t NAME##_persist(int L, int V, const WLaunch& g, cudaStream_t st, const PersistArgs& a) {  \
        switch (8 * L + V) { LIST(PSTD_WCASE_PERSIST) default: return cudaErrorInvalidValue; }           \
    }                                                                                                    \
    cudaError_t NAME##_persist_blocks(int L, int V, int threads, size_t smem, int* blocks) {             \
        switch (8 * L + V) { LIST(PSTD_WCASE_PBLOCKS) default: return cudaErrorInvalidValue; }           \
    }
#define PSTD_WCASE_STEP(LL, VV) case 8 * LL + VV: return wlaunch_step<LL, VV>(s, g, st, a);
#define PSTD_WCASE_GRAD(LL, VV) case 8 * LL + VV: return wlaunch_grad<LL, VV>(s, g, st, a);
#define PSTD_WCASE_SMEM(LL, VV) case 8 * LL + VV: return wset_smem<LL, VV>(bytes);
#define PSTD_WCASE_TW(LL, VV) case 8 * LL + VV: wtwiddles<LL, VV>(out); return true;
#define PSTD_WCASE_PERSIST(LL, VV) case 8 * LL + VV: return wlaunch_persist<LL, VV>(g, st, a);
#define PSTD_WCASE_PBLOCKS(LL, VV) case 8 * LL + VV: return wpersist_blocks<LL, VV>(threads, smem, blocks);

// Lanes per sequence of Sched<L, 2> (fewer, wider passes; 0: none).
inline int wlanes_v2(int L) { return L == 1024 ? 64 : 0; }
// Lanes per sequence of Sched<L, 4> (the latency radices, tables in shared
// memory; 0: none).
inline int wlanes_v4(int L) { return L == 512 || L == 768 ? 64 : (L == 256 ? 32 : 0); }
// Lanes per sequence of Sched<L, 5> (as V = 4, tables read from global memory).
inline int wlanes_v5(int L) { return L == 512 ? 64 : (L == 256 ? 32 : 0); }
// Lanes per sequence of Sched<L, 3> (more lanes, 4 elements each; 0: none).
inline int wlanes_v3(int L) { return L == 1024 ? 256 : (L == 512 ? 128 : 0); }

// Lanes per sequence of the latency schedule Sched<L, 1> (0: none).
inline int wlanes_latency(int L) {
    switch (L) {
        case 256: return 32;
        case 512: return 64;
        case 768: return 64;
        case 1024: return 128;
        default: return 0;
    }
}

// Lanes per sequence of Sched<L, 0> (0: not instantiated).
inline int wlanes(int L) {
    switch (L) {
        case 2: case 4: case 8: case 16: case 32: return 1;
        case 64: return 4;
        case 128: return 8;
        case 256: case 512: return 16;
        case 1024: return 32;
        case 96: return 4;
        case 192: return 8;
        case 384: return 16;
        case 768: return 32;
        default: return 0;
    }
}
inline int wseq_words(int L) { return L + L / 32 + 1; }

}  // namespace pstd
