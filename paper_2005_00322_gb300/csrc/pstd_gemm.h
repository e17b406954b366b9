// pstd_gemm.h -- split-precision dense axis pass (see pstd_gemm.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pstd {

struct GemmAxis {
    int N, lp;                // u and p lengths along the axis
    int MT1, KT1;             // GEMM 1 (D_p): 16-row tiles of N, 16-column tiles of lp
    int MT2, KT2;             // GEMM 2 (D_u): 16-row tiles of lp, 16-column tiles of N
    const uint4* A1h;         // D_p / s1, FP16 hi / lo in fragment order
    const uint4* A1l;
    const uint4* A2h;         // D_u / s2
    const uint4* A2l;
    float s1, s2;             // matrix scales (time-step factors folded in)
    int64_t nlines, inner;    // lines of the axis and its stride
    int G;                    // lines per CTA (multiple of 8, at most 64)
};

struct GemmStep {
    GemmAxis ax;
    const float* p;
    float* u;
    const float* acc_in;
    float* acc_out;
};

cudaError_t launch_gemm_step(unsigned grid, size_t smem, cudaStream_t st, const GemmStep& a);
cudaError_t gemm_set_smem(int bytes);
size_t gemm_smem_bytes(int G, int KT1, int KT2, int N);

}  // namespace pstd
