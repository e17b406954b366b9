// pstd_energy.cu -- the discrete energy of the leapfrog state in FP64 on the GPU.
//
// The scheme of Eq. dtt_pstd_solution conserves, exactly in exact arithmetic,
//     E^n = sum_j w_j (p_j^n)^2 / (2 rho0 c0^2)
//         + (rho0 / 2) sum_i sum_j w_ij u_{i,j}^{n-1/2} u_{i,j}^{n+1/2}
// with tensor-product quadrature weights: 1/2 on a stored pressure node on a
// Neumann wall, 1/2 on the velocity half-node a Dirichlet mid-cell wall passes
// through, 1 elsewhere.  Each field's weighted sum of products is accumulated
// in FP64: per block over a fixed grid-stride share, then the blocks' partial
// sums in a fixed order, so the result does not depend on scheduling.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pstd_energy.h"

namespace pstd {

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_energy_partial(EnergyField f, double* partial) {
    double acc = 0.0;
    const int64_t n = f.n[0] * f.n[1] * f.n[2];
    for (int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * kThreads) {
        const int64_t i2 = idx % f.n[2];
        const int64_t r = idx / f.n[2];
        const int64_t i1 = r % f.n[1];
        const int64_t i0 = r / f.n[1];
        const int64_t ii[3] = {i0, i1, i2};
        double w = 1.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if ((f.first_half >> a) & 1) w *= ii[a] == 0 ? 0.5 : 1.0;
            if ((f.last_half >> a) & 1) w *= ii[a] == f.n[a] - 1 ? 0.5 : 1.0;
        }
        acc += w * (double)f.a[idx] * (double)f.b[idx];
    }
    // block sum in a fixed order: warp shuffles, then the warps' sums
    __shared__ double ws[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) s += ws[i];
        partial[blockIdx.x] = s;
    }
}

// out = sum_f scale[f] * (sum of field f's nblocks partial sums, in order).
__global__ void k_energy_total(const double* partial, int nblocks, int nfields, EnergyScales sc, double* out) {
    __shared__ double fs[4];
    if (threadIdx.x < nfields) {
        double s = 0.0;
        for (int i = 0; i < nblocks; ++i) s += partial[(size_t)threadIdx.x * nblocks + i];
        fs[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double e = 0.0;
        for (int f = 0; f < nfields; ++f) e += sc.s[f] * fs[f];
        *out = e;
    }
}

}  // namespace

cudaError_t energy_launch(const EnergyField* fields, int nfields, const EnergyScales& sc, int nblocks,
                          double* scratch, cudaStream_t st) {
    for (int f = 0; f < nfields; ++f) {
        k_energy_partial<<<nblocks, kThreads, 0, st>>>(fields[f], scratch + (size_t)f * nblocks);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_energy_total<<<1, 32, 0, st>>>(scratch, nblocks, nfields, sc, scratch + (size_t)4 * nblocks);
    return cudaGetLastError();
}

}  // namespace pstd
