// pstd_tc16.h -- BF16 three-way split form of the dense axis pass on the
// 5th-generation tensor cores (see pstd_tc16.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace pstd {

// One dense derivative applied to every line of an axis:
//     Y[line, m] = Cin[line, m] + sum_k D[m, k] X[line, k]
// with line l at (o, i) = (l / inner, l % inner) and element (l, k) of a field
// of length `len` along the axis at  o * len * inner + k * inner + i.
struct Tc16Gemm {
    int K, Mout;          // input and output lengths along the axis
    int MT, KC;           // 128-row output tiles, 16-wide k chunks (an even count)
    int64_t nlines, inner;
    const float* X;
    const float* Cin;
    float* Y;
    int* status;          // set to 1 when a bounded wait gives up
};

// The operator D (Mout x K, FP64) as three BF16 planes [Mpad][Kpad] on the
// device, split per (row, 32-wide k block) so that the main product's block
// sums are exact (pstd_tc16.cu); `planes` receives the device buffer (owned by
// the caller) and `map` its TMA tensor map.  Returns a cudaError_t value, or -1
// when the driver's tensor-map encoder is unavailable.
int tc16_operator(const std::vector<double>& D, int Mout, int K, uint16_t** planes, CUtensorMap* map);
int tc16_chunks(int K);
cudaError_t tc16_launch(const CUtensorMap& map, const Tc16Gemm& g, cudaStream_t st);
cudaError_t tc16_set_smem();
size_t tc16_smem_bytes();

}  // namespace pstd
