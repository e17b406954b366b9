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
// over fields in the plan's padded layout, read and written through tensor
// maps (tc16_field_map).  Lines come in tiles of 128: on the contiguous (last)
// axis consecutive rows; on a strided axis 128 consecutive inner indices of
// one outer block (tpo tiles per outer block).
struct Tc16Gemm {
    int K, Mout;          // input and output lengths along the axis
    int MT, KC;           // 128-row output tiles, 16-wide k chunks (an even count)
    int contiguous;       // 1: the axis is the last one (lines are rows)
    int64_t tiles;        // line tiles
    int64_t tpo;          // strided axes: line tiles per outer block
    const uint8_t* op;    // the operator's slices, tiled (tc16_operator)
    int* status;          // set to 1 when a bounded wait gives up
};

// The operator D (Mout x K, FP64) as three BF16 slices per (row, 32-wide k
// block) power-of-two grid, so that the main product's block sums are exact
// (pstd_tc16.cu), stored on the device chunk by chunk: for output tile mt and
// 16-wide chunk c, 12 KB at (mt * chunks + c) * 12 KB laid out as the MMA
// reads them ([slice][128 rows][16 k], 32-byte swizzle).  `planes` receives
// the device buffer (owned by the caller).  Returns a cudaError_t value.
int tc16_operator(const std::vector<double>& D, int Mout, int K, uint16_t** planes);
int tc16_chunks(int K);
// Tensor map of a padded FP32 field for one axis: contiguous (last) axis: rows
// of `len` values `pitch` floats apart, `lines_or_inner` rows; strided axis:
// (inner, len, outer) with inner = lines_or_inner (a multiple of 4).  ymap:
// the output-tile box (Y / Cin), else the field-block box (X).  0 or -1.
int tc16_field_map(float* base, int contiguous, int64_t len, int64_t lines_or_inner, int64_t outer, int64_t pitch,
                   int ymap, CUtensorMap* map);
cudaError_t tc16_launch(const CUtensorMap& mx, const CUtensorMap& mcin, const CUtensorMap& my, const Tc16Gemm& g,
                        cudaStream_t st);
cudaError_t tc16_set_smem();
size_t tc16_smem_bytes();

}  // namespace pstd
