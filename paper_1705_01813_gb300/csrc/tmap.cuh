// Host helper: TMA tensor maps of row-major BF16 matrices in the 128-byte
// swizzle layout that the tcgen05 shared-memory descriptors (tc.cuh) expect.
#pragma once

#include <cuda.h>  // CUtensorMap and its enums (the encoder comes from cudaGetDriverEntryPointByVersion)
#include <cuda_runtime.h>

#include <stdint.h>

namespace gkm {

// Tensor map of a rows x cols BF16 matrix with a row stride of row_elems
// elements (row_elems * 2 a multiple of 16, base 16-byte aligned): boxes of
// box_cols (<= 64: at most one 128-byte swizzle row) x box_rows elements,
// 128-byte swizzle, L2 promotion of 256 bytes, elements outside the matrix
// read as zeros.  Returns cudaErrorInvalidValue when the CUDA driver rejects it.
cudaError_t bf16_tensor_map(CUtensorMap *tm, const void *base, int64_t cols, int64_t rows, int64_t row_elems,
                            uint32_t box_cols, uint32_t box_rows);

}  // namespace gkm
