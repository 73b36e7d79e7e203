// Tensor maps for the tensor-core kernels outside the trailing update.
#pragma once
#include <cuda.h>
#include <cstdint>

// 2-D tensor map with 128-byte swizzle (FP32 data when f32, else BF16):
// `inner` elements per row (contiguous), `rows` rows `row_bytes` apart, box
// of box_inner x box_rows elements (box_inner x element size = 128 bytes for
// the K-major operand tiles of the tensor cores).  False if the driver entry
// point is missing or rejects the map.
bool encode_2d_sw128(CUtensorMap* m, int f32, const void* base, uint64_t inner, uint64_t rows, uint64_t row_bytes,
                     uint32_t box_inner, uint32_t box_rows);
