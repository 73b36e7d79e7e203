// Tensor-core trailing update of the mixed-precision elimination.
#pragma once
#include "common.cuh"

int tc_panel_width(int precision);
size_t tc_pack_bytes_per_item(int n);
// Returns false (with must_set_error) if the update could not be launched.
// err: device word set to 1 by any CTA whose bounded waits ran out.
bool tc_trailing_update(int precision, float2* A, size_t stride, int ld, int n, int k0, int nbe, int items,
                        char* packs, int* err, cudaStream_t st);

// Tile width (complex columns) of the tensor-core update: 128 or 256.
bool tc_set_tile_n(int bn);
int tc_get_tile_n();
