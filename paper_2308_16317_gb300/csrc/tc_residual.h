// Refinement residual R = E0 - M X on the tensor cores (exact digit split;
// see tc_residual.cu).
#pragma once
#include "common.cuh"

// Bytes of the B-operand buffer (digit tiles of X) for one item.
size_t tc_residual_b_bytes(int n, int kap);

// R = E0 - M X for the items with conv[item] == 0.  M: double-float copy of
// M (float4 per element, column-major, ld, items `stride` elements apart);
// rexp: row exponents of M without its diagonal ([item][n]); fexp: receives
// the column exponents of X ([item][kap]); X, R: [item][kap][n]; bbuf: device
// buffer of items x tc_residual_b_bytes(n, kap) bytes (256-byte aligned).
// err is raised if a bounded wait in the kernel runs out.  Returns false
// (with must_set_error) if a launch failed.
bool tc_residual(const float4* M, size_t stride, int ld, int n, int kap, int items, const int* rexp, int* fexp,
                 const double2* X, double2* R, void* bbuf, const int* conv, int* err, unsigned long long* work,
                 cudaStream_t st);
