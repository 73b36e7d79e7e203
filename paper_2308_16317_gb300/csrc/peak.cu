// Arithmetic peak probes (instrumentation, not part of the paper's method).
//
// The roofline fractions of the FP64 path and of the FP32/integer kernels
// need a measured denominator on this GPU: the nominal FP64 figure of the
// part does not say whether the FP64 tensor instruction (DMMA) runs faster
// than plain DFMA here.  Each probe keeps every lane busy with independent
// dependency chains of one instruction kind and stores the chains' values so
// the compiler keeps the work:
//   kind 0: DFMA, a 4 x 4 register block (16 independent chains per thread);
//   kind 1: DMMA (mma.sync m8n8k4 f64), 8 independent accumulators per warp;
//   kind 2: FFMA, 8 independent chains per thread.
// The caller times the launch (CUDA events on `stream`) and divides the
// returned flop count by it.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "prof.h"

namespace {

__global__ void __launch_bounds__(256) dfma_probe_kernel(double* __restrict__ sink, long long iters) {
  // register-blocked like a GEMM inner loop: a 4 x 4 block of accumulators
  // updated by the outer product of two 4-vectors (16 independent chains)
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double a[4], b[4], c[16];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    a[k] = 0.999999 + 1e-9 * k;
    b[k] = 1e-7 * (k + 1);
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) c[k] = sink[t] + k;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) c[4 * p + q] = fma(a[p], b[q], c[4 * p + q]);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 16; ++k) s += c[k];
  sink[t] = s;
}

__global__ void __launch_bounds__(256) ffma_probe_kernel(double* __restrict__ sink, long long iters) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const float x = 0.9999f + 1e-6f * (t & 7), y = 1e-4f;
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = float(sink[t]) + k;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], x, y);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  sink[t] = s;
}

// D = A B + C on 8x8x4 FP64 tiles; per thread one element of A and B and two
// of each accumulator.
__device__ __forceinline__ void dmma_8x8x4(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(256) dmma_probe_kernel(double* __restrict__ sink, long long iters) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const double a = 1e-3 * ((t & 3) + 1), b = 1e-3 * (((t >> 2) & 3) + 1);
  double c[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) c[k] = sink[t] + k;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) dmma_8x8x4(c[2 * k], c[2 * k + 1], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 16; ++k) s += c[k];
  sink[t] = s;
}

}  // namespace

extern "C" must_status must_peak_probe(int32_t kind, int32_t blocks, int64_t iters, double* sink, double* flops,
                                       void* stream) {
  if (kind < 0 || kind > 2 || blocks < 1 || iters < 1 || !sink || !flops) {
    must_set_error("must_peak_probe: bad argument");
    return MUST_EINVAL;
  }
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, sink) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    must_set_error("must_peak_probe: sink must be device memory (blocks x 256 doubles)");
    return MUST_EINVAL;
  }
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double threads = double(blocks) * 256.0;
  if (kind == 0) {
    dfma_probe_kernel<<<blocks, 256, 0, st>>>(sink, iters);
    *flops = threads * double(iters) * 16.0 * 2.0;
  } else if (kind == 1) {
    dmma_probe_kernel<<<blocks, 256, 0, st>>>(sink, iters);
    // per warp and iteration: 8 MMAs of 8 x 8 x 4 multiply-adds
    *flops = threads / 32.0 * double(iters) * 8.0 * (8.0 * 8.0 * 4.0 * 2.0);
  } else {
    ffma_probe_kernel<<<blocks, 256, 0, st>>>(sink, iters);
    *flops = threads * double(iters) * 8.0 * 2.0;
  }
  prof_launched(PH_OTHER, 1);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    must_set_error("must_peak_probe: launch failed: %s", cudaGetErrorString(e));
    return MUST_ECUDA;
  }
  return MUST_OK;
}
