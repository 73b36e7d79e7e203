// Plain FP64 elimination of the leading r = n - kap columns of a batch of KKR
// matrices (paper Sec. 2.2: only the first block of M^{-1} is needed; Sec. 3.2:
// LU factorisation and solve).  With the central site ordered last, a
// right-looking blocked LU whose pivots are restricted to rows < r leaves the
// kap x kap Schur complement S = D - C A^{-1} B in the bottom-right corner and
// tau_00 = S^{-1}.
//
// Per panel of width nb, batched over every matrix of the chunk:
//   panel64_kernel  one CTA per matrix: pivot search (warp-shuffle argmax of
//                   |z|^2, ties to the lowest row), row swap inside the panel,
//                   scaling, rank-1 updates of the remaining panel columns.
//   laswp64_kernel  the panel's interchanges applied to the other columns.
//   trsm64_kernel   U12 = L11^{-1} A12, one warp per column (lane i holds x_i).
//   gemm64_kernel   A22 -= L21 U12, 64x64 complex tiles, 4x4 complex register
//                   tile per thread, FP64 FMA (GB300's DMMA runs at the same
//                   1.05 TFLOP/s as DFMA, measured).
//   schur_inv_kernel  tau_00 = S^{-1} by Gauss-Jordan with partial pivoting.
#include "common.cuh"
#include "prof.h"

#define LU64_T 256

__device__ __forceinline__ void argmax_merge(double& v, int& i, double v2, int i2) {
  if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
}

__global__ void __launch_bounds__(LU64_T) panel64_kernel(double2* __restrict__ A0, size_t stride, int ld, int n,
                                                         int r, int k0, int nbe, int* __restrict__ piv0,
                                                         int* __restrict__ status) {
  __shared__ double sv[LU64_T / 32];
  __shared__ int si[LU64_T / 32];
  __shared__ int s_p;
  const int item = blockIdx.x;
  cd* A = reinterpret_cast<cd*>(A0 + size_t(item) * stride);
  int* piv = piv0 + size_t(item) * r;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j = 0; j < nbe; ++j) {
    const int c = k0 + j;
    cd* col = A + size_t(c) * ld;
    double best = -1.0;
    int bi = c;
    for (int i = c + tid; i < r; i += LU64_T) argmax_merge(best, bi, cnorm(col[i]), i);
    for (int o = 16; o > 0; o >>= 1) {
      const double v2 = __shfl_down_sync(0xffffffffu, best, o);
      const int i2 = __shfl_down_sync(0xffffffffu, bi, o);
      argmax_merge(best, bi, v2, i2);
    }
    if (lane == 0) { sv[warp] = best; si[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double b = sv[0];
      int p = si[0];
      for (int w = 1; w < LU64_T / 32; ++w) argmax_merge(b, p, sv[w], si[w]);
      if (!(b > 0.0)) status[item] = ST_SINGULAR;
      piv[c] = p;
      s_p = p;
    }
    __syncthreads();
    const int p = s_p;
    if (p != c) {
      for (int cc = k0 + tid; cc < k0 + nbe; cc += LU64_T) {
        cd* cp = A + size_t(cc) * ld;
        const cd t = cp[c];
        cp[c] = cp[p];
        cp[p] = t;
      }
    }
    __syncthreads();
    const cd d = col[c];
    if (cnorm(d) > 0.0) {
      const cd inv = cinv(d);
      for (int i = c + 1 + tid; i < n; i += LU64_T) {
        const cd l = col[i] * inv;
        col[i] = l;
        for (int cc = c + 1; cc < k0 + nbe; ++cc) {
          cd* cp = A + size_t(cc) * ld;
          cfms(cp[i], l, cp[c]);
        }
      }
    }
    __syncthreads();
  }
}

// Apply the panel's interchanges (rows k0..k0+nbe-1 with piv[]) to every
// column outside the panel.
__global__ void laswp64_kernel(double2* __restrict__ A0, size_t stride, int ld, int n, int r, int k0, int nbe,
                               const int* __restrict__ piv0) {
  const int item = blockIdx.y;
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  const int nout = n - nbe;
  if (col >= nout) return;
  if (col >= k0) col += nbe;
  double2* A = A0 + size_t(item) * stride + size_t(col) * ld;
  const int* piv = piv0 + size_t(item) * r;
  for (int j = 0; j < nbe; ++j) {
    const int c = k0 + j, p = piv[c];
    if (p != c) {
      const double2 t = A[c];
      A[c] = A[p];
      A[p] = t;
    }
  }
}

// U12 = L11^{-1} A12 for columns k0+nbe .. n-1 (nbe <= 32): one warp per column.
__global__ void __launch_bounds__(256) trsm64_kernel(double2* __restrict__ A0, size_t stride, int ld, int n,
                                                     int k0, int nbe) {
  __shared__ cd L[32][33];
  const int item = blockIdx.y;
  cd* A = reinterpret_cast<cd*>(A0 + size_t(item) * stride);
  for (int t = threadIdx.x; t < nbe * nbe; t += blockDim.x) {
    const int i = t % nbe, j = t / nbe;
    L[i][j] = A[size_t(k0 + j) * ld + k0 + i];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int col = k0 + nbe + blockIdx.x * 8 + warp;
  if (col >= n) return;
  cd* x = A + size_t(col) * ld + k0;
  cd v = (lane < nbe) ? x[lane] : mk(0.0, 0.0);
  for (int j = 0; j < nbe - 1; ++j) {
    const cd xj = mk(__shfl_sync(0xffffffffu, v.x, j), __shfl_sync(0xffffffffu, v.y, j));
    if (lane > j && lane < nbe) cfms(v, L[lane][j], xj);
  }
  if (lane < nbe) x[lane] = v;
}

// A22 -= L21 U12 on rows/cols [k0+nbe, n): 64x64 complex tile per CTA.
__global__ void __launch_bounds__(256) gemm64_kernel(double2* __restrict__ A0, size_t stride, int ld, int n,
                                                     int k0, int nbe) {
  extern __shared__ cd sm[];
  cd* As = sm;              // [32][64]
  cd* Bs = sm + 32 * 64;    // [32][64]
  const int item = blockIdx.z;
  cd* A = reinterpret_cast<cd*>(A0 + size_t(item) * stride);
  const int base = k0 + nbe;
  const int m0 = base + blockIdx.x * 64, n0 = base + blockIdx.y * 64;
  const int tid = threadIdx.x;
  for (int t = tid; t < nbe * 64; t += 256) {
    const int k = t / 64, i = t % 64;
    const int row = m0 + i;
    As[k * 64 + i] = (row < n) ? A[size_t(k0 + k) * ld + row] : mk(0.0, 0.0);
  }
  for (int t = tid; t < nbe * 64; t += 256) {
    const int j = t / nbe, k = t % nbe;
    const int colg = n0 + j;
    Bs[k * 64 + j] = (colg < n) ? A[size_t(colg) * ld + k0 + k] : mk(0.0, 0.0);
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  cd acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = mk(0.0, 0.0);
  for (int k = 0; k < nbe; ++k) {
    cd a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = As[k * 64 + tx + 16 * i];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = Bs[k * 64 + ty + 16 * j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        acc[i][j].x = fma(a[i].x, b[j].x, acc[i][j].x);
        acc[i][j].x = fma(-a[i].y, b[j].y, acc[i][j].x);
        acc[i][j].y = fma(a[i].x, b[j].y, acc[i][j].y);
        acc[i][j].y = fma(a[i].y, b[j].x, acc[i][j].y);
      }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int colg = n0 + ty + 16 * j;
    if (colg >= n) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int row = m0 + tx + 16 * i;
      if (row < n) {
        cd& c = A[size_t(colg) * ld + row];
        c = c - acc[i][j];
      }
    }
  }
}

// tau_00 = S^{-1}, S = A[r:n, r:n], by Gauss-Jordan with partial pivoting.
// With equilibration (A = D M D) the block is D_c S^{-1} D_c.
// out: item's kap x kap block (column-major) at out0 + out_index[item] * kap^2.
__global__ void __launch_bounds__(256) schur_inv64_kernel(const double2* __restrict__ A0, size_t stride, int ld,
                                                          int n, int kap, const double* __restrict__ scale,
                                                          double2* __restrict__ out0,
                                                          const int* __restrict__ out_index,
                                                          int* __restrict__ status, int* __restrict__ status_out) {
  extern __shared__ cd W[];   // [kap][2 kap] row-major
  __shared__ int s_p;
  const int item = blockIdx.x;
  const cd* A = reinterpret_cast<const cd*>(A0 + size_t(item) * stride);
  const int r = n - kap, w = 2 * kap;
  for (int t = threadIdx.x; t < kap * w; t += blockDim.x) {
    const int i = t / w, j = t % w;
    W[t] = (j < kap) ? A[size_t(r + j) * ld + r + i] : mk(j - kap == i ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  bool fin_in = true;
  for (int t = threadIdx.x; t < kap * w; t += blockDim.x)
    if (!isfinite(W[t].x) || !isfinite(W[t].y)) fin_in = false;
  fin_in = __syncthreads_and(fin_in);
  bool sing = !fin_in;
  for (int k = 0; k < kap && fin_in; ++k) {
    if (threadIdx.x == 0) {
      int p = k;
      double b = cnorm(W[k * w + k]);
      for (int i = k + 1; i < kap; ++i) {
        const double v = cnorm(W[i * w + k]);
        if (v > b) { b = v; p = i; }
      }
      s_p = (b > 0.0) ? p : -1;
    }
    __syncthreads();
    const int p = s_p;
    if (p < 0) { sing = true; break; }
    if (p != k)
      for (int j = threadIdx.x; j < w; j += blockDim.x) {
        const cd t = W[k * w + j];
        W[k * w + j] = W[p * w + j];
        W[p * w + j] = t;
      }
    __syncthreads();
    const cd inv = cinv(W[k * w + k]);
    __syncthreads();
    for (int j = threadIdx.x; j < w; j += blockDim.x) W[k * w + j] = W[k * w + j] * inv;
    __syncthreads();
    for (int t = threadIdx.x; t < kap * w; t += blockDim.x) {
      const int i = t / w, j = t % w;
      if (i == k) continue;
      const cd f = W[i * w + k];
      if (j == k) continue;
      cfms(W[t], f, W[k * w + j]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kap; i += blockDim.x)
      if (i != k) W[i * w + k] = mk(0.0, 0.0);
    __syncthreads();
  }
  const size_t o = size_t(out_index[item]) * kap * kap;
  bool finite = true;
  for (int t = threadIdx.x; t < kap * kap; t += blockDim.x) {
    const int i = t % kap, j = t / kap;   // column-major output
    cd v = !fin_in ? mk(nan(""), nan("")) : (sing ? mk(0.0, 0.0) : W[i * w + kap + j]);
    if (scale) v = (scale[size_t(item) * n + r + i] * scale[size_t(item) * n + r + j]) * v;
    if (!isfinite(v.x) || !isfinite(v.y)) finite = false;
    out0[o + t] = make_double2(v.x, v.y);
  }
  finite = __syncthreads_and(finite);
  if (threadIdx.x == 0 && status_out) {
    int st = status[item];
    if (sing) st = ST_SINGULAR;
    if (!fin_in || !finite) st = ST_NONFINITE;
    status_out[out_index[item]] = st;
  }
}

// ------------------------------------------------------------------------
void lu64_factor(double2* A, size_t stride, int ld, int n, int r, int n_items, int nb, int* piv, int* status,
                 cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(gemm64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 32 * 64 * 16);
    attr = true;
  }
  for (int k0 = 0; k0 < r; k0 += nb) {
    const int nbe = (r - k0 < nb) ? (r - k0) : nb;
    {
      ProfScope ps(PH_PANEL, st);
      panel64_kernel<<<n_items, LU64_T, 0, st>>>(A, stride, ld, n, r, k0, nbe, piv, status);
      prof_launched(PH_PANEL, 1, n_items);
    }
    {
      ProfScope ps(PH_SWAP, st);
      laswp64_kernel<<<dim3((n - nbe + 255) / 256, n_items), 256, 0, st>>>(A, stride, ld, n, r, k0, nbe, piv);
      prof_launched(PH_SWAP, 1, n_items);
    }
    const int rem = n - k0 - nbe;
    if (rem > 0) {
      {
        ProfScope ps(PH_TRSM, st);
        trsm64_kernel<<<dim3((rem + 7) / 8, n_items), 256, 0, st>>>(A, stride, ld, n, k0, nbe);
        prof_launched(PH_TRSM, 1, n_items);
      }
      ProfScope ps(PH_UPDATE, st);
      const int tiles = (rem + 63) / 64;
      gemm64_kernel<<<dim3(tiles, tiles, n_items), 256, 2 * 32 * 64 * 16, st>>>(A, stride, ld, n, k0, nbe);
      prof_launched(PH_UPDATE, 1, n_items);
    }
  }
}

void schur_inv64(const double2* A, size_t stride, int ld, int n, int kap, int n_items, const double* scale,
                 double2* out, const int* out_index, int* status, int* status_out, cudaStream_t st) {
  const size_t smem = size_t(kap) * 2 * kap * 16;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(schur_inv64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 50 * 50 * 16);
    attr = true;
  }
  ProfScope ps(PH_SCHUR, st);
  schur_inv64_kernel<<<n_items, 256, smem, st>>>(A, stride, ld, n, kap, scale, out, out_index, status, status_out);
  prof_launched(PH_SCHUR, 1, n_items);
}
