// Low-precision correction of the mixed path on thread-block clusters:
//   delta = D U^{-1} L^{-1} P (D R),  X += delta,
// for G right-hand sides of one item per cluster of CL = 8 CTAs.
//
// The substitutions run over 32-row blocks; block b of the matrix belongs to
// CTA b mod CL, which keeps the right-hand sides of its rows in shared memory
// ([local block][G][32], FP32 complex).  Each step j (columns 32 j .. 32 j +
// 31 of the eliminated part, the diagonal block of row block j) is:
//   the owner of block j solves its 32 x 32 triangle (4 warps, G / 4
//   right-hand sides each, lane = row, shuffles broadcast solved entries);
//   cluster barrier;
//   every CTA copies the solved block from the owner's shared memory
//   (distributed shared memory) and applies it to the rows it owns below
//   (forward, L) or above (backward, U) the block.
// So every CTA streams only its own rows of L and U and the per-step work
// is spread over 8 SMs; the dependent chain per step is one triangle solve
// and one cluster barrier.  The central block (Schur complement inverse,
// FP64) is applied once per cluster by CTA 0 and shared the same way.
// Same arithmetic as the one-CTA correction (FP32 factors and updates, FP64
// central block and solution update); only the summation order of the block
// updates differs.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"
#include "mixed.h"
#include "prof.h"

namespace cg = cooperative_groups;

namespace {

constexpr int CL = 8;          // CTAs per cluster
constexpr int CT = 256;        // threads per CTA
constexpr int W_BUDGET = 72 * 1024;   // shared memory for the owned rows' right-hand sides

__device__ __forceinline__ cf ldcf(const float2* p) {
  const float2 v = *p;
  return mkf(v.x, v.y);
}

// Apply a solved block xs[jj][c] (jj < bs, G right-hand sides) to the rows of
// one owned row block: w_i -= sum_jj A[col0 + jj][i] xs[jj], for the rows
// i = b 32 + lane of that block with lo <= i < hi.  Warp unit: (block, half
// of the right-hand sides).
template <int G>
__device__ __forceinline__ void apply_block(const cf* __restrict__ A, int ld, cf* __restrict__ Wb, const cf* xs,
                                            int bs, int col0, int i, int lane, int c0, bool active) {
  constexpr int H = G / 2;
  cf acc[H];
  if (active) {
#pragma unroll
    for (int c = 0; c < H; ++c) acc[c] = Wb[(c0 + c) * 32 + lane];
  }
  for (int h = 0; h < bs; h += 8) {
    cf l[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) l[q] = (active && h + q < bs) ? A[size_t(col0 + h + q) * ld + i] : mkf(0.f, 0.f);
    if (active) {
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (h + q < bs)
#pragma unroll
          for (int c = 0; c < H; ++c) cfmsf(acc[c], l[q], xs[(h + q) * G + c0 + c]);
    }
  }
  if (active) {
#pragma unroll
    for (int c = 0; c < H; ++c) Wb[(c0 + c) * 32 + lane] = acc[c];
  }
}

template <int G>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(CT)
    correct_cluster_kernel(const float2* __restrict__ A0, size_t stride, int ld, int n, int kap,
                           const int* __restrict__ perm0, const double* __restrict__ scale0,
                           const double2* __restrict__ Sinv0, const double2* __restrict__ R0,
                           double2* __restrict__ X0, double* __restrict__ norms, const int* __restrict__ conv,
                           int first_all, const int* __restrict__ first_flags, unsigned long long* __restrict__ work) {
  constexpr int RPW = G / 4;   // right-hand sides per warp in the triangle solves
  extern __shared__ __align__(16) uint8_t cc_smem[];
  __shared__ cf Tb[32][33];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = int(cluster.block_rank());
  const int item = blockIdx.y;
  if (conv[item]) return;   // uniform over the cluster (one item)
  const int first = first_flags ? first_flags[item] : first_all;
  if (work && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(work, 1ull);
  const int cb = (blockIdx.x / CL) * G;
  const int ng = min(G, kap - cb);
  const int r = n - kap;
  const int nb = (n + 31) / 32, nlb = (nb + CL - 1) / CL;
  const int nsteps = (r + 31) / 32;
  cf* W = reinterpret_cast<cf*>(cc_smem);          // [nlb][G][32]
  cf* xs = W + size_t(nlb) * G * 32;               // [32][G]
  cf* xcf = xs + 32 * G;                           // [kap][G] central solution (FP32 copy)
  cd* xc = reinterpret_cast<cd*>(xcf + kap * G);   // [kap][G] central solution (FP64, CTA 0)
  const cf* A = reinterpret_cast<const cf*>(A0 + size_t(item) * stride);
  const int* perm = perm0 + size_t(item) * n;
  const double* d = scale0 + size_t(item) * n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // gather w = P (D R) for the owned rows (first solve: P D E0)
  for (int t = tid; t < nlb * G * 32; t += CT) {
    const int lb = t / (G * 32), c = (t / 32) % G, ii = t % 32;
    const int i = (lb * CL + rank) * 32 + ii;
    cf v = mkf(0.f, 0.f);
    if (i < n && c < ng) {
      const int src = perm[i];
      if (first) {
        if (src == r + cb + c) v = mkf(float(d[src]), 0.f);
      } else {
        const double2 rv = R0[size_t(item) * n * kap + size_t(cb + c) * n + src];
        v = mkf(float(d[src] * rv.x), float(d[src] * rv.y));
      }
    }
    W[t] = v;
  }
  __syncthreads();

  // one substitution step: the owner solves its triangle, the cluster
  // shares it, every CTA applies it to its rows in [lo, hi)
  auto step = [&](int j, bool lower) {
    const int owner = j % CL, lbj = j / CL, bs = min(32, r - 32 * j), c0 = 32 * j;
    cf* Wj = W + size_t(lbj) * G * 32;
    if (rank == owner) {
      for (int t = tid; t < 32 * 32; t += CT) {
        const int ii = t & 31, jj = t >> 5;
        if (ii < bs && jj < bs) Tb[ii][jj] = A[size_t(c0 + jj) * ld + c0 + ii];
      }
      __syncthreads();
      if (warp < 4) {
        cf v[RPW];
#pragma unroll
        for (int q = 0; q < RPW; ++q) v[q] = (lane < bs) ? Wj[(warp * RPW + q) * 32 + lane] : mkf(0.f, 0.f);
        if (lower) {
          for (int jj = 0; jj < bs - 1; ++jj) {
            const cf l = (lane > jj && lane < bs) ? Tb[lane][jj] : mkf(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < RPW; ++q) {
              const cf xj = mkf(__shfl_sync(0xffffffffu, v[q].x, jj), __shfl_sync(0xffffffffu, v[q].y, jj));
              cfmsf(v[q], l, xj);
            }
          }
        } else {
          const cf dinv = (lane < bs) ? cinvf(Tb[lane][lane]) : mkf(0.f, 0.f);
          for (int jj = bs - 1; jj >= 0; --jj) {
            if (lane == jj)
#pragma unroll
              for (int q = 0; q < RPW; ++q) v[q] = cmulf(v[q], dinv);
            const cf u = (lane < jj) ? Tb[lane][jj] : mkf(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < RPW; ++q) {
              const cf xj = mkf(__shfl_sync(0xffffffffu, v[q].x, jj), __shfl_sync(0xffffffffu, v[q].y, jj));
              cfmsf(v[q], u, xj);
            }
          }
        }
        if (lane < bs)
#pragma unroll
          for (int q = 0; q < RPW; ++q) Wj[(warp * RPW + q) * 32 + lane] = v[q];
      }
    }
    cluster.sync();
    // the solved block, from the owner's shared memory
    const cf* Wo = cluster.map_shared_rank(Wj, owner);
    for (int t = tid; t < 32 * G; t += CT) {
      const int jj = t / G, c = t % G;
      xs[t] = (jj < bs) ? Wo[c * 32 + jj] : mkf(0.f, 0.f);
    }
    __syncthreads();
    // rows to update: below the block (forward) or above it (backward)
    const int lo = lower ? c0 + bs : 0, hi = lower ? n : c0;
    const int b_lo = lo / 32, b_hi = (hi + 31) / 32;
    // owned blocks b = lb CL + rank in [b_lo, b_hi); warp units (block, RHS half)
    // (b - rank + CL - 1) / CL is ceil((b - rank) / CL) for b - rank >= 1 - CL, here always
    const int lb_lo = (b_lo - rank + CL - 1) / CL;
    const int lb_hi = min(nlb, (b_hi - rank + CL - 1) / CL);
    const int units = max(0, lb_hi - lb_lo) * 2;
    for (int u = warp; u < units; u += CT / 32) {
      const int lb = lb_lo + u / 2, half = u % 2;
      const int i = (lb * CL + rank) * 32 + lane;
      const bool active = i >= lo && i < hi;
      apply_block<G>(A, ld, W + size_t(lb) * G * 32, xs, bs, c0, min(i, n - 1), lane, half * (G / 2), active);
    }
    __syncthreads();
  };

  // forward: unit lower L, columns 0..r-1 (skipped on the first solve: P D E0
  // is zero in rows 0..r-1, since the pivots stay among those rows)
  if (!first)
    for (int j = 0; j < nsteps; ++j) step(j, true);

  // central block: w_c = Sinv w_c (FP64, by CTA 0), shared with the cluster
  cluster.sync();
  if (rank == 0) {
    const double2* Si = Sinv0 + size_t(item) * kap * kap;
    // w_c from the owners of the central rows
    for (int t = tid; t < kap * G; t += CT) {
      const int k = t / G, c = t % G;
      const int i = r + k, b = i / 32;
      const cf* Wo = cluster.map_shared_rank(W + size_t(b / CL) * G * 32, b % CL);
      xcf[t] = Wo[c * 32 + (i % 32)];
    }
    __syncthreads();
    for (int t = tid; t < kap * G; t += CT) {
      const int i = t / G, c = t % G;
      cd acc = mk(0.0, 0.0);
      for (int k = 0; k < kap; ++k) {
        const double2 sv = Si[size_t(i) * kap + k];
        const cf x = xcf[k * G + c];
        acc = acc + mk(sv.x, sv.y) * mk(x.x, x.y);
      }
      xc[t] = acc;
    }
  }
  cluster.sync();
  {
    const cd* xr = cluster.map_shared_rank(xc, 0);
    for (int t = tid; t < kap * G; t += CT) {
      const cd v = xr[t];
      xcf[t] = mkf(float(v.x), float(v.y));
    }
    __syncthreads();
    // the owners store the central rows; w_1 -= U12 w_c for the rows < r
    for (int t = tid; t < nlb * G * 32; t += CT) {
      const int lb = t / (G * 32), c = (t / 32) % G, ii = t % 32;
      const int i = (lb * CL + rank) * 32 + ii;
      if (i >= r && i < n) W[t] = xcf[(i - r) * G + c];
    }
    for (int u = warp; u < nlb * 2; u += CT / 32) {
      const int lb = u / 2, c0 = (u % 2) * (G / 2);
      const int i = (lb * CL + rank) * 32 + lane;
      if (i < r) {
        cf* Wb = W + size_t(lb) * G * 32;
        cf acc[G / 2];
#pragma unroll
        for (int c = 0; c < G / 2; ++c) acc[c] = Wb[(c0 + c) * 32 + lane];
        for (int k = 0; k < kap; ++k) {
          const cf uv = ldcf(reinterpret_cast<const float2*>(A + size_t(r + k) * ld + i));
#pragma unroll
          for (int c = 0; c < G / 2; ++c) cfmsf(acc[c], uv, xcf[k * G + c0 + c]);
        }
#pragma unroll
        for (int c = 0; c < G / 2; ++c) Wb[(c0 + c) * 32 + lane] = acc[c];
      }
    }
    __syncthreads();
  }

  // backward: U11 (non-unit upper), blocks from the bottom
  for (int j = nsteps - 1; j >= 0; --j) step(j, false);

  // X += D w for the owned rows; ||delta||^2, ||X||^2
  double dn = 0.0, xn = 0.0;
  double2* X = X0 + size_t(item) * n * kap;
  for (int t = tid; t < nlb * G * 32; t += CT) {
    const int lb = t / (G * 32), c = (t / 32) % G, ii = t % 32;
    const int i = (lb * CL + rank) * 32 + ii;
    if (i >= n || c >= ng) continue;
    const cf v = W[t];
    const double2 dl = make_double2(d[i] * v.x, d[i] * v.y);
    double2 x = first ? make_double2(0.0, 0.0) : X[size_t(cb + c) * n + i];
    x.x += dl.x;
    x.y += dl.y;
    X[size_t(cb + c) * n + i] = x;
    dn += dl.x * dl.x + dl.y * dl.y;
    xn += x.x * x.x + x.y * x.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    dn += __shfl_down_sync(0xffffffffu, dn, o);
    xn += __shfl_down_sync(0xffffffffu, xn, o);
  }
  if (lane == 0) {
    atomicAdd(&norms[2 * item], dn);
    atomicAdd(&norms[2 * item + 1], xn);
  }
  cluster.sync();   // no CTA leaves while another may still read its shared memory
}

size_t cc_smem_bytes(int n, int kap, int G) {
  const int nb = (n + 31) / 32, nlb = (nb + CL - 1) / CL;
  return size_t(nlb) * G * 32 * 8 + size_t(32) * G * 8 + size_t(kap) * G * 8 + size_t(kap) * G * 16;
}

}  // namespace

int correct_cluster_rhs(int n, int kap) {
  const int nb = (n + 31) / 32, nlb = (nb + CL - 1) / CL;
  for (int G : {16, 8, 4})
    if (size_t(nlb) * G * 32 * 8 <= size_t(W_BUDGET) && cc_smem_bytes(n, kap, G) <= 200 * 1024) return G;
  return 0;
}

bool correct_cluster(const float2* A, size_t stride, int ld, int n, int kap, int items, const int* perm,
                     const double* scale, const double2* Sinv, const double2* R, double2* X, double* norms,
                     const int* conv, int first_all, const int* first_flags, unsigned long long* work,
                     cudaStream_t st) {
  const int G = correct_cluster_rhs(n, kap);
  if (!G) {
    must_set_error("matrix order %d too large for the cluster correction", n);
    return false;
  }
  const size_t smem = cc_smem_bytes(n, kap, G);
  const dim3 grid(CL * ((kap + G - 1) / G), items);
  static size_t set16 = 0, set8 = 0, set4 = 0;
  cudaError_t e = cudaSuccess;
  if (G == 16) {
    if (smem > set16) { e = cudaFuncSetAttribute(correct_cluster_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)); set16 = smem; }
    if (e == cudaSuccess)
      correct_cluster_kernel<16><<<grid, CT, smem, st>>>(A, stride, ld, n, kap, perm, scale, Sinv, R, X, norms, conv,
                                                          first_all, first_flags, work);
  } else if (G == 8) {
    if (smem > set8) { e = cudaFuncSetAttribute(correct_cluster_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)); set8 = smem; }
    if (e == cudaSuccess)
      correct_cluster_kernel<8><<<grid, CT, smem, st>>>(A, stride, ld, n, kap, perm, scale, Sinv, R, X, norms, conv,
                                                         first_all, first_flags, work);
  } else {
    if (smem > set4) { e = cudaFuncSetAttribute(correct_cluster_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)); set4 = smem; }
    if (e == cudaSuccess)
      correct_cluster_kernel<4><<<grid, CT, smem, st>>>(A, stride, ld, n, kap, perm, scale, Sinv, R, X, norms, conv,
                                                         first_all, first_flags, work);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    must_set_error("cluster correction launch failed: %s", cudaGetErrorString(e));
    return false;
  }
  return true;
}
