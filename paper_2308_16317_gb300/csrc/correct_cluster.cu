// Low-precision correction of the mixed path on thread-block clusters:
//   delta = D U^{-1} L^{-1} P (D R),  X += delta,
// for G right-hand sides of one item per cluster of CL CTAs (2 by default).
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
// is spread over CL SMs; the dependent chain per step is one triangle solve
// and one cluster barrier.  The factors are read-only here, so each warp
// issues the loads of its first unit of a step, and the next step's owner
// the loads of its diagonal block, before waiting at the step's barrier.  The central block (Schur complement inverse,
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

constexpr int CT = 256;        // threads per CTA
constexpr int W_BUDGET = 72 * 1024;   // shared memory for the owned rows' right-hand sides
int g_cluster_ctas = 2;        // preferred CTAs per cluster (tuning knob 7)
int g_cluster_rhs = 0;         // right-hand sides per cluster (tuning knob 8; 0: the most within W_BUDGET)

// One warp's unit of a substitution step: the 32 rows of one owned block
// (lane = row) against the G / 2 right-hand sides of one half, for the
// step's columns col0 .. col0 + bs - 1 of L or U.  The row segment of the
// factor is loaded in one batch of 32 independent loads (lrow), so a unit
// costs one memory round trip; units whose rows need no update load zeros.
template <int G>
struct Unit {
  cf l[32];
  __device__ __forceinline__ void load(const cf* __restrict__ A, int ld, int col0, int bs, int i, bool active) {
#pragma unroll
    for (int q = 0; q < 32; ++q) l[q] = (active && q < bs) ? A[size_t(col0 + q) * ld + i] : mkf(0.f, 0.f);
  }
  // w_i -= sum_q l[q] xs[q] for the half's right-hand sides
  __device__ __forceinline__ void apply(cf* __restrict__ Wb, const cf* xs, int lane, int c0, bool active) {
    constexpr int H = G / 2;
    if (!active) return;
    cf acc[H];
#pragma unroll
    for (int c = 0; c < H; ++c) acc[c] = Wb[(c0 + c) * 32 + lane];
#pragma unroll
    for (int q = 0; q < 32; ++q)
#pragma unroll
      for (int c = 0; c < H; ++c) cfmsf(acc[c], l[q], xs[q * G + c0 + c]);
#pragma unroll
    for (int c = 0; c < H; ++c) Wb[(c0 + c) * 32 + lane] = acc[c];
  }
};

template <int G>
__global__ void __launch_bounds__(CT, 2)
    correct_cluster_kernel(const float2* __restrict__ A0, size_t stride, int ld, int n, int kap,
                           const int* __restrict__ perm0, const double* __restrict__ scale0,
                           const double2* __restrict__ Sinv0, const double2* __restrict__ R0,
                           double2* __restrict__ X0, double* __restrict__ norms, const int* __restrict__ conv,
                           int first_all, const int* __restrict__ first_flags, unsigned long long* __restrict__ work) {
  constexpr int RPW = G / 4;   // right-hand sides per warp in the triangle solves
  extern __shared__ __align__(16) uint8_t cc_smem[];
  __shared__ cf Tb[2][32][33];  // diagonal blocks of the current and the next step
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = int(cluster.num_blocks());
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
  // diagonal block of step j (rows and columns 32 j .. 32 j + bs - 1); the
  // factors are read-only here, so a step's block is loaded one step ahead
  auto tb_load = [&](int j, cf* v) {
    const int bs = min(32, r - 32 * j), c0 = 32 * j;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int t = tid + q * CT, ii = t & 31, jj = t >> 5;
      v[q] = (ii < bs && jj < bs) ? A[size_t(c0 + jj) * ld + c0 + ii] : mkf(0.f, 0.f);
    }
  };
  auto tb_store = [&](int buf, const cf* v) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int t = tid + q * CT;
      Tb[buf][t & 31][t >> 5] = v[q];
    }
  };
  __syncthreads();

  // one substitution step: the owner solves its triangle, the cluster
  // shares it, every CTA applies it to its rows in [lo, hi)
  auto step = [&](int j, bool lower, int jnext) {
    const int owner = j % CL, lbj = j / CL, bs = min(32, r - 32 * j), c0 = 32 * j;
    cf* Wj = W + size_t(lbj) * G * 32;
    const int lo = lower ? c0 + bs : 0, hi = lower ? n : c0;
    const int b_lo = lo / 32, b_hi = (hi + 31) / 32;
    // owned blocks b = lb CL + rank in [b_lo, b_hi) ((b - rank + CL - 1) / CL
    // is ceil((b - rank) / CL), as b - rank >= 1 - CL); warp units (block, half)
    const int lb_lo = (b_lo - rank + CL - 1) / CL;
    const int lb_hi = min(nlb, (b_hi - rank + CL - 1) / CL);
    const int units = max(0, lb_hi - lb_lo) * 2;
    // issue the loads of this warp's first unit and of the next step's
    // diagonal block before waiting for the solved block
    Unit<G> un;
    int u = warp;
    auto unit_rows = [&](int uu, int& lb, int& i, bool& active) {
      lb = lb_lo + uu / 2;
      i = (lb * CL + rank) * 32 + lane;
      active = i >= lo && i < hi;
    };
    int ulb = 0, ui = 0;
    bool uact = false;
    if (u < units) {
      unit_rows(u, ulb, ui, uact);
      un.load(A, ld, c0, bs, min(ui, n - 1), uact);
    }
    cf tbn[4];
    const bool pre = jnext >= 0 && rank == jnext % CL;
    if (pre) tb_load(jnext, tbn);
    if (rank == owner) {
      if (warp < 4) {
        cf v[RPW];
#pragma unroll
        for (int q = 0; q < RPW; ++q) v[q] = (lane < bs) ? Wj[(warp * RPW + q) * 32 + lane] : mkf(0.f, 0.f);
        const cf(*T)[33] = Tb[j & 1];
        if (lower) {
          for (int jj = 0; jj < bs - 1; ++jj) {
            const cf l = (lane > jj && lane < bs) ? T[lane][jj] : mkf(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < RPW; ++q) {
              const cf xj = mkf(__shfl_sync(0xffffffffu, v[q].x, jj), __shfl_sync(0xffffffffu, v[q].y, jj));
              cfmsf(v[q], l, xj);
            }
          }
        } else {
          const cf dinv = (lane < bs) ? cinvf(T[lane][lane]) : mkf(0.f, 0.f);
          for (int jj = bs - 1; jj >= 0; --jj) {
            if (lane == jj)
#pragma unroll
              for (int q = 0; q < RPW; ++q) v[q] = cmulf(v[q], dinv);
            const cf uu = (lane < jj) ? T[lane][jj] : mkf(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < RPW; ++q) {
              const cf xj = mkf(__shfl_sync(0xffffffffu, v[q].x, jj), __shfl_sync(0xffffffffu, v[q].y, jj));
              cfmsf(v[q], uu, xj);
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
    if (pre) tb_store(jnext & 1, tbn);
    __syncthreads();
    for (; u < units; u += CT / 32) {
      if (u != warp) {
        unit_rows(u, ulb, ui, uact);
        un.load(A, ld, c0, bs, min(ui, n - 1), uact);
      }
      un.apply(W + size_t(ulb) * G * 32, xs, lane, (u % 2) * (G / 2), uact);
    }
    __syncthreads();
  };

  // forward: unit lower L, columns 0..r-1 (skipped on the first solve: P D E0
  // is zero in rows 0..r-1, since the pivots stay among those rows)
  if (!first && nsteps > 0) {
    if (rank == 0) {
      cf v[4];
      tb_load(0, v);
      tb_store(0, v);
    }
    __syncthreads();
    for (int j = 0; j < nsteps; ++j) step(j, true, j + 1 < nsteps ? j + 1 : -1);
  }

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
          const cf uv = A[size_t(r + k) * ld + i];
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
  if (nsteps > 0) {
    if (rank == (nsteps - 1) % CL) {
      cf v[4];
      tb_load(nsteps - 1, v);
      tb_store((nsteps - 1) & 1, v);
    }
    __syncthreads();
    for (int j = nsteps - 1; j >= 0; --j) step(j, false, j > 0 ? j - 1 : -1);
  }

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

size_t cc_smem_bytes(int n, int kap, int G, int CL) {
  const int nb = (n + 31) / 32, nlb = (nb + CL - 1) / CL;
  return size_t(nlb) * G * 32 * 8 + size_t(32) * G * 8 + size_t(kap) * G * 8 + size_t(kap) * G * 16;
}

template <int G>
cudaError_t launch_cc(int CL, dim3 grid, size_t smem, cudaStream_t st, const float2* A, size_t stride, int ld, int n,
                      int kap, const int* perm, const double* scale, const double2* Sinv, const double2* R,
                      double2* X, double* norms, const int* conv, int first_all, const int* first_flags,
                      unsigned long long* work) {
  static size_t set = 0;
  if (smem > set) {
    const cudaError_t e =
        cudaFuncSetAttribute(correct_cluster_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    set = smem;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(CT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = unsigned(CL);
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, correct_cluster_kernel<G>, A, stride, ld, n, kap, perm, scale, Sinv, R, X, norms,
                            conv, first_all, first_flags, work);
}

}  // namespace

bool correct_cluster_set_ctas(int ctas) {
  if (ctas != 2 && ctas != 4 && ctas != 8) return false;
  g_cluster_ctas = ctas;
  return true;
}

int correct_cluster_get_ctas() { return g_cluster_ctas; }

bool correct_cluster_set_rhs(int rhs) {
  if (rhs != 0 && rhs != 4 && rhs != 8 && rhs != 16) return false;
  g_cluster_rhs = rhs;
  return true;
}

int correct_cluster_get_rhs() { return g_cluster_rhs; }

// Right-hand sides per cluster and CTAs per cluster for order n: the
// preferred cluster size (knob 7) or, when the owned rows' right-hand sides
// do not fit its shared memory even for 4 right-hand sides, the next larger.
static void cc_shape(int n, int kap, int* G_out, int* CL_out) {
  *G_out = 0;
  *CL_out = 0;
  for (int CL = g_cluster_ctas; CL <= 8; CL *= 2) {
    const int nb = (n + 31) / 32, nlb = (nb + CL - 1) / CL;
    for (int G : {16, 8, 4})
      if (g_cluster_rhs ? (G == g_cluster_rhs && cc_smem_bytes(n, kap, G, CL) <= 200 * 1024)
                        : (size_t(nlb) * G * 32 * 8 <= size_t(W_BUDGET) && cc_smem_bytes(n, kap, G, CL) <= 100 * 1024)) {
        *G_out = G;
        *CL_out = CL;
        return;
      }
  }
}

int correct_cluster_rhs(int n, int kap) {
  int G, CL;
  cc_shape(n, kap, &G, &CL);
  return G;
}

bool correct_cluster(const float2* A, size_t stride, int ld, int n, int kap, int items, const int* perm,
                     const double* scale, const double2* Sinv, const double2* R, double2* X, double* norms,
                     const int* conv, int first_all, const int* first_flags, unsigned long long* work,
                     cudaStream_t st, int shape) {
  int G, CL;
  cc_shape(n, kap, &G, &CL);
  if (shape > 0) {   // CL * 100 + G, if its rows fit the shared memory
    const int CLs = shape / 100, Gs = shape % 100;
    if (cc_smem_bytes(n, kap, Gs, CLs) <= 200 * 1024) {
      G = Gs;
      CL = CLs;
    }
  }
  if (!G) {
    must_set_error("matrix order %d too large for the cluster correction", n);
    return false;
  }
  const size_t smem = cc_smem_bytes(n, kap, G, CL);
  const dim3 grid(CL * ((kap + G - 1) / G), items);
  cudaError_t e;
  if (G == 16)
    e = launch_cc<16>(CL, grid, smem, st, A, stride, ld, n, kap, perm, scale, Sinv, R, X, norms, conv, first_all,
                      first_flags, work);
  else if (G == 8)
    e = launch_cc<8>(CL, grid, smem, st, A, stride, ld, n, kap, perm, scale, Sinv, R, X, norms, conv, first_all,
                     first_flags, work);
  else
    e = launch_cc<4>(CL, grid, smem, st, A, stride, ld, n, kap, perm, scale, Sinv, R, X, norms, conv, first_all,
                     first_flags, work);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    must_set_error("cluster correction launch failed: %s", cudaGetErrorString(e));
    return false;
  }
  return true;
}
