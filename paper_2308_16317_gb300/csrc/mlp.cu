// Learned warm start for the refinement (an extension; the paper has no learned part): a small MLP
// (three linear layers with SiLU between them) that predicts tau_00(E_k) from
// tau_00 at the neighbouring contour energies and the LIZ's species
// occupancy.  BF16 weights for the products, FP32 accumulation, FP32 master
// weights and Adam moments; every pass is a hand-written kernel:
//   mlp_tc_gemm_kernel C = op(A) op(B) on the tcgen05 tensor cores (3xTF32
//                      splits packed K-major by tf32_pack_kernel from
//                      arbitrary strides; covers the forward products, the
//                      data gradients and the weight gradients), fused bias /
//                      SiLU / SiLU' epilogues
//   colsum_kernel      bias gradients
//   mse_kernel         loss and dL/dy
//   adam_kernel        Adam (Kingma & Ba) on the master weights, refreshes
//                      the BF16 copies
//   features_kernel    normalised inputs from the neighbouring tau_00
//   apply_kernel       tau^ = interpolation + scale * y
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include "common.cuh"
#include "prof.h"
#include "tc_ptx.cuh"
#include "tmap.h"

struct must_mlp {
  int I, H, O, max_batch;
  size_t nparam;
  float* p;              // master params: W1[H][I] b1[H] W2[H][H] b2[H] W3[O][H] b3[O]
  float* g;              // gradients (same layout)
  float* m;              // Adam first moments
  float* v;              // Adam second moments
  __nv_bfloat16* wb;     // BF16 copies of the params (same layout)
  float* act;            // activations: z1 h1 z2 h2 y dy dh
  double* loss;          // device scalar
  long long step;
  float* pk;             // tensor-core operand packs: A_hi A_lo [pa floats each], B_hi B_lo [pb floats each]
  size_t pa, pb;
  int* err;              // device word raised when a bounded wait of the product kernel runs out
};

namespace {

size_t off_W1(const must_mlp* n) { return 0; }
size_t off_b1(const must_mlp* n) { return size_t(n->H) * n->I; }
size_t off_W2(const must_mlp* n) { return off_b1(n) + n->H; }
size_t off_b2(const must_mlp* n) { return off_W2(n) + size_t(n->H) * n->H; }
size_t off_W3(const must_mlp* n) { return off_b2(n) + n->H; }
size_t off_b3(const must_mlp* n) { return off_W3(n) + size_t(n->O) * n->H; }

__device__ __forceinline__ float ld_elem(const float* p, size_t i) { return p[i]; }
__device__ __forceinline__ float ld_elem(const __nv_bfloat16* p, size_t i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z) {
  const float s = 1.0f / (1.0f + expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

enum { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_SILU = 2, EPI_DSILU = 3 };

// ---------------------------------------------------- tensor-core products --
// C[m][n] = sum_k A(m,k) B(k,n) (+ epilogue) on tcgen05 with kind::tf32 and
// FP32 accumulation in tensor memory.  Operands are first packed K-major
// (row r, K contiguous, zero-padded to 128 x 32 / 64 x 32 tiles) as a TF32
// pair x = hi + lo (hi = x rounded to TF32, lo = the rest rounded to TF32):
//   A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi      (3xTF32, ~FP32 accuracy)
// and the A_hi B_lo product is skipped when B holds the BF16 weights, which
// TF32 represents exactly (B_lo = 0).
constexpr int MG_BM = 128, MG_BN = 64, MG_KB = 32;   // tile rows, columns; K elements per stage (128 B)
constexpr int MG_STAGES = 4;
constexpr int MG_A_BYTES = MG_BM * 128, MG_B_BYTES = MG_BN * 128;
constexpr int MG_STAGE_BYTES = 2 * MG_A_BYTES + 2 * MG_B_BYTES;
constexpr size_t MG_SMEM = size_t(MG_STAGES) * MG_STAGE_BYTES + 1024;
constexpr int MG_THREADS = 192;                       // producer, MMA issuer, 4 epilogue warps

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// dst_hi / dst_lo [Rp][Kp] (row-major) = TF32 split of src(r, k) = src[r rs + k cs]
// for r < R, k < K; zero in the padding.
template <typename T>
__global__ void tf32_pack_kernel(int R, int K, int Rp, int Kp, const T* __restrict__ src, long rs, long cs,
                                 float* __restrict__ hi, float* __restrict__ lo) {
  const size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= size_t(Rp) * Kp) return;
  const int r = int(t / Kp), k = int(t % Kp);
  const float x = (r < R && k < K) ? ld_elem(src, size_t(r) * rs + size_t(k) * cs) : 0.f;
  const float h = tf32_rn(x);
  hi[t] = h;
  lo[t] = tf32_rn(x - h);
}

__device__ __forceinline__ void mg_tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          tcptx::smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(tcptx::smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mg_mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

// One CTA per 128 x 64 tile of C.  Warp 0 streams the four operand tiles of
// each 32-element K step by TMA (4 stages), warp 1 issues the MMAs (four
// K = 8 instructions per stage and product), warps 2-5 read the accumulator
// (one TMEM lane quarter each) and apply the epilogue.  Every wait is bounded;
// on time-out the kernel raises *err, drains its copies and frees its TMEM.
__global__ void __launch_bounds__(MG_THREADS, 1)
    mlp_tc_gemm_kernel(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
                       const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl, int M, int N,
                       int nks, int three, float* __restrict__ C, long ldc, int epi, const float* __restrict__ bias,
                       float* __restrict__ aux, long ldaux, int* __restrict__ err) {
  using namespace tcptx;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full[MG_STAGES], empty[MG_STAGES], done;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * MG_BM, n0 = blockIdx.x * MG_BN;
  if (threadIdx.x == 0) {
    for (int s = 0; s < MG_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(MG_BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  volatile int* fail = &s_fail;
  int issued = 0;
  if (warp == 0) {
    if (lane == 0) {
      for (int ks = 0; ks < nks; ++ks) {
        const int s = ks % MG_STAGES;
        if (ks >= MG_STAGES && !mbar_wait_f(&empty[s], ((ks / MG_STAGES) - 1) & 1, fail)) break;
        uint8_t* st = smem + s * MG_STAGE_BYTES;
        mbar_expect_tx(&full[s], MG_STAGE_BYTES);
        mg_tma_load_2d(st, &tAh, ks * MG_KB, m0, &full[s]);
        mg_tma_load_2d(st + MG_A_BYTES, &tAl, ks * MG_KB, m0, &full[s]);
        mg_tma_load_2d(st + 2 * MG_A_BYTES, &tBh, ks * MG_KB, n0, &full[s]);
        mg_tma_load_2d(st + 2 * MG_A_BYTES + MG_B_BYTES, &tBl, ks * MG_KB, n0, &full[s]);
        ++issued;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // D FP32, A and B TF32, both K-major, N = 64, M = 128
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(MG_BN >> 3) << 17) |
                             (uint32_t(MG_BM >> 4) << 24);
      for (int ks = 0; ks < nks; ++ks) {
        const int s = ks % MG_STAGES;
        if (!mbar_wait_f(&full[s], (ks / MG_STAGES) & 1, fail)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ah = smem_u32(smem + s * MG_STAGE_BYTES), al = ah + MG_A_BYTES;
        const uint32_t bh = ah + 2 * MG_A_BYTES, bl = bh + MG_B_BYTES;
#pragma unroll
        for (int k = 0; k < 4; ++k) {   // four K = 8 steps of 32 bytes per 128-byte row
          mg_mma_tf32(tmem, sdesc(ah + 32 * k), sdesc(bh + 32 * k), idesc, (ks > 0 || k > 0) ? 1u : 0u);
          if (three) mg_mma_tf32(tmem, sdesc(ah + 32 * k), sdesc(bl + 32 * k), idesc, 1u);
          mg_mma_tf32(tmem, sdesc(al + 32 * k), sdesc(bh + 32 * k), idesc, 1u);
        }
        mma_commit(&empty[s]);
      }
      mma_commit(&done);
    }
  } else {
    const int quarter = warp & 3;
    const int m = m0 + quarter * 32 + lane;
    if (mbar_wait_f(&done, 0, fail)) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int h = 0; h < MG_BN; h += 32) {
        uint32_t v[32];
        tmem_ld32(tmem + (uint32_t(quarter * 32) << 16) + uint32_t(h), v);
        if (m < M) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int n = n0 + h + j;
            if (n >= N) continue;
            float x = __uint_as_float(v[j]);
            if (epi == EPI_BIAS || epi == EPI_BIAS_SILU) x += bias[n];
            if (epi == EPI_BIAS_SILU) {
              aux[size_t(m) * ldaux + n] = x;
              x = silu_f(x);
            } else if (epi == EPI_DSILU) {
              x *= dsilu_f(aux[size_t(m) * ldaux + n]);
            }
            C[size_t(m) * ldc + n] = x;
          }
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 32 && !mbar_wait(&done, 0)) s_fail = 1;   // the MMAs have drained
  if (warp == 0 && lane == 0 && *fail)
    for (int ks = (issued > MG_STAGES ? issued - MG_STAGES : 0); ks < issued; ++ks)
      mbar_wait(&full[ks % MG_STAGES], (ks / MG_STAGES) & 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && *fail) atomicExch(err, 1);
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MG_BN));
}

// out[n] = sum_b d[b][n]
__global__ void colsum_kernel(int Bn, int N, const float* __restrict__ d, float* __restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int b = 0; b < Bn; ++b) s += d[size_t(b) * N + n];
  out[n] = s;
}

// loss = sum (y - t)^2 / B, dy = 2 (y - t) / B
__global__ void mse_kernel(int Bn, int O, const float* __restrict__ y, const float* __restrict__ t,
                           float* __restrict__ dy, double* __restrict__ loss) {
  const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  double s = 0.0;
  if (i < size_t(Bn) * O) {
    const float d = y[i] - t[i];
    dy[i] = 2.0f * d / Bn;
    s = double(d) * d / Bn;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s);
}

__global__ void adam_kernel(size_t np, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, __nv_bfloat16* __restrict__ wb, float lr, float c1, float c2) {
  const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float mi = b1 * m[i] + (1.f - b1) * g[i];
  const float vi = b2 * v[i] + (1.f - b2) * g[i] * g[i];
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  wb[i] = __float2bfloat16_rn(pi);
}

__global__ void to_bf16_kernel(size_t np, const float* __restrict__ p, __nv_bfloat16* __restrict__ wb) {
  const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < np) wb[i] = __float2bfloat16_rn(p[i]);
}

size_t rup(size_t x, size_t m) { return (x + m - 1) / m * m; }

// C = A B (+ epilogue) on the tensor cores: A(m,k) = A[m ars + k acs], B(k,n) =
// B[k brs + n bcs].  b_exact: B holds BF16 values (exact in TF32), so its low
// TF32 part is zero and the A_hi B_lo product is skipped.
template <typename TA, typename TB>
bool gemm(const must_mlp* net, int M, int N, int K, const TA* A, long ars, long acs, const TB* B, long brs, long bcs,
          float* C, long ldc, int epi, const float* bias, float* aux, long ldaux, bool b_exact, cudaStream_t st) {
  const int Mp = int(rup(M, MG_BM)), Np = int(rup(N, MG_BN)), Kp = int(rup(K, MG_KB));
  if (size_t(Mp) * Kp > net->pa || size_t(Np) * Kp > net->pb) return false;
  float* ah = net->pk;
  float* al = ah + net->pa;
  float* bh = al + net->pa;
  float* bl = bh + net->pb;
  const size_t na = size_t(Mp) * Kp, nb = size_t(Np) * Kp;
  tf32_pack_kernel<TA><<<unsigned((na + 255) / 256), 256, 0, st>>>(M, K, Mp, Kp, A, ars, acs, ah, al);
  tf32_pack_kernel<TB><<<unsigned((nb + 255) / 256), 256, 0, st>>>(N, K, Np, Kp, B, bcs, brs, bh, bl);
  CUtensorMap mAh, mAl, mBh, mBl;
  const uint64_t rb = uint64_t(Kp) * 4;
  if (!encode_2d_sw128(&mAh, 1, ah, Kp, Mp, rb, MG_KB, MG_BM) || !encode_2d_sw128(&mAl, 1, al, Kp, Mp, rb, MG_KB, MG_BM) ||
      !encode_2d_sw128(&mBh, 1, bh, Kp, Np, rb, MG_KB, MG_BN) || !encode_2d_sw128(&mBl, 1, bl, Kp, Np, rb, MG_KB, MG_BN))
    return false;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(mlp_tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(MG_SMEM));
    attr = true;
  }
  const dim3 grid(Np / MG_BN, Mp / MG_BM);
  mlp_tc_gemm_kernel<<<grid, MG_THREADS, MG_SMEM, st>>>(mAh, mAl, mBh, mBl, M, N, Kp / MG_KB, b_exact ? 0 : 1, C, ldc,
                                                        epi, bias, aux, ldaux, net->err);
  prof_launched(PH_OTHER, 3);
  return true;
}

// activations layout inside act: z1 h1 z2 h2 [B][H] each, y dy [B][O], dh [B][H]
struct Act {
  float *z1, *h1, *z2, *h2, *y, *dy, *dh;
};
Act acts(const must_mlp* n) {
  Act a;
  const size_t BH = size_t(n->max_batch) * n->H, BO = size_t(n->max_batch) * n->O;
  a.z1 = n->act;
  a.h1 = a.z1 + BH;
  a.z2 = a.h1 + BH;
  a.h2 = a.z2 + BH;
  a.y = a.h2 + BH;
  a.dy = a.y + BO;
  a.dh = a.dy + BO;
  return a;
}

bool forward(const must_mlp* n, int Bn, const float* x, float* y, cudaStream_t st) {
  const Act a = acts(n);
  const __nv_bfloat16* w = n->wb;
  const float* p = n->p;
  // z1 = x W1^T + b1 ; h1 = silu(z1)     (B(k=i, n=h) = W1[h][i])
  return gemm(n, Bn, n->H, n->I, x, n->I, 1, w + off_W1(n), 1, n->I, a.h1, n->H, EPI_BIAS_SILU, p + off_b1(n), a.z1,
              n->H, true, st) &&
         gemm(n, Bn, n->H, n->H, a.h1, n->H, 1, w + off_W2(n), 1, n->H, a.h2, n->H, EPI_BIAS_SILU, p + off_b2(n),
              a.z2, n->H, true, st) &&
         gemm(n, Bn, n->O, n->H, a.h2, n->H, 1, w + off_W3(n), 1, n->H, y, n->O, EPI_BIAS, p + off_b3(n), nullptr, 0,
              true, st);
}

// gradients of the mean-squared loss into n->g; dy must hold dL/dy
bool backward(must_mlp* n, int Bn, const float* x, cudaStream_t st) {
  const Act a = acts(n);
  const __nv_bfloat16* w = n->wb;
  float* g = n->g;
  const int H = n->H, O = n->O, I = n->I;
  // dW3[o][h] = sum_b dy[b][o] h2[b][h]
  if (!gemm(n, O, H, Bn, a.dy, 1, O, a.h2, H, 1, g + off_W3(n), H, EPI_STORE, nullptr, nullptr, 0, false, st))
    return false;
  colsum_kernel<<<(O + 255) / 256, 256, 0, st>>>(Bn, O, a.dy, g + off_b3(n));
  // dz2 = (dy W3) * silu'(z2)        (B(k=o, n=h) = W3[o][h])
  if (!gemm(n, Bn, H, O, a.dy, O, 1, w + off_W3(n), H, 1, a.dh, H, EPI_DSILU, nullptr, a.z2, H, true, st) ||
      !gemm(n, H, H, Bn, a.dh, 1, H, a.h1, H, 1, g + off_W2(n), H, EPI_STORE, nullptr, nullptr, 0, false, st))
    return false;
  colsum_kernel<<<(H + 255) / 256, 256, 0, st>>>(Bn, H, a.dh, g + off_b2(n));
  // dz1 = (dz2 W2) * silu'(z1); reuse h2 as the buffer for dz1
  if (!gemm(n, Bn, H, H, a.dh, H, 1, w + off_W2(n), H, 1, a.h2, H, EPI_DSILU, nullptr, a.z1, H, true, st) ||
      !gemm(n, H, I, Bn, a.h2, 1, H, x, I, 1, g + off_W1(n), I, EPI_STORE, nullptr, nullptr, 0, false, st))
    return false;
  colsum_kernel<<<(H + 255) / 256, 256, 0, st>>>(Bn, H, a.h2, g + off_b1(n));
  prof_launched(PH_OTHER, 3);
  return true;
}

}  // namespace

// --------------------------------------------------------------------------
extern "C" {

must_status must_mlp_create(int32_t n_in, int32_t hidden, int32_t n_out, int32_t max_batch, uint64_t seed,
                            must_mlp** out) {
  if (!out || n_in < 1 || hidden < 1 || n_out < 1 || max_batch < 1) {
    must_set_error("must_mlp_create: bad argument");
    return MUST_EINVAL;
  }
  *out = nullptr;
  must_mlp* n = new must_mlp();
  n->I = n_in; n->H = hidden; n->O = n_out; n->max_batch = max_batch; n->step = 0;
  n->nparam = size_t(hidden) * n_in + hidden + size_t(hidden) * hidden + hidden + size_t(n_out) * hidden + n_out;
  const size_t np = n->nparam;
  const size_t nact = size_t(max_batch) * (5 * size_t(hidden) + 2 * size_t(n_out));
  // operand packs of the tensor-core products: every product's rows, columns
  // and K are among the batch, the input, hidden and output widths
  const size_t mmax = std::max({size_t(max_batch), size_t(hidden), size_t(n_out)});
  const size_t nmax = std::max({size_t(hidden), size_t(n_out), size_t(n_in)});
  const size_t kmax = std::max({size_t(n_in), size_t(hidden), size_t(max_batch), size_t(n_out)});
  n->pa = rup(mmax, MG_BM) * rup(kmax, MG_KB);
  n->pb = rup(nmax, MG_BN) * rup(kmax, MG_KB);
  n->pk = nullptr;
  n->err = nullptr;
  bool ok = cudaMalloc(&n->p, np * 4) == cudaSuccess && cudaMalloc(&n->g, np * 4) == cudaSuccess &&
            cudaMalloc(&n->m, np * 4) == cudaSuccess && cudaMalloc(&n->v, np * 4) == cudaSuccess &&
            cudaMalloc(&n->wb, np * 2) == cudaSuccess && cudaMalloc(&n->act, nact * 4) == cudaSuccess &&
            cudaMalloc(&n->loss, 8) == cudaSuccess && cudaMalloc(&n->pk, 2 * (n->pa + n->pb) * 4) == cudaSuccess &&
            cudaMalloc(&n->err, 4) == cudaSuccess;
  if (!ok) {
    must_set_error("must_mlp_create: device allocation failed");
    cudaFree(n->p); cudaFree(n->g); cudaFree(n->m); cudaFree(n->v); cudaFree(n->wb); cudaFree(n->act);
    cudaFree(n->loss); cudaFree(n->pk); cudaFree(n->err);
    delete n;
    return MUST_ENOMEM;
  }
  cudaMemset(n->err, 0, 4);
  // He-style uniform initialisation from the seed (host), zero biases
  std::vector<float> h(np, 0.f);
  std::mt19937_64 rng(seed);
  auto fill = [&](size_t off, int rows, int cols) {
    const float a = std::sqrt(6.0f / float(cols));
    std::uniform_real_distribution<float> U(-a, a);
    for (size_t i = 0; i < size_t(rows) * cols; ++i) h[off + i] = U(rng);
  };
  fill(off_W1(n), hidden, n_in);
  fill(off_W2(n), hidden, hidden);
  fill(off_W3(n), n_out, hidden);
  for (size_t i = 0; i < size_t(n_out) * hidden; ++i) h[off_W3(n) + i] *= 0.1f;   // small initial correction
  cudaMemcpy(n->p, h.data(), np * 4, cudaMemcpyHostToDevice);
  cudaMemset(n->m, 0, np * 4);
  cudaMemset(n->v, 0, np * 4);
  to_bf16_kernel<<<unsigned((np + 255) / 256), 256>>>(np, n->p, n->wb);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    must_set_error("must_mlp_create: initialisation failed");
    return MUST_ECUDA;
  }
  *out = n;
  return MUST_OK;
}

void must_mlp_free(must_mlp* n) {
  if (!n) return;
  cudaFree(n->p); cudaFree(n->g); cudaFree(n->m); cudaFree(n->v); cudaFree(n->wb); cudaFree(n->act);
  cudaFree(n->loss); cudaFree(n->pk); cudaFree(n->err);
  delete n;
}

size_t must_mlp_param_count(const must_mlp* n) { return n ? n->nparam : 0; }

must_status must_mlp_get_params(const must_mlp* n, float* params, void* stream) {
  if (!n || !params) { must_set_error("must_mlp_get_params: NULL"); return MUST_EINVAL; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(params, n->p, n->nparam * 4, cudaMemcpyDefault, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    must_set_error("must_mlp_get_params: copy failed");
    return MUST_ECUDA;
  }
  return MUST_OK;
}

must_status must_mlp_set_params(must_mlp* n, const float* params, void* stream) {
  if (!n || !params) { must_set_error("must_mlp_set_params: NULL"); return MUST_EINVAL; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(n->p, params, n->nparam * 4, cudaMemcpyDefault, st) != cudaSuccess) {
    must_set_error("must_mlp_set_params: copy failed");
    return MUST_ECUDA;
  }
  cudaMemsetAsync(n->m, 0, n->nparam * 4, st);
  cudaMemsetAsync(n->v, 0, n->nparam * 4, st);
  to_bf16_kernel<<<unsigned((n->nparam + 255) / 256), 256, 0, st>>>(n->nparam, n->p, n->wb);
  n->step = 0;
  return cudaStreamSynchronize(st) == cudaSuccess ? MUST_OK : MUST_ECUDA;
}

must_status must_mlp_forward(const must_mlp* n, int32_t batch, const float* x, float* y, void* stream) {
  if (!n || !x || !y || batch < 1 || batch > n->max_batch) {
    must_set_error("must_mlp_forward: bad argument (batch must be in [1, max_batch])");
    return MUST_EINVAL;
  }
  if (!forward(n, batch, x, y, static_cast<cudaStream_t>(stream))) {
    must_set_error("must_mlp_forward: tensor-core product could not be launched");
    return MUST_ECUDA;
  }
  return cudaGetLastError() == cudaSuccess ? MUST_OK : MUST_ECUDA;
}

// Loss and gradients of the mean (over the batch) squared error; grads (host
// or device, param_count floats) and loss (host or device double) optional.
must_status must_mlp_gradients(must_mlp* n, int32_t batch, const float* x, const float* target, float* grads,
                               double* loss, void* stream) {
  if (!n || !x || !target || batch < 1 || batch > n->max_batch) {
    must_set_error("must_mlp_gradients: bad argument");
    return MUST_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Act a = acts(n);
  if (!forward(n, batch, x, a.y, st)) {
    must_set_error("must_mlp_gradients: tensor-core product could not be launched");
    return MUST_ECUDA;
  }
  cudaMemsetAsync(n->loss, 0, 8, st);
  const size_t cnt = size_t(batch) * n->O;
  mse_kernel<<<unsigned((cnt + 255) / 256), 256, 0, st>>>(batch, n->O, a.y, target, a.dy, n->loss);
  if (!backward(n, batch, x, st)) {
    must_set_error("must_mlp_gradients: tensor-core product could not be launched");
    return MUST_ECUDA;
  }
  if (grads) cudaMemcpyAsync(grads, n->g, n->nparam * 4, cudaMemcpyDefault, st);
  if (loss) cudaMemcpyAsync(loss, n->loss, 8, cudaMemcpyDefault, st);
  return cudaGetLastError() == cudaSuccess ? MUST_OK : MUST_ECUDA;
}

must_status must_mlp_train_step(must_mlp* n, int32_t batch, const float* x, const float* target, float lr,
                                double* loss, void* stream) {
  must_status s = must_mlp_gradients(n, batch, x, target, nullptr, loss, stream);
  if (s != MUST_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  n->step += 1;
  const float c1 = 1.0f - std::pow(0.9f, float(n->step)), c2 = 1.0f - std::pow(0.999f, float(n->step));
  adam_kernel<<<unsigned((n->nparam + 255) / 256), 256, 0, st>>>(n->nparam, n->p, n->g, n->m, n->v, n->wb, lr, c1,
                                                                  c2);
  prof_launched(PH_OTHER, 1);
  return cudaGetLastError() == cudaSuccess ? MUST_OK : MUST_ECUDA;
}

// Checkpoint: header (I, H, O, step) then params, Adam moments (FP32).
must_status must_mlp_save(const must_mlp* n, const char* path) {
  if (!n || !path) { must_set_error("must_mlp_save: NULL"); return MUST_EINVAL; }
  std::vector<float> buf(3 * n->nparam);
  cudaMemcpy(buf.data(), n->p, n->nparam * 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(buf.data() + n->nparam, n->m, n->nparam * 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(buf.data() + 2 * n->nparam, n->v, n->nparam * 4, cudaMemcpyDeviceToHost);
  FILE* f = std::fopen(path, "wb");
  if (!f) { must_set_error("must_mlp_save: cannot open %s", path); return MUST_EINVAL; }
  const long long hdr[5] = {0x4d4c5031LL, n->I, n->H, n->O, n->step};
  bool ok = std::fwrite(hdr, sizeof(hdr), 1, f) == 1 && std::fwrite(buf.data(), 4, buf.size(), f) == buf.size();
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) { must_set_error("must_mlp_save: write failed"); return MUST_EINVAL; }
  return MUST_OK;
}

must_status must_mlp_load(must_mlp* n, const char* path) {
  if (!n || !path) { must_set_error("must_mlp_load: NULL"); return MUST_EINVAL; }
  FILE* f = std::fopen(path, "rb");
  if (!f) { must_set_error("must_mlp_load: cannot open %s", path); return MUST_EINVAL; }
  long long hdr[5];
  std::vector<float> buf(3 * n->nparam);
  bool ok = std::fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == 0x4d4c5031LL && hdr[1] == n->I && hdr[2] == n->H &&
            hdr[3] == n->O && std::fread(buf.data(), 4, buf.size(), f) == buf.size();
  std::fclose(f);
  if (!ok) { must_set_error("must_mlp_load: %s is not a checkpoint of this network", path); return MUST_EINVAL; }
  cudaMemcpy(n->p, buf.data(), n->nparam * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(n->m, buf.data() + n->nparam, n->nparam * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(n->v, buf.data() + 2 * n->nparam, n->nparam * 4, cudaMemcpyHostToDevice);
  to_bf16_kernel<<<unsigned((n->nparam + 255) / 256), 256>>>(n->nparam, n->p, n->wb);
  n->step = hdr[4];
  return cudaDeviceSynchronize() == cudaSuccess ? MUST_OK : MUST_ECUDA;
}

}  // extern "C"

// --------------------------------------------------------------------------
// Features and prediction.  For each sample: neighbours tau_- = tau(E_{k-1}),
// tau_+ = tau(E_{k+1}) (kap x kap complex, column-major), interpolation
// m = (tau_- + tau_+)/2, half-difference d = (tau_+ - tau_-)/2 with RMS s_d,
// RMS s_m of m.  x = [d/s_d (2 kap^2), m/s_m (2 kap^2), occupancy (n_occ),
// Re/Im E_-, E, E_+, spin sign, log10(s_d/s_m)].  The network predicts
// (tau - m)/s_d.
__global__ void features_kernel(int n, int kap, const double2* __restrict__ tm, const double2* __restrict__ tp,
                                const double2* __restrict__ E3, const float* __restrict__ spin,
                                const float* __restrict__ occ, int n_occ, int n_in, float* __restrict__ x,
                                float* __restrict__ scale, double2* __restrict__ interp) {
  __shared__ double red[2][8];
  const int sidx = blockIdx.x;
  const int kk = kap * kap;
  const double2* a = tm + size_t(sidx) * kk;
  const double2* b = tp + size_t(sidx) * kk;
  double sd = 0.0, sm = 0.0;
  for (int t = threadIdx.x; t < kk; t += blockDim.x) {
    const double dx = 0.5 * (b[t].x - a[t].x), dy = 0.5 * (b[t].y - a[t].y);
    const double mx = 0.5 * (b[t].x + a[t].x), my = 0.5 * (b[t].y + a[t].y);
    sd += dx * dx + dy * dy;
    sm += mx * mx + my * my;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sd += __shfl_down_sync(0xffffffffu, sd, o);
    sm += __shfl_down_sync(0xffffffffu, sm, o);
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { red[0][warp] = sd; red[1][warp] = sm; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double A = 0, Bv = 0;
    for (int w = 0; w < (int(blockDim.x) + 31) / 32; ++w) { A += red[0][w]; Bv += red[1][w]; }
    red[0][0] = sqrt(A / kk) + 1e-300;
    red[1][0] = sqrt(Bv / kk) + 1e-300;
  }
  __syncthreads();
  const double s_d = red[0][0], s_m = red[1][0];
  float* xs = x + size_t(sidx) * n_in;
  for (int t = threadIdx.x; t < kk; t += blockDim.x) {
    const double dx = 0.5 * (b[t].x - a[t].x), dy = 0.5 * (b[t].y - a[t].y);
    const double mx = 0.5 * (b[t].x + a[t].x), my = 0.5 * (b[t].y + a[t].y);
    xs[2 * t] = float(dx / s_d);
    xs[2 * t + 1] = float(dy / s_d);
    xs[2 * kk + 2 * t] = float(mx / s_m);
    xs[2 * kk + 2 * t + 1] = float(my / s_m);
    interp[size_t(sidx) * kk + t] = make_double2(mx, my);
  }
  for (int t = threadIdx.x; t < n_occ; t += blockDim.x) xs[4 * kk + t] = occ[size_t(sidx) * n_occ + t];
  if (threadIdx.x == 0) {
    float* sc = xs + 4 * kk + n_occ;
    for (int q = 0; q < 3; ++q) {
      sc[2 * q] = float(E3[size_t(sidx) * 3 + q].x);
      sc[2 * q + 1] = float(E3[size_t(sidx) * 3 + q].y);
    }
    sc[6] = spin[sidx];
    sc[7] = float(log10(s_d / s_m));
    scale[sidx] = float(s_d);
  }
}

__global__ void apply_kernel(int n, int kk, const float* __restrict__ y, int n_out, const float* __restrict__ scale,
                             const double2* __restrict__ interp, double2* __restrict__ pred) {
  const size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= size_t(n) * kk) return;
  const size_t sidx = t / kk, e = t % kk;
  const double s = scale[sidx];
  const float* ys = y + sidx * n_out;
  const double2 m = interp[t];
  pred[t] = make_double2(m.x + s * ys[2 * e], m.y + s * ys[2 * e + 1]);
}

// target y = (tau - m)/s_d for training
__global__ void target_kernel(int n, int kk, const double2* __restrict__ tau, const float* __restrict__ scale,
                              const double2* __restrict__ interp, float* __restrict__ y, int n_out) {
  const size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= size_t(n) * kk) return;
  const size_t sidx = t / kk, e = t % kk;
  const double s = scale[sidx];
  y[sidx * n_out + 2 * e] = float((tau[t].x - interp[t].x) / s);
  y[sidx * n_out + 2 * e + 1] = float((tau[t].y - interp[t].y) / s);
}

extern "C" {

must_status must_mlp_features(int32_t n, int32_t kap, const double* tau_prev, const double* tau_next,
                              const double* E3, const float* spin, const float* occ, int32_t n_occ, int32_t n_in,
                              float* x, float* scale, double* interp, void* stream) {
  if (n < 1 || kap < 1 || !tau_prev || !tau_next || !E3 || !spin || !x || !scale || !interp ||
      n_in != 4 * kap * kap + n_occ + 8 || (n_occ > 0 && !occ)) {
    must_set_error("must_mlp_features: bad argument (n_in must be 4 kap^2 + n_occ + 8)");
    return MUST_EINVAL;
  }
  features_kernel<<<n, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      n, kap, reinterpret_cast<const double2*>(tau_prev), reinterpret_cast<const double2*>(tau_next),
      reinterpret_cast<const double2*>(E3), spin, occ, n_occ, n_in, x, scale, reinterpret_cast<double2*>(interp));
  prof_launched(PH_OTHER, 1);
  return cudaGetLastError() == cudaSuccess ? MUST_OK : MUST_ECUDA;
}

must_status must_mlp_apply(int32_t n, int32_t kap, const float* y, int32_t n_out, const float* scale,
                           const double* interp, double* tau_pred, void* stream) {
  if (n < 1 || !y || !scale || !interp || !tau_pred || n_out != 2 * kap * kap) {
    must_set_error("must_mlp_apply: bad argument (n_out must be 2 kap^2)");
    return MUST_EINVAL;
  }
  const size_t cnt = size_t(n) * kap * kap;
  apply_kernel<<<unsigned((cnt + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      n, kap * kap, y, n_out, scale, reinterpret_cast<const double2*>(interp), reinterpret_cast<double2*>(tau_pred));
  prof_launched(PH_OTHER, 1);
  return cudaGetLastError() == cudaSuccess ? MUST_OK : MUST_ECUDA;
}

must_status must_mlp_targets(int32_t n, int32_t kap, const double* tau, const float* scale, const double* interp,
                             float* y, int32_t n_out, void* stream) {
  if (n < 1 || !tau || !scale || !interp || !y || n_out != 2 * kap * kap) {
    must_set_error("must_mlp_targets: bad argument");
    return MUST_EINVAL;
  }
  const size_t cnt = size_t(n) * kap * kap;
  target_kernel<<<unsigned((cnt + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      n, kap * kap, reinterpret_cast<const double2*>(tau), scale, reinterpret_cast<const double2*>(interp), y, n_out);
  prof_launched(PH_OTHER, 1);
  return cudaGetLastError() == cudaSuccess ? MUST_OK : MUST_ECUDA;
}

}  // extern "C"
