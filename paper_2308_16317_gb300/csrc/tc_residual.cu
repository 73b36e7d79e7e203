// Refinement residual R = E0 - M X on the tensor cores, exact to ~2^-48 of
// the row scale: an Ozaki-style error-free split (Ozaki, Ogita, Oishi &
// Rump, Numer. Algorithms 59, 2012) of M and X into fixed-point BF16 digits,
// digit products on tcgen05 with FP32 accumulation in tensor memory that is
// exact by construction, and the partial sums combined in integers.
//
// Scaling and digits.  Row i of M without its diagonal entry has exponent
// e_i (|M_ik| < 2^(e_i - 1)); column c of X has f_c.  With H = M 2^(8 - e_i)
// (|H| < 128) and likewise for X, each real number is expanded as
//   H = sum_{s=0}^{5} d_s 2^(-8 s) + O(2^-41),   d_s integers, |d_s| <= 256,
// by repeated round-to-nearest (d = rint(x), x = (x - d) 256); the low word
// of M's double-float copy is folded in after the third digit, where FP32
// still holds it to 2^-17 of a digit.  Every digit is an integer of at most
// 9 bits and so is exact in BF16.
//
// Products.  Complex M X in real form: A = [Mr Mi] (row i, K index 2k, 2k+1)
// times B with B[2k][c] = Xr, B[2k+1][c] = -Xi (real part of column c) and
// B[2k][16+c] = Xi, B[2k+1][16+c] = Xr (imaginary part), 16 right-hand sides
// per group.  The B tile stacks the six X digit slices along N; the MMA of M
// digit slice s takes B slices 0 .. 5-s and accumulates into tensor-memory
// columns starting at 32 s, so level l = s + t (weight 2^(-8 l)) collects
// every digit pair of that weight in one FP32 accumulator.  A level holds at
// most 8 x 2^14 per K element (the digits after the folded low word reach
// 256), so over a chunk of 128 real K elements every partial sum is an
// integer below 2^24: FP32 accumulation is exact.  After each chunk the
// epilogue warps move the six levels to registers: levels 0-2 into one
// 64-bit integer (exact), levels 3-5 (below 2^-24 of the total) into FP32.
// The diagonal entry (t^-1, often far above the rest of its row) is left out
// of the digits and added in FP64, as is E0.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "prof.h"
#include "tc_ptx.cuh"
#include "tc_residual.h"

namespace {

using namespace tcptx;

constexpr int RT_ROWS = 128;                    // complex rows of M per CTA (TMEM lanes)
constexpr int RT_KC = 16;                       // complex columns of M per K block (32 real K, 64-byte rows)
constexpr int RT_RHS = 16;                      // right-hand sides per group
constexpr int RT_SLICES = 6;                    // digits per number
constexpr int RT_N = 2 * RT_RHS;                // real accumulator columns per level
constexpr int RT_ROWB = 64;                     // bytes per operand row of a K block (64-byte swizzle)
constexpr int RT_A_SLICE = RT_ROWS * RT_ROWB;   // bytes of one A digit slice of a K block (8 KB)
constexpr int RT_A_BYTES = RT_SLICES * RT_A_SLICE;           // 48 KB
constexpr int RT_A_STAGES = 3;
constexpr int RT_B_BYTES = RT_SLICES * RT_N * RT_ROWB;       // 12 KB: B tile of a K block
constexpr int RT_B_STAGES = 3;
constexpr int RT_CHUNK_KB = 4;                  // K blocks per exact accumulation chunk (128 real K)
constexpr int RT_ACC_COLS = 256;                // tensor-memory columns per accumulator buffer
constexpr int RT_CONV_WARPS = 8;
constexpr int RT_EPI_WARPS = 8;
constexpr int RT_THREADS = 32 * (2 + RT_CONV_WARPS + RT_EPI_WARPS);
constexpr size_t RT_SMEM = size_t(RT_A_STAGES) * RT_A_BYTES + RT_B_STAGES * RT_B_BYTES + 1024;

// Six fixed-point digits of H + L (|H| < 128, L the low word scaled alike).
__device__ __forceinline__ void digits6(float H, float L, float d[RT_SLICES]) {
  float x = H;
  d[0] = rintf(x);
  x = (x - d[0]) * 256.f;
  d[1] = rintf(x);
  x = (x - d[1]) * 256.f;
  d[2] = rintf(x);
  x = fmaf(L, 16777216.f, (x - d[2]) * 256.f);
  d[3] = rintf(x);
  x = (x - d[3]) * 256.f;
  d[4] = rintf(x);
  x = (x - d[4]) * 256.f;
  d[5] = rintf(x);
}

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // integers of <= 9 bits: exact
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Byte offset of the 4-byte pair (real K elements 2k, 2k+1) of row r in a
// 64-byte-swizzled K-major tile: rows 64 bytes apart, the 16-byte chunk
// index XOR (row / 2) mod 4 (the pattern repeats every 8 rows, 512 bytes).
__device__ __forceinline__ uint32_t swz(int r, int k) {
  return uint32_t(r) * RT_ROWB + uint32_t(((k >> 2) ^ ((r >> 1) & 3)) << 4) + uint32_t(k & 3) * 4u;
}

// Shared-memory matrix descriptor of such a tile: K-major, 64-byte swizzle,
// 8-row groups 512 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc64(uint32_t addr) {
  return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t(1) << 16) | (uint64_t(512 >> 4) << 32) | (uint64_t(1) << 46) |
         (uint64_t(4) << 61);
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace

namespace {

struct RtParams {
  const float4* M;      // double-float copy of M (hi.re, hi.im, lo.re, lo.im), column-major
  size_t stride;        // elements between items
  int ld, n, kap, nkb, ngroups;
  const int* rexp;      // [item][n] row exponents (diagonal excluded)
  const int* fexp;      // [item][kap] column exponents of X
  const uint8_t* B;     // [item][group][kb] B tiles of RT_B_BYTES
  const double2* X;     // [item][kap][n]
  double2* R;           // [item][kap][n]
  const int* conv;      // converged items are skipped
  int* err;             // raised when a bounded wait runs out
  unsigned long long* work;
};

// One CTA per (128-row tile, item, group of 16 right-hand sides).  Warp 0
// streams the B tiles (bulk copies, three stages), warp 1 allocates tensor
// memory and issues the MMAs, warps 2-9 convert the M tile of each K block
// into six swizzled digit slices in shared memory (three stages, so the
// conversion of the next blocks overlaps the MMAs of this one; each
// converter loads the next block's M entries before converting this one's),
// warps 10-17 drain the two accumulator buffers (one per chunk of four K
// blocks) and write R.
__global__ void __launch_bounds__(RT_THREADS, 1) residual_tc_kernel(RtParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + RT_A_STAGES * RT_A_BYTES;
  __shared__ __align__(8) uint64_t a_full[RT_A_STAGES], a_empty[RT_A_STAGES], mma_done;
  __shared__ __align__(8) uint64_t b_full[RT_B_STAGES], b_empty[RT_B_STAGES];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;

  const int item = blockIdx.y, g = blockIdx.z, row0 = blockIdx.x * RT_ROWS;
  if (P.conv[item]) return;   // uniform over the CTA
  if (P.work && blockIdx.x == 0 && g == 0 && threadIdx.x == 0) atomicAdd(P.work, 1ull);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = P.n, nkb = P.nkb, nchunks = (nkb + RT_CHUNK_KB - 1) / RT_CHUNK_KB;

  if (threadIdx.x == 0) {
    for (int s = 0; s < RT_A_STAGES; ++s) {
      mbar_init(&a_full[s], RT_CONV_WARPS);
      mbar_init(&a_empty[s], 1);
    }
    mbar_init(&mma_done, 1);
    for (int s = 0; s < RT_B_STAGES; ++s) {
      mbar_init(&b_full[s], 1);
      mbar_init(&b_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], RT_EPI_WARPS);
    }
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(2 * RT_ACC_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  volatile int* fail = &s_fail;
  int b_issued = 0;

  if (warp == 0) {
    if (lane == 0) {
      const uint8_t* src = P.B + (size_t(item) * P.ngroups + g) * size_t(nkb) * RT_B_BYTES;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % RT_B_STAGES;
        if (kb >= RT_B_STAGES && !mbar_wait_f(&b_empty[s], ((kb / RT_B_STAGES) - 1) & 1, fail)) break;
        mbar_expect_tx(&b_full[s], RT_B_BYTES);
        bulk_load(sB + s * RT_B_BYTES, src + size_t(kb) * RT_B_BYTES, RT_B_BYTES, &b_full[s]);
        ++b_issued;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // instruction descriptors: D FP32, A and B BF16, both K-major, M = 128, N = 32 (6 - s)
      uint32_t idesc[RT_SLICES];
#pragma unroll
      for (int s = 0; s < RT_SLICES; ++s)
        idesc[s] = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t((RT_N * (RT_SLICES - s)) >> 3) << 17) |
                   (uint32_t(RT_ROWS >> 4) << 24);
      for (int kb = 0; kb < nkb; ++kb) {
        const int c = kb / RT_CHUNK_KB, buf = c & 1;
        const bool cfirst = (kb % RT_CHUNK_KB) == 0;
        const bool clast = (kb % RT_CHUNK_KB) == RT_CHUNK_KB - 1 || kb == nkb - 1;
        if (cfirst && c >= 2 && !mbar_wait_f(&acc_empty[buf], ((c >> 1) - 1) & 1, fail)) break;
        const int sa = kb % RT_A_STAGES;
        if (!mbar_wait_f(&a_full[sa], (kb / RT_A_STAGES) & 1, fail)) break;
        if (!mbar_wait_f(&b_full[kb % RT_B_STAGES], (kb / RT_B_STAGES) & 1, fail)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = smem_u32(sA + sa * RT_A_BYTES), b0 = smem_u32(sB + (kb % RT_B_STAGES) * RT_B_BYTES);
        const uint32_t d0 = tmem + uint32_t(buf * RT_ACC_COLS);
#pragma unroll
        for (int ks = 0; ks < RT_ROWB / 32; ++ks)   // K = 16 BF16 (32 bytes) per MMA
#pragma unroll
          for (int s = 0; s < RT_SLICES; ++s)
            mma_bf16(d0 + uint32_t(RT_N * s), sdesc64(a0 + s * RT_A_SLICE + 32 * ks), sdesc64(b0 + 32 * ks),
                     idesc[s], (cfirst && ks == 0 && s == 0) ? 0u : 1u);
        mma_commit(&a_empty[sa]);
        mma_commit(&b_empty[kb % RT_B_STAGES]);
        if (clast) mma_commit(&acc_full[buf]);
      }
      mma_commit(&mma_done);   // arrives once every MMA issued above has completed
    }
  } else if (warp < 2 + RT_CONV_WARPS) {
    // Converter warp cw owns row octets 2cw, 2cw + 1 of the tile; lane l takes
    // row 8 octet + (l & 7) and complex column 4 kq + (l >> 3) of each K-quad
    // kq, so that a warp's global loads read 128 contiguous bytes per column
    // and its 4-byte digit stores hit 32 distinct banks.
    const int cw = warp - 2;
    const float4* M = P.M + size_t(item) * P.stride;
    int grow[2];
    float sc[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      grow[h] = row0 + 8 * (2 * cw + h) + (lane & 7);
      const int e = (grow[h] < n) ? P.rexp[size_t(item) * n + grow[h]] : 0;
      sc[h] = __int_as_float((127 + 8 - e) << 23);   // 2^(8 - e), exact
    }
    auto load_block = [&](int kb, float4* v) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int h = j >> 2, kq = j & 3;
        const int gk = kb * RT_KC + 4 * kq + (lane >> 3);
        const bool ok = kb < nkb && grow[h] < n && gk < n && gk != grow[h];
        v[j] = ok ? M[size_t(gk) * P.ld + grow[h]] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    float4 va[8], vb[8];
    load_block(0, va);
    for (int kb = 0; kb < nkb; kb += 2) {
#pragma unroll
      for (int half = 0; half < 2; ++half) {   // blocks kb (registers va) and kb + 1 (vb)
        const int b = kb + half;
        if (b >= nkb) break;
        float4* cur = half ? vb : va;
        float4* nxt = half ? va : vb;
        load_block(b + 1, nxt);   // in flight while this block is converted
        const int sa = b % RT_A_STAGES;
        if (b >= RT_A_STAGES && !mbar_wait_f(&a_empty[sa], ((b / RT_A_STAGES) - 1) & 1, fail)) { kb = nkb; break; }
        uint8_t* dst = sA + sa * RT_A_BYTES;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int h = j >> 2, kq = j & 3;
          const int r = 8 * (2 * cw + h) + (lane & 7), k = 4 * kq + (lane >> 3);
          float dr[RT_SLICES], di[RT_SLICES];
          digits6(cur[j].x * sc[h], cur[j].z * sc[h], dr);
          digits6(cur[j].y * sc[h], cur[j].w * sc[h], di);
          const uint32_t off = swz(r, k);
#pragma unroll
          for (int s = 0; s < RT_SLICES; ++s)
            *reinterpret_cast<uint32_t*>(dst + s * RT_A_SLICE + off) = bf16x2(dr[s], di[s]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor-core reads
        __syncwarp();
        if (lane == 0) mbar_arrive(&a_full[sa]);
      }
    }
  } else {
    // Epilogue warp: TMEM lane quarter (warp % 4), accumulator half (16 real
    // columns: the real parts of the group's 16 right-hand sides, or their
    // imaginary parts).
    const int ew = warp - 2 - RT_CONV_WARPS;
    const int quarter = warp & 3, half = ew >> 2;
    long long acc[16];
    float accf[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      acc[j] = 0;
      accf[j] = 0.f;
    }
    for (int c = 0; c < nchunks; ++c) {
      const int buf = c & 1;
      if (!mbar_wait_f(&acc_full[buf], (c >> 1) & 1, fail)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = tmem + (uint32_t(quarter * 32) << 16) + uint32_t(buf * RT_ACC_COLS + 16 * half);
      uint32_t v[16];
#pragma unroll
      for (int l = 0; l < 3; ++l) {   // levels 0-2: exact integers below 2^24
        tmem_ld16(base + uint32_t(RT_N * l), v);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] += (long long)__float2int_rn(__uint_as_float(v[j])) << (16 - 8 * l);
      }
#pragma unroll
      for (int l = 3; l < RT_SLICES; ++l) {   // levels 3-5: below 2^-24 of the total
        tmem_ld16(base + uint32_t(RT_N * l), v);
        tmem_wait_ld();
        const float w = (l == 3) ? 1.f : (l == 4) ? 0.00390625f : 1.52587890625e-05f;
#pragma unroll
        for (int j = 0; j < 16; ++j) accf[j] = fmaf(__uint_as_float(v[j]), w, accf[j]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
    const int gr = row0 + quarter * 32 + lane;
    if (!*fail && gr < n) {
      const int e = P.rexp[size_t(item) * n + gr];
      const float4 dm = P.M[size_t(item) * P.stride + size_t(gr) * P.ld + gr];
      const double mr = double(dm.x) + double(dm.z), mi = double(dm.y) + double(dm.w);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = RT_RHS * g + j;
        if (c >= P.kap) break;
        const int f = P.fexp[size_t(item) * P.kap + c];
        // digit-product units: levels 0-2 carry 2^16, levels 3-5 2^-24 (relative to level 0)
        double t = double(acc[j]) * 1.52587890625e-05 + double(accf[j]) * 5.9604644775390625e-08;
        t = ldexp(t, e + f - 16);
        const size_t o = (size_t(item) * P.kap + c) * n + gr;
        const double2 xv = P.X[o];
        const double dg = half == 0 ? mr * xv.x - mi * xv.y : mr * xv.y + mi * xv.x;
        const double e0 = (half == 0 && gr == n - P.kap + c) ? 1.0 : 0.0;
        reinterpret_cast<double*>(P.R + o)[half] = e0 - (t + dg);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 32) {   // the MMA issuer's warp: wait (bounded) for the MMAs to drain
    if (!mbar_wait(&mma_done, 0)) s_fail = 1;
  }
  if (warp == 0 && lane == 0 && *fail) {
    // drain the bulk copies this CTA armed (bounded)
    for (int kb = (b_issued > RT_B_STAGES ? b_issued - RT_B_STAGES : 0); kb < b_issued; ++kb)
      mbar_wait(&b_full[kb % RT_B_STAGES], (kb / RT_B_STAGES) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*fail && threadIdx.x == 0) atomicExch(P.err, 1);
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * RT_ACC_COLS));
}

}  // namespace

namespace {

// B tiles of the residual from X: one CTA per (right-hand side slot, item);
// slot c of group c / 16 is column c of X (slots c >= kap are zero).  Column
// exponent f_c (|X_kc| < 2^(f_c - 1)), then six digits of every entry of
// X 2^(8 - f_c), written into the swizzled K-major tile of its K block:
// row j = c % 16 takes (digit of Xr, digit of -Xi) at real K 2k, 2k + 1,
// row 16 + j takes (Xi, Xr); slice t of a tile occupies rows 32 t .. 32 t + 31.
__global__ void __launch_bounds__(256) split_xo_kernel(const double2* __restrict__ X0, int n, int kap, int nkb,
                                                       int ngroups, uint8_t* __restrict__ B0, int* __restrict__ fexp0,
                                                       const int* __restrict__ conv) {
  __shared__ double red[8];
  const int slot = blockIdx.x, item = blockIdx.y;
  if (conv[item]) return;
  const int g = slot / RT_RHS, j = slot % RT_RHS;
  uint8_t* B = B0 + (size_t(item) * ngroups + g) * size_t(nkb) * RT_B_BYTES;
  const bool live = slot < kap;
  const double2* X = X0 + (size_t(item) * kap + (live ? slot : 0)) * n;
  int f = 0;
  if (live) {
    double mx = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) mx = fmax(mx, fmax(fabs(X[k].x), fabs(X[k].y)));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = red[0];
    for (int w = 1; w < int(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
    f = (mx > 0.0 && mx <= 1e300) ? ilogb(mx) + 2 : 0;
    f = min(max(f, -90), 120);
    if (threadIdx.x == 0) fexp0[size_t(item) * kap + slot] = f;
  }
  const double s = ldexp(1.0, 8 - f);
  for (int k = threadIdx.x; k < nkb * RT_KC; k += blockDim.x) {
    float dr[RT_SLICES], di[RT_SLICES];
    if (live && k < n) {
      const double xr = X[k].x * s, xi = X[k].y * s;
      const float hr = float(xr), hi = float(xi);
      digits6(hr, float(xr - double(hr)), dr);
      digits6(hi, float(xi - double(hi)), di);
    } else {
#pragma unroll
      for (int t = 0; t < RT_SLICES; ++t) dr[t] = di[t] = 0.f;
    }
    uint8_t* tile = B + size_t(k / RT_KC) * RT_B_BYTES;
    const int kk = k % RT_KC;
#pragma unroll
    for (int t = 0; t < RT_SLICES; ++t) {
      *reinterpret_cast<uint32_t*>(tile + swz(RT_N * t + j, kk)) = bf16x2(dr[t], -di[t]);
      *reinterpret_cast<uint32_t*>(tile + swz(RT_N * t + RT_RHS + j, kk)) = bf16x2(di[t], dr[t]);
    }
  }
}

}  // namespace

size_t tc_residual_b_bytes(int n, int kap) {
  const size_t nkb = (size_t(n) + RT_KC - 1) / RT_KC, ng = (size_t(kap) + RT_RHS - 1) / RT_RHS;
  return ng * nkb * RT_B_BYTES;
}

bool tc_residual(const float4* M, size_t stride, int ld, int n, int kap, int items, const int* rexp, int* fexp,
                 const double2* X, double2* R, void* bbuf, const int* conv, int* err, unsigned long long* work,
                 cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(residual_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(RT_SMEM)) !=
        cudaSuccess) {
      must_set_error("tensor-core residual: shared-memory attribute rejected");
      return false;
    }
    attr = true;
  }
  const int nkb = (n + RT_KC - 1) / RT_KC, ng = (kap + RT_RHS - 1) / RT_RHS;
  uint8_t* B = static_cast<uint8_t*>(bbuf);
  split_xo_kernel<<<dim3(ng * RT_RHS, items), 256, 0, st>>>(X, n, kap, nkb, ng, B, fexp, conv);
  RtParams P;
  P.M = M;
  P.stride = stride;
  P.ld = ld;
  P.n = n;
  P.kap = kap;
  P.nkb = nkb;
  P.ngroups = ng;
  P.rexp = rexp;
  P.fexp = fexp;
  P.B = B;
  P.X = X;
  P.R = R;
  P.conv = conv;
  P.err = err;
  P.work = work;
  residual_tc_kernel<<<dim3((n + RT_ROWS - 1) / RT_ROWS, items, ng), RT_THREADS, RT_SMEM, st>>>(P);
  prof_launched(PH_RESIDUAL, 2);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    must_set_error("tensor-core residual launch failed: %s", cudaGetErrorString(e));
    return false;
  }
  return true;
}
