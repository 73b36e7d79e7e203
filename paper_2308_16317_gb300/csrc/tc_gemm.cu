// Tensor-core trailing update of the mixed-precision elimination,
//   A22 -= L21 U12   (complex FP32 storage, column-major),
// on the 5th-generation tensor cores: tcgen05.mma with operands staged in
// shared memory by TMA (cp.async.bulk.tensor, 128-byte swizzle) and FP32
// accumulators in tensor memory, read back with tcgen05.ld for the epilogue.
//
// Complex -> real block form, row-interleaved so the epilogue is coalesced:
//   A'[2i]   = [Lr(i,p), -Li(i,p)]_p     A'[2i+1] = [Li(i,p), Lr(i,p)]_p
//   B'[j]    = [Ur(p,j),  Ui(p,j)]_p     (K index 2p, 2p+1)
//   C'[2i][j] = Re(L U)(i,j),  C'[2i+1][j] = Im(L U)(i,j).
// Split products (Henry, Tang & Heinecke, ARITH 2019 for BF16; the same
// three-term scheme with TF32 halves): x = x_hi + x_lo, and
//   A'B'^T ~ A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T
// accumulated in one FP32 TMEM accumulator (the lo*lo term is dropped).
//
// Kernels sharing this scheme (knob 2 of must_tune_set picks one):
//  - streamed kernels: each CTA takes a run of 128-row x 64-column tiles of
//    one column block, with the U block (B_hi, B_lo) resident in shared
//    memory, the A rows streaming through a TMA ring and two TMEM
//    accumulators, so that the MMAs of tile t+1 overlap the epilogue of tile
//    t.  The update is HBM-bound, so they differ in how C moves:
//      tc_update_tmac (default): a loader warp brings C tiles into three
//        shared-memory buffers by TMA; the epilogue forms C - A'B' and stores
//        it from registers (coalesced 128-byte column segments);
//      tc_update_regc: C loaded and stored from registers, two tiles ahead;
//      tc_update_streamed: C loaded by TMA, updated in shared memory and
//        stored by TMA.
//    All three issue the same MMAs and subtract the same way, so their
//    results are identical.
//  - the per-tile kernel (one CTA per tile), used for 256-column tiles and
//    the TF32 splits.
//
// Per-tile kernel: one CTA (256 threads) computes a 128 x BN tile of C' (64 complex rows x BN
// complex columns): warp 0 lane 0 issues TMA loads into a STAGES-deep ring,
// warp 1 lane 0 issues the MMAs (one per 32 bytes of K), and all eight warps
// (two per TMEM lane quarter, one per column half) update C in place.  Every mbarrier wait is
// bounded; on time-out the kernel raises the workspace error word, drains its
// own copies, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "tc_gemm.h"
#include "tc_ptx.cuh"
#include "prof.h"

namespace {

using namespace tcptx;

constexpr int BM = 128;                // real rows per tile (= TMEM lanes)
constexpr int KB = 128;                // bytes of K per stage (one swizzle row)
constexpr int PANEL_NB = 64;           // complex panel width of the mixed path

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int c0, int c1, int c2) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(map), "r"(c0),
               "r"(c1), "r"(c2), "r"(smem_u32(src))
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ void mma_issue(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc,
                                          int kind_tf32) {
  if (kind_tf32)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

struct TcParams {
  float2* C;
  size_t stride;
  int ld, n;
  int base;      // first trailing row/column (k0 + nbe)
  int ksteps;    // K stages per split pass
  int* err;      // workspace error word
  int tf32;
  int col_tile0; // first column tile of this launch
  int aoff;      // first row of the A operand's slot in the pack (0 or rows_pad)
};

template <int BN, int STAGES>
__global__ void __launch_bounds__(256, 1)
    tc_update_kernel(const __grid_constant__ CUtensorMap tA_hi, const __grid_constant__ CUtensorMap tA_lo,
                     const __grid_constant__ CUtensorMap tB_hi, const __grid_constant__ CUtensorMap tB_lo,
                     TcParams P) {
  constexpr int A_BYTES = BM * KB;          // 16 KB
  constexpr int B_BYTES = BN * KB;
  constexpr int ST_BYTES = A_BYTES + B_BYTES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full[STAGES];
  __shared__ __align__(8) uint64_t empty[STAGES];
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = blockIdx.z;
  const int row0 = blockIdx.x * BM;     // real rows of C' relative to the trailing block
  const int col0 = (blockIdx.y + P.col_tile0) * BN;   // complex columns relative to the trailing block
  const int nsteps = 3 * P.ksteps;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  int issued = 0;   // producer: TMA stages issued
  if (warp == 0 && lane == 0) {
    const int kstep_elems = P.tf32 ? KB / 4 : KB / 2;
    for (int step = 0; step < nsteps; ++step) {
      const int s = step % STAGES;
      const uint32_t ph = (step / STAGES) & 1;
      if (step >= STAGES && !mbar_wait(&empty[s], ph ^ 1)) { s_fail = 1; break; }
      const int pass = step / P.ksteps, kb = step % P.ksteps;
      const CUtensorMap* ma = (pass == 2) ? &tA_lo : &tA_hi;
      const CUtensorMap* mb = (pass == 1) ? &tB_lo : &tB_hi;
      uint8_t* sa = smem + s * ST_BYTES;
      mbar_expect_tx(&full[s], ST_BYTES);
      tma_load_3d(sa, ma, kb * kstep_elems, P.aoff + 2 * P.base + row0, item, &full[s]);
      tma_load_3d(sa + A_BYTES, mb, kb * kstep_elems, P.base + col0, item, &full[s]);
      ++issued;
    }
  } else if (warp == 1 && lane == 0) {
    // instruction descriptor: D F32, A/B BF16 (f16 kind) or TF32, K-major, N, M
    const uint32_t fmt = P.tf32 ? 2u : 1u;
    const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (uint32_t(BN >> 3) << 17) | (uint32_t(BM >> 4) << 24);
    bool ok = true;
    for (int step = 0; step < nsteps && ok; ++step) {
      const int s = step % STAGES;
      const uint32_t ph = (step / STAGES) & 1;
      if (!mbar_wait(&full[s], ph)) { ok = false; s_fail = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(smem + s * ST_BYTES), b0 = a0 + A_BYTES;
#pragma unroll
      for (int k = 0; k < KB / 32; ++k)
        mma_issue(tmem, sdesc(a0 + 32 * k), sdesc(b0 + 32 * k), idesc, (step > 0 || k > 0) ? 1u : 0u, P.tf32);
      mma_commit(&empty[s]);
    }
    mma_commit(&done);
  }
  __syncthreads();   // roles finished issuing (s_fail visible); the MMAs may still run
  // Epilogue mapping: warp w reads TMEM lane quarter (w % 4) and the column
  // half (w / 4) of the tile.  Real row rr of the tile is complex row i,
  // component comp (re/im), so consecutive lanes hit consecutive floats of a
  // column (coalesced).  The C segment is prefetched while the MMAs run.
  constexpr int HALF = BN / 2;
  const int quarter = warp & 3, half = warp >> 2;
  const int rr = row0 + quarter * 32 + lane;
  const int i = P.base + (rr >> 1);
  const int comp = rr & 1;
  const int cbase = P.base + col0 + half * HALF;
  float* Cc = reinterpret_cast<float*>(P.C + size_t(item) * P.stride);
  float cv[HALF];
  if (i < P.n) {
#pragma unroll
    for (int j = 0; j < HALF; ++j) {
      const int col = cbase + j;
      cv[j] = (col < P.n) ? Cc[2 * (size_t(col) * P.ld + i) + comp] : 0.f;
    }
  }
  const bool have = mbar_wait(&done, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (have && !s_fail) {
#pragma unroll
    for (int cc = 0; cc < HALF; cc += 32) {
      uint32_t v[32];
      tmem_ld32(tmem + (uint32_t(quarter * 32) << 16) + half * HALF + cc, v);
      if (i < P.n) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = cbase + cc + j;
          if (col < P.n) Cc[2 * (size_t(col) * P.ld + i) + comp] = cv[cc + j] - __uint_as_float(v[j]);
        }
      }
    }
  }
  if (!have || s_fail) {
    if (threadIdx.x == 0) atomicExch(P.err, 1);
    // drain: wait (bounded) for every TMA stage this CTA armed
    if (warp == 0 && lane == 0)
      for (int step = (issued > STAGES ? issued - STAGES : 0); step < issued; ++step)
        mbar_wait(&full[step % STAGES], (step / STAGES) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
}

// ------------------------------------------------------- streamed kernel --
// Tiles of 128 real rows x 64 complex columns.  A CTA takes a run of up to
// P.run consecutive row tiles of one column tile: the column block of U
// (B_hi and B_lo for all K, 32 KB) is loaded once and stays in shared memory,
// the A rows stream through a 3-stage ring (A_hi and A_lo of one 128-byte K
// step per stage, so A_hi is fetched once for both products that use it), and
// C tiles stream through 3 buffers: a C-mover warp keeps two C loads in
// flight, and stores each tile once the epilogue warps have updated it, so
// the epilogue never waits on a store.
constexpr int SBN = 64;                        // complex columns per tile
constexpr int S_STAGES = 3;                    // A ring depth
constexpr int S_CBUF = 3;                      // C tile buffers
constexpr int C_TILE_BYTES = BM * SBN * 4;     // 128 floats x 64 columns
constexpr int S_THREADS = 352;                 // producer, MMA, 8 epilogue warps, C mover
constexpr int S_KSTEPS = 2;                    // 128-byte K steps per product (K = 2 x 64 complex)
constexpr int SA_BYTES = BM * KB;              // one A operand K step
constexpr int SB_BYTES = SBN * KB;             // one B operand K step
constexpr int S_STAGE_BYTES = 2 * SA_BYTES;    // A_hi + A_lo
constexpr int S_B_BYTES = 2 * S_KSTEPS * SB_BYTES;
constexpr size_t S_SMEM = size_t(S_STAGES) * S_STAGE_BYTES + S_B_BYTES + size_t(S_CBUF) * C_TILE_BYTES + 1024;

struct TcsParams {
  float* C;      // C as floats (tmem-C kernel only): item `stride2` floats apart, columns ld2 floats apart
  size_t stride2;
  int ld2, n;
  int base;      // first trailing row/column (k0 + nbe)
  int abase;     // base rounded down to even: row origin of the tiles (16-byte TMA rule)
  int rt, ct;    // row tiles, column tiles of this launch
  int col_tile0; // first column tile
  int run;       // row tiles per CTA
  int rruns;     // runs per column tile
  int* err;
  int tf32;
  int aoff;      // first row of the A operand's slot in the pack (0 or rows_pad)
  int boff;      // ... of the B operand's slot
  int aoff2, boff2;   // the second step's slots (tmac kernel with K = 128 only)
};

// CTA b: item, column tile and first row tile of its run; runs of one item
// are numbered consecutively so the CTAs resident at a time share an item
// and its packed operands stay in L2.
__device__ __forceinline__ void run_coords(const TcsParams& P, int b, int& rt0, int& ntile, int& col0, int& item) {
  const int rr = b % P.rruns;
  const int c = (b / P.rruns) % P.ct;
  item = b / (P.rruns * P.ct);
  rt0 = rr * P.run;
  ntile = min(P.run, P.rt - rt0);
  col0 = (c + P.col_tile0) * SBN;
}

__global__ void __launch_bounds__(S_THREADS, 1)
    tc_update_streamed(const __grid_constant__ CUtensorMap tA_hi, const __grid_constant__ CUtensorMap tA_lo,
                       const __grid_constant__ CUtensorMap tB_hi, const __grid_constant__ CUtensorMap tB_lo,
                       const __grid_constant__ CUtensorMap tC, TcsParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* bres = smem + S_STAGES * S_STAGE_BYTES;   // [hi k0, hi k1, lo k0, lo k1]
  uint8_t* cbuf = bres + S_B_BYTES;
  __shared__ __align__(8) uint64_t full[S_STAGES];
  __shared__ __align__(8) uint64_t empty[S_STAGES];
  __shared__ __align__(8) uint64_t bfull;        // resident B landed
  __shared__ __align__(8) uint64_t cfull[S_CBUF]; // C tile landed
  __shared__ __align__(8) uint64_t cdone[S_CBUF]; // C tile updated by the epilogue (8 warps)
  __shared__ __align__(8) uint64_t afull[2];     // accumulator ready
  __shared__ __align__(8) uint64_t aempty[2];    // accumulator read out
  __shared__ __align__(8) uint64_t mdone;        // every MMA of this CTA retired
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail_raw;
  volatile int* s_fail = &s_fail_raw;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int rt0, ntile, col0, item;
  run_coords(P, blockIdx.x, rt0, ntile, col0, item);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < S_CBUF; ++b) {
      mbar_init(&cfull[b], 1);
      mbar_init(&cdone[b], 8);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&afull[b], 1);
      mbar_init(&aempty[b], 8);
    }
    mbar_init(&bfull, 1);
    mbar_init(&mdone, 1);
    s_fail_raw = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(2 * SBN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const int kstep_elems = P.tf32 ? KB / 4 : KB / 2;

  if (warp == 0 && lane == 0) {
    // producer: the resident B block once, then two A stages per tile
    mbar_expect_tx(&bfull, S_B_BYTES);
    for (int kb = 0; kb < S_KSTEPS; ++kb) {
      tma_load_3d(bres + kb * SB_BYTES, &tB_hi, kb * kstep_elems, P.base + col0, item, &bfull);
      tma_load_3d(bres + (S_KSTEPS + kb) * SB_BYTES, &tB_lo, kb * kstep_elems, P.base + col0, item, &bfull);
    }
    int gs = 0;
    for (int lt = 0; lt < ntile; ++lt) {
      const int row0 = (rt0 + lt) * BM;
      bool ok = true;
      for (int kb = 0; kb < S_KSTEPS; ++kb, ++gs) {
        const int s = gs % S_STAGES;
        if (gs >= S_STAGES && !mbar_wait_f(&empty[s], ((gs / S_STAGES) - 1) & 1, s_fail)) { ok = false; break; }
        uint8_t* sa = smem + s * S_STAGE_BYTES;
        mbar_expect_tx(&full[s], S_STAGE_BYTES);
        tma_load_3d(sa, &tA_hi, kb * kstep_elems, P.aoff + 2 * P.abase + row0, item, &full[s]);
        tma_load_3d(sa + SA_BYTES, &tA_lo, kb * kstep_elems, P.aoff + 2 * P.abase + row0, item, &full[s]);
      }
      if (!ok) break;
    }
    if (*s_fail) {
      // drain: the last load armed on each barrier must land before the CTA exits
      volatile int dummy = 0;
      mbar_wait_f(&bfull, 0, &dummy);
      for (int s = 0; s < S_STAGES && s < gs; ++s) {
        const int cnt = (gs - s + S_STAGES - 1) / S_STAGES;   // loads armed on full[s]
        mbar_wait_f(&full[s], (cnt - 1) & 1, &dummy);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: per K step, A_hi B_hi + A_hi B_lo + A_lo B_hi into accumulator lt & 1
    const uint32_t fmt = P.tf32 ? 2u : 1u;
    const uint32_t idesc =
        (1u << 4) | (fmt << 7) | (fmt << 10) | (uint32_t(SBN >> 3) << 17) | (uint32_t(BM >> 4) << 24);
    bool ok = mbar_wait_f(&bfull, 0, s_fail);
    const uint32_t bh = smem_u32(bres), bl = bh + S_KSTEPS * SB_BYTES;
    int gs = 0;
    for (int lt = 0; lt < ntile && ok; ++lt) {
      const int ab = lt & 1;
      if (lt >= 2 && !mbar_wait_f(&aempty[ab], ((lt >> 1) - 1) & 1, s_fail)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t acc = tmem + uint32_t(ab * SBN);
      for (int kb = 0; kb < S_KSTEPS; ++kb, ++gs) {
        const int s = gs % S_STAGES;
        if (!mbar_wait_f(&full[s], (gs / S_STAGES) & 1, s_fail)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ah = smem_u32(smem + s * S_STAGE_BYTES), al = ah + SA_BYTES;
        const uint32_t bhk = bh + kb * SB_BYTES, blk = bl + kb * SB_BYTES;
#pragma unroll
        for (int kk = 0; kk < KB / 32; ++kk) {
          mma_issue(acc, sdesc(ah + 32 * kk), sdesc(bhk + 32 * kk), idesc, (kb > 0 || kk > 0) ? 1u : 0u, P.tf32);
          mma_issue(acc, sdesc(ah + 32 * kk), sdesc(blk + 32 * kk), idesc, 1u, P.tf32);
          mma_issue(acc, sdesc(al + 32 * kk), sdesc(bhk + 32 * kk), idesc, 1u, P.tf32);
        }
        mma_commit(&empty[s]);
      }
      if (ok) mma_commit(&afull[ab]);
    }
    // TMEM is freed only after every MMA issued here has retired
    mma_commit(&mdone);
    volatile int dummy = 0;
    mbar_wait_f(&mdone, 0, &dummy);
  } else if (warp >= 2 && warp < 10) {
    // epilogue: warp w reads TMEM lane quarter w % 4 and column half (w - 2) / 4;
    // thread = one real row of the tile; C tile in shared memory [column][128 floats].
    // It never waits for stores: the C mover (warp 10) takes the tile from here.
    const int ew = warp - 2, quarter = warp & 3, half = ew >> 2;
    const int x = quarter * 32 + lane;
    for (int lt = 0; lt < ntile; ++lt) {
      const int cb = lt % S_CBUF, ab = lt & 1;
      if (!mbar_wait_f(&cfull[cb], (lt / S_CBUF) & 1, s_fail)) break;
      if (!mbar_wait_f(&afull[ab], (lt >> 1) & 1, s_fail)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int row0 = (rt0 + lt) * BM;
      float* cs = reinterpret_cast<float*>(cbuf + cb * C_TILE_BYTES);
      const bool live = (2 * P.abase + row0 + x) >= 2 * P.base;   // rows above base stay as they are
      uint32_t v[32];
      tmem_ld32(tmem + (uint32_t(quarter * 32) << 16) + uint32_t(ab * SBN + half * 32), v);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&aempty[ab]);
      if (live) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          float* e = cs + (half * 32 + j) * BM + x;
          *e = *e - __uint_as_float(v[j]);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&cdone[cb]);
    }
  } else if (warp == 10 && lane == 0) {
    // C mover: the first S_CBUF tile loads, then per tile: wait for the
    // epilogue, store the tile, and once the store has read the buffer, load
    // the tile S_CBUF ahead into it
    int c_issued = 0;
    for (; c_issued < S_CBUF && c_issued < ntile; ++c_issued) {
      const int cb = c_issued;
      mbar_expect_tx(&cfull[cb], C_TILE_BYTES);
      tma_load_3d(cbuf + cb * C_TILE_BYTES, &tC, 2 * P.abase + (rt0 + c_issued) * BM, P.base + col0, item,
                  &cfull[cb]);
    }
    for (int lt = 0; lt < ntile; ++lt) {
      const int cb = lt % S_CBUF;
      if (!mbar_wait_f(&cdone[cb], (lt / S_CBUF) & 1, s_fail)) break;
      float* cs = reinterpret_cast<float*>(cbuf + cb * C_TILE_BYTES);
      tma_store_3d(&tC, cs, 2 * P.abase + (rt0 + lt) * BM, P.base + col0, item);   // returns once read
      if (c_issued < ntile) {
        mbar_expect_tx(&cfull[cb], C_TILE_BYTES);
        tma_load_3d(cs, &tC, 2 * P.abase + (rt0 + c_issued) * BM, P.base + col0, item, &cfull[cb]);
        ++c_issued;
      }
    }
    if (*s_fail) {
      // drain the C loads still in flight
      volatile int dummy = 0;
      for (int cb = 0; cb < S_CBUF && cb < c_issued; ++cb) {
        const int cnt = (c_issued - cb + S_CBUF - 1) / S_CBUF;
        mbar_wait_f(&cfull[cb], (cnt - 1) & 1, &dummy);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && *s_fail) atomicExch(P.err, 1);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * SBN));
}

// ------------------------------------------ streamed, C through registers --
// Same runs, operands and resident B block as the streamed kernel, but C never
// passes through shared memory: the epilogue warps load a tile of C from
// global memory into registers ahead of time, read the tile's accumulator
// once its MMAs are done, and store C - A'B' straight to global memory.  The
// products are still summed from zero in TMEM (adding them onto C there would
// round each partial sum at the scale of C).  Shared memory then carries only
// the MMA operands, which leaves room for a deeper A ring (or two CTAs per SM).
// KS = 4: two paired panel steps per pass (as in the TMA-C kernel below), with
// the deeper A ring that the K = 128 pass needs to keep its A loads in flight.
template <int STAGES, int KS = 2>
struct RegcCfg {
  static constexpr int THREADS = 320;   // producer, MMA, 8 epilogue warps
  static constexpr int B_BYTES = 2 * KS * SB_BYTES;
  static constexpr size_t SMEM = size_t(STAGES) * S_STAGE_BYTES + B_BYTES + 1024;
};
static_assert(RegcCfg<5, 4>::SMEM <= 227 * 1024, "regc shared memory");

template <int STAGES, int KS = 2>
__global__ void __launch_bounds__(RegcCfg<STAGES, KS>::THREADS, RegcCfg<STAGES, KS>::SMEM * 2 <= 227 * 1024 ? 2 : 1)
    tc_update_regc(const __grid_constant__ CUtensorMap tA_hi, const __grid_constant__ CUtensorMap tA_lo,
                    const __grid_constant__ CUtensorMap tB_hi, const __grid_constant__ CUtensorMap tB_lo, TcsParams P) {
  constexpr int R_B_BYTES = RegcCfg<STAGES, KS>::B_BYTES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* bres = smem + STAGES * S_STAGE_BYTES;   // [hi k0 .. k(KS-1), lo k0 .. k(KS-1)]
  __shared__ __align__(8) uint64_t full[STAGES];
  __shared__ __align__(8) uint64_t empty[STAGES];
  __shared__ __align__(8) uint64_t bfull;        // resident B landed
  __shared__ __align__(8) uint64_t aempty[2];    // accumulator read out (8 epilogue warps)
  __shared__ __align__(8) uint64_t afull[2];     // accumulator ready
  __shared__ __align__(8) uint64_t mdone;        // every MMA of this CTA retired
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail_raw;
  volatile int* s_fail = &s_fail_raw;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int rt0, ntile, col0, item;
  run_coords(P, blockIdx.x, rt0, ntile, col0, item);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&aempty[b], 8);
      mbar_init(&afull[b], 1);
    }
    mbar_init(&bfull, 1);
    mbar_init(&mdone, 1);
    s_fail_raw = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(2 * SBN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const int kstep_elems = KB / 2;

  if (warp == 0 && lane == 0) {
    // producer: the resident B block once, then KS A stages per tile (K
    // steps 2-3 of a paired pass from the second step's operand slots)
    mbar_expect_tx(&bfull, R_B_BYTES);
    for (int kb = 0; kb < KS; ++kb) {
      const int brow = (kb < 2 ? P.boff : P.boff2) + P.base + col0, kc = (kb & 1) * kstep_elems;
      tma_load_3d(bres + kb * SB_BYTES, &tB_hi, kc, brow, item, &bfull);
      tma_load_3d(bres + (KS + kb) * SB_BYTES, &tB_lo, kc, brow, item, &bfull);
    }
    int gs = 0;
    for (int lt = 0; lt < ntile; ++lt) {
      const int row0 = (rt0 + lt) * BM;
      bool ok = true;
      for (int kb = 0; kb < KS; ++kb, ++gs) {
        const int s = gs % STAGES;
        if (gs >= STAGES && !mbar_wait_f(&empty[s], ((gs / STAGES) - 1) & 1, s_fail)) { ok = false; break; }
        uint8_t* sa = smem + s * S_STAGE_BYTES;
        const int arow = (kb < 2 ? P.aoff : P.aoff2) + 2 * P.abase + row0, kc = (kb & 1) * kstep_elems;
        mbar_expect_tx(&full[s], S_STAGE_BYTES);
        tma_load_3d(sa, &tA_hi, kc, arow, item, &full[s]);
        tma_load_3d(sa + SA_BYTES, &tA_lo, kc, arow, item, &full[s]);
      }
      if (!ok) break;
    }
    if (*s_fail) {
      volatile int dummy = 0;
      mbar_wait_f(&bfull, 0, &dummy);
      for (int s = 0; s < STAGES && s < gs; ++s) {
        const int cnt = (gs - s + STAGES - 1) / STAGES;   // loads armed on full[s]
        mbar_wait_f(&full[s], (cnt - 1) & 1, &dummy);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: per K step A_hi B_hi + A_hi B_lo + A_lo B_hi into accumulator lt & 1
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(SBN >> 3) << 17) | (uint32_t(BM >> 4) << 24);
    bool ok = mbar_wait_f(&bfull, 0, s_fail);
    const uint32_t bh = smem_u32(bres), bl = bh + KS * SB_BYTES;
    int gs = 0;
    for (int lt = 0; lt < ntile && ok; ++lt) {
      const int ab = lt & 1;
      if (lt >= 2 && !mbar_wait_f(&aempty[ab], ((lt >> 1) - 1) & 1, s_fail)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t acc = tmem + uint32_t(ab * SBN);
      for (int kb = 0; kb < KS; ++kb, ++gs) {
        const int s = gs % STAGES;
        if (!mbar_wait_f(&full[s], (gs / STAGES) & 1, s_fail)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ah = smem_u32(smem + s * S_STAGE_BYTES), al = ah + SA_BYTES;
        const uint32_t bhk = bh + kb * SB_BYTES, blk = bl + kb * SB_BYTES;
#pragma unroll
        for (int kk = 0; kk < KB / 32; ++kk) {
          mma_issue(acc, sdesc(ah + 32 * kk), sdesc(bhk + 32 * kk), idesc, (kb > 0 || kk > 0) ? 1u : 0u, 0);
          mma_issue(acc, sdesc(ah + 32 * kk), sdesc(blk + 32 * kk), idesc, 1u, 0);
          mma_issue(acc, sdesc(al + 32 * kk), sdesc(bhk + 32 * kk), idesc, 1u, 0);
        }
        mma_commit(&empty[s]);
      }
      if (ok) mma_commit(&afull[ab]);
    }
    mma_commit(&mdone);
    volatile int dummy = 0;
    mbar_wait_f(&mdone, 0, &dummy);
  } else if (warp >= 2) {
    // epilogue: warp w owns TMEM lane quarter w % 4 (float rows x of the
    // tile) and column half (w - 2) / 4; the C of tile t + 1 is in registers
    // (and that of t + 2 on its way) while tile t is finished
    const int ew = warp - 2, quarter = warp & 3, half = ew >> 2;
    const int x = quarter * 32 + lane;
    const int colb = P.base + col0 + half * 32;
    float* Cg = P.C + size_t(item) * P.stride2;
    const uint32_t lane_off = uint32_t(quarter * 32) << 16;
    auto load_tile = [&](int lt, float* c) {
      const int gr = 2 * P.abase + (rt0 + lt) * BM + x;
      const bool ok = lt < ntile && gr < 2 * P.n;
#pragma unroll
      for (int j = 0; j < 32; ++j)
        c[j] = (ok && colb + j < P.n) ? __ldcs(Cg + size_t(colb + j) * P.ld2 + gr) : 0.f;
    };
    // finish tile lt with its C in c: returns false when a wait gave up
    auto finish = [&](int lt, const float* c) {
      const int ab = lt & 1;
      if (!mbar_wait_f(&afull[ab], (lt >> 1) & 1, s_fail)) return false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint32_t v[32];
      tmem_ld32(tmem + lane_off + uint32_t(ab * SBN + half * 32), v);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&aempty[ab]);
      const int gr = 2 * P.abase + (rt0 + lt) * BM + x;
      if (gr >= 2 * P.base && gr < 2 * P.n) {   // rows above base stay as they are
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (colb + j < P.n) __stcs(Cg + size_t(colb + j) * P.ld2 + gr, c[j] - __uint_as_float(v[j]));
      }
      return true;
    };
    // two register sets used in turn (no copies between them, so a set's
    // loads are first needed two tiles after they were issued)
    float c0[32], c1[32];
    load_tile(0, c0);
    load_tile(1, c1);
    for (int lt = 0; lt < ntile; lt += 2) {
      if (!finish(lt, c0)) break;
      load_tile(lt + 2, c0);
      if (lt + 1 < ntile) {
        if (!finish(lt + 1, c1)) break;
        load_tile(lt + 3, c1);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && *s_fail) atomicExch(P.err, 1);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * SBN));
}

// Variant of the register kernel whose C tiles come in by TMA (a loader warp
// keeps up to T_CBUF tiles in flight in shared memory); the epilogue reads
// them from there and stores C - A'B' straight to global memory.
// KS = 2: one panel step (K = 64 complex, two 128-byte K steps); KS = 4: two
// panel steps applied in one pass (K = 128 complex: K steps 0-1 from the
// first step's operands, 2-3 from the second's, at the row offsets
// aoff/boff and aoff2/boff2 of their pack slots), which halves the C traffic
// of the pair; its larger resident B block leaves room for two C buffers.
template <int KS>
struct TmacCfg {
  static constexpr int CBUF = KS == 2 ? 3 : 2;
  static constexpr int STAGES = 3;
  static constexpr int B_BYTES = 2 * KS * SB_BYTES;
  static constexpr size_t SMEM =
      size_t(STAGES) * S_STAGE_BYTES + B_BYTES + size_t(CBUF) * C_TILE_BYTES + 1024;
};
constexpr int T_THREADS = 352;                 // producer, MMA, 8 epilogue warps, C loader
static_assert(TmacCfg<2>::SMEM <= 227 * 1024 && TmacCfg<4>::SMEM <= 227 * 1024, "tmac shared memory");

template <int KS>
__global__ void __launch_bounds__(T_THREADS, 1)
    tc_update_tmac(const __grid_constant__ CUtensorMap tA_hi, const __grid_constant__ CUtensorMap tA_lo,
                   const __grid_constant__ CUtensorMap tB_hi, const __grid_constant__ CUtensorMap tB_lo,
                   const __grid_constant__ CUtensorMap tC, TcsParams P) {
  constexpr int T_CBUF = TmacCfg<KS>::CBUF, T_STAGES = TmacCfg<KS>::STAGES, T_B_BYTES = TmacCfg<KS>::B_BYTES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* bres = smem + T_STAGES * S_STAGE_BYTES;   // [hi k0 .. k(KS-1), lo k0 .. k(KS-1)]
  uint8_t* cbuf = bres + T_B_BYTES;
  __shared__ __align__(8) uint64_t full[T_STAGES];
  __shared__ __align__(8) uint64_t empty[T_STAGES];
  __shared__ __align__(8) uint64_t bfull;
  __shared__ __align__(8) uint64_t cfull[T_CBUF];   // C tile landed
  __shared__ __align__(8) uint64_t cfree[T_CBUF];   // C tile read by the epilogue (8 warps)
  __shared__ __align__(8) uint64_t aempty[2];
  __shared__ __align__(8) uint64_t afull[2];
  __shared__ __align__(8) uint64_t mdone;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail_raw;
  volatile int* s_fail = &s_fail_raw;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int rt0, ntile, col0, item;
  run_coords(P, blockIdx.x, rt0, ntile, col0, item);

  if (threadIdx.x == 0) {
    for (int s = 0; s < T_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < T_CBUF; ++b) {
      mbar_init(&cfull[b], 1);
      mbar_init(&cfree[b], 8);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&aempty[b], 8);
      mbar_init(&afull[b], 1);
    }
    mbar_init(&bfull, 1);
    mbar_init(&mdone, 1);
    s_fail_raw = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(2 * SBN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const int kstep_elems = KB / 2;

  if (warp == 0 && lane == 0) {
    mbar_expect_tx(&bfull, T_B_BYTES);
    for (int kb = 0; kb < KS; ++kb) {
      const int brow = (kb < 2 ? P.boff : P.boff2) + P.base + col0, kc = (kb & 1) * kstep_elems;
      tma_load_3d(bres + kb * SB_BYTES, &tB_hi, kc, brow, item, &bfull);
      tma_load_3d(bres + (KS + kb) * SB_BYTES, &tB_lo, kc, brow, item, &bfull);
    }
    int gs = 0;
    for (int lt = 0; lt < ntile; ++lt) {
      const int row0 = (rt0 + lt) * BM;
      bool ok = true;
      for (int kb = 0; kb < KS; ++kb, ++gs) {
        const int s = gs % T_STAGES;
        if (gs >= T_STAGES && !mbar_wait_f(&empty[s], ((gs / T_STAGES) - 1) & 1, s_fail)) { ok = false; break; }
        uint8_t* sa = smem + s * S_STAGE_BYTES;
        const int arow = (kb < 2 ? P.aoff : P.aoff2) + 2 * P.abase + row0, kc = (kb & 1) * kstep_elems;
        mbar_expect_tx(&full[s], S_STAGE_BYTES);
        tma_load_3d(sa, &tA_hi, kc, arow, item, &full[s]);
        tma_load_3d(sa + SA_BYTES, &tA_lo, kc, arow, item, &full[s]);
      }
      if (!ok) break;
    }
    if (*s_fail) {
      volatile int dummy = 0;
      mbar_wait_f(&bfull, 0, &dummy);
      for (int s = 0; s < T_STAGES && s < gs; ++s) {
        const int cnt = (gs - s + T_STAGES - 1) / T_STAGES;
        mbar_wait_f(&full[s], (cnt - 1) & 1, &dummy);
      }
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(SBN >> 3) << 17) | (uint32_t(BM >> 4) << 24);
    bool ok = mbar_wait_f(&bfull, 0, s_fail);
    const uint32_t bh = smem_u32(bres), bl = bh + KS * SB_BYTES;
    int gs = 0;
    for (int lt = 0; lt < ntile && ok; ++lt) {
      const int ab = lt & 1;
      if (lt >= 2 && !mbar_wait_f(&aempty[ab], ((lt >> 1) - 1) & 1, s_fail)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t acc = tmem + uint32_t(ab * SBN);
      for (int kb = 0; kb < KS; ++kb, ++gs) {
        const int s = gs % T_STAGES;
        if (!mbar_wait_f(&full[s], (gs / T_STAGES) & 1, s_fail)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ah = smem_u32(smem + s * S_STAGE_BYTES), al = ah + SA_BYTES;
        const uint32_t bhk = bh + kb * SB_BYTES, blk = bl + kb * SB_BYTES;
#pragma unroll
        for (int kk = 0; kk < KB / 32; ++kk) {
          mma_issue(acc, sdesc(ah + 32 * kk), sdesc(bhk + 32 * kk), idesc, (kb > 0 || kk > 0) ? 1u : 0u, 0);
          mma_issue(acc, sdesc(ah + 32 * kk), sdesc(blk + 32 * kk), idesc, 1u, 0);
          mma_issue(acc, sdesc(al + 32 * kk), sdesc(bhk + 32 * kk), idesc, 1u, 0);
        }
        mma_commit(&empty[s]);
      }
      if (ok) mma_commit(&afull[ab]);
    }
    mma_commit(&mdone);
    volatile int dummy = 0;
    mbar_wait_f(&mdone, 0, &dummy);
  } else if (warp >= 2 && warp < 10) {
    // epilogue: C from the shared-memory tile, result stored to global memory
    const int ew = warp - 2, quarter = warp & 3, half = ew >> 2;
    const int x = quarter * 32 + lane;
    const int colb = P.base + col0 + half * 32;
    float* Cg = P.C + size_t(item) * P.stride2;
    const uint32_t lane_off = uint32_t(quarter * 32) << 16;
    for (int lt = 0; lt < ntile; ++lt) {
      const int ab = lt & 1, cb = lt % T_CBUF;
      if (!mbar_wait_f(&afull[ab], (lt >> 1) & 1, s_fail)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint32_t v[32];
      tmem_ld32(tmem + lane_off + uint32_t(ab * SBN + half * 32), v);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&aempty[ab]);
      if (!mbar_wait_f(&cfull[cb], (lt / T_CBUF) & 1, s_fail)) break;
      const float* cs = reinterpret_cast<const float*>(cbuf + cb * C_TILE_BYTES);
      // C - A'B' is formed before the buffer is handed back: the loader's
      // next TMA write into it (async proxy) must not overtake these reads
      // (generic proxy), so the values are consumed and the reads fenced
      // against the async proxy before the release.  (Without this, tiles
      // came out stale when other kernels ran concurrently on the GPU.)
      float c[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) c[j] = cs[(half * 32 + j) * BM + x] - __uint_as_float(v[j]);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&cfree[cb]);
      const int gr = 2 * P.abase + (rt0 + lt) * BM + x;
      if (gr >= 2 * P.base && gr < 2 * P.n) {   // rows above base stay as they are
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (colb + j < P.n) __stcs(Cg + size_t(colb + j) * P.ld2 + gr, c[j]);
      }
    }
  } else if (warp == 10 && lane == 0) {
    // C loader: tile lt into buffer lt % T_CBUF once the epilogue has read tile lt - T_CBUF from it
    int issued = 0;
    for (; issued < ntile; ++issued) {
      const int cb = issued % T_CBUF;
      if (issued >= T_CBUF && !mbar_wait_f(&cfree[cb], ((issued / T_CBUF) - 1) & 1, s_fail)) break;
      mbar_expect_tx(&cfull[cb], C_TILE_BYTES);
      tma_load_3d(cbuf + cb * C_TILE_BYTES, &tC, 2 * P.abase + (rt0 + issued) * BM, P.base + col0, item, &cfull[cb]);
    }
    if (*s_fail) {
      volatile int dummy = 0;
      for (int cb = 0; cb < T_CBUF && cb < issued; ++cb) {
        const int cnt = (issued - cb + T_CBUF - 1) / T_CBUF;
        mbar_wait_f(&cfull[cb], (cnt - 1) & 1, &dummy);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && *s_fail) atomicExch(P.err, 1);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * SBN));
}

// ---------------------------------------------------------------- packing --
__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16_raw& hi, __nv_bfloat16_raw& lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
  hi = static_cast<__nv_bfloat16_raw>(h);
  lo = static_cast<__nv_bfloat16_raw>(l);
}

__device__ __forceinline__ float tf32_rna(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

// A'-pack rows 2i, 2i+1 for matrix rows i in [base, n); K = 2p, 2p+1 for
// panel column p < nbe, zero for p in [nbe, Kp/2).  Layout [item][row][Kp].
template <typename T>
__global__ void pack_a_kernel(const float2* __restrict__ C0, size_t stride, int ld, int n, int k0, int nbe, int base,
                              int Kp, int rows_pad, T* __restrict__ hi0, T* __restrict__ lo0, int tf32) {
  const int item = blockIdx.y;
  const int half = Kp / 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = base + t / half, p = t % half;
  if (i >= n) return;
  float2 v = make_float2(0.f, 0.f);
  if (p < nbe) v = C0[size_t(item) * stride + size_t(k0 + p) * ld + i];
  const float e[4] = {v.x, -v.y, v.y, v.x};   // row 2i: (Lr, -Li); row 2i+1: (Li, Lr)
  T* hi = hi0 + size_t(item) * rows_pad * Kp;
  T* lo = lo0 + size_t(item) * rows_pad * Kp;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const size_t off = size_t(2 * i + (q >> 1)) * Kp + 2 * p + (q & 1);
    if constexpr (sizeof(T) == 2) {
      __nv_bfloat16_raw h, l;
      split_bf16(e[q], h, l);
      hi[off] = *reinterpret_cast<T*>(&h);
      lo[off] = *reinterpret_cast<T*>(&l);
    } else {
      const float h = tf32_rna(e[q]);
      hi[off] = h;
      lo[off] = tf32_rna(e[q] - h);
    }
  }
}

// The same A'-pack for the BF16 splits through a shared-memory tile of
// PACK_ROWS matrix rows x the panel's K per CTA: read down the columns
// (consecutive threads take consecutive rows of one column) and written along
// K as BF16 pairs (consecutive threads take consecutive K pairs of one row),
// so both sides are coalesced; every element is split exactly as above.
constexpr int PACK_ROWS = 16;

__global__ void __launch_bounds__(256) pack_a_bf16_tiled_kernel(const float2* __restrict__ C0, size_t stride, int ld,
                                                                int n, int k0, int nbe, int base, int Kp, int rows_pad,
                                                                uint16_t* __restrict__ hi0, uint16_t* __restrict__ lo0) {
  __shared__ float2 tile[64][PACK_ROWS + 1];   // [p][row]
  const int item = blockIdx.y;
  const int half = Kp / 2;                     // complex K of the pack (<= 64)
  const int i0 = base + blockIdx.x * PACK_ROWS;
  const float2* C = C0 + size_t(item) * stride;
  for (int t = threadIdx.x; t < half * PACK_ROWS; t += blockDim.x) {
    const int p = t / PACK_ROWS, r = t % PACK_ROWS, i = i0 + r;
    float2 v = make_float2(0.f, 0.f);
    if (p < nbe && i < n) v = C[size_t(k0 + p) * ld + i];
    tile[p][r] = v;
  }
  __syncthreads();
  uint16_t* hi = hi0 + size_t(item) * rows_pad * Kp;
  uint16_t* lo = lo0 + size_t(item) * rows_pad * Kp;
  for (int t = threadIdx.x; t < PACK_ROWS * half; t += blockDim.x) {
    const int r = t / half, p = t % half, i = i0 + r;
    if (i >= n) continue;
    const float2 v = tile[p][r];
    const float e[4] = {v.x, -v.y, v.y, v.x};   // row 2i: (Lr, -Li); row 2i+1: (Li, Lr)
    __nv_bfloat16_raw h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) split_bf16(e[q], h[q], l[q]);
    const size_t o0 = size_t(2 * i) * Kp + 2 * p, o1 = o0 + Kp;
    *reinterpret_cast<uint32_t*>(hi + o0) = uint32_t(h[0].x) | (uint32_t(h[1].x) << 16);
    *reinterpret_cast<uint32_t*>(lo + o0) = uint32_t(l[0].x) | (uint32_t(l[1].x) << 16);
    *reinterpret_cast<uint32_t*>(hi + o1) = uint32_t(h[2].x) | (uint32_t(h[3].x) << 16);
    *reinterpret_cast<uint32_t*>(lo + o1) = uint32_t(l[2].x) | (uint32_t(l[3].x) << 16);
  }
}

// B'-pack row j (matrix column j in [base, n)): K = 2p -> Ur(p,j), 2p+1 -> Ui(p,j).
template <typename T>
__global__ void pack_b_kernel(const float2* __restrict__ C0, size_t stride, int ld, int n, int k0, int nbe, int base,
                              int Kp, int rows_pad, T* __restrict__ hi0, T* __restrict__ lo0, int tf32) {
  const int item = blockIdx.y;
  const int half = Kp / 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = base + t / half, p = t % half;
  if (j >= n) return;
  float2 v = make_float2(0.f, 0.f);
  if (p < nbe) v = C0[size_t(item) * stride + size_t(j) * ld + k0 + p];
  const float e[2] = {v.x, v.y};
  T* hi = hi0 + size_t(item) * rows_pad * Kp;
  T* lo = lo0 + size_t(item) * rows_pad * Kp;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const size_t off = size_t(j) * Kp + 2 * p + q;
    if constexpr (sizeof(T) == 2) {
      __nv_bfloat16_raw h, l;
      split_bf16(e[q], h, l);
      hi[off] = *reinterpret_cast<T*>(&h);
      lo[off] = *reinterpret_cast<T*>(&l);
    } else {
      const float h = tf32_rna(e[q]);
      hi[off] = h;
      lo[off] = tf32_rna(e[q] - h);
    }
  }
}

// Row interchanges of a later panel step applied to the A operand of an
// earlier one: pack rows (2c, 2c+1) <-> (2p, 2p+1) for c in [c0, c0 + nsw),
// p = piv[c], in order (as the interchanges were applied to the matrix).
// One CTA per item, one thread per 32-bit word column of the hi and lo rows.
__global__ void pack_swap_kernel(uint32_t* __restrict__ hi0, uint32_t* __restrict__ lo0, size_t item_words, int KW,
                                 const int* __restrict__ piv0, int r, int c0, int nsw) {
  const int item = blockIdx.x, t = threadIdx.x;
  if (t >= 4 * KW) return;
  const int arr = t / (2 * KW), sub = (t / KW) & 1, w = t % KW;
  uint32_t* P = (arr ? lo0 : hi0) + size_t(item) * item_words;
  const int* piv = piv0 + size_t(item) * r;
  for (int j = 0; j < nsw; ++j) {
    const int c = c0 + j, p = piv[c];
    if (p != c) {
      uint32_t* x = P + size_t(2 * c + sub) * KW + w;
      uint32_t* y = P + size_t(2 * p + sub) * KW + w;
      const uint32_t v = *x;
      *x = *y;
      *y = v;
    }
  }
}

// ------------------------------------------------------------- host side --
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

bool get_encoder() {
  static std::once_flag once;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  return g_encode != nullptr;
}

bool make_map(CUtensorMap* m, void* base, bool tf32, int Kp, int rows, int items, int box_rows) {
  const int es = tf32 ? 4 : 2;
  cuuint64_t dims[3] = {cuuint64_t(Kp), cuuint64_t(rows), cuuint64_t(items)};
  cuuint64_t strides[2] = {cuuint64_t(Kp) * es, cuuint64_t(Kp) * es * rows};
  cuuint32_t box[3] = {cuuint32_t(KB / es), cuuint32_t(box_rows), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool make_c_map(CUtensorMap* m, float2* C, int ld, size_t stride, int n, int items) {
  cuuint64_t dims[3] = {cuuint64_t(2) * n, cuuint64_t(n), cuuint64_t(items)};
  cuuint64_t strides[2] = {cuuint64_t(ld) * 8, cuuint64_t(stride) * 8};
  cuuint32_t box[3] = {cuuint32_t(BM), cuuint32_t(SBN), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, C, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

constexpr int TC_STAGES = 3;
int g_tile_n = 128;   // 128 or 256 complex columns per tile (autotuned)
int g_streamed = 3;   // BF16 splits, streamed runs: 3: C loaded by TMA, stored from registers; 2: C loaded
                      // and stored through registers; 1: C through shared memory both ways; 0: per-tile kernel
int g_run = 32;       // row tiles per CTA of the streamed kernel
int g_pair_kernel = 3;   // kernel of the paired (K = 128) pass: 3 TMA-C, 2 register-C with a 5-stage A ring

template <int BN>
void launch_tc(const CUtensorMap& mah, const CUtensorMap& mal, const CUtensorMap& mbh, const CUtensorMap& mbl,
               const TcParams& P, int m, int items, int col_tiles, cudaStream_t st) {
  constexpr size_t smem = size_t(TC_STAGES) * (BM * KB + BN * KB) + 1024;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc_update_kernel<BN, TC_STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    attr = true;
  }
  dim3 grid((2 * m + BM - 1) / BM, col_tiles, items);
  tc_update_kernel<BN, TC_STAGES><<<grid, 256, smem, st>>>(mah, mal, mbh, mbl, P);
}

void launch_tc_streamed(const CUtensorMap& mah, const CUtensorMap& mal, const CUtensorMap& mbh,
                        const CUtensorMap& mbl, const CUtensorMap& mc, const TcsParams& P, int items,
                        cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc_update_streamed, cudaFuncAttributeMaxDynamicSharedMemorySize, int(S_SMEM));
    attr = true;
  }
  const int grid = P.rruns * P.ct * items;
  tc_update_streamed<<<grid, S_THREADS, S_SMEM, st>>>(mah, mal, mbh, mbl, mc, P);
}

template <int STAGES, int KS = 2>
void launch_tc_regc(const CUtensorMap& mah, const CUtensorMap& mal, const CUtensorMap& mbh, const CUtensorMap& mbl,
                     const TcsParams& P, int items, cudaStream_t st) {
  using Cfg = RegcCfg<STAGES, KS>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc_update_regc<STAGES, KS>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Cfg::SMEM));
    attr = true;
  }
  const int grid = P.rruns * P.ct * items;
  tc_update_regc<STAGES, KS><<<grid, Cfg::THREADS, Cfg::SMEM, st>>>(mah, mal, mbh, mbl, P);
}

template <int KS>
void launch_tc_tmac(const CUtensorMap& mah, const CUtensorMap& mal, const CUtensorMap& mbh, const CUtensorMap& mbl,
                    const CUtensorMap& mc, const TcsParams& P, int items, cudaStream_t st) {
  constexpr size_t smem = TmacCfg<KS>::SMEM;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc_update_tmac<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    attr = true;
  }
  const int grid = P.rruns * P.ct * items;
  tc_update_tmac<KS><<<grid, T_THREADS, smem, st>>>(mah, mal, mbh, mbl, mc, P);
}

int kp_of(bool tf32) {
  // K elements per pass padded to whole 128-byte stages
  const int per = tf32 ? KB / 4 : KB / 2;
  return ((2 * PANEL_NB + per - 1) / per) * per;
}

}  // namespace

int tc_panel_width(int) { return PANEL_NB; }

bool tc_set_tile_n(int bn) {
  if (bn != 128 && bn != 256) return false;
  g_tile_n = bn;
  return true;
}

int tc_get_tile_n() { return g_tile_n; }

bool tc_set_streamed(int on) {
  if (on < 0 || on > 3) return false;
  g_streamed = on;
  return true;
}
int tc_get_streamed() { return g_streamed; }

bool tc_set_run(int run) {
  if (run < 1 || run > 64) return false;
  g_run = run;
  return true;
}
int tc_get_run() { return g_run; }

bool tc_set_pair_kernel(int k) {
  if (k != 2 && k != 3) return false;
  g_pair_kernel = k;
  return true;
}
int tc_get_pair_kernel() { return g_pair_kernel; }

size_t tc_pack_bytes_per_item(int n) {
  const int rows_pad = 2 * ((n + 127) / 128) * 128;
  const size_t kp = size_t(kp_of(true));   // 4-byte elements: the larger of the two
  return 4 * a256(size_t(rows_pad) * kp * 4);
}

int tc_tile_n() { return g_tile_n; }

namespace {
struct PackGeom {
  bool tf32;
  int base, m, rows_pad, Kp, es, item_rows;
  size_t pbytes;
  char *pa_hi, *pa_lo, *pb_hi, *pb_lo;
};
PackGeom pack_geom(int precision, int n, int k0, int nbe, int items, char* packs) {
  PackGeom g;
  g.tf32 = (precision == MUST_MIXED_TF32X3);
  g.base = k0 + nbe;
  g.m = n - g.base;
  g.rows_pad = 2 * ((n + 127) / 128) * 128;
  g.Kp = kp_of(g.tf32);
  g.es = g.tf32 ? 4 : 2;
  g.pbytes = a256(size_t(g.rows_pad) * g.Kp * 4);
  g.pa_hi = packs;
  g.pa_lo = packs + size_t(items) * g.pbytes;
  g.pb_hi = packs + 2 * size_t(items) * g.pbytes;
  g.pb_lo = packs + 3 * size_t(items) * g.pbytes;
  g.item_rows = int(g.pbytes / (size_t(g.Kp) * g.es));
  return g;
}
}  // namespace

bool tc_pack_b_target(int precision, int n, int k0, int nbe, int items, char* packs, PackB* out, int slot) {
  const PackGeom g = pack_geom(precision, n, k0, nbe, items, packs);
  if (g.tf32 || slot < 0 || slot > 1) return false;
  const size_t boff = size_t(slot) * g.rows_pad * g.Kp;
  out->hi = reinterpret_cast<uint16_t*>(g.pb_hi) + boff;
  out->lo = reinterpret_cast<uint16_t*>(g.pb_lo) + boff;
  out->Kp = g.Kp;
  out->item_rows = g.item_rows;
  return true;
}

int tc_pack_slots(int precision) { return precision == MUST_MIXED_TF32X3 ? 1 : 2; }

bool tc_pack_swap_rows(int precision, int n, int k0, int nbe, int slot, int items, char* packs, const int* piv, int r,
                       int c0, int nsw, cudaStream_t st) {
  const PackGeom g = pack_geom(precision, n, k0, nbe, items, packs);
  if (g.tf32 || slot < 0 || slot > 1 || c0 < g.base || nsw < 0) {
    must_set_error("tc_pack_swap_rows: bad arguments");
    return false;
  }
  if (nsw == 0 || g.m <= 0) return true;
  const size_t aoff = size_t(slot) * g.rows_pad * g.Kp;   // BF16 elements
  const int KW = g.Kp / 2;
  ProfScope ps(PH_SWAP, st);
  pack_swap_kernel<<<items, 4 * KW, 0, st>>>(reinterpret_cast<uint32_t*>(reinterpret_cast<uint16_t*>(g.pa_hi) + aoff),
                                             reinterpret_cast<uint32_t*>(reinterpret_cast<uint16_t*>(g.pa_lo) + aoff),
                                             size_t(g.item_rows) * KW, KW, piv, r, c0, nsw);
  prof_launched(PH_SWAP, 1, items);
  return true;
}

bool tc_pack_a_target(int precision, int n, int k0, int nbe, int items, char* packs, int slot, PackB* out) {
  const PackGeom g = pack_geom(precision, n, k0, nbe, items, packs);
  if (g.tf32 || slot < 0 || slot >= tc_pack_slots(precision)) return false;
  const size_t aoff = size_t(slot) * g.rows_pad * g.Kp;
  out->hi = reinterpret_cast<uint16_t*>(g.pa_hi) + aoff;
  out->lo = reinterpret_cast<uint16_t*>(g.pa_lo) + aoff;
  out->Kp = g.Kp;
  out->item_rows = g.item_rows;
  return true;
}

bool tc_pack(int precision, float2* A, size_t stride, int ld, int n, int k0, int nbe, int items, char* packs,
             cudaStream_t st, bool with_b, int slot) {
  const PackGeom g = pack_geom(precision, n, k0, nbe, items, packs);
  if (g.m <= 0) return true;
  if (slot < 0 || slot >= tc_pack_slots(precision) || (slot && with_b)) {
    must_set_error("tc_pack: bad operand slot %d", slot);
    return false;
  }
  const size_t aoff = size_t(slot) * g.rows_pad * g.Kp;   // elements: slot 1 starts rows_pad rows in
  ProfScope ps(PH_PACK, st);
  const int half = g.Kp / 2;
  const int ta = g.m * half;
  dim3 grid((ta + 255) / 256, items);
  if (!with_b) {
    if (g.tf32)
      pack_a_kernel<float><<<grid, 256, 0, st>>>(A, stride, ld, n, k0, nbe, g.base, g.Kp, g.item_rows,
                                                 reinterpret_cast<float*>(g.pa_hi), reinterpret_cast<float*>(g.pa_lo),
                                                 1);
    else
      pack_a_bf16_tiled_kernel<<<dim3((g.m + PACK_ROWS - 1) / PACK_ROWS, items), 256, 0, st>>>(
          A, stride, ld, n, k0, nbe, g.base, g.Kp, g.item_rows, reinterpret_cast<uint16_t*>(g.pa_hi) + aoff,
          reinterpret_cast<uint16_t*>(g.pa_lo) + aoff);
    prof_launched(PH_PACK, 1, items);
    return true;
  }
  if (g.tf32) {
    pack_a_kernel<float><<<grid, 256, 0, st>>>(A, stride, ld, n, k0, nbe, g.base, g.Kp, g.item_rows,
                                               reinterpret_cast<float*>(g.pa_hi), reinterpret_cast<float*>(g.pa_lo), 1);
    pack_b_kernel<float><<<grid, 256, 0, st>>>(A, stride, ld, n, k0, nbe, g.base, g.Kp, g.item_rows,
                                               reinterpret_cast<float*>(g.pb_hi), reinterpret_cast<float*>(g.pb_lo), 1);
  } else {
    pack_a_bf16_tiled_kernel<<<dim3((g.m + PACK_ROWS - 1) / PACK_ROWS, items), 256, 0, st>>>(
        A, stride, ld, n, k0, nbe, g.base, g.Kp, g.item_rows, reinterpret_cast<uint16_t*>(g.pa_hi),
        reinterpret_cast<uint16_t*>(g.pa_lo));
    pack_b_kernel<uint16_t><<<grid, 256, 0, st>>>(A, stride, ld, n, k0, nbe, g.base, g.Kp, g.item_rows,
                                                  reinterpret_cast<uint16_t*>(g.pb_hi),
                                                  reinterpret_cast<uint16_t*>(g.pb_lo), 0);
  }
  prof_launched(PH_PACK, 2, items);
  return true;
}

bool tc_update(int precision, float2* A, size_t stride, int ld, int n, int k0, int nbe, int items, char* packs,
               int* err, int col_lo, int col_hi, cudaStream_t st, int slot) {
  return tc_update_steps(precision, A, stride, ld, n, TcStep{k0, nbe, slot, 0}, nullptr, items, packs, err, col_lo,
                         col_hi, -1, st);
}

bool tc_update_steps(int precision, float2* A, size_t stride, int ld, int n, TcStep s1, const TcStep* s2, int items,
                     char* packs, int* err, int col_lo, int col_hi, int row_tiles, cudaStream_t st) {
  if (!get_encoder()) {
    must_set_error("cuTensorMapEncodeTiled is not available");
    return false;
  }
  // the trailing block starts after the last step's panel
  const TcStep& last = s2 ? *s2 : s1;
  const PackGeom g = pack_geom(precision, n, last.k0, last.nbe, items, packs);
  if (g.m <= 0) return true;
  const int nslots = tc_pack_slots(precision);
  if (s1.slot < 0 || s1.slot >= nslots || s1.bslot < 0 || s1.bslot >= nslots ||
      (s2 && (s2->slot < 0 || s2->slot >= nslots || s2->bslot < 0 || s2->bslot >= nslots ||
              s2->k0 != s1.k0 + s1.nbe || s1.nbe != PANEL_NB))) {
    must_set_error("tc_update: bad operand slots or steps");
    return false;
  }
  if ((s2 || s1.bslot || row_tiles >= 0) && !(g_streamed == 3 && !g.tf32)) {
    must_set_error("tc_update: paired steps, B slots and row limits need the TMA-C streamed kernel (knob 2 = 3)");
    return false;
  }
  // The streamed kernel serves the BF16 splits (K = 2 x 128-byte steps per
  // product); TF32 splits and 256-column tiles use the per-tile kernel.
  const bool streamed = g_streamed && !g.tf32;
  const int bn = streamed ? SBN : g_tile_n;
  const int tiles = (g.m + bn - 1) / bn;
  const int t0 = col_lo / bn;
  const int t1 = (col_hi < 0) ? tiles : std::min(tiles, (col_hi + bn - 1) / bn);
  if (t1 <= t0) return true;
  CUtensorMap mah, mal, mbh, mbl;
  if (!make_map(&mah, g.pa_hi, g.tf32, g.Kp, g.item_rows, items, BM) ||
      !make_map(&mal, g.pa_lo, g.tf32, g.Kp, g.item_rows, items, BM) ||
      !make_map(&mbh, g.pb_hi, g.tf32, g.Kp, g.item_rows, items, bn) ||
      !make_map(&mbl, g.pb_lo, g.tf32, g.Kp, g.item_rows, items, bn)) {
    must_set_error("tensor map encoding failed");
    return false;
  }
  if (streamed) {
    if (g.Kp * g.es / KB != S_KSTEPS) {
      must_set_error("streamed update: unexpected K steps");
      return false;
    }
    // rows of the tiles start at base rounded down to even, so that the
    // first coordinate of every C tile (2 * abase + row0 floats) is a
    // multiple of 16 bytes; a row above base is written back unchanged
    const int abase = g.base & ~1;
    CUtensorMap mc;
    if (!make_c_map(&mc, A, ld, stride, n, items)) {
      must_set_error("tensor map encoding failed (C)");
      return false;
    }
    TcsParams S;
    S.C = reinterpret_cast<float*>(A);
    S.stride2 = 2 * stride;
    S.ld2 = 2 * ld;
    S.n = n;
    S.base = g.base;
    S.abase = abase;
    S.rt = (2 * (n - abase) + BM - 1) / BM;
    if (row_tiles >= 0) S.rt = std::min(S.rt, row_tiles);
    if (S.rt <= 0) return true;
    S.ct = t1 - t0;
    S.col_tile0 = t0;
    // runs of at most g_run row tiles, evenly split, and enough of them for
    // two CTAs per SM when few column tiles are updated (the look-ahead's
    // first-tile launch, the last panel steps)
    {
      static int sms = 0;
      if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
      }
      const int per_col = items * S.ct;
      int rruns = (S.rt + g_run - 1) / g_run;
      rruns = std::max(rruns, (2 * sms + per_col - 1) / per_col);
      rruns = std::min(rruns, S.rt);
      S.run = (S.rt + rruns - 1) / rruns;
      S.rruns = (S.rt + S.run - 1) / S.run;
    }
    S.err = err;
    S.tf32 = 0;
    S.aoff = s1.slot * g.rows_pad;
    S.boff = s1.bslot * g.rows_pad;
    S.aoff2 = s2 ? s2->slot * g.rows_pad : 0;
    S.boff2 = s2 ? s2->bslot * g.rows_pad : 0;
    ProfScope ps(PH_UPDATE, st);
    if (g_streamed == 2)
      launch_tc_regc<6>(mah, mal, mbh, mbl, S, items, st);
    else if (s2 && g_pair_kernel == 2)
      launch_tc_regc<5, 4>(mah, mal, mbh, mbl, S, items, st);
    else if (g_streamed == 3 && s2)
      launch_tc_tmac<4>(mah, mal, mbh, mbl, mc, S, items, st);
    else if (g_streamed == 3)
      launch_tc_tmac<2>(mah, mal, mbh, mbl, mc, S, items, st);
    else
      launch_tc_streamed(mah, mal, mbh, mbl, mc, S, items, st);
    prof_launched(PH_UPDATE, 1, items);
    return true;
  }
  TcParams P;
  P.C = A;
  P.stride = stride;
  P.ld = ld;
  P.n = n;
  P.base = g.base;
  P.ksteps = g.Kp * g.es / KB;
  P.err = err;
  P.tf32 = g.tf32 ? 1 : 0;
  P.col_tile0 = t0;
  P.aoff = s1.slot * g.rows_pad;
  ProfScope ps(PH_UPDATE, st);
  if (bn == 256)
    launch_tc<256>(mah, mal, mbh, mbl, P, g.m, items, t1 - t0, st);
  else
    launch_tc<128>(mah, mal, mbh, mbl, P, g.m, items, t1 - t0, st);
  prof_launched(PH_UPDATE, 1, items);
  return true;
}

bool tc_trailing_update(int precision, float2* A, size_t stride, int ld, int n, int k0, int nbe, int items,
                        char* packs, int* err, cudaStream_t st) {
  return tc_pack(precision, A, stride, ld, n, k0, nbe, items, packs, st) &&
         tc_update(precision, A, stride, ld, n, k0, nbe, items, packs, err, 0, -1, st);
}
