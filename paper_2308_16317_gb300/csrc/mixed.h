// Mixed-precision path: FP32 factors with tensor-core trailing updates and
// FP64 residual refinement.
#pragma once
#include "common.cuh"
#include "solver.h"

struct MixedChunk {
  AsmChunk asmc;
  int n, ld, kap, items;
  double2* M64;
  size_t stride;
  int* piv;
  int* status;
  const int* out_index;
  double2* tau;
  int* status_out;
  char* ws;
  must_solve_opts opts;
  // learned warm start (NULL when absent): per output block, indexed like tau
  const double2* seed;      // [n_out*nE][kap][kap] column-major
  const int* seed_mask;     // 1 = try the seed
  int* seed_used;           // 1 = the seed passed the residual gate
};

size_t mixed_item_bytes(int n, int ld, int kap);
must_status mixed_solve_chunk(const MixedChunk& c, cudaStream_t st);

// Tuning knob 4: 1 (default) factor panel k+1 on a high-priority side stream
// while the rest of step k's trailing update runs; 0 keeps one stream.
extern int g_lookahead;
// Tuning knob 5: right-hand sides per CTA of the correction solve (2, 4 or 8;
// 0 = the most that fit: 8 up to order 3200, 4 up to 6400, else 2).
extern int g_corr_rhs;
// Tuning knob 6: 1 (default) runs the correction solve on thread-block
// clusters (correct_cluster.cu), 0 on one CTA per item and RHS group.
extern int g_corr_cluster;

// Correction delta = D U^{-1} L^{-1} P (D R), X += delta, on clusters of
// CTAs (knob 7) per item and group of right-hand sides (correct_cluster.cu).  Same
// arguments as the one-CTA kernel; false (with must_set_error) if the order
// is too large for its shared memory or the launch failed.
int correct_cluster_rhs(int n, int kap);
// Tuning knob 7: preferred CTAs per cluster of the cluster correction (2, 4
// or 8; a larger one is taken when the rows do not fit).
bool correct_cluster_set_ctas(int ctas);
int correct_cluster_get_ctas();
// Tuning knob 8: right-hand sides per cluster of the cluster correction (4, 8
// or 16; 0, the default: the most whose rows fit a 72 KB share of shared
// memory, so that two CTAs fit an SM).
bool correct_cluster_set_rhs(int rhs);
int correct_cluster_get_rhs();
bool correct_cluster(const float2* A, size_t stride, int ld, int n, int kap, int items, const int* perm,
                     const double* scale, const double2* Sinv, const double2* R, double2* X, double* norms,
                     const int* conv, int first_all, const int* first_flags, unsigned long long* work,
                     cudaStream_t st, int shape = 0);
// Tuning knob 12: shape of the cluster correction from the third
// correction on, when few items are still iterating and each item's chain
// of substitution steps, not the batch, sets the time: CTAs per cluster *
// 100 + right-hand sides per cluster (204, 404, 408, 804, 808, ...), or 0 for
// the shape of the first corrections.  Default 408: on the 135-site LIZ the
// correction phase drops from 4.89 to 4.65 ms per step (404: 5.06, 804: 5.21,
// 808: 4.95, 204: 4.93).
extern int g_corr_late;

// Tuning knob 9: 1 (default) runs U12 = L11^{-1} A12 with persistent CTAs
// (contiguous runs of column tiles, the next tile copied by cp.async while
// the current one is multiplied), 0 with one CTA per column tile.
extern int g_trsm_persist;
// Tuning knob 10: where the A operand (L21 as BF16 hi/lo pairs) of each
// panel step is packed: 0 a pack kernel on the main stream; 1 a pack kernel
// on the side stream right after the next panel (needs the look-ahead, knob
// 4); 2 the panel kernel itself, at its end.  1 and 2 alternate the pack's
// two A buffers so that step k+1's operand is written while step k's update
// still reads the other.  All three write the same values.  Default 0: on
// the 135-site LIZ 1 measured 1 % slower (the concurrent pack kernel slows
// the bandwidth-bound trailing update) and 2 measured 2.4 % slower (the pack
// adds ~90 us to each panel on its single SM per item).
extern int g_pack_side;
// Tuning knob 11: paired panel steps.  While the trailing block left after
// two panels has at least this many rows, steps k and k+1 are applied to it
// in one pass of the tensor-core update (K = 128 instead of two passes with
// K = 64), at the price of factoring panel k+1 with nothing to overlap it;
// 0 pairs no steps.  Needs the BF16 splits and the TMA-C streamed update
// kernel (knob 2 = 3); the A pack placement (knob 10) is then 0.  Default
// 1536: on the 135-site LIZ (with the faster panel) thresholds 1024 / 1536 /
// 1792 / 1900 give 2252 / 2262 / 2256 / 2257 against 2239 solves/s unpaired:
// pairing cuts the trailing update from 13.6 to 10.9-12.7 ms per step, but
// each pair's second panel runs with nothing to overlap it, so only the
// earliest steps, where the update dominates, gain.
extern int g_pair_rows;
