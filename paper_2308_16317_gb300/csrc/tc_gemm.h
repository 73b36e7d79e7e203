// Tensor-core trailing update of the mixed-precision elimination.
#pragma once
#include "common.cuh"

int tc_panel_width(int precision);
size_t tc_pack_bytes_per_item(int n);
// Returns false (with must_set_error) if the update could not be launched.
// err: device word set to 1 by any CTA whose bounded waits ran out.
// The update is split in two calls: tc_pack (operands of panel step k0) and
// tc_update over the complex columns [base + col_lo, base + col_hi) of the
// trailing block (col_hi < 0: to the end); col_lo/col_hi are rounded to the
// tile width, which tc_tile_n() returns.
// with_b = false: only the A operand (L21); the caller wrote the B operand
// itself into the target tc_pack_b_target() describes.
// slot: which of the A operand's buffers to write (tc_pack_slots(): 2 for
// the BF16 splits, whose rows take half of the TF32-sized pack, 1 for TF32),
// so that the A operand of the next panel step can be packed while the
// current one is still being read; slot > 0 only with with_b = false.
int tc_pack_slots(int precision);
bool tc_pack(int precision, float2* A, size_t stride, int ld, int n, int k0, int nbe, int items, char* packs,
             cudaStream_t st, bool with_b = true, int slot = 0);
// B-operand (U12) pack of panel step k0 in BF16 hi/lo pairs: matrix column j,
// panel row p -> element j * Kp + 2p (re) and + 1 (im) of item `item_rows *
// Kp` elements apart; rows p >= nbe are zero.  False for the TF32 splits
// (those keep the separate pack kernel).
struct PackB {
  uint16_t *hi, *lo;
  int Kp, item_rows;
};
// slot: which of the B operand's two buffers (BF16 splits) to target.
bool tc_pack_b_target(int precision, int n, int k0, int nbe, int items, char* packs, PackB* out, int slot = 0);
// A-operand (L21) pack target of panel step k0 in the given slot, same
// layout as tc_pack writes (rows 2i, 2i+1 for matrix rows i >= k0 + nbe;
// item `item_rows * Kp` elements apart; hi/lo already offset to the slot).
// False for the TF32 splits.
bool tc_pack_a_target(int precision, int n, int k0, int nbe, int items, char* packs, int slot, PackB* out);
bool tc_update(int precision, float2* A, size_t stride, int ld, int n, int k0, int nbe, int items, char* packs,
               int* err, int col_lo, int col_hi, cudaStream_t st, int slot = 0);
// A panel step's operands in the pack: the step (k0, nbe), and the buffers
// (slots) holding its A and B operands.
struct TcStep {
  int k0, nbe, slot, bslot;
};
// Trailing update by one panel step (s2 == nullptr), or by two consecutive
// steps s1, s2 in one pass (K = 128; s1.nbe must be the panel width): the
// trailing block starts after the last step's panel.  row_tiles >= 0 limits
// the update to the first row_tiles tiles of 64 rows of that block (-1: all).
// Pairs, B slots and row limits need the BF16 splits and the TMA-C streamed
// kernel (knob 2 = 3).
bool tc_update_steps(int precision, float2* A, size_t stride, int ld, int n, TcStep s1, const TcStep* s2, int items,
                     char* packs, int* err, int col_lo, int col_hi, int row_tiles, cudaStream_t st);
// Applies the row interchanges piv[c] <-> c, c in [c0, c0 + nsw) (in order,
// piv indexed per item with stride r) to the A operand of step (k0, nbe)
// held in `slot`: the operand of an earlier step whose rows a later panel
// has permuted.  BF16 splits only.
bool tc_pack_swap_rows(int precision, int n, int k0, int nbe, int slot, int items, char* packs, const int* piv, int r,
                       int c0, int nsw, cudaStream_t st);
int tc_tile_n();
bool tc_trailing_update(int precision, float2* A, size_t stride, int ld, int n, int k0, int nbe, int items,
                        char* packs, int* err, cudaStream_t st);

// Tile width (complex columns) of the tensor-core update: 128 or 256.
bool tc_set_tile_n(int bn);
int tc_get_tile_n();

// Trailing-update kernel for 128-column tiles: 1 = streamed (C staged through
// shared memory by TMA, double-buffered accumulators), 0 = one CTA per tile.
bool tc_set_streamed(int on);
int tc_get_streamed();
// Tiles per CTA of the streamed kernel (1..64).
bool tc_set_run(int run);
int tc_get_run();
// Kernel of the paired (K = 128) pass: 3 (default) the TMA-C kernel (two C
// buffers, three A stages), 2 the register-C kernel (five A stages; measured
// slower on the 135-site LIZ: 2249 against 2273 solves/s).
bool tc_set_pair_kernel(int k);
int tc_get_pair_kernel();
