// Internal launch interfaces shared by the library's translation units.
#pragma once
#include "common.cuh"

bool must_is_device_ptr(const void* p);

// assemble.cu
struct AsmArgs;
void launch_geom(int N, int lmax, const double* pos_perm, const int2* pq, int n_pairs, double* d, double* Y,
                 cudaStream_t st);
void launch_tinv(int nE, const double2* E, int n_pot, const double* V, double a, int lmax, double2* out,
                 cudaStream_t st);

// Assembly of one chunk of energies e0 .. e0+nEc-1 of one LIZ.
struct AsmChunk {
  const must_liz* liz;
  int e0, nEc, nE, nspin, n_species;
  const double2* E;
  const double2* tinv;
  double2* M64;
  float2* M32;
  int ld;
  size_t stride;
  double* scale;
  int scale64;      // equilibrate the FP64 copy as well (FP64 path)
  int m64_df;       // store the unscaled matrix as FP32 pairs (double-float residual)
};
void launch_assemble_chunk(const AsmChunk& c, cudaStream_t st);

// lu64.cu
void lu64_factor(double2* A, size_t stride, int ld, int n, int r, int n_items, int nb, int* piv, int* status,
                 cudaStream_t st);
void schur_inv64(const double2* A, size_t stride, int ld, int n, int kap, int n_items, const double* scale,
                 double2* out, const int* out_index, int* status, int* status_out, cudaStream_t st);

// solve.cu: out_index[it] = spin * nE + e0 + e_local, status[it] = 0
void launch_chunk_index(int* out_index, int* status, int items, int ne, int nE, int e0, int canted, cudaStream_t st);
