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

// Assembly of one chunk: energies e0 .. e0+nEc-1 of n_lz LIZs that share the
// (padded) matrix order n.  LIZ j of the chunk occupies items
// (j * items_per_e + spin) * nEc + e_local; its sites are placed after pad[j]
// decoupled identity sites, so smaller LIZs can share launches with larger
// ones without changing their Schur complement.
#define MUST_CHUNK_LIZ 64
struct AsmChunk {
  int n_lz;
  const must_liz* lz[MUST_CHUNK_LIZ];
  int pad[MUST_CHUNK_LIZ];          // identity sites before the LIZ's own sites
  int n;                            // chunk matrix order (kap * (N + pad), equal for all)
  int e0, nEc, nE, nspin, n_species;
  const double2* E;
  const double2* tinv;
  double2* M64;
  float2* M32;
  int ld;
  size_t stride;
  double* scale;
  float* scale32;   // FP32 copy of scale (mixed path; NULL otherwise)
  int scale64;      // equilibrate the FP64 copy as well (FP64 path)
  int m64_df;       // store the unscaled matrix as FP32 pairs (double-float residual)
  int* rowmax;      // NULL, or [item][n] zeroed ints that receive (atomic max) the bits of the largest
                    // |hi.re|, |hi.im| of each row without its diagonal entry (row scales of the residual)
};
void launch_assemble_chunk(const AsmChunk& c, cudaStream_t st);

// lu64.cu
void lu64_factor(double2* A, size_t stride, int ld, int n, int r, int n_items, int nb, int* piv, int* status,
                 cudaStream_t st);
void schur_inv64(const double2* A, size_t stride, int ld, int n, int kap, int n_items, const double* scale,
                 double2* out, const int* out_index, int* status, int* status_out, cudaStream_t st);

// solve.cu: out_index[it] = (liz_global * n_out + spin) * nE + e0 + e_local, status[it] = 0
struct ChunkIndex {
  int n_lz, ipe, ne, nE, e0, n_out;
  int liz_global[MUST_CHUNK_LIZ];
};
void launch_chunk_index(int* out_index, int* status, int items, const ChunkIndex& ci, cudaStream_t st);

void launch_site_charge(int lmax, int nE, const double2* E, const double2* w, int n_out, const double* V, double a,
                        const double2* tau, int kap, double* nE_out, double* N_out, cudaStream_t st);
void launch_site_density(int lmax, int nE, const double2* E, const double2* w, int n_out, const double* V, double a,
                         const double2* tau, int kap, int n_r, const double* r, double* out, cudaStream_t st);
