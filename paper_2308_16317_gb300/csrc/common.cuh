// Shared device/host definitions of the GB300 tau_00 library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/must.h"

#define MUST_MAX_LMAX 4
#define MUST_MAX_NL ((MUST_MAX_LMAX + 1) * (MUST_MAX_LMAX + 1))
#define MUST_MAX_NL2 ((2 * MUST_MAX_LMAX + 1) * (2 * MUST_MAX_LMAX + 1))

// ---------------------------------------------------------------- complex --
struct cd { double x, y; };
struct cf { float x, y; };

__host__ __device__ __forceinline__ cd mk(double a, double b) { cd r; r.x = a; r.y = b; return r; }
__host__ __device__ __forceinline__ cd operator+(cd a, cd b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cd operator-(cd a, cd b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cd operator-(cd a) { return mk(-a.x, -a.y); }
__host__ __device__ __forceinline__ cd operator*(cd a, cd b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ __forceinline__ cd operator*(double s, cd a) { return mk(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ cd cconj(cd a) { return mk(a.x, -a.y); }
__host__ __device__ __forceinline__ double cnorm(cd a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ cd cinv(cd a) {
  // 1/a with Smith's scaling (avoids overflow in |a|^2)
  if (fabs(a.x) >= fabs(a.y)) {
    double r = a.y / a.x, d = a.x + a.y * r;
    return mk(1.0 / d, -r / d);
  } else {
    double r = a.x / a.y, d = a.x * r + a.y;
    return mk(r / d, -1.0 / d);
  }
}
__host__ __device__ __forceinline__ cd cdiv(cd a, cd b) { return a * cinv(b); }
// a -= b * c
__host__ __device__ __forceinline__ void cfms(cd& a, cd b, cd c) {
  a.x = fma(-b.x, c.x, a.x);
  a.x = fma(b.y, c.y, a.x);
  a.y = fma(-b.x, c.y, a.y);
  a.y = fma(-b.y, c.x, a.y);
}
// principal square root (branch cut on the negative real axis, Re >= 0)
__host__ __device__ __forceinline__ cd csqrt_p(cd z) {
  double r = hypot(z.x, z.y);
  if (r == 0.0) return mk(0.0, 0.0);
  if (z.x >= 0.0) {
    double u = sqrt(0.5 * (r + z.x));
    return mk(u, z.y / (2.0 * u));
  }
  double v = copysign(sqrt(0.5 * (r - z.x)), z.y);
  return mk(z.y / (2.0 * v), v);
}
// exp(i z)
__device__ __forceinline__ cd cexpi(cd z) {
  double s, c;
  sincos(z.x, &s, &c);
  double m = exp(-z.y);
  return mk(m * c, m * s);
}

__host__ __device__ __forceinline__ cf mkf(float a, float b) { cf r; r.x = a; r.y = b; return r; }
__device__ __forceinline__ void cfmsf(cf& a, cf b, cf c) {
  a.x = fmaf(-b.x, c.x, a.x);
  a.x = fmaf(b.y, c.y, a.x);
  a.y = fmaf(-b.x, c.y, a.y);
  a.y = fmaf(-b.y, c.x, a.y);
}
// a += b c
__device__ __forceinline__ void cfmaf_acc(cf& a, cf b, cf c) {
  a.x = fmaf(b.x, c.x, a.x);
  a.x = fmaf(-b.y, c.y, a.x);
  a.y = fmaf(b.x, c.y, a.y);
  a.y = fmaf(b.y, c.x, a.y);
}
__device__ __forceinline__ cf cmulf(cf a, cf b) { return mkf(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ cf cinvf(cf a) {
  if (fabsf(a.x) >= fabsf(a.y)) {
    float r = a.y / a.x, d = a.x + a.y * r;
    return mkf(1.0f / d, -r / d);
  } else {
    float r = a.x / a.y, d = a.x * r + a.y;
    return mkf(r / d, -1.0f / d);
  }
}

// ------------------------------------------------------------- LIZ handle --
struct must_liz {
  int N, lmax, nL, nL2, canted, kap, n, n_pairs, device;
  // host copies (for validation / batching)
  int* h_species_perm;   // species of the site at permuted position p (centre last)
  // device tables
  int* d_species_perm;   // [N]
  double* d_dirs_perm;   // [N][3] (canted) or NULL
  int2* d_pair_pq;       // [n_pairs] permuted positions (p, q), p < q
  double* d_pair_d;      // [n_pairs] |R_pq|
  double* d_pair_Y;      // [n_pairs][nL2] Y_L''(R_pq^), R_pq = pos(p) - pos(q)
  int* d_g_start;        // [nL*nL + 1] CSR rows of the sparse Gaunt contraction
  int* d_g_L2;           // [nnz]
  double* d_g_c;         // [nnz] i^{l-l'+l''} C(L,L',L'') (real: l-l'+l'' is even)
  int g_nnz;
};

// Per-call description of one chunk of matrices on the device.
struct MatBatch {
  int n_items;          // matrices in the chunk
  int n;                // order
  int ld;               // leading dimension (elements)
  size_t stride;        // elements between consecutive matrices
};

// Internal status words written by kernels (per item).
enum { ST_OK = 0, ST_SINGULAR = 4, ST_NOCONV = 5, ST_NONFINITE = 6 };

// Host helpers (api.cu)
void must_set_error(const char* fmt, ...);
