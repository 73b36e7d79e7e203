// C-ABI entry points of the GB300 LSMS tau_00 library (declared in
// include/must.h).  Host code here validates arguments, builds the per-LIZ
// device tables, carves the caller's workspace and enqueues the kernels; all
// arithmetic of the path runs in the device kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "solver.h"

void must_gaunt_csr(int lmax, std::vector<int>& start, std::vector<int>& L2s, std::vector<double>& coef);

static thread_local char g_err[512] = "";

void must_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

#define CUDA_TRY(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      must_set_error("%s failed: %s", #call, cudaGetErrorString(e_));                   \
      return MUST_ECUDA;                                                                 \
    }                                                                                    \
  } while (0)

bool must_is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

extern "C" {

void must_default_opts(must_solve_opts* o) {
  if (!o) return;
  o->precision = MUST_FP64;
  o->tol = 1e-10;
  o->max_iter = 10;
  o->warm_start = 0;
  o->deterministic = 0;
  o->equilibrate = 1;
  o->residual = 0;
}

const char* must_status_string(must_status s) {
  switch (s) {
    case MUST_OK: return "MUST_OK";
    case MUST_EINVAL: return "MUST_EINVAL";
    case MUST_ENOMEM: return "MUST_ENOMEM";
    case MUST_ECUDA: return "MUST_ECUDA";
    case MUST_ESINGULAR: return "MUST_ESINGULAR";
    case MUST_ENOCONV: return "MUST_ENOCONV";
    case MUST_ENONFINITE: return "MUST_ENONFINITE";
    case MUST_ETIMEOUT: return "MUST_ETIMEOUT";
    case MUST_EUNSUPPORTED: return "MUST_EUNSUPPORTED";
  }
  return "MUST_<unknown>";
}

const char* must_last_error(void) { return g_err; }

void must_liz_free(must_liz* z) {
  if (!z) return;
  cudaFree(z->d_species_perm);
  cudaFree(z->d_dirs_perm);
  cudaFree(z->d_pair_pq);
  cudaFree(z->d_pair_d);
  cudaFree(z->d_pair_Y);
  cudaFree(z->d_g_start);
  cudaFree(z->d_g_L2);
  cudaFree(z->d_g_c);
  delete[] z->h_species_perm;
  delete z;
}

int32_t must_liz_order(const must_liz* z) { return z ? z->n : 0; }
int32_t must_liz_kappa(const must_liz* z) { return z ? z->kap : 0; }

must_status must_liz_build(const double* pos, const int32_t* species, int32_t N, int32_t lmax,
                           const double* dirs, void* stream, must_liz** out) {
  if (!out) { must_set_error("must_liz_build: out is NULL"); return MUST_EINVAL; }
  *out = nullptr;
  if (!pos || !species) { must_set_error("must_liz_build: pos/species NULL"); return MUST_EINVAL; }
  if (N < 1 || N > 100000) { must_set_error("must_liz_build: n_sites=%d out of range", N); return MUST_EINVAL; }
  if (lmax < 0 || lmax > MUST_MAX_LMAX) { must_set_error("must_liz_build: lmax=%d not in [0,%d]", lmax, MUST_MAX_LMAX); return MUST_EINVAL; }
  for (int i = 0; i < N; ++i) {
    if (species[i] < 0) { must_set_error("must_liz_build: species[%d] < 0", i); return MUST_EINVAL; }
    for (int c = 0; c < 3; ++c)
      if (!std::isfinite(pos[3 * i + c])) { must_set_error("must_liz_build: non-finite position"); return MUST_EINVAL; }
    if (dirs) {
      const double n2 = dirs[3 * i] * dirs[3 * i] + dirs[3 * i + 1] * dirs[3 * i + 1] + dirs[3 * i + 2] * dirs[3 * i + 2];
      if (!(std::fabs(n2 - 1.0) < 1e-6)) { must_set_error("must_liz_build: spin_dirs[%d] not a unit vector", i); return MUST_EINVAL; }
    }
  }
  // site order with the central atom (row 0) last
  std::vector<int> order(N);
  for (int p = 0; p < N - 1; ++p) order[p] = p + 1;
  order[N - 1] = 0;
  std::vector<double> pos_perm(3 * N), dirs_perm(dirs ? 3 * N : 0);
  std::vector<int> sp_perm(N);
  for (int p = 0; p < N; ++p) {
    for (int c = 0; c < 3; ++c) pos_perm[3 * p + c] = pos[3 * order[p] + c];
    if (dirs) for (int c = 0; c < 3; ++c) dirs_perm[3 * p + c] = dirs[3 * order[p] + c];
    sp_perm[p] = species[order[p]];
  }
  std::vector<int2> pq;
  pq.reserve(size_t(N) * (N - 1) / 2);
  for (int p = 0; p < N; ++p)
    for (int q = p + 1; q < N; ++q) {
      const double dx = pos_perm[3 * p] - pos_perm[3 * q], dy = pos_perm[3 * p + 1] - pos_perm[3 * q + 1],
                   dz = pos_perm[3 * p + 2] - pos_perm[3 * q + 2];
      if (dx * dx + dy * dy + dz * dz < 1e-12) { must_set_error("must_liz_build: coincident sites"); return MUST_EINVAL; }
      pq.push_back(make_int2(p, q));
    }
  std::vector<int> gs, gl;
  std::vector<double> gc;
  must_gaunt_csr(lmax, gs, gl, gc);

  must_liz* z = new must_liz();
  std::memset(z, 0, sizeof(*z));
  z->N = N; z->lmax = lmax; z->nL = (lmax + 1) * (lmax + 1); z->nL2 = (2 * lmax + 1) * (2 * lmax + 1);
  z->canted = dirs ? 1 : 0;
  z->kap = z->nL * (dirs ? 2 : 1);
  z->n = N * z->kap;
  z->n_pairs = int(pq.size());
  z->g_nnz = int(gl.size());
  cudaGetDevice(&z->device);
  z->h_species_perm = new int[N];
  std::memcpy(z->h_species_perm, sp_perm.data(), sizeof(int) * N);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* d_pos = nullptr;
  auto fail = [&](cudaError_t e) {
    must_set_error("must_liz_build: %s", cudaGetErrorString(e));
    cudaFree(d_pos);
    must_liz_free(z);
    return (e == cudaErrorMemoryAllocation) ? MUST_ENOMEM : MUST_ECUDA;
  };
  cudaError_t e;
#define TRYB(x) do { e = (x); if (e != cudaSuccess) return fail(e); } while (0)
  TRYB(cudaMalloc(&d_pos, sizeof(double) * 3 * N));
  TRYB(cudaMalloc(&z->d_species_perm, sizeof(int) * N));
  if (dirs) TRYB(cudaMalloc(&z->d_dirs_perm, sizeof(double) * 3 * N));
  const size_t np = std::max<size_t>(pq.size(), 1);
  TRYB(cudaMalloc(&z->d_pair_pq, sizeof(int2) * np));
  TRYB(cudaMalloc(&z->d_pair_d, sizeof(double) * np));
  TRYB(cudaMalloc(&z->d_pair_Y, sizeof(double) * np * z->nL2));
  TRYB(cudaMalloc(&z->d_g_start, sizeof(int) * gs.size()));
  TRYB(cudaMalloc(&z->d_g_L2, sizeof(int) * std::max<size_t>(gl.size(), 1)));
  TRYB(cudaMalloc(&z->d_g_c, sizeof(double) * std::max<size_t>(gc.size(), 1)));
  TRYB(cudaMemcpyAsync(d_pos, pos_perm.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice, st));
  TRYB(cudaMemcpyAsync(z->d_species_perm, sp_perm.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  if (dirs) TRYB(cudaMemcpyAsync(z->d_dirs_perm, dirs_perm.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice, st));
  if (!pq.empty()) TRYB(cudaMemcpyAsync(z->d_pair_pq, pq.data(), sizeof(int2) * pq.size(), cudaMemcpyHostToDevice, st));
  TRYB(cudaMemcpyAsync(z->d_g_start, gs.data(), sizeof(int) * gs.size(), cudaMemcpyHostToDevice, st));
  if (!gl.empty()) {
    TRYB(cudaMemcpyAsync(z->d_g_L2, gl.data(), sizeof(int) * gl.size(), cudaMemcpyHostToDevice, st));
    TRYB(cudaMemcpyAsync(z->d_g_c, gc.data(), sizeof(double) * gc.size(), cudaMemcpyHostToDevice, st));
  }
  launch_geom(N, lmax, d_pos, z->d_pair_pq, z->n_pairs, z->d_pair_d, z->d_pair_Y, st);
  TRYB(cudaGetLastError());
  TRYB(cudaStreamSynchronize(st));
#undef TRYB
  cudaFree(d_pos);
  *out = z;
  return MUST_OK;
}

must_status must_tinv_square_well(int32_t nE, const double* E, int32_t n_pot, const double* V, double r_mt,
                                  int32_t lmax, double* tinv, void* stream) {
  if (nE < 0 || n_pot < 0 || !E || !V || !tinv) { must_set_error("must_tinv_square_well: bad argument"); return MUST_EINVAL; }
  if (lmax < 0 || lmax > MUST_MAX_LMAX || !(r_mt > 0.0)) { must_set_error("must_tinv_square_well: lmax/r_mt"); return MUST_EINVAL; }
  if (nE == 0 || n_pot == 0) return MUST_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool dE = must_is_device_ptr(E), dV = must_is_device_ptr(V), dT = must_is_device_ptr(tinv);
  const size_t bE = sizeof(double2) * nE, bV = sizeof(double) * n_pot, bT = sizeof(double2) * nE * n_pot * (lmax + 1);
  char* tmp = nullptr;
  const size_t need = (dE ? 0 : align256(bE)) + (dV ? 0 : align256(bV)) + (dT ? 0 : align256(bT));
  if (need) CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&tmp), need, st));
  char* cur = tmp;
  const double2* Ed = reinterpret_cast<const double2*>(E);
  const double* Vd = V;
  double2* Td = reinterpret_cast<double2*>(tinv);
  if (!dE) { CUDA_TRY(cudaMemcpyAsync(cur, E, bE, cudaMemcpyHostToDevice, st)); Ed = reinterpret_cast<double2*>(cur); cur += align256(bE); }
  if (!dV) { CUDA_TRY(cudaMemcpyAsync(cur, V, bV, cudaMemcpyHostToDevice, st)); Vd = reinterpret_cast<double*>(cur); cur += align256(bV); }
  if (!dT) { Td = reinterpret_cast<double2*>(cur); }
  launch_tinv(nE, Ed, n_pot, Vd, r_mt, lmax, Td, st);
  CUDA_TRY(cudaGetLastError());
  if (!dT) {
    CUDA_TRY(cudaMemcpyAsync(tinv, Td, bT, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
  }
  if (tmp) CUDA_TRY(cudaFreeAsync(tmp, st));
  return MUST_OK;
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton's method on P_n (three-term recurrence).
static void gauss_legendre_host(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

must_status must_contour_weights(int32_t n_e, double e_bot, double e_f, double* E, double* w) {
  if (n_e < 1 || !E || !w || !(e_f > e_bot)) { must_set_error("must_contour_weights: bad argument"); return MUST_EINVAL; }
  std::vector<double> x, W;
  gauss_legendre_host(n_e, x, W);
  const double c = 0.5 * (e_bot + e_f), r = 0.5 * (e_f - e_bot);
  for (int k = 0; k < n_e; ++k) {
    const double th = 0.5 * M_PI * (1.0 - x[k]);     // from pi (e_bot) to 0 (e_f)
    const double ct = std::cos(th), st = std::sin(th);
    E[2 * k] = c + r * ct;
    E[2 * k + 1] = r * st;
    // w = W (dtheta/dx) (dE/dtheta) = W (-pi/2) (i r e^{i theta})
    const double f = -0.5 * M_PI * W[k] * r;
    w[2 * k] = -f * st;
    w[2 * k + 1] = f * ct;
  }
  return MUST_OK;
}

must_status must_site_charge(int32_t lmax, int32_t nE, const double* E, const double* w, int32_t n_out,
                             const double* V, double r_mt, const double* tau00, double* n_of_E, double* N,
                             void* stream) {
  if (nE < 1 || n_out < 1 || !E || !w || !V || !tau00 || !N) {
    must_set_error("must_site_charge: bad argument");
    return MUST_EINVAL;
  }
  if (lmax < 0 || lmax > MUST_MAX_LMAX || !(r_mt > 0.0)) { must_set_error("must_site_charge: lmax/r_mt"); return MUST_EINVAL; }
  const void* ptrs[6] = {E, w, V, tau00, N, n_of_E};
  for (int i = 0; i < 6; ++i)
    if (ptrs[i] && !must_is_device_ptr(ptrs[i])) {
      must_set_error("must_site_charge: every array must be device memory");
      return MUST_EINVAL;
    }
  const int kap = (lmax + 1) * (lmax + 1);
  launch_site_charge(lmax, nE, reinterpret_cast<const double2*>(E), reinterpret_cast<const double2*>(w), n_out, V,
                     r_mt, reinterpret_cast<const double2*>(tau00), kap, n_of_E, N, static_cast<cudaStream_t>(stream));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { must_set_error("must_site_charge: %s", cudaGetErrorString(e)); return MUST_ECUDA; }
  return MUST_OK;
}

must_status must_site_density(int32_t lmax, int32_t nE, const double* E, const double* w, int32_t n_out,
                              const double* V, double r_mt, const double* tau00, int32_t n_r, const double* r,
                              double* n_of_r, void* stream) {
  if (nE < 1 || n_out < 1 || n_r < 1 || !E || !w || !V || !tau00 || !r || !n_of_r) {
    must_set_error("must_site_density: bad argument");
    return MUST_EINVAL;
  }
  if (lmax < 0 || lmax > MUST_MAX_LMAX || !(r_mt > 0.0)) { must_set_error("must_site_density: lmax/r_mt"); return MUST_EINVAL; }
  const void* ptrs[6] = {E, w, V, tau00, r, n_of_r};
  for (int i = 0; i < 6; ++i)
    if (!must_is_device_ptr(ptrs[i])) {
      must_set_error("must_site_density: every array must be device memory");
      return MUST_EINVAL;
    }
  const int kap = (lmax + 1) * (lmax + 1);
  launch_site_density(lmax, nE, reinterpret_cast<const double2*>(E), reinterpret_cast<const double2*>(w), n_out, V,
                      r_mt, reinterpret_cast<const double2*>(tau00), kap, n_r, r, n_of_r,
                      static_cast<cudaStream_t>(stream));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { must_set_error("must_site_density: %s", cudaGetErrorString(e)); return MUST_ECUDA; }
  return MUST_OK;
}

}  // extern "C"

// Gauss-Legendre rule for other translation units (C++ linkage).
void must_gauss_legendre_nodes(int n, std::vector<double>& x, std::vector<double>& w) { gauss_legendre_host(n, x, w); }
