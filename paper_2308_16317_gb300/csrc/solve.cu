// Orchestration of must_tau00_solve / must_tau00_batch: workspace layout,
// staging of host buffers, chunking over energies and the launch sequence
//   assemble (M on the device) -> eliminate the leading n - kap columns ->
//   tau_00 = S^{-1} (FP64 path), or the mixed-precision path in mixed.cu.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "solver.h"
#include "mixed.h"
#include "prof.h"
#include "tc_gemm.h"

namespace {

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

int ld_of(int n) { return (n + 31) & ~31; }

struct Layout {
  int n, ld, r, kap, items_per_e, n_out;
  int precision;
  size_t per_item;      // bytes per matrix item
  size_t staging;       // bytes for staged inputs/outputs (independent of chunk)
};

size_t item_bytes(int n, int ld, int kap, int precision) {
  const size_t mat64 = a256(size_t(ld) * n * 16);
  // status and output index are carved as two separate 256-byte-rounded
  // arrays per chunk: 2 x 256 bytes per item covers their rounding for any
  // item count >= 1
  size_t b = mat64 + a256(size_t(n) * 4) /*piv*/ + a256(size_t(n) * 8) /*scale*/ + 512 /*status+index*/;
  if (precision != MUST_FP64) b += mixed_item_bytes(n, ld, kap);
  return b;
}

Layout make_layout(const must_liz* z, int nE, int nspin, int n_species, int precision, bool stage_E, bool stage_t,
                   bool stage_tau, bool stage_st) {
  Layout L;
  L.n = z->n;
  L.ld = ld_of(z->n);
  L.kap = z->kap;
  L.r = z->n - z->kap;
  L.items_per_e = z->canted ? 1 : nspin;
  L.n_out = z->canted ? 1 : nspin;
  L.precision = precision;
  L.per_item = item_bytes(L.n, L.ld, L.kap, precision);
  size_t s = 0;
  if (stage_E) s += a256(size_t(nE) * 16);
  if (stage_t) s += a256(size_t(nspin) * n_species * nE * (z->lmax + 1) * 16);
  if (stage_tau) s += a256(size_t(L.n_out) * nE * L.kap * L.kap * 16);
  if (stage_st) s += a256(size_t(L.n_out) * nE * 4);
  L.staging = s;
  return L;
}

int check_opts(const must_solve_opts* o) {
  if (o->precision < MUST_FP64 || o->precision > MUST_MIXED_TF32X3) return 0;
  if (o->precision != MUST_FP64 && (o->max_iter < 0 || !(o->tol > 0.0))) return 0;
  if (o->residual < 0 || o->residual > 3) return 0;
  return 1;
}

}  // namespace

extern "C" size_t must_workspace_bytes(const must_liz* z, int32_t n_items, const must_solve_opts* opts) {
  if (!z || n_items < 1) return 0;
  must_solve_opts o;
  must_default_opts(&o);
  if (opts) o = *opts;
  const int ld = ld_of(z->n);
  // staging assumes host inputs/outputs (an upper bound); 2 species, 2 spins
  const size_t stage = a256(size_t(n_items) * 16) + a256(size_t(n_items) * 4 * (z->lmax + 1) * 16) +
                       a256(size_t(n_items) * z->kap * z->kap * 16) + a256(size_t(n_items) * 4);
  return stage + size_t(n_items) * item_bytes(z->n, ld, z->kap, o.precision) + 4096;
}

// Seeds of must_tau00_solve_seeded for the call in progress on this thread.
struct SeedArgs {
  const double2* seed;
  const int* mask;
  int* used;
};
static thread_local const SeedArgs* g_seed = nullptr;

// One chunk: items (LIZ j, spin, energy) of the (padded) order c.n, all in
// the workspace `ws`.  Carves per-item storage, assembles, eliminates and
// writes tau_00 / status through out_index.
static must_status run_chunk(AsmChunk c, int items, const ChunkIndex& ci, const must_solve_opts& o, char* ws,
                             size_t ws_left, double2* tau_dev, int* status_dev, cudaStream_t st) {
  const int n = c.n, ld = ld_of(n), kap = c.lz[0]->kap, r = n - kap;
  char* cur = ws;
  double2* M64 = reinterpret_cast<double2*>(cur);
  const size_t stride = size_t(ld) * n;
  cur += a256(size_t(items) * stride * 16);
  int* piv = reinterpret_cast<int*>(cur);
  cur += a256(size_t(items) * n * 4);
  int* st_item = reinterpret_cast<int*>(cur);
  cur += a256(size_t(items) * 4);
  int* out_index = reinterpret_cast<int*>(cur);
  cur += a256(size_t(items) * 4);
  double* scale64 = reinterpret_cast<double*>(cur);
  cur += a256(size_t(items) * n * 8);
  char* mixed_ws = cur;
  const size_t mixed_bytes = (o.precision != MUST_FP64) ? size_t(items) * mixed_item_bytes(n, ld, kap) : 0;
  if (size_t(cur - ws) + mixed_bytes > ws_left) {
    must_set_error("workspace layout overflow");
    return MUST_ENOMEM;
  }
  launch_chunk_index(out_index, st_item, items, ci, st);
  c.M64 = M64;
  c.ld = ld;
  c.stride = stride;
  if (o.precision == MUST_FP64) {
    c.M32 = nullptr;
    c.scale32 = nullptr;
    c.scale = o.equilibrate ? scale64 : nullptr;
    c.scale64 = o.equilibrate ? 1 : 0;
    c.m64_df = 0;
    launch_assemble_chunk(c, st);
    lu64_factor(M64, stride, ld, n, r, items, 32, piv, st_item, st);
    schur_inv64(M64, stride, ld, n, kap, items, c.scale, tau_dev, out_index, st_item, status_dev, st);
  } else {
    c.scale64 = 0;
    c.m64_df = o.residual >= 1 ? 1 : 0;
    MixedChunk mc;
    mc.asmc = c; mc.n = n; mc.ld = ld; mc.kap = kap; mc.items = items; mc.M64 = M64; mc.stride = stride;
    mc.piv = piv; mc.status = st_item; mc.out_index = out_index; mc.tau = tau_dev; mc.status_out = status_dev;
    mc.ws = mixed_ws; mc.opts = o;
    mc.seed = g_seed ? g_seed->seed : nullptr;
    mc.seed_mask = g_seed ? g_seed->mask : nullptr;
    mc.seed_used = g_seed ? g_seed->used : nullptr;
    must_status s = mixed_solve_chunk(mc, st);
    if (s != MUST_OK) return s;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { must_set_error("kernel launch failed: %s", cudaGetErrorString(e)); return MUST_ECUDA; }
  return MUST_OK;
}

// LIZs lz[0..count) padded to the common order n (pad[j] identity sites in
// front of LIZ j's own sites), every energy and spin, in chunks that fit the
// workspace: several whole LIZs per chunk when they fit, else one LIZ's
// energies in pieces.  tau_dev/status_dev are the call's whole output arrays.
static must_status solve_group(const must_liz* const* lz, const int* liz_global, const int* pad, int count, int n,
                               int nE, const double2* E_dev, const double2* tinv_dev, int n_species, int nspin,
                               const must_solve_opts& o, char* ws, size_t ws_left, double2* tau_dev, int* status_dev,
                               cudaStream_t st) {
  const int kap = lz[0]->kap, ld = ld_of(n);
  const int ipe = lz[0]->canted ? 1 : nspin, n_out = lz[0]->canted ? 1 : nspin;
  const size_t per = item_bytes(n, ld, kap, o.precision);
  const size_t cap = ws_left / per;
  if (cap < size_t(ipe)) {
    must_set_error("workspace too small: need at least %zu bytes for one energy", per * ipe);
    return MUST_ENOMEM;
  }
  AsmChunk c;
  c.rowmax = nullptr;
  c.n = n; c.nE = nE; c.nspin = nspin; c.n_species = n_species; c.E = E_dev; c.tinv = tinv_dev;
  ChunkIndex ci;
  ci.ipe = ipe; ci.nE = nE; ci.n_out = n_out;
  if (cap >= size_t(ipe) * nE) {
    const int per_chunk = int(std::min<size_t>(MUST_CHUNK_LIZ, cap / (size_t(ipe) * nE)));
    for (int j0 = 0; j0 < count; j0 += per_chunk) {
      const int m = std::min(per_chunk, count - j0);
      c.n_lz = m; c.e0 = 0; c.nEc = nE;
      ci.n_lz = m; ci.ne = nE; ci.e0 = 0;
      for (int j = 0; j < m; ++j) {
        c.lz[j] = lz[j0 + j];
        c.pad[j] = pad[j0 + j];
        ci.liz_global[j] = liz_global[j0 + j];
      }
      must_status s = run_chunk(c, m * ipe * nE, ci, o, ws, ws_left, tau_dev, status_dev, st);
      if (s != MUST_OK) return s;
    }
    return MUST_OK;
  }
  const int nEc = int(cap / ipe);
  for (int j = 0; j < count; ++j)
    for (int e0 = 0; e0 < nE; e0 += nEc) {
      const int ne = std::min(nEc, nE - e0);
      c.n_lz = 1; c.lz[0] = lz[j]; c.pad[0] = pad[j]; c.e0 = e0; c.nEc = ne;
      ci.n_lz = 1; ci.liz_global[0] = liz_global[j]; ci.ne = ne; ci.e0 = e0;
      must_status s = run_chunk(c, ne * ipe, ci, o, ws, ws_left, tau_dev, status_dev, st);
      if (s != MUST_OK) return s;
    }
  return MUST_OK;
}

// One LIZ, all energies (no padding).
static must_status solve_one(const must_liz* z, int nE, const double2* E_dev, const double2* tinv_dev,
                             int n_species, int nspin, const must_solve_opts& o, char* ws, size_t ws_left,
                             double2* tau_dev, int* status_dev, cudaStream_t st) {
  const int zero = 0;
  return solve_group(&z, &zero, &zero, 1, z->n, nE, E_dev, tinv_dev, n_species, nspin, o, ws, ws_left, tau_dev,
                     status_dev, st);
}

// Sites per padding quantum for the batched call (LIZ sizes are rounded up to
// a multiple so that LIZs of nearby size share launches).
static int g_bucket_sites = 4;

static must_status solve_common(int n_liz, const must_liz* const* lizs, int nE, const double* E, const double* tinv,
                                int n_species, int nspin, const must_solve_opts* opts, void* workspace,
                                size_t ws_bytes, double* tau00, int32_t* status, void* stream) {
  if (n_liz < 1 || !lizs || nE < 1 || !E || !tinv || !tau00 || !workspace) {
    must_set_error("must_tau00_solve: NULL argument or empty size");
    return MUST_EINVAL;
  }
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) { must_set_error("workspace not 256-byte aligned"); return MUST_EINVAL; }
  if (n_species < 1 || nspin < 1 || nspin > 2) { must_set_error("n_species/nspin out of range"); return MUST_EINVAL; }
  must_solve_opts o;
  must_default_opts(&o);
  if (opts) o = *opts;
  if (!check_opts(&o)) { must_set_error("invalid must_solve_opts"); return MUST_EINVAL; }
  const int lmax = lizs[0]->lmax, canted = lizs[0]->canted, kap = lizs[0]->kap;
  for (int i = 0; i < n_liz; ++i) {
    if (!lizs[i]) { must_set_error("NULL handle"); return MUST_EINVAL; }
    if (lizs[i]->lmax != lmax || lizs[i]->canted != canted) { must_set_error("handles differ in lmax/canting"); return MUST_EINVAL; }
    for (int p = 0; p < lizs[i]->N; ++p)
      if (lizs[i]->h_species_perm[p] >= n_species) { must_set_error("species index >= n_species"); return MUST_EINVAL; }
  }
  if (canted && nspin != 2) { must_set_error("canted handles need nspin == 2"); return MUST_EINVAL; }
  if (!must_is_device_ptr(workspace)) { must_set_error("workspace must be device memory"); return MUST_EINVAL; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n_out = canted ? 1 : nspin;
  const bool dE = must_is_device_ptr(E), dT = must_is_device_ptr(tinv), dTau = must_is_device_ptr(tau00);
  const bool dSt = status ? must_is_device_ptr(status) : true;
  // staging region
  char* ws = static_cast<char*>(workspace);
  char* cur = ws;
  const size_t bE = size_t(nE) * 16, bT = size_t(nspin) * n_species * nE * (lmax + 1) * 16;
  const size_t bTau = size_t(n_liz) * n_out * nE * kap * kap * 16, bSt = size_t(n_liz) * n_out * nE * 4;
  size_t stage = (dE ? 0 : a256(bE)) + (dT ? 0 : a256(bT)) + (dTau ? 0 : a256(bTau)) + (dSt ? 0 : a256(bSt));
  if (stage >= ws_bytes) { must_set_error("workspace too small for staging (%zu bytes)", stage); return MUST_ENOMEM; }
  const double2* Ed = reinterpret_cast<const double2*>(E);
  const double2* Td = reinterpret_cast<const double2*>(tinv);
  double2* Taud = reinterpret_cast<double2*>(tau00);
  int* Std = status;
#define TRYC(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { must_set_error("%s: %s", #x, cudaGetErrorString(e_)); return MUST_ECUDA; } } while (0)
  if (!dE) { TRYC(cudaMemcpyAsync(cur, E, bE, cudaMemcpyHostToDevice, st)); Ed = reinterpret_cast<double2*>(cur); cur += a256(bE); }
  if (!dT) { TRYC(cudaMemcpyAsync(cur, tinv, bT, cudaMemcpyHostToDevice, st)); Td = reinterpret_cast<double2*>(cur); cur += a256(bT); }
  if (!dTau) { Taud = reinterpret_cast<double2*>(cur); cur += a256(bTau); }
  if (!dSt) { Std = reinterpret_cast<int*>(cur); cur += a256(bSt); }
  const size_t left = ws_bytes - size_t(cur - ws);
  if (n_liz == 1) {
    must_status s = solve_one(lizs[0], nE, Ed, Td, n_species, nspin, o, cur, left, Taud, Std, st);
    if (s != MUST_OK) return s;
  } else {
    // buckets of equal padded order, largest first
    std::vector<int> idx(n_liz);
    for (int i = 0; i < n_liz; ++i) idx[i] = i;
    const int q = std::max(1, g_bucket_sites);
    auto padded_sites = [&](int i) { return ((lizs[i]->N + q - 1) / q) * q; };
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return padded_sites(a) > padded_sites(b); });
    size_t b0 = 0;
    while (b0 < idx.size()) {
      size_t b1 = b0;
      const int Np = padded_sites(idx[b0]);
      while (b1 < idx.size() && padded_sites(idx[b1]) == Np) ++b1;
      std::vector<const must_liz*> g;
      std::vector<int> gi, gp;
      for (size_t k = b0; k < b1; ++k) {
        g.push_back(lizs[idx[k]]);
        gi.push_back(idx[k]);
        gp.push_back(Np - lizs[idx[k]]->N);
      }
      must_status s = solve_group(g.data(), gi.data(), gp.data(), int(g.size()), Np * kap, nE, Ed, Td, n_species,
                                  nspin, o, cur, left, Taud, Std, st);
      if (s != MUST_OK) return s;
      b0 = b1;
    }
  }
  if (!dTau) TRYC(cudaMemcpyAsync(tau00, Taud, bTau, cudaMemcpyDeviceToHost, st));
  if (!dSt && status) TRYC(cudaMemcpyAsync(status, Std, bSt, cudaMemcpyDeviceToHost, st));
  if (!dTau || (!dSt && status)) TRYC(cudaStreamSynchronize(st));
#undef TRYC
  return MUST_OK;
}

extern "C" must_status must_tau00_solve(const must_liz* liz, int32_t nE, const double* E, const double* tinv,
                                        int32_t n_species, int32_t nspin, const must_solve_opts* opts,
                                        void* workspace, size_t ws_bytes, double* tau00, int32_t* status,
                                        void* stream) {
  if (!liz) { must_set_error("must_tau00_solve: NULL handle"); return MUST_EINVAL; }
  const must_liz* arr[1] = {liz};
  return solve_common(1, arr, nE, E, tinv, n_species, nspin, opts, workspace, ws_bytes, tau00, status, stream);
}

extern "C" must_status must_tau00_batch(int32_t n_liz, const must_liz* const* lizs, int32_t nE, const double* E,
                                        const double* tinv, int32_t n_species, int32_t nspin,
                                        const must_solve_opts* opts, void* workspace, size_t ws_bytes,
                                        double* tau00, int32_t* status, void* stream) {
  return solve_common(n_liz, lizs, nE, E, tinv, n_species, nspin, opts, workspace, ws_bytes, tau00, status, stream);
}

extern "C" size_t must_batch_workspace_bytes(int32_t n_liz, const must_liz* const* lizs, int32_t n_items_per_liz,
                                             const must_solve_opts* opts) {
  if (n_liz < 1 || !lizs || n_items_per_liz < 1) return 0;
  must_solve_opts o;
  must_default_opts(&o);
  if (opts) o = *opts;
  const int q = std::max(1, g_bucket_sites);
  int Nmax = 0;
  for (int i = 0; i < n_liz; ++i) Nmax = std::max(Nmax, ((lizs[i]->N + q - 1) / q) * q);
  const int kap = lizs[0]->kap, n = Nmax * kap;
  const size_t per = item_bytes(n, ld_of(n), kap, o.precision);
  // one whole LIZ (all its items) at the largest padded order, plus staging
  // of every LIZ's outputs; more workspace lets several LIZs share launches
  return size_t(n_items_per_liz) * per + a256(size_t(n_items_per_liz) * 16) +
         a256(size_t(n_items_per_liz) * 4 * (lizs[0]->lmax + 1) * 16) +
         a256(size_t(n_liz) * n_items_per_liz * kap * kap * 16) + a256(size_t(n_liz) * n_items_per_liz * 4) + 4096;
}

__global__ void chunk_index_kernel(int* out_index, int* status, int items, ChunkIndex ci) {
  const int it = blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= items) return;
  const int el = it % ci.ne;
  const int grp = it / ci.ne;            // lz * ipe + spin
  const int lz = grp / ci.ipe, s = grp % ci.ipe;
  out_index[it] = (ci.liz_global[lz] * ci.n_out + s) * ci.nE + ci.e0 + el;
  status[it] = 0;
}

void launch_chunk_index(int* out_index, int* status, int items, const ChunkIndex& ci, cudaStream_t st) {
  chunk_index_kernel<<<(items + 127) / 128, 128, 0, st>>>(out_index, status, items, ci);
  prof_launched(PH_OTHER, 1);
}

// --------------------------------------------------------------------------
// Allocation-free entry point (no counterpart in the paper).
//
// Some callers cannot allocate device memory while they run: a host code that
// has handed all device memory to its own pool allocator, a solver called
// from inside a region where allocation is forbidden (another library's
// callback, a real-time loop that must not block on the allocator), or a
// language binding with no way to obtain a device buffer.  For them the FP64
// solve can run in a scratch area that lives in the library itself: a
// file-scope device array of MUST_STATIC_SCRATCH_BYTES, allocated when the
// library's GPU code is loaded on a device and held until the process exits.
//
// The array's name is only a host-side stand-in in host code, so its device
// address is looked up with cudaGetSymbolAddress once per device (with that
// device current) on the first call made on that device; make that first call
// before any stream capture.  All calls share the one array and it keeps the
// last call's contents, so two calls whose GPU work overlaps (different
// streams, or different host threads) race on it: serialise them.
#define MUST_STATIC_SCRATCH_BYTES (size_t(160) << 20)

static __device__ __align__(256) unsigned char g_must_static_scratch[MUST_STATIC_SCRATCH_BYTES];

static void* static_scratch_address(must_status* err) {
  static std::mutex mu;
  static void* addr[256] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    must_set_error("must_tau00_solve_static: no current CUDA device");
    *err = MUST_ECUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_must_static_scratch);
    if (e != cudaSuccess || !p) {
      must_set_error("must_tau00_solve_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      *err = MUST_ECUDA;
      return nullptr;
    }
    addr[dev] = p;
  }
  return addr[dev];
}

extern "C" size_t must_static_scratch_bytes(void) { return MUST_STATIC_SCRATCH_BYTES; }

extern "C" must_status must_tau00_solve_static(const must_liz* z, int32_t nE, const double* E, const double* tinv,
                                               int32_t n_species, int32_t nspin, double* tau00, int32_t* status,
                                               void* stream) {
  if (!z || nE < 1 || !E || !tinv || !tau00) {
    must_set_error("must_tau00_solve_static: NULL argument or empty size");
    return MUST_EINVAL;
  }
  if (n_species < 1 || nspin < 1 || nspin > 2 || (z->canted && nspin != 2)) {
    must_set_error("must_tau00_solve_static: n_species/nspin out of range");
    return MUST_EINVAL;
  }
  for (int p = 0; p < z->N; ++p)
    if (z->h_species_perm[p] >= n_species) {
      must_set_error("must_tau00_solve_static: species index >= n_species");
      return MUST_EINVAL;
    }
  if (!must_is_device_ptr(E) || !must_is_device_ptr(tinv) || !must_is_device_ptr(tau00) ||
      (status && !must_is_device_ptr(status))) {
    must_set_error("must_tau00_solve_static: E, tinv, tau00 and status must be device memory");
    return MUST_EINVAL;
  }
  // one energy (both spins of a collinear LIZ) must fit in the scratch
  const int ld = ld_of(z->n), ipe = z->canted ? 1 : nspin;
  const size_t need = size_t(ipe) * item_bytes(z->n, ld, z->kap, MUST_FP64) + 4 * 256;
  if (need > MUST_STATIC_SCRATCH_BYTES) {
    must_set_error("must_tau00_solve_static: matrix order %d needs %zu bytes of scratch per energy, more than the "
                   "%zu-byte static scratch; use must_tau00_solve with a caller workspace",
                   z->n, need, size_t(MUST_STATIC_SCRATCH_BYTES));
    return MUST_EINVAL;
  }
  must_status err = MUST_OK;
  char* ws = static_cast<char*>(static_scratch_address(&err));
  if (!ws) return err;
  must_solve_opts o;
  must_default_opts(&o);   // FP64 path with equilibration
  return solve_one(z, nE, reinterpret_cast<const double2*>(E), reinterpret_cast<const double2*>(tinv), n_species,
                   nspin, o, ws, MUST_STATIC_SCRATCH_BYTES, reinterpret_cast<double2*>(tau00), status,
                   static_cast<cudaStream_t>(stream));
}

// --------------------------------------------------------------------------
// Batched plans: the whole launch sequence of one must_tau00_batch call with
// fixed (device) arguments captured once into a CUDA graph and replayed.
struct must_plan {
  cudaGraphExec_t exec;
  cudaGraph_t graph;
  long long kernels;      // kernel nodes per replay (for the launch counter)
};

extern "C" must_status must_plan_batch(int32_t n_liz, const must_liz* const* lizs, int32_t nE, const double* E,
                                       const double* tinv, int32_t n_species, int32_t nspin,
                                       const must_solve_opts* opts, void* workspace, size_t ws_bytes, double* tau00,
                                       int32_t* status, must_plan** out) {
  if (!out) { must_set_error("must_plan_batch: out is NULL"); return MUST_EINVAL; }
  *out = nullptr;
  if (!E || !tinv || !tau00 || !workspace || !must_is_device_ptr(E) || !must_is_device_ptr(tinv) ||
      !must_is_device_ptr(tau00) || !must_is_device_ptr(workspace) || (status && !must_is_device_ptr(status))) {
    must_set_error("must_plan_batch: E, tinv, tau00, status and workspace must be device memory");
    return MUST_EINVAL;
  }
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    must_set_error("must_plan_batch: cannot create a capture stream");
    return MUST_ECUDA;
  }
  const int prof_was_on = prof_suspend();
  const long long l0 = must_launch_count();
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
  must_status st = MUST_ECUDA;
  cudaGraph_t g = nullptr;
  if (e == cudaSuccess) {
    st = solve_common(n_liz, lizs, nE, E, tinv, n_species, nspin, opts, workspace, ws_bytes, tau00, status, s);
    e = cudaStreamEndCapture(s, &g);
  }
  const long long kernels = must_launch_count() - l0;
  prof_resume(prof_was_on);
  prof_add_launches(-kernels);   // capture enqueued nothing; replays count them
  cudaStreamDestroy(s);
  if (st != MUST_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    if (st == MUST_OK) {
      must_set_error("must_plan_batch: stream capture failed: %s", cudaGetErrorString(e));
      st = MUST_ECUDA;
    }
    return st;
  }
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    must_set_error("must_plan_batch: graph instantiation failed: %s", cudaGetErrorString(e));
    return MUST_ECUDA;
  }
  must_plan* p = new must_plan();
  p->exec = x;
  p->graph = g;
  p->kernels = kernels;
  *out = p;
  return MUST_OK;
}

extern "C" must_status must_plan_launch(const must_plan* p, void* stream) {
  if (!p) { must_set_error("must_plan_launch: NULL plan"); return MUST_EINVAL; }
  const cudaError_t e = cudaGraphLaunch(p->exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    must_set_error("must_plan_launch: %s", cudaGetErrorString(e));
    return MUST_ECUDA;
  }
  prof_add_launches(p->kernels);
  return MUST_OK;
}

extern "C" void must_plan_free(must_plan* p) {
  if (!p) return;
  cudaGraphExecDestroy(p->exec);
  cudaGraphDestroy(p->graph);
  delete p;
}

// Tuning knobs (set by the autotuner).
extern "C" must_status must_tune_set(int32_t knob, int32_t value) {
  switch (knob) {
    case 0:   // sites per padding quantum of the batched call
      if (value < 1 || value > 64) { must_set_error("bucket sites must be in [1, 64]"); return MUST_EINVAL; }
      g_bucket_sites = value;
      return MUST_OK;
    case 1:   // tensor-core tile width (complex columns)
      if (!tc_set_tile_n(value)) { must_set_error("tile width must be 128 or 256"); return MUST_EINVAL; }
      return MUST_OK;
    case 2:   // streamed trailing-update kernel on/off
      if (!tc_set_streamed(value)) { must_set_error("trailing-update kernel must be 0..3"); return MUST_EINVAL; }
      return MUST_OK;
    case 3:   // tiles per CTA of the streamed kernel
      if (!tc_set_run(value)) { must_set_error("tiles per CTA must be in [1, 64]"); return MUST_EINVAL; }
      return MUST_OK;
    case 4:   // panel look-ahead on a side stream
      if (value != 0 && value != 1) { must_set_error("look-ahead switch must be 0 or 1"); return MUST_EINVAL; }
      g_lookahead = value;
      return MUST_OK;
    case 5:   // right-hand sides per CTA of the correction solve
      if (value != 0 && value != 2 && value != 4 && value != 8) {
        must_set_error("correction right-hand sides per CTA must be 0, 2, 4 or 8");
        return MUST_EINVAL;
      }
      g_corr_rhs = value;
      return MUST_OK;
    case 6:   // correction kernel: 1 = thread-block clusters, 0 = one CTA per item and RHS group
      if (value != 0 && value != 1) { must_set_error("correction kernel must be 0 or 1"); return MUST_EINVAL; }
      g_corr_cluster = value;
      return MUST_OK;
    case 7:   // CTAs per cluster of the cluster correction
      if (!correct_cluster_set_ctas(value)) { must_set_error("cluster CTAs must be 2, 4 or 8"); return MUST_EINVAL; }
      return MUST_OK;
    case 9:   // U12 solve: persistent CTAs with copies overlapped (1) or one CTA per tile (0)
      if (value != 0 && value != 1) { must_set_error("U12 solve kernel must be 0 or 1"); return MUST_EINVAL; }
      g_trsm_persist = value;
      return MUST_OK;
    case 8:   // right-hand sides per cluster of the cluster correction
      if (!correct_cluster_set_rhs(value)) { must_set_error("cluster right-hand sides must be 0, 4, 8 or 16"); return MUST_EINVAL; }
      return MUST_OK;
    case 11:  // paired panel steps while the trailing block has at least this many rows (0: never)
      if (value < 0 || value > (1 << 20)) { must_set_error("pairing rows must be in [0, 2^20]"); return MUST_EINVAL; }
      g_pair_rows = value;
      return MUST_OK;
    case 12: {  // cluster correction shape from the third correction on: CL * 100 + G, or 0
      const int CLs = value / 100, Gs = value % 100;
      if (value != 0 && !((CLs == 2 || CLs == 4 || CLs == 8) && (Gs == 4 || Gs == 8 || Gs == 16))) {
        must_set_error("late correction shape must be 0 or CTAs * 100 + right-hand sides (CTAs 2, 4, 8; RHS 4, 8, 16)");
        return MUST_EINVAL;
      }
      g_corr_late = value;
      return MUST_OK;
    }
    case 13:  // kernel of the paired pass
      if (!tc_set_pair_kernel(value)) { must_set_error("paired-pass kernel must be 2 or 3"); return MUST_EINVAL; }
      return MUST_OK;
    case 10:  // where the A operand is packed: main stream, side stream, inside the panel kernel
      if (value < 0 || value > 2) { must_set_error("A pack placement must be 0, 1 or 2"); return MUST_EINVAL; }
      g_pack_side = value;
      return MUST_OK;
  }
  must_set_error("unknown tuning knob %d", knob);
  return MUST_EINVAL;
}

extern "C" int32_t must_tune_get(int32_t knob) {
  switch (knob) {
    case 0: return g_bucket_sites;
    case 1: return tc_get_tile_n();
    case 2: return tc_get_streamed();
    case 3: return tc_get_run();
    case 4: return g_lookahead;
    case 5: return g_corr_rhs;
    case 6: return g_corr_cluster;
    case 7: return correct_cluster_get_ctas();
    case 8: return correct_cluster_get_rhs();
    case 9: return g_trsm_persist;
    case 10: return g_pack_side;
    case 11: return g_pair_rows;
    case 12: return g_corr_late;
    case 13: return tc_get_pair_kernel();
  }
  return -1;
}

// --------------------------------------------------------------------------
// Seeded solve (learned warm start): see include/must.h.
extern "C" must_status must_tau00_solve_seeded(const must_liz* liz, int32_t nE, const double* E, const double* tinv,
                                               int32_t n_species, int32_t nspin, const must_solve_opts* opts,
                                               void* workspace, size_t ws_bytes, const double* tau_seed,
                                               const int32_t* seed_mask, double* tau00, int32_t* status,
                                               int32_t* seed_used, void* stream) {
  must_solve_opts o;
  must_default_opts(&o);
  if (opts) o = *opts;
  if (o.precision == MUST_FP64) {
    must_set_error("must_tau00_solve_seeded: the seed enters the refinement of a mixed-precision path");
    return MUST_EINVAL;
  }
  if (!liz || !tau_seed || !seed_mask || !must_is_device_ptr(tau_seed) || !must_is_device_ptr(seed_mask) ||
      (seed_used && !must_is_device_ptr(seed_used)) || !must_is_device_ptr(tau00)) {
    must_set_error("must_tau00_solve_seeded: tau_seed, seed_mask, seed_used and tau00 must be device memory");
    return MUST_EINVAL;
  }
  SeedArgs a{reinterpret_cast<const double2*>(tau_seed), seed_mask, seed_used};
  g_seed = &a;
  const must_liz* arr[1] = {liz};
  must_status s = solve_common(1, arr, nE, E, tinv, n_species, nspin, &o, workspace, ws_bytes, tau00, status,
                               stream);
  g_seed = nullptr;
  return s;
}
