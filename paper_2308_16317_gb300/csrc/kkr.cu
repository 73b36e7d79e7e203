// Full KKR for a periodic crystal (the paper's Sec. 5: the KKR matrix inverse
// of the original method, built and inverted on the GPU).
//
// N_b sites b_s per cell of the lattice {R}.  The structure constants of
// Eq. (4) summed over the lattice with Bloch phases,
//   G^{st}_{LL'}(k) = sum_{R: rho != 0} e^{ik.R} g0_{LL'}(rho),  rho = b_s - b_t - R,
// give the KKR matrix M(k) = t^{-1} - G(k) of order N_b (lmax+1)^2 (Sec. 2.1),
// and the site-diagonal scattering-path block is its Brillouin-zone average
//   tau^{ss}(E) = (1/N_k) sum_k [M(k)^{-1}]^{ss}
// over a Gamma-centred uniform mesh of n_k^3 points.
//
// Lattice sums by Ewald's split.  With D^{st}_L(k) = sum_R e^{ik.R}
// h_l(kappa|rho|) Y_L(rho^), so that G^{st}_{LL'} = -4 pi i kappa
// sum_L'' i^{l-l'+l''} C(L,L',L'') D^{st}_L'':
//   D_L = (-kappa)^{-l} (-i/kappa) [A_L + B_L + C_L]
//   A_L = (4 pi/Omega) i^l sum_K e^{iq.x} YS_L(q) e^{(E-q^2)/eta} / (q^2 - E),   q = k + K
//   B_L = (2/sqrt pi) (-2)^l sum_{R: rho != 0} e^{ik.R} YS_L(rho) I_l(|rho|)
//   C_0 = -(1/sqrt(4 pi)) [i kappa - sqrt(eta/pi) sum_n (E/eta)^n / (n! (2n-1))]   (s = t only)
// with x = b_s - b_t, YS_L(v) = |v|^l Y_L(v^) the real solid harmonics and
//   I_l(rho) = int_{sqrt(eta)/2}^inf xi^{2l} exp(-rho^2 xi^2 + E/(4 xi^2)) d xi.
// This follows from h_l(kappa r) Y_L(r^) = (-kappa)^{-l} YS_L(grad) h_0(kappa r),
// h_0(z) = -i e^{iz}/z and e^{i kappa r}/r = (2/sqrt pi) int_0^inf
// exp(-r^2 xi^2 + E/(4 xi^2)) d xi, split at xi0 = sqrt(eta)/2: the part below
// xi0 is summed over the reciprocal lattice (Poisson), the part above in real
// space.  I_l is evaluated after the substitution u = rho^2 (xi^2 - xi0^2),
//   I_l = e^{-rho^2 xi0^2} / (2 rho^2) int_0^inf e^{-u} xi^{2l-1} e^{E/(4 xi^2)} du,
// by 16-point Gauss-Legendre rules on the graded panels [0,1], [1,2], [2,4], ...,
// [32,60] of u (the integrand's singularity at u = -rho^2 xi0^2 can lie close to
// u = 0 for near-neighbour rho and small eta, which a Gauss-Laguerre rule
// resolves only to ~1e-11; the graded panels reach ~1e-15).
//
// Only part of the mesh is evaluated: one point per orbit of the crystal's
// point group (operations that map each site onto a site of its class; the sum
// symmetrised at the end with the real-harmonic representation D(g)), or, when
// only the identity qualifies, one point of each pair {k, -k} (M(-k) = M(k)^T,
// its blocks added transposed).
//
// Kernels (all FP64):
//   kkr_real_terms_kernel  per (item, real-space point): the k-independent factor of B_L
//   kkr_recip_table_kernel at build, per k: the energy-independent factors of every
//                          reciprocal term, e^{-q^2/eta} YS_L(q), cos(q.x), sin(q.x), q^2
//   kkr_recip_kernel       per (k, group of items): A_L + C_L for every displacement (x and -x paired)
//   kkr_realsum_kernel     per (item, displacement group, 32 k points): adds B_L
//   kkr_invert_kernel      per (item, group of <= 8 k points): M(k) by the Gaunt contraction,
//                          equilibrated, in-place Gauss-Jordan with partial pivoting in
//                          shared memory (up to 8 small M(k) side by side), diagonal blocks
//                          of M(k)^{-1} summed over the group in a fixed order
//   kkr_bz_sum_kernel      per output element: the groups summed in a fixed order, / N_k
//   kkr_symmetrise_kernel  per (site, item), point-group mode: (1/|G|) sum_g D(g) S^{t_g(s)} D(g)^T
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "solver.h"
#include "prof.h"

void must_gaunt_csr(int lmax, std::vector<int>& start, std::vector<int>& L2s, std::vector<double>& coef);
void must_gauss_legendre_nodes(int n, std::vector<double>& x, std::vector<double>& w);

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int KKR_MAX_N = 64;          // largest M(k) order (one CTA's shared memory)
constexpr int KKR_MAX_L2 = 8;          // l'' <= 2 lmax
constexpr int KKR_MAX_NL2 = (KKR_MAX_L2 + 1) * (KKR_MAX_L2 + 1);
constexpr int KKR_MAX_DISP = 32;       // distinct displacements b_s - b_t
constexpr int KKR_QUAD = 112;          // quadrature nodes for I_l (7 panels x 16)
constexpr int KKR_KCHUNK = 64;         // reciprocal vectors per shared-memory chunk
constexpr int KKR_KB = 32;             // k points per real-space block
constexpr int KKR_RCHUNK = 32;         // real-space points per chunk
constexpr int KKR_KG_MAX = 8;          // most k points per inversion CTA
constexpr double KKR_CUT = 40.0;       // both sums cut where their Gaussian factor < e^{-cut}
constexpr double KKR_ECAP = 1.5;       // sums are cut for Re E <= KKR_ECAP (Ry)
constexpr size_t KKR_TAB_CAP = size_t(512) << 20;   // largest reciprocal-term table kept on the device

__device__ __forceinline__ int l_of_L(int L) {
  int l = 0;
  while ((l + 1) * (l + 1) <= L) ++l;
  return l;
}

// Normalisation of the real harmonics, c_ynorm[l*l + l + m] for m >= 0:
// sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), times sqrt2 for m > 0 (set by must_kkr_build).
__constant__ double c_ynorm[KKR_MAX_NL2];
// 1/n for n = 0..KKR_MAX_L2 (entry 0 unused): the recurrence below divides by l - m
__constant__ double c_recip[KKR_MAX_L2 + 1];

// One column m >= 0 of the real solid harmonics YS_L(v) = |v|^l Y_L(v^)
// (same basis as the library's Y_L, no Condon-Shortley phase), l = m..lmax,
// evaluated as polynomials so that v = 0 needs no special case:
//   YS_lm = c_ynorm {Re (x+iy)^m | Im (x+iy)^|m|} q_l^m(z, r^2),
//   q_m^m = (2m-1)!!, q_{m+1}^m = (2m+1) z q_m^m,
//   q_l^m = [(2l-1) z q_{l-1}^m - (l+m-1) r^2 q_{l-2}^m] / (l-m).
// emit(l, L, value) receives YS_L for L = l*l + l + m and l*l + l - m.
template <class Emit>
__device__ __forceinline__ void solid_harmonic_column(int lmax, int m, double x, double y, double z, double r2,
                                                      Emit emit) {
  double cr = 1.0, ci = 0.0, dfact = 1.0;   // (x + i y)^m, (2m-1)!!
  for (int p = 1; p <= m; ++p) {
    const double nr = cr * x - ci * y, ni = cr * y + ci * x;
    cr = nr;
    ci = ni;
    dfact *= (2.0 * p - 1.0);
  }
  double qm2 = 0.0, qm1 = 0.0;
  for (int l = m; l <= lmax; ++l) {
    double q;
    if (l == m) q = dfact;
    else if (l == m + 1) q = (2.0 * m + 1.0) * z * dfact;
    else q = ((2.0 * l - 1.0) * z * qm1 - (l + m - 1.0) * r2 * qm2) * c_recip[l - m];
    qm2 = qm1;
    qm1 = q;
    const double nq = c_ynorm[l * l + l + m] * q;
    if (m == 0) {
      emit(l, l * l + l, nq);
    } else {
      emit(l, l * l + l + m, nq * cr);
      emit(l, l * l + l - m, nq * ci);
    }
  }
}

__device__ void solid_harmonics(int lmax, double x, double y, double z, double* out) {
  const double r2 = x * x + y * y + z * z;
  for (int m = 0; m <= lmax; ++m)
    solid_harmonic_column(lmax, m, x, y, z, r2, [&](int, int L, double v) { out[L] = v; });
}

__device__ __forceinline__ cd cexp_d(cd z) {
  double s, c;
  sincos(z.y, &s, &c);
  const double m = exp(z.x);
  return mk(m * c, m * s);
}

// i^l
__device__ __forceinline__ cd ipow_d(int l) {
  switch (l & 3) {
    case 0: return mk(1.0, 0.0);
    case 1: return mk(0.0, 1.0);
    case 2: return mk(-1.0, 0.0);
    default: return mk(0.0, -1.0);
  }
}

struct KkrDev {
  int nb, lmax, nL, l2max, nL2, n, n_kpts, n_disp, n_pts, n_kg;
  int kg;                 // k points per inversion CTA (a multiple of the matrices per pass)
  int n_mesh;             // n_k^3: the mesh the average is taken over
  double eta, omega;
  const double* kpts;     // [n_kpts][3]: one point of each pair {k, -k} of the mesh
  const int* kpair;       // [n_kpts]: 1 if -k is a different mesh point (counted as the transpose)
  const int* kwt;         // [n_kpts]: orbit size of the point under the point group (point-group mode)
  int n_ops;              // point-group operations (0: k / -k pairing only)
  const double* Dop;      // [n_ops][nL][nL]: real-harmonic representation of each operation
  const int* op_src;      // [n_ops][nb]: site t with g b_t = b_s (mod lattice), for each site s
  const int* site_class;  // [nb]: sites of one class carry equal t^-1 (checked per item)
  const double* Kvec;     // [nK][3]
  const int* kK_start;    // [n_kpts + 1]
  const int* kK_idx;      // reciprocal vectors of each k with |k + K|^2 <= qmax^2
  const double* disp;     // [n_disp][3], disp 0 = 0
  const int* pair_disp;   // [nb * nb]
  const int* pt_start;    // [n_groups + 1]: points of each displacement group
  const double* pt_R;     // [n_pts][3] lattice vector R
  const double* pt_rho;   // [n_pts][4] rho = x - R and |rho|
  const double* quad_u;   // [KKR_QUAD] nodes in u
  const double* quad_w;   // weights times e^{-u}
  const int* g_start;     // Gaunt CSR, rows (L, L')
  const int* g_L2;
  const double* g_c;
  const double* tab;      // [n_kK][tab_w] or NULL: per (k, K) term, e^{-q^2/eta} YS_L(q) (nL2),
                          // cos(q.x), sin(q.x) of each pair group's x, then q^2
  int tab_w;              // nL2 + 2 (n_groups - 1) + 1
};

// -------------------------------------------------------------------------
// B_L's k-independent factor of every (item, real-space point):
//   T[item][pt][L] = (2/sqrt pi) (-2)^l YS_L(rho) I_l(|rho|)
__global__ void kkr_real_terms_kernel(KkrDev K, int items, const double2* __restrict__ E,
                                      double2* __restrict__ T, int* __restrict__ status) {
  const int pt = blockIdx.x * blockDim.x + threadIdx.x;
  const int it = blockIdx.y;
  if (pt >= K.n_pts || it >= items) return;
  const cd e = mk(E[it].x, E[it].y);
  if (!(e.x <= KKR_ECAP) || !isfinite(e.y)) {
    if (pt == 0) atomicMax(status + it, int(MUST_EUNSUPPORTED));
  }
  const double* pr = K.pt_rho + size_t(pt) * 4;
  const double r = pr[3], r2 = r * r, inv_r2 = 1.0 / r2;
  const double xi02 = 0.25 * K.eta;
  cd I[KKR_MAX_L2 + 1];
  for (int l = 0; l <= K.l2max; ++l) I[l] = mk(0.0, 0.0);
  for (int j = 0; j < KKR_QUAD; ++j) {
    const double xi2 = xi02 + K.quad_u[j] * inv_r2;
    const double inv_xi2 = 1.0 / xi2;
    const cd g = K.quad_w[j] * cexp_d(mk(0.25 * e.x * inv_xi2, 0.25 * e.y * inv_xi2));
    double p = rsqrt(xi2);               // xi^{2l-1}, l = 0
    for (int l = 0; l <= K.l2max; ++l) {
      I[l] = I[l] + p * g;
      p *= xi2;
    }
  }
  const double pref = exp(-r2 * xi02) / (2.0 * r2) * (2.0 / sqrt(kPi));
  double Y[KKR_MAX_NL2];
  solid_harmonics(K.l2max, pr[0], pr[1], pr[2], Y);
  double2* out = T + (size_t(it) * K.n_pts + pt) * K.nL2;
  double m2l = 1.0;                      // (-2)^l
  for (int l = 0; l <= K.l2max; ++l) {
    const cd f = (pref * m2l) * I[l];
    for (int m = -l; m <= l; ++m) {
      const int L = l * l + l + m;
      out[L] = make_double2(f.x * Y[L], f.y * Y[L]);
    }
    m2l *= -2.0;
  }
}

// -------------------------------------------------------------------------
// Displacement groups.  Displacement 0 is x = 0; the others come in pairs
// (x, -x) at indices 2g-1, 2g (group g >= 1).  Both sums use the pairing:
// with the real solid harmonics YS_L(-v) = (-1)^l YS_L(v),
//   reciprocal:  A^{x}_L = i^l (U_L + i V_L),  A^{-x}_L = i^l (U_L - i V_L),
//                U_L = sum_K cos(q.x) w_K YS_L(q), V_L = sum_K sin(q.x) w_K YS_L(q);
//   real space:  the points of -x are those of x negated, so with
//                C_L = sum_R cos(k.R) T_L(R), S_L = sum_R sin(k.R) T_L(R) over the points of x,
//                B^{x}_L = C_L + i S_L,  B^{-x}_L = (-1)^l (C_L - i S_L);
//                for x = 0 only one point of each pair {R, -R} is kept and
//                B^{0}_L = 2 C_L (l even), 2 i S_L (l odd).
// Every accumulation is then a real coefficient times a complex term (or a
// complex coefficient times a real harmonic): two FMAs instead of four.

// -------------------------------------------------------------------------
// A_L + C_L for every displacement, one CTA per (k, group of IB items):
//   Dk[item][k][d][L] = (4 pi/Omega) i^l sum_K e^{iq.x_d} YS_L(q) e^{(E-q^2)/eta}/(q^2-E) + C_L
// Per chunk of KKR_KCHUNK reciprocal vectors: the harmonics come from the
// table (or are formed, four m columns per vector), shared by the CTA's
// items; each (item, vector) gets its weight and its coefficients (w for
// group 0, cos(q.x) w and sin(q.x) w for the pairs); then each thread
// accumulates its outputs (item, group, L) -- over every vector of the
// chunk, or, when the outputs are fewer than the threads, over one of G
// interleaved subsets, the G partial sums being added in order at the end.
// IB is fixed per handle, so an item's summation order does not depend on
// the other items of the call.
constexpr int RECIP_THREADS = 256;

// The energy-independent factors of the reciprocal terms, one row per (k, K)
// in the order of kK_idx: e^{-q^2/eta} YS_L(q) for every L, then cos(q.x) and
// sin(q.x) for the x of each pair group, then q^2.  One CTA per k point.  The
// items of every call then form only 1/(q^2 - E) per term.
constexpr int TAB_THREADS = 128;
__global__ void __launch_bounds__(TAB_THREADS) kkr_recip_table_kernel(KkrDev K, double* __restrict__ tab) {
  const int ik = blockIdx.x;
  const double* kp = K.kpts + size_t(ik) * 3;
  const int k0 = K.kK_start[ik], k1 = K.kK_start[ik + 1];
  const int n_groups = 1 + (K.n_disp - 1) / 2;
  const double inv_eta = 1.0 / K.eta;
  for (int p = k0 + threadIdx.x; p < k1; p += TAB_THREADS) {
    const double* Kv = K.Kvec + size_t(K.kK_idx[p]) * 3;
    const double q0 = kp[0] + Kv[0], q1 = kp[1] + Kv[1], q2v = kp[2] + Kv[2];
    const double qq = q0 * q0 + q1 * q1 + q2v * q2v;
    const double g = exp(-qq * inv_eta);
    double* row = tab + size_t(p) * K.tab_w;
    for (int m = 0; m <= K.l2max; ++m)
      solid_harmonic_column(K.l2max, m, q0, q1, q2v, qq, [&](int, int L, double v) { row[L] = g * v; });
    for (int gi = 1; gi < n_groups; ++gi) {
      const double* x = K.disp + (2 * gi - 1) * 3;
      double sn, cs;
      sincos(q0 * x[0] + q1 * x[1] + q2v * x[2], &sn, &cs);
      row[K.nL2 + 2 * (gi - 1)] = cs;
      row[K.nL2 + 2 * (gi - 1) + 1] = sn;
    }
    row[K.tab_w - 1] = qq;
  }
}

constexpr int KKR_MAX_GROUPS = 1 + (KKR_MAX_DISP - 1) / 2;
constexpr int RECIP_OUT = 6;        // outputs (item, group, L) per thread at most
constexpr int RECIP_IB_MAX = 8;     // items per CTA at most
constexpr int RECIP_MPARTS = RECIP_THREADS / KKR_KCHUNK;
static_assert(KKR_MAX_GROUPS * KKR_MAX_NL2 <= RECIP_OUT * RECIP_THREADS, "one item's outputs per CTA");

__global__ void __launch_bounds__(RECIP_THREADS) kkr_recip_kernel(KkrDev K, int items, int IB,
                                                                  const double2* __restrict__ E,
                                                                  double2* __restrict__ Dk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double2 s_e[RECIP_IB_MAX], s_pre[RECIP_IB_MAX];   // E and (4 pi/Omega) e^{E/eta} of each item
  const int n_groups = 1 + (K.n_disp - 1) / 2;
  const int n_out = n_groups * K.nL2;             // outputs of one item
  const int n_tot = IB * n_out;                   // outputs of the CTA, item-major
  double* Y = reinterpret_cast<double*>(smem_raw);                    // [KCHUNK][nL2] real harmonics
  double* qv = Y + KKR_KCHUNK * K.nL2;                                // [KCHUNK][5]: q, |q|^2, Gaussian
  double2* W = reinterpret_cast<double2*>(qv + 5 * KKR_KCHUNK);       // [IB][n_disp][KCHUNK] coefficients
  double2* wv = W + size_t(IB) * K.n_disp * KKR_KCHUNK;               // [IB][KCHUNK]
  double2* red = wv + IB * KKR_KCHUNK;                                // [2][RECIP_THREADS] partial sums
  const int ik = blockIdx.x, it0 = blockIdx.y * IB, tid = threadIdx.x;
  const int nb_here = min(IB, items - it0);
  const double* kp = K.kpts + size_t(ik) * 3;
  const int k0 = K.kK_start[ik], k1 = K.kK_start[ik + 1];
  const int G = (n_tot <= RECIP_THREADS) ? RECIP_THREADS / n_tot : 1;
  const double inv_eta = 1.0 / K.eta;
  if (tid < IB) {
    const double2 ev = E[it0 + min(tid, nb_here - 1)];
    const cd e = mk(ev.x, ev.y);
    // (4 pi / Omega) e^{E/eta}; each term then needs the real e^{-q^2/eta}
    const cd wpre = (4.0 * kPi / K.omega) * cexp_d(mk(e.x * inv_eta, e.y * inv_eta));
    s_e[tid] = ev;
    s_pre[tid] = make_double2(wpre.x, wpre.y);
  }
  __syncthreads();
  cd accU[RECIP_OUT], accV[RECIP_OUT];
#pragma unroll
  for (int j = 0; j < RECIP_OUT; ++j) { accU[j] = mk(0.0, 0.0); accV[j] = mk(0.0, 0.0); }
  for (int c0 = k0; c0 < k1; c0 += KKR_KCHUNK) {
    const int cn = min(KKR_KCHUNK, k1 - c0);
    const double* trow = K.tab ? K.tab + size_t(c0) * K.tab_w : nullptr;   // the chunk's table rows
    if (tid < KKR_KCHUNK) {
      double q0 = 0.0, q1 = 0.0, q2v = 0.0, qq = 0.0, gq = 0.0;
      if (tid < cn) {
        if (trow) {
          qq = trow[size_t(tid) * K.tab_w + K.tab_w - 1];
          gq = 1.0;   // e^{-q^2/eta} is in the tabulated harmonics
        } else {
          const double* Kv = K.Kvec + size_t(K.kK_idx[c0 + tid]) * 3;
          q0 = kp[0] + Kv[0]; q1 = kp[1] + Kv[1]; q2v = kp[2] + Kv[2];
          qq = q0 * q0 + q1 * q1 + q2v * q2v;
          gq = exp(-qq * inv_eta);
        }
      }
      qv[tid * 5] = q0; qv[tid * 5 + 1] = q1; qv[tid * 5 + 2] = q2v; qv[tid * 5 + 3] = qq; qv[tid * 5 + 4] = gq;
    }
    if (trow) {
      // the chunk's harmonic rows: cn x nL2 doubles copied as they lie in the table
      for (int i = tid; i < cn * K.nL2; i += RECIP_THREADS) {
        const int j = i / K.nL2, L = i - j * K.nL2;
        Y[i] = trow[size_t(j) * K.tab_w + L];
      }
    }
    __syncthreads();
    // w = (4 pi / Omega) e^{(E - q^2)/eta} / (q^2 - E) per (item, vector); zero past the chunk's end
    for (int p = tid; p < IB * KKR_KCHUNK; p += RECIP_THREADS) {
      const int b = p / KKR_KCHUNK, j = p - b * KKR_KCHUNK;
      cd w = mk(0.0, 0.0);
      if (j < cn && b < nb_here) {
        const double2 ev = s_e[b], pr = s_pre[b];
        w = qv[j * 5 + 4] * (mk(pr.x, pr.y) * cinv(mk(qv[j * 5 + 3] - ev.x, -ev.y)));
      }
      wv[p] = make_double2(w.x, w.y);
    }
    if (!trow) {
      const int j = tid % KKR_KCHUNK, part = tid / KKR_KCHUNK;
      double* y = Y + j * K.nL2;
      for (int m = part; m <= K.l2max; m += RECIP_MPARTS)
        solid_harmonic_column(K.l2max, m, qv[j * 5], qv[j * 5 + 1], qv[j * 5 + 2], qv[j * 5 + 3],
                              [&](int, int L, double v) { y[L] = v; });
    }
    __syncthreads();
    for (int p = tid; p < IB * K.n_disp * KKR_KCHUNK; p += RECIP_THREADS) {
      const int b = p / (K.n_disp * KKR_KCHUNK), r = p - b * (K.n_disp * KKR_KCHUNK);
      const int d = r / KKR_KCHUNK, j = r - d * KKR_KCHUNK;
      const double2 w = wv[b * KKR_KCHUNK + j];
      if (d == 0) {
        W[p] = w;
      } else {
        double f;   // row 2g-1: cos(q.x), row 2g: sin(q.x)
        if (trow) {
          f = (j < cn) ? trow[size_t(j) * K.tab_w + K.nL2 + 2 * ((d - 1) / 2) + ((d & 1) ? 0 : 1)] : 0.0;
        } else {
          const double* x = K.disp + ((d - 1) / 2 * 2 + 1) * 3;   // the x of the pair
          double sn, cs;
          sincos(qv[j * 5] * x[0] + qv[j * 5 + 1] * x[1] + qv[j * 5 + 2] * x[2], &sn, &cs);
          f = (d & 1) ? cs : sn;
        }
        W[p] = make_double2(f * w.x, f * w.y);
      }
    }
    __syncthreads();
    const int sub = (G > 1) ? tid / n_tot : 0;
    const int nloop = (G > 1) ? 1 : RECIP_OUT;
#pragma unroll
    for (int jj = 0; jj < RECIP_OUT; ++jj) {
      if (jj >= nloop) break;
      const int ot = (G > 1) ? tid % n_tot : tid + jj * RECIP_THREADS;
      if (ot >= n_tot || (G > 1 && tid >= G * n_tot)) continue;
      const int b = ot / n_out, o = ot - b * n_out;
      const int g = o / K.nL2, L = o - g * K.nL2;
      const int step = (G > 1) ? G : 1;
      const double2* Wb = W + size_t(b) * K.n_disp * KKR_KCHUNK;
      if (g == 0) {
        cd u = accU[jj];
        for (int j = sub; j < cn; j += step) {
          const double yv = Y[j * K.nL2 + L];
          const double2 c = Wb[j];
          u.x = fma(c.x, yv, u.x);
          u.y = fma(c.y, yv, u.y);
        }
        accU[jj] = u;
      } else {
        cd u = accU[jj], v = accV[jj];
        const double2* Wc = Wb + (2 * g - 1) * KKR_KCHUNK;
        const double2* Ws = Wc + KKR_KCHUNK;
        for (int j = sub; j < cn; j += step) {
          const double yv = Y[j * K.nL2 + L];
          const double2 c = Wc[j], sv = Ws[j];
          u.x = fma(c.x, yv, u.x);
          u.y = fma(c.y, yv, u.y);
          v.x = fma(sv.x, yv, v.x);
          v.y = fma(sv.y, yv, v.y);
        }
        accU[jj] = u;
        accV[jj] = v;
      }
    }
    __syncthreads();
  }
  if (G > 1) {
    // partial sums of the G subsets, added in order
    if (tid < G * n_tot) {
      red[tid] = make_double2(accU[0].x, accU[0].y);
      red[RECIP_THREADS + tid] = make_double2(accV[0].x, accV[0].y);
    }
    __syncthreads();
    if (tid < n_tot) {
      cd u = mk(0.0, 0.0), v = mk(0.0, 0.0);
      for (int g = 0; g < G; ++g) {
        u = u + mk(red[g * n_tot + tid].x, red[g * n_tot + tid].y);
        v = v + mk(red[RECIP_THREADS + g * n_tot + tid].x, red[RECIP_THREADS + g * n_tot + tid].y);
      }
      accU[0] = u;
      accV[0] = v;
    }
  }
  const int nwrite = (G > 1) ? 1 : RECIP_OUT;
#pragma unroll
  for (int jj = 0; jj < RECIP_OUT; ++jj) {
    if (jj >= nwrite) break;
    const int ot = tid + jj * RECIP_THREADS;
    if (ot >= n_tot) continue;
    const int b = ot / n_out, o = ot - b * n_out;
    if (b >= nb_here) continue;
    const int g = o / K.nL2, L = o - g * K.nL2, l = l_of_L(L);
    const cd il = ipow_d(l);
    double2* out = Dk + (size_t(it0 + b) * K.n_kpts + ik) * K.n_disp * K.nL2;
    if (g == 0) {
      cd a = il * accU[jj];
      if (L == 0) {
        // C_0 of displacement 0 (x = 0): the R = 0 term of the reciprocal sum removed
        const cd e = mk(s_e[b].x, s_e[b].y);
        const cd kap = csqrt_p(e);
        const cd z = mk(e.x * inv_eta, e.y * inv_eta);
        cd sm = mk(0.0, 0.0), term = mk(1.0, 0.0);   // (E/eta)^n / n!
        for (int n = 0; n < 400; ++n) {
          const cd add = (1.0 / double(2 * n - 1)) * term;
          sm = sm + add;
          if (n > 4 && cnorm(add) < 1e-36 * cnorm(sm)) break;
          term = (1.0 / double(n + 1)) * (term * z);
        }
        const cd f1 = mk(-kap.y, kap.x) - sqrt(K.eta / kPi) * sm;
        a = a - (1.0 / sqrt(4.0 * kPi)) * f1;
      }
      out[L] = make_double2(a.x, a.y);
    } else {
      const cd u = accU[jj], v = accV[jj];
      const cd p = il * mk(u.x - v.y, u.y + v.x);   // i^l (U + i V)
      const cd m = il * mk(u.x + v.y, u.y - v.x);   // i^l (U - i V)
      out[(2 * g - 1) * K.nL2 + L] = make_double2(p.x, p.y);
      out[(2 * g) * K.nL2 + L] = make_double2(m.x, m.y);
    }
  }
}

// -------------------------------------------------------------------------
// Adds B_L, one CTA per (block of KKR_KB k points, displacement group, item):
// the cosine and sine sums C_L, S_L of the group's points (see above).
constexpr int RSUM_THREADS = 256;
constexpr int RSUM_OUT = (KKR_KB * KKR_MAX_NL2 + RSUM_THREADS - 1) / RSUM_THREADS;

__global__ void __launch_bounds__(RSUM_THREADS) kkr_realsum_kernel(KkrDev K, int items,
                                                                   const double2* __restrict__ T,
                                                                   double2* __restrict__ Dk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* Ts = reinterpret_cast<double2*>(smem_raw);   // [RCHUNK][nL2]
  double2* ph = Ts + KKR_RCHUNK * K.nL2;                 // [KB][RCHUNK]: (cos, sin)
  const int kb = blockIdx.x, g = blockIdx.y, it = blockIdx.z, tid = threadIdx.x;
  const int kbase = kb * KKR_KB;
  const int nkb = min(KKR_KB, K.n_kpts - kbase);
  const int p0 = K.pt_start[g], p1 = K.pt_start[g + 1];
  const int n_out = nkb * K.nL2;
  cd accC[RSUM_OUT], accS[RSUM_OUT];
#pragma unroll
  for (int j = 0; j < RSUM_OUT; ++j) { accC[j] = mk(0.0, 0.0); accS[j] = mk(0.0, 0.0); }
  const double2* Tit = T + size_t(it) * K.n_pts * K.nL2;
  for (int c0 = p0; c0 < p1; c0 += KKR_RCHUNK) {
    const int cn = min(KKR_RCHUNK, p1 - c0);
    for (int q = tid; q < cn * K.nL2; q += RSUM_THREADS) Ts[q] = Tit[size_t(c0) * K.nL2 + q];
    for (int q = tid; q < KKR_KB * KKR_RCHUNK; q += RSUM_THREADS) {
      const int kk = q / KKR_RCHUNK, j = q % KKR_RCHUNK;
      if (kk < nkb && j < cn) {
        const double* kp = K.kpts + size_t(kbase + kk) * 3;
        const double* R = K.pt_R + size_t(c0 + j) * 3;
        double sn, cs;
        sincos(kp[0] * R[0] + kp[1] * R[1] + kp[2] * R[2], &sn, &cs);
        ph[q] = make_double2(cs, sn);
      }
    }
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < RSUM_OUT; ++jj) {
      const int o = tid + jj * RSUM_THREADS;
      if (o < n_out) {
        const int kk = o / K.nL2, L = o % K.nL2;
        if (g == 0) {
          // x = 0: only the cosine sum (l even) or the sine sum (l odd) is needed
          const int odd = l_of_L(L) & 1;
          cd a = accC[jj];
          for (int j = 0; j < cn; ++j) {
            const double2 pp = ph[kk * KKR_RCHUNK + j], tt = Ts[j * K.nL2 + L];
            const double f = odd ? pp.y : pp.x;
            a.x = fma(f, tt.x, a.x);
            a.y = fma(f, tt.y, a.y);
          }
          accC[jj] = a;
        } else {
          cd a = accC[jj], b = accS[jj];
          for (int j = 0; j < cn; ++j) {
            const double2 pp = ph[kk * KKR_RCHUNK + j], tt = Ts[j * K.nL2 + L];
            a.x = fma(pp.x, tt.x, a.x);
            a.y = fma(pp.x, tt.y, a.y);
            b.x = fma(pp.y, tt.x, b.x);
            b.y = fma(pp.y, tt.y, b.y);
          }
          accC[jj] = a;
          accS[jj] = b;
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int jj = 0; jj < RSUM_OUT; ++jj) {
    const int o = tid + jj * RSUM_THREADS;
    if (o < n_out) {
      const int kk = o / K.nL2, L = o % K.nL2, l = l_of_L(L);
      double2* row = Dk + (size_t(it) * K.n_kpts + kbase + kk) * K.n_disp * K.nL2;
      const cd c = accC[jj], sv = accS[jj];
      if (g == 0) {
        const cd add = (l & 1) ? mk(-2.0 * c.y, 2.0 * c.x) : mk(2.0 * c.x, 2.0 * c.y);   // 2 i S or 2 C
        const double2 v = row[L];
        row[L] = make_double2(v.x + add.x, v.y + add.y);
      } else {
        const cd plus = mk(c.x - sv.y, c.y + sv.x);             // C + i S
        const double sg = (l & 1) ? -1.0 : 1.0;
        const cd minus = mk(sg * (c.x + sv.y), sg * (c.y - sv.x));   // (-1)^l (C - i S)
        double2* dp = row + (2 * g - 1) * K.nL2 + L;
        double2* dm = row + (2 * g) * K.nL2 + L;
        const double2 vp = *dp, vm = *dm;
        *dp = make_double2(vp.x + plus.x, vp.y + plus.y);
        *dm = make_double2(vm.x + minus.x, vm.y + minus.y);
      }
    }
  }
}

// -------------------------------------------------------------------------
// M(k) = t^{-1} - G(k) in shared memory, inverted in place; the diagonal
// blocks of M(k)^{-1} of K.kg k points summed in order into
//   part[item][group][s][L][L'].
// NM matrices (NM = kkr_matrices_per_pass(n): 1 at n = 64, up to 8 for n <= 22)
// are factored side by side so that small orders still fill the CTA: warp m
// searches matrix m's pivot column, and each matrix's update is spread over
// 256 / NM threads (column j, rows rg, rg + RG, ..., four at a time).
constexpr int INV_THREADS = 256;
constexpr int INV_ACC = (KKR_MAX_N * 25 + INV_THREADS - 1) / INV_THREADS;   // nb nL^2 <= n nL <= 64 x 25

__host__ __device__ inline int kkr_matrices_per_pass(int n) {
  int nm = 8;
  while (nm > 1 && (nm * n * n > KKR_MAX_N * KKR_MAX_N || INV_THREADS / nm < n)) nm >>= 1;
  return nm;
}

__global__ void __launch_bounds__(INV_THREADS) kkr_invert_kernel(KkrDev K, int items, const double2* __restrict__ E,
                                                                 const double2* __restrict__ tinv,
                                                                 const double2* __restrict__ Dk,
                                                                 double2* __restrict__ part, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = K.n, ldA = n + 1, nn = n * ldA;
  const int NM = kkr_matrices_per_pass(n);
  const int TPM = INV_THREADS / NM;                          // threads per matrix
  const int RG = TPM / n;                                    // row groups of the update (>= 1)
  const int nDL = K.n_disp * K.nL2;
  double2* A = reinterpret_cast<double2*>(smem_raw);        // [NM][n][n+1] row-major
  double2* colk = A + NM * nn;                               // [NM][n]
  double2* pinv_s = colk + NM * n;                           // [NM]
  double* sc = reinterpret_cast<double*>(pinv_s + NM);       // [NM][n]
  int* perm = reinterpret_cast<int*>(sc + NM * n);           // [NM][n]
  int* sigma = perm + NM * n;                                // [NM][n]
  int* piv_s = sigma + NM * n;                               // [NM]
  __shared__ double2 fl[KKR_MAX_L2 + 1];
  __shared__ double2 ti_s[KKR_MAX_N];
  __shared__ int singular;
  const int g = blockIdx.x, it = blockIdx.y, tid = threadIdx.x;
  const int nL = K.nL, nb = K.nb;
  const cd e = mk(E[it].x, E[it].y);
  const cd kap = csqrt_p(e);
  if (tid <= K.l2max) {
    // f_l = (-kappa)^{-l} (-i/kappa), times the -4 pi i kappa of G: -4 pi (-kappa)^{-l}
    cd p = mk(-4.0 * kPi, 0.0);
    const cd mik = cinv(mk(-kap.x, -kap.y));
    for (int l = 0; l < tid; ++l) p = p * mik;
    fl[tid] = make_double2(p.x, p.y);
  }
  if (tid < n) {
    const int s = tid / nL, L = tid % nL, l = l_of_L(L);
    ti_s[tid] = tinv[(size_t(it) * nb + s) * (K.lmax + 1) + l];
  }
  // the sum of the diagonal blocks, element q = tid + u * INV_THREADS of [nb][nL][nL]
  cd acc[INV_ACC];
#pragma unroll
  for (int u = 0; u < INV_ACC; ++u) acc[u] = mk(0.0, 0.0);
  if (tid == 0) singular = 0;
  __syncthreads();
  const int kbeg = g * K.kg, kend = min(K.n_kpts, kbeg + K.kg);
  for (int kb = kbeg; kb < kend; kb += NM) {
    const int nm = min(NM, kend - kb);
    // A = t^{-1} - G, G_{LL'} = sum_{L''} c f_{l''} D_{L''} (D read from the lattice sums)
    for (int q = tid; q < nm * n * n; q += INV_THREADS) {
      const int m = q / (n * n), i = (q / n) % n, j = q % n;
      const int s = i / nL, L = i % nL, t = j / nL, Lp = j % nL;
      const double2* Dd = Dk + (size_t(it) * K.n_kpts + kb + m) * nDL + K.pair_disp[s * nb + t] * K.nL2;
      cd gsum = mk(0.0, 0.0);
      for (int p = K.g_start[L * nL + Lp]; p < K.g_start[L * nL + Lp + 1]; ++p) {
        const int L2 = K.g_L2[p];
        const double2 dv = Dd[L2];
        const double2 f = fl[l_of_L(L2)];
        const cd v = K.g_c[p] * (mk(dv.x, dv.y) * mk(f.x, f.y));
        gsum = gsum + v;
      }
      cd a = mk(-gsum.x, -gsum.y);
      if (i == j) a = a + mk(ti_s[i].x, ti_s[i].y);
      A[m * nn + i * ldA + j] = make_double2(a.x, a.y);
    }
    __syncthreads();
    // symmetric equilibration D A D, D = |diag A|^{-1/2}
    for (int q = tid; q < nm * n; q += INV_THREADS) {
      const int m = q / n, i = q % n;
      const double2 d = A[m * nn + i * ldA + i];
      const double mg = sqrt(d.x * d.x + d.y * d.y);
      sc[q] = (mg > 0.0 && isfinite(mg)) ? 1.0 / sqrt(mg) : 1.0;
    }
    __syncthreads();
    for (int q = tid; q < nm * n * n; q += INV_THREADS) {
      const int m = q / (n * n), i = (q / n) % n, j = q % n;
      const double f = sc[m * n + i] * sc[m * n + j];
      double2 v = A[m * nn + i * ldA + j];
      A[m * nn + i * ldA + j] = make_double2(v.x * f, v.y * f);
    }
    __syncthreads();
    // Gauss-Jordan in place with partial (row) pivoting, all nm matrices in step
    for (int k = 0; k < n; ++k) {
      {
        const int w = tid >> 5, lane = tid & 31;
        if (w < nm) {
          const double2* Am = A + w * nn;
          double best = -1.0;
          int bi = k;
          for (int i = k + lane; i < n; i += 32) {
            const double2 v = Am[i * ldA + k];
            const double mg = fabs(v.x) + fabs(v.y);
            if (mg > best) { best = mg; bi = i; }
          }
          for (int off = 16; off > 0; off >>= 1) {
            const double ob = __shfl_down_sync(0xffffffffu, best, off);
            const int oi = __shfl_down_sync(0xffffffffu, bi, off);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
          }
          if (lane == 0) {
            piv_s[w] = bi;
            perm[w * n + k] = bi;
            if (!(best > 0.0)) singular = 1;
            // the pivot's reciprocal, formed once (read before the interchange)
            const double2 pv = Am[bi * ldA + k];
            const cd r = (pv.x == 0.0 && pv.y == 0.0) ? mk(0.0, 0.0) : cinv(mk(pv.x, pv.y));
            pinv_s[w] = make_double2(r.x, r.y);
          }
        }
      }
      __syncthreads();
      for (int q = tid; q < nm * n; q += INV_THREADS) {
        const int m = q / n, j = q % n, p = piv_s[m];
        if (p != k) {
          double2* Am = A + m * nn;
          const double2 t0 = Am[k * ldA + j];
          Am[k * ldA + j] = Am[p * ldA + j];
          Am[p * ldA + j] = t0;
        }
      }
      __syncthreads();
      for (int q = tid; q < nm * n; q += INV_THREADS) {
        const int m = q / n, j = q % n;
        double2* Am = A + m * nn;
        if (j != k) {
          const cd v = mk(Am[k * ldA + j].x, Am[k * ldA + j].y) * mk(pinv_s[m].x, pinv_s[m].y);
          Am[k * ldA + j] = make_double2(v.x, v.y);
        }
        colk[q] = Am[j * ldA + k];
      }
      __syncthreads();
      // every row i != k: A[i][j] -= colk[i] A[k][j] (j != k), A[i][k] = -colk[i] / pivot
      {
        const int m = tid / TPM, r = tid % TPM;
        if (m < nm && r < RG * n) {
          double2* Am = A + m * nn;
          const double2* cm = colk + m * n;
          const cd pinv = mk(pinv_s[m].x, pinv_s[m].y);
          const int j = r % n, rg = r / n;
          if (j == k) {
            for (int i = rg; i < n; i += RG) {
              if (i == k) {
                Am[k * ldA + k] = make_double2(pinv.x, pinv.y);
              } else {
                const cd v = mk(cm[i].x, cm[i].y) * pinv;
                Am[i * ldA + k] = make_double2(-v.x, -v.y);
              }
            }
          } else {
            const cd rk = mk(Am[k * ldA + j].x, Am[k * ldA + j].y);
            int i = rg;
            for (; i + 3 * RG < n; i += 4 * RG) {
              double2 a[4], c[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                a[u] = Am[(i + u * RG) * ldA + j];
                c[u] = cm[i + u * RG];
              }
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                if (i + u * RG == k) continue;
                cd v = mk(a[u].x, a[u].y);
                cfms(v, mk(c[u].x, c[u].y), rk);
                Am[(i + u * RG) * ldA + j] = make_double2(v.x, v.y);
              }
            }
            for (; i < n; i += RG) {
              if (i == k) continue;
              cd v = mk(Am[i * ldA + j].x, Am[i * ldA + j].y);
              cfms(v, mk(cm[i].x, cm[i].y), rk);
              Am[i * ldA + j] = make_double2(v.x, v.y);
            }
          }
        }
      }
      __syncthreads();
    }
    // column j of the inverse is column sigma(j) of the in-place result
    for (int q = tid; q < nm * n; q += INV_THREADS) {
      const int m = q / n;
      int v = q % n;
      for (int k = 0; k < n; ++k) {
        const int pk = perm[m * n + k];
        if (v == k) v = pk;
        else if (v == pk) v = k;
      }
      sigma[q] = v;
    }
    __syncthreads();
    // [M(k)^{-1}]^{ss}, and for a paired point also [M(-k)^{-1}]^{ss} = ([M(k)^{-1}]^{ss})^T
    // (M(-k) = M(k)^T by the reciprocity G_{LL'}(rho) = G_{L'L}(-rho)); k points in order
#pragma unroll
    for (int u = 0; u < INV_ACC; ++u) {
      const int q = tid + u * INV_THREADS;
      if (q >= nb * nL * nL) break;
      const int s = q / (nL * nL), L = (q / nL) % nL, Lp = q % nL;
      const int i = s * nL + L, j = s * nL + Lp;
      double ax = acc[u].x, ay = acc[u].y;
      for (int m = 0; m < nm; ++m) {
        const double2* Am = A + m * nn;
        const int* sg = sigma + m * n;
        const double f = sc[m * n + i] * sc[m * n + j];
        const double2 x = Am[i * ldA + sg[j]];
        if (K.n_ops > 0) {
          // point-group mode: the point stands for its orbit (symmetrised at the end)
          const double fw = f * double(K.kwt[kb + m]);
          ax += fw * x.x;
          ay += fw * x.y;
        } else {
          ax += f * x.x;
          ay += f * x.y;
          if (K.kpair[kb + m]) {
            const double2 y = Am[j * ldA + sg[i]];
            ax += f * y.x;
            ay += f * y.y;
          }
        }
      }
      acc[u] = mk(ax, ay);
    }
    __syncthreads();
  }
  double2* dst = part + (size_t(it) * K.n_kg + g) * nb * nL * nL;
#pragma unroll
  for (int u = 0; u < INV_ACC; ++u) {
    const int q = tid + u * INV_THREADS;
    if (q < nb * nL * nL) dst[q] = make_double2(acc[u].x, acc[u].y);
  }
  if (tid == 0 && singular) atomicMax(status + it, int(MUST_ESINGULAR));
}

// Sum of the k groups in a fixed order, / N_k: written as tau[item][s]
// (column-major kap x kap), or, in point-group mode, as the orbit-weighted sum
// S[item][s] (row-major) that kkr_symmetrise_kernel turns into tau.
__global__ void kkr_bz_sum_kernel(KkrDev K, int items, const double2* __restrict__ part, double2* __restrict__ tau,
                                  double2* __restrict__ S, int* __restrict__ status) {
  const int nLL = K.nL * K.nL;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= items * K.nb * nLL) return;
  const int it = q / (K.nb * nLL), r = q % (K.nb * nLL);
  const int s = r / nLL, L = (r / K.nL) % K.nL, Lp = r % K.nL;
  double sx = 0.0, sy = 0.0;
  for (int g = 0; g < K.n_kg; ++g) {
    const double2 v = part[(size_t(it) * K.n_kg + g) * K.nb * nLL + r];
    sx += v.x;
    sy += v.y;
  }
  const double w = 1.0 / double(K.n_mesh);
  sx *= w;
  sy *= w;
  if (!isfinite(sx) || !isfinite(sy)) atomicMax(status + it, int(MUST_ENONFINITE));
  if (K.n_ops > 0) S[size_t(it) * K.nb * nLL + r] = make_double2(sx, sy);
  else tau[(size_t(it) * K.nb + s) * nLL + L + Lp * K.nL] = make_double2(sx, sy);
}

// Point-group mode: tau^{s} = (1/|G|) sum_g D(g) S^{t_g(s)} D(g)^T, t_g(s) the site
// that g carries onto s ([M(gk)^{-1}]^{ss'} blocks of sites related by g are
// D(g) [M(k)^{-1}]^{tt} D(g)^T: the Bloch phases of the permutation cancel on the
// diagonal).  Also checks, per item, that sites of one class carry equal t^-1.
// One CTA per (site, item).
constexpr int SYM_THREADS = 256;
constexpr int SYM_OUT = (25 * 25 + SYM_THREADS - 1) / SYM_THREADS;

__global__ void __launch_bounds__(SYM_THREADS) kkr_symmetrise_kernel(KkrDev K, int items,
                                                                      const double2* __restrict__ S,
                                                                      const double2* __restrict__ tinv,
                                                                      double2* __restrict__ tau,
                                                                      int* __restrict__ status) {
  __shared__ double2 Ssrc[25 * 25];
  __shared__ double2 T[25 * 25];
  const int nL = K.nL, nLL = nL * nL;
  const int s = blockIdx.x, it = blockIdx.y, tid = threadIdx.x;
  if (s == 0 && tid == 0) {
    // the promise the symmetry rests on: equal t^-1 within each class
    bool ok = true;
    for (int a = 0; a < K.nb; ++a)
      for (int b2 = a + 1; b2 < K.nb; ++b2)
        if (K.site_class[a] == K.site_class[b2])
          for (int l = 0; l <= K.lmax; ++l) {
            const double2 x = tinv[(size_t(it) * K.nb + a) * (K.lmax + 1) + l];
            const double2 y = tinv[(size_t(it) * K.nb + b2) * (K.lmax + 1) + l];
            if (x.x != y.x || x.y != y.y) ok = false;
          }
    if (!ok) atomicMax(status + it, int(MUST_EINVAL));
  }
  double2 out[SYM_OUT];
#pragma unroll
  for (int u = 0; u < SYM_OUT; ++u) out[u] = make_double2(0.0, 0.0);
  for (int op = 0; op < K.n_ops; ++op) {
    const int t = K.op_src[op * K.nb + s];
    const double2* St = S + (size_t(it) * K.nb + t) * nLL;
    for (int r = tid; r < nLL; r += SYM_THREADS) Ssrc[r] = St[r];
    __syncthreads();
    const double* D = K.Dop + size_t(op) * nLL;
    for (int r = tid; r < nLL; r += SYM_THREADS) {   // T = D S
      const int L = r / nL, B = r % nL;
      double tx = 0.0, ty = 0.0;
      for (int A = 0; A < nL; ++A) {
        const double d = D[L * nL + A];
        tx = fma(d, Ssrc[A * nL + B].x, tx);
        ty = fma(d, Ssrc[A * nL + B].y, ty);
      }
      T[r] = make_double2(tx, ty);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < SYM_OUT; ++u) {              // out += T D^T
      const int r = tid + u * SYM_THREADS;
      if (r < nLL) {
        const int L = r / nL, Lp = r % nL;
        double ox = out[u].x, oy = out[u].y;
        for (int B = 0; B < nL; ++B) {
          const double d = D[Lp * nL + B];
          ox = fma(T[L * nL + B].x, d, ox);
          oy = fma(T[L * nL + B].y, d, oy);
        }
        out[u] = make_double2(ox, oy);
      }
    }
    __syncthreads();
  }
  const double scale = 1.0 / double(K.n_ops);
#pragma unroll
  for (int u = 0; u < SYM_OUT; ++u) {
    const int r = tid + u * SYM_THREADS;
    if (r < nLL) {
      const int L = r / nL, Lp = r % nL;
      tau[(size_t(it) * K.nb + s) * nLL + L + Lp * nL] = make_double2(out[u].x * scale, out[u].y * scale);
    }
  }
}

__global__ void kkr_status_init_kernel(int items, int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < items) status[i] = 0;
}

__global__ void kkr_status_out_kernel(int items, const int* status, int* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < items) out[i] = status[i];
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// Nodes and weights (times e^{-u}) of 16-point Gauss-Legendre rules on the
// graded panels [0,1], [1,2], [2,4], [4,8], [8,16], [16,32], [32,60] of u.
void quadrature_u(std::vector<double>& u, std::vector<double>& w) {
  std::vector<double> x, wx;
  must_gauss_legendre_nodes(16, x, wx);
  const double edges[8] = {0.0, 1.0, 2.0, 4.0, 8.0, 16.0, 32.0, 60.0};
  u.clear();
  w.clear();
  for (int p = 0; p < 7; ++p) {
    const double lo = edges[p], hi = edges[p + 1], h = 0.5 * (hi - lo);
    for (int j = 0; j < 16; ++j) {
      const double uj = lo + h * (x[j] + 1.0);
      u.push_back(uj);
      w.push_back(h * wx[j] * std::exp(-uj));
    }
  }
}

double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
double norm3(const double* a) { return std::sqrt(dot3(a, a)); }

// All n1 V0 + n2 V1 + n3 V2 with |c + v| <= rmax; W: dual rows (a_i . b_j = 2 pi delta).
void points_within(const double V[3][3], const double W[3][3], const double* c, double rmax,
                   std::vector<double>& out) {
  int nmax[3];
  const double cn = norm3(c);
  for (int i = 0; i < 3; ++i) nmax[i] = int(std::ceil((rmax + cn) * norm3(W[i]) / (2.0 * kPi))) + 1;
  out.clear();
  for (int n1 = -nmax[0]; n1 <= nmax[0]; ++n1)
    for (int n2 = -nmax[1]; n2 <= nmax[1]; ++n2)
      for (int n3 = -nmax[2]; n3 <= nmax[2]; ++n3) {
        double v[3], w[3];
        for (int d = 0; d < 3; ++d) {
          v[d] = n1 * V[0][d] + n2 * V[1][d] + n3 * V[2][d];
          w[d] = c[d] + v[d];
        }
        if (norm3(w) <= rmax) out.insert(out.end(), v, v + 3);
      }
}


// Real spherical harmonics on the host (the library's basis: no Condon-Shortley
// phase, sqrt2 cos / sin combinations), for the point-group matrices only.
void ylm_host(int lmax, double x, double y, double z, double* out) {
  const double r = std::sqrt(x * x + y * y + z * z);
  const double ct = z / r, rho = std::sqrt(x * x + y * y), st = rho / r;
  const double phi = rho > 0.0 ? std::atan2(y, x) : 0.0;
  for (int m = 0; m <= lmax; ++m) {
    double pmm = 1.0;
    for (int i = 1; i <= m; ++i) pmm *= (2.0 * i - 1.0) * st;
    double p2 = 0.0, p1 = pmm;
    for (int l = m; l <= lmax; ++l) {
      double pl;
      if (l == m) pl = pmm;
      else if (l == m + 1) pl = (2.0 * m + 1.0) * ct * pmm;
      else pl = ((2.0 * l - 1.0) * ct * p1 - (l + m - 1.0) * p2) / double(l - m);
      if (l > m) { p2 = p1; p1 = pl; }
      double ratio = 1.0;
      for (int q = l - m + 1; q <= l + m; ++q) ratio /= double(q);
      const double N = std::sqrt((2.0 * l + 1.0) / (4.0 * kPi) * ratio);
      if (m == 0) {
        out[l * l + l] = N * pl;
      } else {
        out[l * l + l + m] = std::sqrt(2.0) * N * pl * std::cos(m * phi);
        out[l * l + l - m] = std::sqrt(2.0) * N * pl * std::sin(m * phi);
      }
    }
  }
}

// D(g)_{LM} = int Y_L(g r) Y_M(r) dOmega for l <= lmax (exact product rule:
// Gauss-Legendre in cos theta, uniform in phi).
void harmonic_rep(int lmax, const double g[3][3], std::vector<double>& D) {
  const int nL = (lmax + 1) * (lmax + 1);
  const int nt = lmax + 2, np = 2 * lmax + 3;
  std::vector<double> xt, wt;
  must_gauss_legendre_nodes(nt, xt, wt);
  D.assign(size_t(nL) * nL, 0.0);
  std::vector<double> Ya(nL), Yb(nL);
  for (int a = 0; a < nt; ++a) {
    const double ct = xt[a], st = std::sqrt(1.0 - ct * ct);
    for (int b = 0; b < np; ++b) {
      const double ph = 2.0 * kPi * b / np, w = wt[a] * 2.0 * kPi / np;
      const double r[3] = {st * std::cos(ph), st * std::sin(ph), ct};
      double gr[3];
      for (int i = 0; i < 3; ++i) gr[i] = g[i][0] * r[0] + g[i][1] * r[1] + g[i][2] * r[2];
      ylm_host(lmax, gr[0], gr[1], gr[2], Ya.data());
      ylm_host(lmax, r[0], r[1], r[2], Yb.data());
      for (int L = 0; L < nL; ++L)
        for (int M = 0; M < nL; ++M) D[size_t(L) * nL + M] += w * Ya[L] * Yb[M];
    }
  }
  for (double& v : D)
    if (std::fabs(v) < 1e-14) v = 0.0;
}

}  // namespace

struct must_kkr {
  int nb, lmax, nL, l2max, nL2, n, n_k, n_kpts, n_mesh, n_disp, n_pts, n_pts0, n_K, n_kK, n_kg, kg, n_ops, device;
  double eta, omega;
  double* d_kpts;
  int* d_kpair;
  int* d_kwt;
  double* d_Dop;
  int* d_op_src;
  int* d_class;
  double* d_K;
  int* d_kK_start;
  int* d_kK_idx;
  double* d_disp;
  int* d_pair_disp;
  int* d_pt_start;
  double* d_pt_R;
  double* d_pt_rho;
  double* d_quad_u;
  double* d_quad_w;
  int* d_g_start;
  int* d_g_L2;
  double* d_g_c;
  double* d_tab;          // reciprocal-term table (NULL: the terms are formed per item)
  int tab_w;
  size_t tab_bytes;
};

namespace {

KkrDev dev_view(const must_kkr* h) {
  KkrDev K;
  K.nb = h->nb; K.lmax = h->lmax; K.nL = h->nL; K.l2max = h->l2max; K.nL2 = h->nL2; K.n = h->n;
  K.n_kpts = h->n_kpts; K.n_mesh = h->n_mesh; K.n_disp = h->n_disp; K.n_pts = h->n_pts; K.n_kg = h->n_kg; K.kg = h->kg;
  K.eta = h->eta; K.omega = h->omega;
  K.kpts = h->d_kpts; K.kpair = h->d_kpair; K.kwt = h->d_kwt; K.n_ops = h->n_ops; K.Dop = h->d_Dop; K.op_src = h->d_op_src; K.site_class = h->d_class; K.Kvec = h->d_K; K.kK_start = h->d_kK_start; K.kK_idx = h->d_kK_idx;
  K.disp = h->d_disp; K.pair_disp = h->d_pair_disp; K.pt_start = h->d_pt_start; K.pt_R = h->d_pt_R;
  K.pt_rho = h->d_pt_rho; K.quad_u = h->d_quad_u; K.quad_w = h->d_quad_w;
  K.g_start = h->d_g_start; K.g_L2 = h->d_g_L2; K.g_c = h->d_g_c;
  K.tab = h->d_tab; K.tab_w = h->tab_w;
  return K;
}

size_t recip_smem_ib(const must_kkr* h, int ib) {
  return sizeof(double) * (size_t(KKR_KCHUNK) * h->nL2 + 5 * KKR_KCHUNK) +
         sizeof(double2) * (size_t(ib) * (size_t(h->n_disp) + 1) * KKR_KCHUNK + 2 * RECIP_THREADS);
}

// Items per CTA of the reciprocal sums: as many as the output registers
// (RECIP_OUT per thread) and ~100 KB of shared memory (two CTAs per SM) allow,
// at most RECIP_IB_MAX.
int recip_ib(const must_kkr* h) {
  const int n_out = (1 + (h->n_disp - 1) / 2) * h->nL2;
  int ib = std::max(1, std::min(RECIP_IB_MAX, (RECIP_OUT * RECIP_THREADS) / n_out));
  while (ib > 1 && recip_smem_ib(h, ib) > size_t(100) * 1024) --ib;
  return ib;
}

size_t recip_smem(const must_kkr* h) { return recip_smem_ib(h, recip_ib(h)); }

size_t realsum_smem(const must_kkr* h) {
  return sizeof(double2) * (size_t(KKR_RCHUNK) * h->nL2 + size_t(KKR_KB) * KKR_RCHUNK);
}

size_t invert_smem(const must_kkr* h) {
  const size_t NM = size_t(kkr_matrices_per_pass(h->n)), n = size_t(h->n);
  return sizeof(double2) * (NM * n * (n + 1) + NM * n + NM) + sizeof(double) * NM * n + sizeof(int) * (2 * NM * n + NM);
}

struct KkrWs {
  double2* T;
  double2* Dk;
  double2* part;
  double2* S;
  int* status;
  size_t bytes;
};

KkrWs carve(const must_kkr* h, int items, char* base) {
  KkrWs w;
  size_t off = 0;
  auto take = [&](size_t b) { char* p = base ? base + off : nullptr; off += a256(b); return p; };
  w.T = reinterpret_cast<double2*>(take(sizeof(double2) * size_t(items) * h->n_pts * h->nL2));
  w.Dk = reinterpret_cast<double2*>(take(sizeof(double2) * size_t(items) * h->n_kpts * h->n_disp * h->nL2));
  w.part = reinterpret_cast<double2*>(take(sizeof(double2) * size_t(items) * h->n_kg * h->nb * h->nL * h->nL));
  w.S = reinterpret_cast<double2*>(take(sizeof(double2) * size_t(items) * h->nb * h->nL * h->nL));
  w.status = reinterpret_cast<int*>(take(sizeof(int) * size_t(items)));
  w.bytes = off;
  return w;
}

size_t staging_bytes(const must_kkr* h, int items) {
  return a256(sizeof(double2) * size_t(items)) + a256(sizeof(double2) * size_t(items) * h->nb * (h->lmax + 1)) +
         a256(sizeof(double2) * size_t(items) * h->nb * h->nL * h->nL) + a256(sizeof(int) * size_t(items));
}

}  // namespace

// The host set-up (argument checks, lattice, point group, mesh and its orbits,
// reciprocal and real-space vector lists, quadrature, Gaunt table), then the
// device tables.  With dry_info the set-up's sizes are returned instead and no
// CUDA call is made (must_kkr_geometry).
static must_status kkr_build_impl(const double* lattice, const double* basis, const int32_t* site_class,
                                  int32_t n_basis, int32_t lmax, int32_t n_k, double eta, int32_t flags,
                                  void* stream, must_kkr** out, int32_t* dry_info, double* dry_eta) {
  if (!out && !dry_info) { must_set_error("must_kkr_build: out is NULL"); return MUST_EINVAL; }
  if (out) *out = nullptr;
  if (!lattice || !basis || n_basis < 1 || lmax < 0 || lmax > 4 || n_k < 1 || n_k > 64 || !(eta >= 0.0) ||
      (flags & ~(MUST_KKR_NO_SYMMETRY | MUST_KKR_NO_TABLE))) {
    must_set_error("must_kkr_build: bad argument (lattice/basis NULL, n_basis < 1, lmax outside 0..4, n_k outside "
                   "1..64 or eta < 0)");
    return MUST_EINVAL;
  }
  const int nL = (lmax + 1) * (lmax + 1);
  if (n_basis * nL > KKR_MAX_N) {
    must_set_error("must_kkr_build: order n_basis (lmax+1)^2 = %d exceeds %d", n_basis * nL, KKR_MAX_N);
    return MUST_EINVAL;
  }
  for (int i = 0; i < 9; ++i)
    if (!std::isfinite(lattice[i])) { must_set_error("must_kkr_build: non-finite lattice"); return MUST_EINVAL; }
  for (int i = 0; i < 3 * n_basis; ++i)
    if (!std::isfinite(basis[i])) { must_set_error("must_kkr_build: non-finite basis"); return MUST_EINVAL; }
  double A[3][3], B[3][3], C[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) A[i][j] = lattice[3 * i + j];
  auto cross = [](const double* u, const double* v, double* w) {
    w[0] = u[1] * v[2] - u[2] * v[1];
    w[1] = u[2] * v[0] - u[0] * v[2];
    w[2] = u[0] * v[1] - u[1] * v[0];
  };
  cross(A[1], A[2], C[0]);
  cross(A[2], A[0], C[1]);
  cross(A[0], A[1], C[2]);
  const double vol = dot3(A[0], C[0]);
  const double scale = norm3(A[0]) * norm3(A[1]) * norm3(A[2]);
  if (!(std::fabs(vol) > 1e-8 * scale)) { must_set_error("must_kkr_build: degenerate lattice"); return MUST_EINVAL; }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) B[i][j] = 2.0 * kPi * C[i][j] / vol;
  const double omega = std::fabs(vol);
  // distinct basis sites modulo the lattice
  for (int s = 0; s < n_basis; ++s)
    for (int t = s + 1; t < n_basis; ++t) {
      double f[3];
      for (int i = 0; i < 3; ++i) {
        const double x[3] = {basis[3 * s] - basis[3 * t], basis[3 * s + 1] - basis[3 * t + 1],
                             basis[3 * s + 2] - basis[3 * t + 2]};
        f[i] = dot3(x, B[i]) / (2.0 * kPi);
      }
      if (std::fabs(f[0] - std::round(f[0])) < 1e-9 && std::fabs(f[1] - std::round(f[1])) < 1e-9 &&
          std::fabs(f[2] - std::round(f[2])) < 1e-9) {
        must_set_error("must_kkr_build: basis sites %d and %d coincide modulo the lattice", s, t);
        return MUST_EINVAL;
      }
    }
  if (eta == 0.0) {
    // 4 pi / Omega^(2/3) makes the two sums about equally long; with one site per
    // cell the real-space side is the cheaper one (x = 0 only, points paired), and
    // 0.7 of it measured fastest (fcc primitive cell: 1174 vs 976 tau solves/s;
    // the 4-site cell was fastest at 1.0; below ~0.4 e^{E/eta} costs accuracy)
    eta = 4.0 * kPi / std::pow(omega, 2.0 / 3.0) * (n_basis == 1 ? 0.7 : 1.0);
  }
  const int l2max = 2 * lmax, nL2 = (l2max + 1) * (l2max + 1);
  // distinct displacements: 0 first, then each x != 0 followed by -x
  std::vector<double> disp = {0.0, 0.0, 0.0};
  std::vector<int> pair_disp(size_t(n_basis) * n_basis);
  auto find_disp = [&](const double* x) {
    for (size_t d = 0; d < disp.size() / 3; ++d)
      if (disp[3 * d] == x[0] && disp[3 * d + 1] == x[1] && disp[3 * d + 2] == x[2]) return int(d);
    return -1;
  };
  for (int s = 0; s < n_basis; ++s)
    for (int t = 0; t < n_basis; ++t) {
      const double x[3] = {basis[3 * s] - basis[3 * t], basis[3 * s + 1] - basis[3 * t + 1],
                           basis[3 * s + 2] - basis[3 * t + 2]};
      int found = find_disp(x);
      if (found < 0) {
        // fl(b_t - b_s) = -fl(b_s - b_t) exactly, so -x is the displacement of (t, s)
        const double mx[3] = {-x[0], -x[1], -x[2]};
        found = int(disp.size() / 3);
        disp.insert(disp.end(), x, x + 3);
        disp.insert(disp.end(), mx, mx + 3);
      }
      pair_disp[size_t(s) * n_basis + t] = found;
    }
  const int n_disp = int(disp.size() / 3);
  if (n_disp > KKR_MAX_DISP) {
    must_set_error("must_kkr_build: %d distinct site displacements exceed %d", n_disp, KKR_MAX_DISP);
    return MUST_EINVAL;
  }
  // Point group: the signed permutations g of the Cartesian axes that map the
  // lattice onto itself and every site onto a site of its class (modulo the
  // lattice); sites of one class are promised equal t^-1 (checked per item).
  // Without classes every site is its own class.  Q_g[i][j] = (g b*_i).a_j / 2 pi
  // is g's integer action on mesh coordinates; src_g[s] the site t with
  // g b_t = b_s (mod lattice).
  std::vector<int> cls(n_basis);
  for (int i = 0; i < n_basis; ++i) cls[i] = site_class ? site_class[i] : i;
  std::vector<std::array<int, 9>> Qops;
  std::vector<double> Dops;
  std::vector<int> src_ops;
  if (!(flags & MUST_KKR_NO_SYMMETRY)) {
    const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int pi = 0; pi < 6; ++pi)
      for (int sg = 0; sg < 8; ++sg) {
        double g[3][3] = {{0.0}};
        for (int r = 0; r < 3; ++r) g[r][perms[pi][r]] = ((sg >> r) & 1) ? -1.0 : 1.0;
        bool ok = true;
        std::array<int, 9> Q{};
        for (int i = 0; i < 3 && ok; ++i) {
          double ga[3], gb[3];
          for (int r = 0; r < 3; ++r) {
            ga[r] = g[r][0] * A[i][0] + g[r][1] * A[i][1] + g[r][2] * A[i][2];
            gb[r] = g[r][0] * B[i][0] + g[r][1] * B[i][1] + g[r][2] * B[i][2];
          }
          for (int j = 0; j < 3 && ok; ++j) {
            const double ca = dot3(ga, B[j]) / (2.0 * kPi), cb = dot3(gb, A[j]) / (2.0 * kPi);
            if (std::fabs(ca - std::round(ca)) > 1e-8 || std::fabs(cb - std::round(cb)) > 1e-8) ok = false;
            Q[3 * i + j] = int(std::lround(cb));
          }
        }
        std::vector<int> src(n_basis, -1);
        for (int t = 0; t < n_basis && ok; ++t) {
          double gbt[3];
          for (int r = 0; r < 3; ++r)
            gbt[r] = g[r][0] * basis[3 * t] + g[r][1] * basis[3 * t + 1] + g[r][2] * basis[3 * t + 2];
          int hit = -1;
          for (int u = 0; u < n_basis && hit < 0; ++u) {
            const double d[3] = {gbt[0] - basis[3 * u], gbt[1] - basis[3 * u + 1], gbt[2] - basis[3 * u + 2]};
            bool lat = true;
            for (int j = 0; j < 3; ++j) {
              const double f = dot3(d, B[j]) / (2.0 * kPi);
              if (std::fabs(f - std::round(f)) > 1e-8) lat = false;
            }
            if (lat) hit = u;
          }
          if (hit < 0 || cls[hit] != cls[t] || src[hit] >= 0) ok = false;
          else src[hit] = t;
        }
        if (!ok) continue;
        Qops.push_back(Q);
        src_ops.insert(src_ops.end(), src.begin(), src.end());
        std::vector<double> D;
        harmonic_rep(lmax, g, D);
        Dops.insert(Dops.end(), D.begin(), D.end());
      }
  }
  if (Qops.size() <= 1) { Qops.clear(); Dops.clear(); src_ops.clear(); }   // identity only: k / -k pairing
  const int n_ops = int(Qops.size());
  // Gamma-centred mesh, folded to m_i in (-n_k/2, n_k/2].  Point-group mode: one
  // point of each orbit, weighted by the orbit's size.  Otherwise one point of
  // each pair {m, -m mod n_k} (M(-k) = M(k)^T), flagged when -m differs.
  std::vector<double> kpts;
  std::vector<int> kpair, kwt;
  double kmax = 0.0;
  std::vector<char> seen(size_t(n_k) * n_k * n_k, 0);
  for (int m1 = 0; m1 < n_k; ++m1)
    for (int m2 = 0; m2 < n_k; ++m2)
      for (int m3 = 0; m3 < n_k; ++m3) {
        const int idx = (m1 * n_k + m2) * n_k + m3;
        if (n_ops > 0) {
          if (seen[idx]) continue;
          int orbit = 0;
          const int mv[3] = {m1, m2, m3};
          for (const auto& Q : Qops) {
            int mm[3];
            for (int j = 0; j < 3; ++j) {
              long v = 0;
              for (int i = 0; i < 3; ++i) v += long(mv[i]) * Q[3 * i + j];
              mm[j] = int(((v % n_k) + n_k) % n_k);
            }
            const int id2 = (mm[0] * n_k + mm[1]) * n_k + mm[2];
            if (!seen[id2]) { seen[id2] = 1; ++orbit; }
          }
          kwt.push_back(orbit);
          kpair.push_back(0);
        } else {
          const int nidx = (((n_k - m1) % n_k) * n_k + (n_k - m2) % n_k) * n_k + (n_k - m3) % n_k;
          if (nidx < idx) continue;   // its partner is kept
          kpair.push_back(nidx != idx ? 1 : 0);
          kwt.push_back(1);
        }
        const int f1 = (2 * m1 > n_k) ? m1 - n_k : m1, f2 = (2 * m2 > n_k) ? m2 - n_k : m2,
                  f3 = (2 * m3 > n_k) ? m3 - n_k : m3;
        double k[3];
        for (int d = 0; d < 3; ++d) k[d] = (f1 * B[0][d] + f2 * B[1][d] + f3 * B[2][d]) / n_k;
        kmax = std::max(kmax, norm3(k));
        kpts.insert(kpts.end(), k, k + 3);
      }
  if (n_ops > 0) {
    long total = 0;
    for (int v : kwt) total += v;
    if (total != long(n_k) * n_k * n_k) {
      must_set_error("must_kkr_build: point-group orbits do not cover the mesh");
      return MUST_EINVAL;
    }
  }
  const int n_kpts = int(kpair.size());
  // reciprocal vectors: |k + K|^2 <= eta cut + E_cap for each k
  const double qmax = std::sqrt(eta * KKR_CUT + KKR_ECAP);
  std::vector<double> Kv;
  const double zero[3] = {0.0, 0.0, 0.0};
  points_within(B, A, zero, qmax + kmax, Kv);
  const int n_K = int(Kv.size() / 3);
  std::vector<int> kK_start(n_kpts + 1, 0), kK_idx;
  for (int ik = 0; ik < n_kpts; ++ik) {
    kK_start[ik] = int(kK_idx.size());
    const double* k = &kpts[3 * ik];
    for (int j = 0; j < n_K; ++j) {
      const double q[3] = {k[0] + Kv[3 * j], k[1] + Kv[3 * j + 1], k[2] + Kv[3 * j + 2]};
      if (dot3(q, q) <= qmax * qmax) kK_idx.push_back(j);
    }
  }
  kK_start[n_kpts] = int(kK_idx.size());
  // real-space points per displacement group: for x = 0 one point of each pair
  // {R, -R} with 0 < |R| <= rho_max (the first nonzero coordinate positive); for
  // a pair (x, -x) the points of x, 0 < |x - R| <= rho_max (those of -x are
  // their negatives)
  const double rho_max = std::sqrt(4.0 * (KKR_CUT + KKR_ECAP / eta) / eta);
  const int n_groups = 1 + (n_disp - 1) / 2;
  std::vector<int> pt_start(n_groups + 1, 0);
  std::vector<double> pt_R, pt_rho, pts;
  for (int g = 0; g < n_groups; ++g) {
    pt_start[g] = int(pt_R.size() / 3);
    const double* x = &disp[3 * (g == 0 ? 0 : 2 * g - 1)];
    const double mx[3] = {-x[0], -x[1], -x[2]};
    points_within(A, B, mx, rho_max, pts);
    const double tiny = 1e-9 * norm3(A[0]);
    for (size_t p = 0; p < pts.size(); p += 3) {
      const double rho[3] = {x[0] - pts[p], x[1] - pts[p + 1], x[2] - pts[p + 2]};
      const double r = norm3(rho);
      if (r < 1e-10) continue;
      if (g == 0) {
        const double* R = &pts[p];
        const int lead = (std::fabs(R[0]) > tiny) ? 0 : (std::fabs(R[1]) > tiny) ? 1 : 2;
        if (R[lead] < 0.0) continue;   // its partner -R is kept
      }
      pt_R.insert(pt_R.end(), pts.begin() + p, pts.begin() + p + 3);
      pt_rho.push_back(rho[0]);
      pt_rho.push_back(rho[1]);
      pt_rho.push_back(rho[2]);
      pt_rho.push_back(r);
    }
  }
  const int n_pts = int(pt_R.size() / 3);
  pt_start[n_groups] = n_pts;
  std::vector<double> lu, lw;
  quadrature_u(lu, lw);
  if (int(lu.size()) != KKR_QUAD) { must_set_error("must_kkr_build: quadrature size"); return MUST_ECUDA; }
  std::vector<int> gs, gl;
  std::vector<double> gc;
  must_gaunt_csr(lmax, gs, gl, gc);

  // k points per inversion CTA: whole passes of side-by-side matrices, at most
  // KKR_KG_MAX, and few enough that small (symmetry-reduced) meshes still give
  // each item ~32 CTAs
  int kg_val;
  {
    const int nm = kkr_matrices_per_pass(n_basis * nL);
    const int want = nm * ((n_kpts + 32 * nm - 1) / (32 * nm));
    kg_val = std::max(nm, std::min(std::max(KKR_KG_MAX, nm), want));
  }
  if (dry_info) {
    dry_info[0] = n_basis * nL;
    dry_info[1] = n_kpts;
    dry_info[2] = n_disp;
    dry_info[3] = n_pts;
    dry_info[4] = int(kK_idx.size());
    dry_info[5] = (n_kpts + kg_val - 1) / kg_val;
    dry_info[6] = n_k * n_k * n_k;
    dry_info[7] = pt_start[1];
    dry_info[8] = n_ops;
    if (dry_eta) *dry_eta = eta;
    return MUST_OK;
  }

  must_kkr* h = new must_kkr();
  std::memset(h, 0, sizeof(*h));
  h->nb = n_basis; h->lmax = lmax; h->nL = nL; h->l2max = l2max; h->nL2 = nL2; h->n = n_basis * nL;
  h->n_k = n_k; h->n_kpts = n_kpts; h->n_mesh = n_k * n_k * n_k; h->n_disp = n_disp; h->n_pts0 = pt_start[1]; h->n_pts = n_pts; h->n_K = n_K;
  h->kg = kg_val;
  h->n_kK = int(kK_idx.size()); h->n_kg = (n_kpts + h->kg - 1) / h->kg; h->n_ops = n_ops;
  h->eta = eta; h->omega = omega;
  cudaGetDevice(&h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  auto up = [&](void** dst, const void* src, size_t bytes) {
    if (e != cudaSuccess) return;
    e = cudaMalloc(dst, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, st);
  };
  up(reinterpret_cast<void**>(&h->d_kpts), kpts.data(), sizeof(double) * kpts.size());
  up(reinterpret_cast<void**>(&h->d_kpair), kpair.data(), sizeof(int) * kpair.size());
  up(reinterpret_cast<void**>(&h->d_kwt), kwt.data(), sizeof(int) * kwt.size());
  up(reinterpret_cast<void**>(&h->d_Dop), Dops.data(), sizeof(double) * Dops.size());
  up(reinterpret_cast<void**>(&h->d_op_src), src_ops.data(), sizeof(int) * src_ops.size());
  up(reinterpret_cast<void**>(&h->d_class), cls.data(), sizeof(int) * cls.size());
  up(reinterpret_cast<void**>(&h->d_K), Kv.data(), sizeof(double) * Kv.size());
  up(reinterpret_cast<void**>(&h->d_kK_start), kK_start.data(), sizeof(int) * kK_start.size());
  up(reinterpret_cast<void**>(&h->d_kK_idx), kK_idx.data(), sizeof(int) * kK_idx.size());
  up(reinterpret_cast<void**>(&h->d_disp), disp.data(), sizeof(double) * disp.size());
  up(reinterpret_cast<void**>(&h->d_pair_disp), pair_disp.data(), sizeof(int) * pair_disp.size());
  up(reinterpret_cast<void**>(&h->d_pt_start), pt_start.data(), sizeof(int) * pt_start.size());
  up(reinterpret_cast<void**>(&h->d_pt_R), pt_R.data(), sizeof(double) * pt_R.size());
  up(reinterpret_cast<void**>(&h->d_pt_rho), pt_rho.data(), sizeof(double) * pt_rho.size());
  up(reinterpret_cast<void**>(&h->d_quad_u), lu.data(), sizeof(double) * lu.size());
  up(reinterpret_cast<void**>(&h->d_quad_w), lw.data(), sizeof(double) * lw.size());
  up(reinterpret_cast<void**>(&h->d_g_start), gs.data(), sizeof(int) * gs.size());
  up(reinterpret_cast<void**>(&h->d_g_L2), gl.data(), sizeof(int) * gl.size());
  up(reinterpret_cast<void**>(&h->d_g_c), gc.data(), sizeof(double) * gc.size());
  if (e == cudaSuccess) {
    double ynorm[KKR_MAX_NL2] = {0.0};
    for (int l = 0; l <= KKR_MAX_L2; ++l)
      for (int m = 0; m <= l; ++m) {
        double ratio = 1.0;
        for (int q = l - m + 1; q <= l + m; ++q) ratio /= double(q);
        ynorm[l * l + l + m] = std::sqrt((2.0 * l + 1.0) / (4.0 * kPi) * ratio) * (m > 0 ? std::sqrt(2.0) : 1.0);
      }
    e = cudaMemcpyToSymbolAsync(c_ynorm, ynorm, sizeof(ynorm), 0, cudaMemcpyHostToDevice, st);
    double rec[KKR_MAX_L2 + 1] = {0.0};
    for (int q = 1; q <= KKR_MAX_L2; ++q) rec[q] = 1.0 / q;
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_recip, rec, sizeof(rec), 0, cudaMemcpyHostToDevice, st);
  }
  {
    // reciprocal-term table, unless asked not to or larger than KKR_TAB_CAP
    const int n_groups = 1 + (n_disp - 1) / 2;
    h->tab_w = nL2 + 2 * (n_groups - 1) + 1;
    const size_t tb = sizeof(double) * size_t(h->n_kK) * size_t(h->tab_w);
    if (e == cudaSuccess && !(flags & MUST_KKR_NO_TABLE) && h->n_kK > 0 && tb <= KKR_TAB_CAP) {
      e = cudaMalloc(reinterpret_cast<void**>(&h->d_tab), tb);
      if (e == cudaErrorMemoryAllocation) {
        // no room for the table: the items form the factors themselves
        cudaGetLastError();
        h->d_tab = nullptr;
        e = cudaSuccess;
      } else if (e == cudaSuccess) {
        h->tab_bytes = tb;
        KkrDev K = dev_view(h);
        K.tab = nullptr;   // the kernel writes the table through its own argument
        kkr_recip_table_kernel<<<h->n_kpts, TAB_THREADS, 0, st>>>(K, h->d_tab);
        e = cudaGetLastError();
      }
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) {
    // dynamic shared memory: raised to this handle's need per device, never
    // lowered (a handle built later must not cut the limit an earlier one uses)
    const size_t need[3] = {recip_smem(h), invert_smem(h), realsum_smem(h)};
    if (need[0] > 227 * 1024 || need[1] > 227 * 1024 || need[2] > 227 * 1024) {
      must_set_error("must_kkr_build: shared memory per CTA exceeded");
      must_kkr_free(h);
      return MUST_EINVAL;
    }
    static std::mutex mu;
    static size_t granted[64][3] = {};
    std::lock_guard<std::mutex> lock(mu);
    const int dv = (h->device >= 0 && h->device < 64) ? h->device : 0;
    const void* fns[3] = {reinterpret_cast<const void*>(kkr_recip_kernel),
                          reinterpret_cast<const void*>(kkr_invert_kernel),
                          reinterpret_cast<const void*>(kkr_realsum_kernel)};
    for (int f = 0; f < 3 && e == cudaSuccess; ++f)
      if (need[f] > granted[dv][f]) {
        e = cudaFuncSetAttribute(fns[f], cudaFuncAttributeMaxDynamicSharedMemorySize, int(need[f]));
        if (e == cudaSuccess) granted[dv][f] = need[f];
      }
  }
  if (e != cudaSuccess) {
    must_set_error("must_kkr_build: %s", cudaGetErrorString(e));
    const must_status s = (e == cudaErrorMemoryAllocation) ? MUST_ENOMEM : MUST_ECUDA;
    must_kkr_free(h);
    return s;
  }
  *out = h;
  return MUST_OK;
}

extern "C" must_status must_kkr_build(const double* lattice, const double* basis, const int32_t* site_class,
                                      int32_t n_basis, int32_t lmax, int32_t n_k, double eta, int32_t flags,
                                      void* stream, must_kkr** out) {
  return kkr_build_impl(lattice, basis, site_class, n_basis, lmax, n_k, eta, flags, stream, out, nullptr, nullptr);
}

extern "C" must_status must_kkr_geometry(const double* lattice, const double* basis, const int32_t* site_class,
                                         int32_t n_basis, int32_t lmax, int32_t n_k, double eta, int32_t flags,
                                         int32_t* info, double* eta_used) {
  if (!info) { must_set_error("must_kkr_geometry: info is NULL"); return MUST_EINVAL; }
  return kkr_build_impl(lattice, basis, site_class, n_basis, lmax, n_k, eta, flags, nullptr, nullptr, info,
                        eta_used);
}

extern "C" void must_kkr_free(must_kkr* h) {
  if (!h) return;
  void* ptrs[] = {h->d_kpts, h->d_kpair, h->d_kwt, h->d_Dop, h->d_op_src, h->d_class, h->d_K, h->d_kK_start, h->d_kK_idx, h->d_disp, h->d_pair_disp, h->d_pt_start,
                  h->d_pt_R, h->d_pt_rho, h->d_quad_u, h->d_quad_w, h->d_g_start, h->d_g_L2, h->d_g_c, h->d_tab};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete h;
}

extern "C" size_t must_kkr_table_bytes(const must_kkr* h) { return h ? h->tab_bytes : 0; }

extern "C" must_status must_kkr_info(const must_kkr* h, int32_t* info) {
  if (!h || !info) { must_set_error("must_kkr_info: NULL argument"); return MUST_EINVAL; }
  info[0] = h->n;
  info[1] = h->n_kpts;
  info[2] = h->n_disp;
  info[3] = h->n_pts;
  info[4] = h->n_kK;
  info[5] = h->n_kg;
  info[6] = h->n_mesh;
  info[7] = h->n_pts0;
  info[8] = h->n_ops;
  return MUST_OK;
}

extern "C" double must_kkr_eta(const must_kkr* h) { return h ? h->eta : 0.0; }

extern "C" size_t must_kkr_workspace_bytes(const must_kkr* h, int32_t n_items) {
  if (!h || n_items < 1) return 0;
  return carve(h, n_items, nullptr).bytes + staging_bytes(h, n_items) + 256;
}

extern "C" must_status must_kkr_tau(const must_kkr* h, int32_t n_items, const double* E, const double* tinv,
                                    void* workspace, size_t workspace_bytes, double* tau, int32_t* status,
                                    void* stream) {
  if (!h || n_items < 0 || (n_items > 0 && (!E || !tinv || !tau || !workspace))) {
    must_set_error("must_kkr_tau: bad argument");
    return MUST_EINVAL;
  }
  if (n_items == 0) return MUST_OK;
  if (n_items > 65535) {   // items are a grid dimension of every launch
    must_set_error("must_kkr_tau: at most 65535 items per call");
    return MUST_EINVAL;
  }
  if (workspace_bytes < must_kkr_workspace_bytes(h, n_items)) {
    must_set_error("must_kkr_tau: workspace too small: need %zu bytes", must_kkr_workspace_bytes(h, n_items));
    return MUST_ENOMEM;
  }
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != h->device) {
    must_set_error("must_kkr_tau: handle built on device %d, current device is %d", h->device, dev);
    return MUST_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(workspace) + 255) & ~uintptr_t(255));
  KkrWs w = carve(h, n_items, base);
  char* stage = base + w.bytes;
  const size_t bE = sizeof(double2) * n_items, bT = sizeof(double2) * size_t(n_items) * h->nb * (h->lmax + 1);
  const size_t bTau = sizeof(double2) * size_t(n_items) * h->nb * h->nL * h->nL, bS = sizeof(int) * n_items;
  const double2* Ed = reinterpret_cast<const double2*>(E);
  const double2* Td = reinterpret_cast<const double2*>(tinv);
  double2* taud = reinterpret_cast<double2*>(tau);
  int* std_ = status;
  const bool hostE = !must_is_device_ptr(E), hostT = !must_is_device_ptr(tinv), hostTau = !must_is_device_ptr(tau);
  const bool hostS = status && !must_is_device_ptr(status);
  cudaError_t e = cudaSuccess;
  if (hostE) {
    e = cudaMemcpyAsync(stage, E, bE, cudaMemcpyHostToDevice, st);
    Ed = reinterpret_cast<const double2*>(stage);
  }
  stage += a256(bE);
  if (e == cudaSuccess && hostT) {
    e = cudaMemcpyAsync(stage, tinv, bT, cudaMemcpyHostToDevice, st);
    Td = reinterpret_cast<const double2*>(stage);
  }
  stage += a256(bT);
  if (hostTau) taud = reinterpret_cast<double2*>(stage);
  stage += a256(bTau);
  if (hostS) std_ = reinterpret_cast<int*>(stage);
  if (e != cudaSuccess) { must_set_error("must_kkr_tau: %s", cudaGetErrorString(e)); return MUST_ECUDA; }

  const KkrDev K = dev_view(h);
  kkr_status_init_kernel<<<(n_items + 255) / 256, 256, 0, st>>>(n_items, w.status);
  prof_launched(PH_OTHER, 1);
  {
    ProfScope ps(PH_KKR_TERMS, st);
    dim3 g0((h->n_pts + 127) / 128, n_items);
    kkr_real_terms_kernel<<<g0, 128, 0, st>>>(K, n_items, Ed, w.T, w.status);
    prof_launched(PH_KKR_TERMS, 1, n_items);
  }
  {
    ProfScope ps(PH_KKR_RECIP, st);
    const int ib = recip_ib(h);
    dim3 g1(h->n_kpts, (n_items + ib - 1) / ib);
    kkr_recip_kernel<<<g1, RECIP_THREADS, recip_smem(h), st>>>(K, n_items, ib, Ed, w.Dk);
    prof_launched(PH_KKR_RECIP, 1, n_items);
  }
  {
    ProfScope ps(PH_KKR_REALSUM, st);
    dim3 g2((h->n_kpts + KKR_KB - 1) / KKR_KB, 1 + (h->n_disp - 1) / 2, n_items);
    kkr_realsum_kernel<<<g2, RSUM_THREADS, realsum_smem(h), st>>>(K, n_items, w.T, w.Dk);
    prof_launched(PH_KKR_REALSUM, 1, n_items);
  }
  {
    ProfScope ps(PH_KKR_INVERT, st);
    dim3 g3(h->n_kg, n_items);
    kkr_invert_kernel<<<g3, INV_THREADS, invert_smem(h), st>>>(K, n_items, Ed, Td, w.Dk, w.part, w.status);
    const int tot = n_items * h->nb * h->nL * h->nL;
    kkr_bz_sum_kernel<<<(tot + 255) / 256, 256, 0, st>>>(K, n_items, w.part, taud, w.S, w.status);
    if (h->n_ops > 0) {
      dim3 g4(h->nb, n_items);
      kkr_symmetrise_kernel<<<g4, SYM_THREADS, 0, st>>>(K, n_items, w.S, Td, taud, w.status);
    }
    prof_launched(PH_KKR_INVERT, h->n_ops > 0 ? 3 : 2, n_items);
  }
  if (std_) {
    kkr_status_out_kernel<<<(n_items + 255) / 256, 256, 0, st>>>(n_items, w.status, std_);
    prof_launched(PH_OTHER, 1);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess && hostTau) e = cudaMemcpyAsync(tau, taud, bTau, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && hostS) e = cudaMemcpyAsync(status, std_, bS, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && (hostTau || hostS)) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { must_set_error("must_kkr_tau: %s", cudaGetErrorString(e)); return MUST_ECUDA; }
  return MUST_OK;
}
