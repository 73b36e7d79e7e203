// KKR matrix assembly on the device (paper Sec. 5: "construct the KKR matrix on
// GPUs"; Eq. (4): M = t^{-1} - g0, g0 between different sites only).
//
//   geom_kernel     once per LIZ: pair distances and real Y_L'' of each pair
//                   direction (R_pq = pos(p) - pos(q), p < q in the permuted
//                   order with the central site last).
//   tinv_kernel     square-well t^{-1}_l(E) fixture (log-derivative matching).
//   scale_kernel    |M_aa|^{-1/2} for the symmetric equilibration of the
//                   low-precision factorisation.
//   assemble_kernel one warp per unordered site pair (or diagonal site) and
//                   energy: Hankel functions h_l''(kappa d), the sparse Gaunt
//                   contraction into a kap x kap block, written for both
//                   pair orders (parity: G^{qp}_{LL'} = (-1)^{l+l'} G^{pq}_{LL'})
//                   and every spin that shares the energy; column-major,
//                   16-byte complex stores, consecutive lanes on consecutive
//                   rows.
#include <algorithm>

#include "common.cuh"
#include "solver.h"
#include "prof.h"

namespace {

__device__ __forceinline__ int l_of(int L) {
  int l = 0;
  while ((l + 1) * (l + 1) <= L) ++l;
  return l;
}

// Real spherical harmonics Y_L(v^), L = l*l+l+m < (lmax+1)^2, no Condon-Shortley
// phase: Y_lm = N_lm P_l^|m|(cos th) {sqrt2 cos m phi | 1 | sqrt2 sin |m| phi}.
__device__ void ylm_real(int lmax, double x, double y, double z, double* out) {
  const double r = sqrt(x * x + y * y + z * z);
  const double rho = sqrt(x * x + y * y);
  const double ct = z / r, st = rho / r;
  double cph = 1.0, sph = 0.0;
  if (rho > 0.0) { cph = x / rho; sph = y / rho; }
  double cm = 1.0, sm = 0.0;   // cos(m phi), sin(m phi)
  double pmm = 1.0;            // P_m^m = (2m-1)!! st^m
  for (int m = 0; m <= lmax; ++m) {
    if (m > 0) {
      const double c2 = cm * cph - sm * sph, s2 = sm * cph + cm * sph;
      cm = c2; sm = s2;
      pmm *= (2.0 * m - 1.0) * st;
    }
    double p_lm2 = 0.0, p_lm1 = pmm;
    for (int l = m; l <= lmax; ++l) {
      double p;
      if (l == m) p = pmm;
      else if (l == m + 1) p = ct * (2.0 * m + 1.0) * pmm;
      else p = ((2.0 * l - 1.0) * ct * p_lm1 - (l + m - 1.0) * p_lm2) / double(l - m);
      if (l > m) { p_lm2 = p_lm1; p_lm1 = p; }
      // N_lm = sqrt((2l+1)/(4pi) (l-m)!/(l+m)!)
      double ratio = 1.0;
      for (int k = l - m + 1; k <= l + m; ++k) ratio /= double(k);
      const double N = sqrt((2.0 * l + 1.0) / (4.0 * 3.14159265358979323846) * ratio);
      if (m == 0) {
        out[l * l + l] = N * p;
      } else {
        out[l * l + l + m] = 1.41421356237309504880 * N * p * cm;
        out[l * l + l - m] = 1.41421356237309504880 * N * p * sm;
      }
    }
  }
}

// h_l(z), l = 0..lmax, outgoing spherical Hankel functions by upward recurrence
// from h_0 = -i e^{iz}/z and h_1 = -e^{iz} (z + i)/z^2.
__device__ void hankel_up(int lmax, cd z, cd* h) {
  const cd e = cexpi(z);
  const cd iz = cinv(z);
  h[0] = mk(e.y, -e.x) * iz;                       // -i e / z
  if (lmax >= 1) h[1] = -(e * (z + mk(0.0, 1.0))) * (iz * iz);
  for (int l = 1; l < lmax; ++l) h[l + 1] = (2.0 * l + 1.0) * (iz * h[l]) - h[l - 1];
}

// j_l(z), l = 0..lmax (lmax >= 1): power series for |z| < 1, else Miller's downward
// recurrence normalised to sin z / z (or to j_1 where j_0 is the smaller).
__device__ void bessel_j(int lmax, cd z, cd* j) {
  const double az = sqrt(cnorm(z));
  if (az < 1.0) {
    const cd q = -0.5 * (z * z);
    cd zl = mk(1.0, 0.0);
    double df = 1.0;
    for (int l = 0; l <= lmax; ++l) {
      if (l > 0) { zl = zl * z; df *= (2.0 * l + 1.0); }
      cd term = mk(1.0, 0.0), sum = mk(1.0, 0.0);
      for (int k = 1; k < 40; ++k) {
        term = (1.0 / (double(k) * (2.0 * l + 2.0 * k + 1.0))) * (term * q);
        sum = sum + term;
        if (cnorm(term) < 1e-36 * cnorm(sum)) break;
      }
      j[l] = (1.0 / df) * (zl * sum);
    }
    return;
  }
  const cd iz = cinv(z);
  const int top = lmax + 24 + int(1.5 * az);
  cd fp1 = mk(0.0, 0.0), f = mk(1e-200, 0.0);
  for (int l = top; l >= 1; --l) {
    const cd fm1 = (2.0 * l + 1.0) * (iz * f) - fp1;
    fp1 = f;
    f = fm1;
    if (cnorm(f) > 1e200) {       // rescale the recurrence and every value kept so far
      const double s = 1e-100;
      f = s * f;
      fp1 = s * fp1;
      for (int m = l; m <= lmax; ++m) j[m] = s * j[m];
    }
    if (l - 1 <= lmax) j[l - 1] = f;
  }
  const cd f0 = j[0], f1 = j[1];
  const cd e = cexpi(z);                                  // e^{iz}
  const cd emi = cinv(e);                                 // e^{-iz}
  const cd sz = mk(0.0, -0.5) * (e - emi);                // sin z = (e^{iz} - e^{-iz}) / (2i)
  const cd cz = 0.5 * (e + emi);
  const cd j0 = sz * iz;
  const cd j1 = (sz * iz - cz) * iz;
  const cd sc = (cnorm(j0) >= cnorm(j1)) ? cdiv(j0, f0) : cdiv(j1, f1);
  for (int l = 0; l <= lmax; ++l) j[l] = sc * j[l];
}

}  // namespace

// ------------------------------------------------------------------------
__global__ void geom_kernel(int N, int nL2, int l2max, const double* __restrict__ pos_perm,
                            const int2* __restrict__ pq, int n_pairs, double* __restrict__ d_out,
                            double* __restrict__ Y_out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_pairs) return;
  const int2 e = pq[t];
  const double x = pos_perm[3 * e.x] - pos_perm[3 * e.y];
  const double y = pos_perm[3 * e.x + 1] - pos_perm[3 * e.y + 1];
  const double z = pos_perm[3 * e.x + 2] - pos_perm[3 * e.y + 2];
  d_out[t] = sqrt(x * x + y * y + z * z);
  double Y[MUST_MAX_NL2];
  ylm_real(l2max, x, y, z, Y);
  for (int L = 0; L < nL2; ++L) Y_out[size_t(t) * nL2 + L] = Y[L];
}

// t^{-1}_l = i k [k h'(ka) j(qa) - q j'(qa) h(ka)] / [k j'(ka) j(qa) - q j'(qa) j(ka)],
// with f_l' = f_{l-1} - (l+1)/z f_l and f_0' = -f_1.
__global__ void tinv_kernel(int nE, const double2* __restrict__ E, int n_pot, const double* __restrict__ V,
                            double a, int lmax, double2* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nE * n_pot) return;
  const int p = t / nE, e = t % nE;
  const cd Ec = mk(E[e].x, E[e].y);
  const cd k = csqrt_p(Ec);
  const cd q = csqrt_p(Ec - mk(V[p], 0.0));
  const cd ka = a * k, qa = a * q;
  cd jk[MUST_MAX_LMAX + 2], hk[MUST_MAX_LMAX + 2], jq[MUST_MAX_LMAX + 2];
  bessel_j(lmax + 1, ka, jk);
  hankel_up(lmax + 1, ka, hk);
  bessel_j(lmax + 1, qa, jq);
  const cd ika = cinv(ka), iqa = cinv(qa);
  for (int l = 0; l <= lmax; ++l) {
    cd djk, dhk, djq;
    if (l == 0) { djk = -jk[1]; dhk = -hk[1]; djq = -jq[1]; }
    else {
      djk = jk[l - 1] - (l + 1.0) * (ika * jk[l]);
      dhk = hk[l - 1] - (l + 1.0) * (ika * hk[l]);
      djq = jq[l - 1] - (l + 1.0) * (iqa * jq[l]);
    }
    const cd num = mk(0.0, 1.0) * k * (k * dhk * jq[l] - q * djq * hk[l]);
    const cd den = k * djk * jq[l] - q * djq * jk[l];
    const cd r = cdiv(num, den);
    out[size_t(p) * nE * (lmax + 1) + size_t(e) * (lmax + 1) + l] = make_double2(r.x, r.y);
  }
}

// ------------------------------------------------------------------------
// Site charge inside the sphere (Eq. 2-3) for the square-well single-site
// problem.  Per energy: int_sphere G(r,r;E) d^3r = sum_L tau_LL F_l - sum_l
// (2l+1) I_l with F_l = int_0^a Z_l^2 r^2 dr, I_l = int_0^a Z_l J_l r^2 dr;
// Z_l = c_l j_l(q r) inside, matched in value to j_l(kappa a)/t_l - i kappa
// h_l(kappa a); J_l = alpha j_l(q r) + beta y_l(q r), matched in value and
// slope to j_l(kappa r).  Radial integrals by the Lommel identity.
namespace {

// j_l, y_l for l = -1 .. lmax + 1 at z (index l + 1)
__device__ void bessel_jy_ext(int lmax, cd z, cd* j, cd* y) {
  cd jj[MUST_MAX_LMAX + 3], hh[MUST_MAX_LMAX + 3];
  bessel_j(lmax + 1, z, jj);
  hankel_up(lmax + 1, z, hh);
  const cd iz = cinv(z);
  const cd e = cexpi(z), emi = cinv(e);
  j[0] = (0.5 * (e + emi)) * iz;                     // j_{-1} = cos z / z
  y[0] = (mk(0.0, -0.5) * (e - emi)) * iz;           // y_{-1} = sin z / z
  for (int l = 0; l <= lmax + 1; ++l) {
    j[l + 1] = jj[l];
    y[l + 1] = mk(0.0, -1.0) * (hh[l] - jj[l]);      // y = (h - j) / i
  }
}

// (x^3/2)[u_l v_l - (u_{l-1} v_{l+1} + u_{l+1} v_{l-1})/2], u, v indexed l + 1
__device__ __forceinline__ cd lommel(int l, cd x, const cd* u, const cd* v) {
  const int k = l + 1;
  return (0.5 * (x * x * x)) * (u[k] * v[k] - 0.5 * (u[k - 1] * v[k + 1] + u[k + 1] * v[k - 1]));
}

// Inside the well (square well of depth V, radius a) at energy E, per l:
// Z_l = c_l j_l(q r) (value matched to j_l/t_l - i kappa h_l at r = a) and
// J_l = alpha_l j_l(q r) + beta_l y_l(q r) (value and slope matched to j_l).
// Also returns j_l(qa), y_l(qa) (indexed l + 1, l = -1 .. lmax + 1) and q.
__device__ void well_coefficients(int lmax, cd E, double V, double a, cd* c, cd* alpha, cd* beta, cd* jq, cd* yq,
                                  cd& q_out) {
  const cd kp = csqrt_p(E), q = csqrt_p(E - mk(V, 0.0));
  const cd ka = a * kp, qa = a * q;
  cd jk[MUST_MAX_LMAX + 3], yk[MUST_MAX_LMAX + 3];
  bessel_jy_ext(lmax, ka, jk, yk);
  bessel_jy_ext(lmax, qa, jq, yq);
  const cd ika = cinv(ka), iqa = cinv(qa);
  for (int l = 0; l <= lmax; ++l) {
    const int k = l + 1;
    const cd hk = jk[k] + mk(0.0, 1.0) * yk[k];
    const cd hkm = jk[k - 1] + mk(0.0, 1.0) * yk[k - 1];
    const cd djk = jk[k - 1] - (l + 1.0) * (ika * jk[k]);
    const cd dhk = hkm - (l + 1.0) * (ika * hk);
    const cd djq = jq[k - 1] - (l + 1.0) * (iqa * jq[k]);
    const cd dyq = yq[k - 1] - (l + 1.0) * (iqa * yq[k]);
    // t_l of the well (log-derivative matching), as in tinv_kernel but inverted
    const cd num = mk(0.0, 1.0) * kp * (kp * dhk * jq[k] - q * djq * hk);
    const cd den = kp * djk * jq[k] - q * djq * jk[k];
    const cd tinv = cdiv(num, den);
    c[l] = cdiv(jk[k] * tinv - mk(0.0, 1.0) * kp * hk, jq[k]);
    const cd det = q * (jq[k] * dyq - yq[k] * djq);
    alpha[l] = cdiv(q * (jk[k] * dyq) - kp * (djk * yq[k]), det);
    beta[l] = cdiv(kp * (djk * jq[k]) - q * (jk[k] * djq), det);
  }
  q_out = q;
}

// sum over m of tau_LL for each l (tau column-major kap x kap)
__device__ __forceinline__ cd tau_diag_l(const double2* tau, int kap, int l) {
  cd dsum = mk(0.0, 0.0);
  for (int m = -l; m <= l; ++m) {
    const int L = l * l + l + m;
    const double2 tv = tau[size_t(L) * kap + L];
    dsum = dsum + mk(tv.x, tv.y);
  }
  return dsum;
}

__device__ cd site_integrand(int lmax, cd E, double V, double a, const double2* tau, int kap) {
  cd c[MUST_MAX_LMAX + 1], al[MUST_MAX_LMAX + 1], be[MUST_MAX_LMAX + 1];
  cd jq[MUST_MAX_LMAX + 3], yq[MUST_MAX_LMAX + 3], q;
  well_coefficients(lmax, E, V, a, c, al, be, jq, yq, q);
  const cd qa = a * q, iq3 = cinv(q * q * q);
  cd g = mk(0.0, 0.0);
  for (int l = 0; l <= lmax; ++l) {
    const cd ljj = iq3 * lommel(l, qa, jq, jq);
    const cd ljy = iq3 * (lommel(l, qa, jq, yq) - mk((2.0 * l + 1.0) / 4.0, 0.0));
    const cd F = c[l] * c[l] * ljj;
    const cd I = c[l] * (al[l] * ljj + be[l] * ljy);
    g = g + tau_diag_l(tau, kap, l) * F - (2.0 * l + 1.0) * I;
  }
  return g;
}

}  // namespace

__global__ void site_charge_kernel(int lmax, int nE, const double2* __restrict__ E, const double2* __restrict__ w,
                                   const double* __restrict__ V, double a, const double2* __restrict__ tau, int kap,
                                   double* __restrict__ nE_out, double* __restrict__ N_out) {
  __shared__ double red[32];
  const int s = blockIdx.x;
  double acc = 0.0;
  for (int k = threadIdx.x; k < nE; k += blockDim.x) {
    const cd g = site_integrand(lmax, mk(E[k].x, E[k].y), V[s], a, tau + (size_t(s) * nE + k) * kap * kap, kap);
    if (nE_out) nE_out[size_t(s) * nE + k] = -g.y / 3.14159265358979323846;
    acc += (mk(w[k].x, w[k].y) * g).y;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) t += red[i];
    N_out[s] = -t / 3.14159265358979323846;
  }
}

void launch_site_charge(int lmax, int nE, const double2* E, const double2* w, int n_out, const double* V, double a,
                        const double2* tau, int kap, double* nE_out, double* N_out, cudaStream_t st) {
  site_charge_kernel<<<n_out, 128, 0, st>>>(lmax, nE, E, w, V, a, tau, kap, nE_out, N_out);
  prof_launched(PH_OTHER, 1);
}

// Radial density inside the sphere: one thread per (radius, output block),
// the contour sum over energies in order:
//   n(r) = -(1/pi) Im sum_k w_k (1/4pi) [sum_L tau_LL Z_l(r)^2 - sum_l (2l+1) Z_l(r) J_l(r)].
// Radii outside (0, a] give NaN.
__global__ void site_density_kernel(int lmax, int nE, const double2* __restrict__ E, const double2* __restrict__ w,
                                    const double* __restrict__ V, double a, const double2* __restrict__ tau, int kap,
                                    int n_r, const double* __restrict__ r, double* __restrict__ out) {
  const int s = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_r) return;
  const double ri = r[i];
  if (!(ri > 0.0 && ri <= a)) {
    out[size_t(s) * n_r + i] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  double acc = 0.0;
  for (int k = 0; k < nE; ++k) {
    cd c[MUST_MAX_LMAX + 1], al[MUST_MAX_LMAX + 1], be[MUST_MAX_LMAX + 1];
    cd jq[MUST_MAX_LMAX + 3], yq[MUST_MAX_LMAX + 3], q;
    well_coefficients(lmax, mk(E[k].x, E[k].y), V[s], a, c, al, be, jq, yq, q);
    cd jr[MUST_MAX_LMAX + 3], yr[MUST_MAX_LMAX + 3];
    bessel_jy_ext(lmax, ri * q, jr, yr);
    const double2* tk = tau + (size_t(s) * nE + k) * kap * kap;
    cd g = mk(0.0, 0.0);
    for (int l = 0; l <= lmax; ++l) {
      const cd Z = c[l] * jr[l + 1];
      const cd J = al[l] * jr[l + 1] + be[l] * yr[l + 1];
      g = g + tau_diag_l(tk, kap, l) * (Z * Z) - (2.0 * l + 1.0) * (Z * J);
    }
    acc += (mk(w[k].x, w[k].y) * g).y;
  }
  out[size_t(s) * n_r + i] = -acc / (4.0 * 3.14159265358979323846 * 3.14159265358979323846);
}

void launch_site_density(int lmax, int nE, const double2* E, const double2* w, int n_out, const double* V, double a,
                         const double2* tau, int kap, int n_r, const double* r, double* out, cudaStream_t st) {
  site_density_kernel<<<dim3((n_r + 63) / 64, n_out), 64, 0, st>>>(lmax, nE, E, w, V, a, tau, kap, n_r, r, out);
  prof_launched(PH_OTHER, 1);
}

// ------------------------------------------------------------------------
struct LizDev {
  int N, n_pairs, pad;
  const int* species;     // [N] permuted
  const double* dirs;     // [N][3] permuted (canted)
  const int2* pair_pq;
  const double* pair_d;
  const double* pair_Y;
};

struct AsmArgs {
  int nL, nL2, lmax, kap, n, canted, n_lz;
  LizDev L[MUST_CHUNK_LIZ];
  const int* g_start;
  const int* g_L2;
  const double* g_c;
  int g_nnz;
  int e0, nEc, nE, nspin, n_species;
  const double2* E;       // [nE]
  const double2* tinv;    // [nspin][n_species][nE][lmax+1]
  double2* M64;           // item matrices (may be NULL)
  float2* M32;            // equilibrated FP32 copies (may be NULL)
  int ld;
  size_t stride;          // elements between items (both copies)
  const double* scale;    // [item][n] (required when M32 != NULL or scale64)
  const float* scale32;   // [item][n] FP32 copy of scale (mixed path)
  int items_per_e;        // nspin (collinear) or 1 (canted)
  int scale64;            // 1: the FP64 copy is equilibrated too (D M D)
  int m64_df;             // 1: the M64 buffer holds M as FP32 pairs (hi.re, hi.im, lo.re, lo.im)
  int* rowmax;            // NULL or [item][n]: atomic max of the float bits of max(|hi.re|, |hi.im|) over
                          // the off-diagonal entries of each row (needs the double-float split)
};

// M_aa of item `it` at row a (for the equilibration scale); 1 on padding sites.
__device__ __forceinline__ cd diag_entry(const AsmArgs& A, int it, int a) {
  const int el = it % A.nEc;
  const int grp = it / A.nEc;               // lz * items_per_e + spin
  const int lz = grp / A.items_per_e, s = A.canted ? 0 : grp % A.items_per_e;
  const LizDev& Lz = A.L[lz];
  const int e = A.e0 + el;
  const int p = a / A.kap - Lz.pad, w = a % A.kap;
  if (p < 0) return mk(1.0, 0.0);
  const int sp = Lz.species[p];
  if (!A.canted) {
    const int l = l_of(w);
    const double2 v = A.tinv[((size_t(s) * A.n_species + sp) * A.nE + e) * (A.lmax + 1) + l];
    return mk(v.x, v.y);
  }
  const int sg = w / A.nL, l = l_of(w % A.nL);
  const double2 u = A.tinv[((size_t(0) * A.n_species + sp) * A.nE + e) * (A.lmax + 1) + l];
  const double2 d = A.tinv[((size_t(1) * A.n_species + sp) * A.nE + e) * (A.lmax + 1) + l];
  const double ez = Lz.dirs[3 * p + 2];
  const cd av = mk(u.x, u.y), bv = mk(d.x, d.y);
  return 0.5 * (av + bv) + (sg == 0 ? 0.5 * ez : -0.5 * ez) * (av - bv);
}

__global__ void scale_kernel(AsmArgs A, double* __restrict__ scale, float* __restrict__ scale32) {
  const int it = blockIdx.y;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < A.n; a += gridDim.x * blockDim.x) {
    const double m = sqrt(sqrt(cnorm(diag_entry(A, it, a))));
    const double sc = (m > 0.0 && isfinite(m)) ? 1.0 / m : 1.0;
    scale[size_t(it) * A.n + a] = sc;
    if (scale32) scale32[size_t(it) * A.n + a] = float(sc);
  }
}

// v -> (hi, lo) with hi + lo carrying 24 + 24 significant bits, built from the
// bit fields of the double with integer operations (hi: v truncated to a
// float's significand; lo: the remaining 29 bits, rounded to a float), so
// the split costs no FP64-pipe conversions.  Values outside the normal float
// range fall back to the conversion instructions.
// Out-of-range values (rare): the conversion instructions.  Kept out of line
// so that the common path of split_df carries no FP64 instructions.
__device__ __noinline__ float2 split_df_slow(double v) {
  const float hi = float(v);
  return make_float2(hi, float(v - double(hi)));
}

__device__ __forceinline__ void split_df(double v, float& hi, float& lo) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  const int e = int((b >> 52) & 0x7FF);
  if (e >= 949 && e <= 1150) {
    const unsigned sign = unsigned(b >> 63) << 31;
    hi = __uint_as_float(sign | (unsigned(e - 896) << 23) | unsigned((b >> 29) & 0x7FFFFF));
    const float m = __uint2float_rn(unsigned(b & 0x1FFFFFFFull));            // low 29 bits
    const float p2 = __uint_as_float(unsigned(e - 948) << 23);                // 2^(e - 1075)
    lo = __uint_as_float(__float_as_uint(m * p2) | sign);
  } else if (e < 949) {   // |v| < 2^-74: negligible next to any row of M
    hi = __uint_as_float(unsigned(b >> 63) << 31);
    lo = 0.f;
  } else {
    const float2 r = split_df_slow(v);
    hi = r.x;
    lo = r.y;
  }
}

// (re_hi, im_hi, re_lo, im_lo) of v.
__device__ __forceinline__ float4 split_cd(cd v) {
  float hr, lr, hi, li;
  split_df(v.x, hr, lr);
  split_df(v.y, hi, li);
  return make_float4(hr, hi, lr, li);
}

__device__ __forceinline__ bool need_df(const AsmArgs& A) { return A.M32 || (A.M64 && A.m64_df); }

// Double-float arithmetic (value = hi + lo, |lo| <= ulp(hi) / 2) for the
// Gaunt contraction of the mixed path, whose M is kept as a double-float copy
// and whose residual resolves M to ~2^-48 of each row scale anyway: the FP32
// pipes carry it at several times the rate of the FP64 pipe.
// acc += c * w with c, w double-floats: the product by Dekker's method with
// FMA (Dekker, Numer. Math. 18, 1971), the sum by Knuth's two-sum, then the
// result renormalised.
__device__ __forceinline__ void df_mac(float& ah, float& al, float ch, float cl, float wh, float wl) {
  const float ph = ch * wh;
  const float pl = fmaf(ch, wl, fmaf(cl, wh, fmaf(ch, wh, -ph)));
  const float sh = ah + ph;
  const float v = sh - ah;
  const float e = ((ah - (sh - v)) + (ph - v)) + (al + pl);
  ah = sh + e;
  al = e - (ah - sh);
}

// Store entry (row, col) of item it: v in FP64 and, when a FP32 copy or the
// double-float M is kept, its split f = split_cd(v).
__device__ __forceinline__ void store_elem(const AsmArgs& A, int it, int row, int col, cd v, float4 f) {
  const size_t off = size_t(it) * A.stride + size_t(col) * A.ld + row;
  if (A.M64 && A.M32 && !A.m64_df) A.M64[off] = make_double2(v.x, v.y);   // FP64 residual copy
  if (need_df(A)) {
    if (A.M64 && A.m64_df) reinterpret_cast<float4*>(A.M64)[off] = f;
    if (A.M32) {
      const float s = A.scale32[size_t(it) * A.n + row] * A.scale32[size_t(it) * A.n + col];
      A.M32[off] = make_float2(f.x * s + f.z * s, f.y * s + f.w * s);
    }
    return;
  }
  if (A.M64) {
    if (A.scale64) {
      const double s = A.scale[size_t(it) * A.n + row] * A.scale[size_t(it) * A.n + col];
      A.M64[off] = make_double2(s * v.x, s * v.y);
    } else {
      A.M64[off] = make_double2(v.x, v.y);
    }
  }
}

__device__ __forceinline__ void store_elem(const AsmArgs& A, int it, int row, int col, cd v) {
  store_elem(A, it, row, col, v, need_df(A) ? split_cd(v) : make_float4(0.f, 0.f, 0.f, 0.f));
}

// Grid (blocks, energy, LIZ of the chunk).  The first blocks of a LIZ take
// PAIRS_PER_BLOCK site pairs p < q each: one thread per pair evaluates the
// Hankel functions (FP64 exp/sincos/division: computed once per pair, not by
// every lane), then each warp contracts the Gaunt table for its pairs.  The
// remaining blocks give one warp to each diagonal site and each padding site
// (identity block; their off-diagonal blocks are zero-filled before the
// launch).
constexpr int PAIRS_PER_BLOCK = 64;

// Byte offset of the float-pair copy of the Gaunt coefficients in the pair
// blocks' dynamic shared memory (after the FP64 coefficients, the L''
// indices and the row starts), rounded up to 8 bytes.
__host__ __device__ inline size_t gaunt_cf_offset(int g_nnz, int nL) {
  return (size_t(g_nnz) * 12 + size_t(nL * nL + 1) * 4 + 7) & ~size_t(7);
}

__host__ __device__ inline int asm_pair_blocks(int n_pairs) { return (n_pairs + PAIRS_PER_BLOCK - 1) / PAIRS_PER_BLOCK; }

__device__ __forceinline__ int absmax_bits(float4 f) { return __float_as_int(fmaxf(fabsf(f.x), fabsf(f.y))); }

__global__ void __launch_bounds__(256) assemble_kernel(AsmArgs A) {
  __shared__ cd wsh[8][MUST_MAX_NL2];
  __shared__ cd hsh[PAIRS_PER_BLOCK][2 * MUST_MAX_LMAX + 1];
  __shared__ int rmx[8][MUST_MAX_NL];   // per warp: row maxima of the current pair block (float bits)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int el = blockIdx.y;
  const int lz = blockIdx.z;
  const LizDev& Lz = A.L[lz];
  const int e = A.e0 + el;
  const cd Ec = mk(A.E[e].x, A.E[e].y);
  const int nL = A.nL, kap = A.kap, off = Lz.pad;
  auto item_of = [&](int ii) { return (lz * A.items_per_e + ii) * A.nEc + el; };
  const int pb = asm_pair_blocks(Lz.n_pairs);
  if (int(blockIdx.x) < pb) {
    const int u0 = blockIdx.x * PAIRS_PER_BLOCK;
    const int np = min(PAIRS_PER_BLOCK, Lz.n_pairs - u0);
    const int l2max = 2 * A.lmax;
    // the Gaunt table in shared memory: [g_nnz] coefficients, [g_nnz] L'', [nL^2 + 1] row starts, and
    // (double-float contraction) the coefficients as (hi, lo) float pairs
    extern __shared__ double gsm[];
    double* gs_c = gsm;
    int* gs_L2 = reinterpret_cast<int*>(gs_c + A.g_nnz);
    int* gs_start = gs_L2 + A.g_nnz;
    float2* gs_cf = reinterpret_cast<float2*>(reinterpret_cast<char*>(gsm) + gaunt_cf_offset(A.g_nnz, nL));
    const bool dfc = A.M32 && A.M64 && A.m64_df;   // mixed path with the double-float M
    for (int i = threadIdx.x; i < A.g_nnz; i += blockDim.x) {
      gs_c[i] = A.g_c[i];
      gs_L2[i] = A.g_L2[i];
      if (dfc) {
        const float h = float(A.g_c[i]);
        gs_cf[i] = make_float2(h, float(A.g_c[i] - double(h)));
      }
    }
    for (int i = threadIdx.x; i <= nL * nL; i += blockDim.x) gs_start[i] = A.g_start[i];
    if (int(threadIdx.x) < np) {
      // 4 pi i kappa h_l''(kappa d), so that the block entry -G = sum c Y w
      const cd k = csqrt_p(Ec);
      const double d = Lz.pair_d[u0 + threadIdx.x];
      cd h[2 * MUST_MAX_LMAX + 1];
      hankel_up(l2max, d * k, h);
      const cd f = mk(0.0, 4.0 * 3.14159265358979323846) * k;
      for (int l = 0; l <= l2max; ++l) hsh[threadIdx.x][l] = f * h[l];
    }
    __syncthreads();
    for (int pi = warp; pi < np; pi += 8) {
      const int unit = u0 + pi;
      const int2 pq = Lz.pair_pq[unit];
      for (int L2 = lane; L2 < A.nL2; L2 += 32) {
        const double y = Lz.pair_Y[size_t(unit) * A.nL2 + L2];
        const cd w = y * hsh[pi][l_of(L2)];
        if (dfc)   // (re hi, im hi, re lo, im lo) in the same 16 bytes
          reinterpret_cast<float4*>(&wsh[warp][0])[L2] = split_cd(w);
        else
          wsh[warp][L2] = w;
      }
      if (lane < nL) rmx[warp][lane] = 0;
      __syncwarp();
      const int p = pq.x + off, q = pq.y + off;
      for (int ent = lane; ent < nL * nL; ent += 32) {
        const int L = ent % nL, Lp = ent / nL;
        cd v = mk(0.0, 0.0);
        const int b = gs_start[L * nL + Lp], t = gs_start[L * nL + Lp + 1];
        float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
        if (dfc) {
          const float4* wf = reinterpret_cast<const float4*>(&wsh[warp][0]);
          for (int i = b; i < t; ++i) {
            const float2 c = gs_cf[i];
            const float4 w = wf[gs_L2[i]];
            df_mac(f.x, f.z, c.x, c.y, w.x, w.z);
            df_mac(f.y, f.w, c.x, c.y, w.y, w.w);
          }
          // (v, the FP64 value, is stored only without the double-float copy)
        } else {
          for (int i = b; i < t; ++i) {
            const double c = gs_c[i];
            const cd w = wsh[warp][gs_L2[i]];
            v.x = fma(c, w.x, v.x);
            v.y = fma(c, w.y, v.y);
          }
          if (need_df(A)) f = split_cd(v);
        }
        // the transposed block by parity: G^{qp}_{LL'} = (-1)^{l+l'} G^{pq}_{LL'} (exact sign flips)
        const bool odd = (l_of(L) + l_of(Lp)) & 1;
        const cd vt = odd ? -v : v;
        const float4 ft = odd ? make_float4(-f.x, -f.y, -f.z, -f.w) : f;
        if (A.rowmax) atomicMax(&rmx[warp][L], absmax_bits(f));
        const cd z0 = mk(0.0, 0.0);
        const float4 f0 = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int ii = 0; ii < A.items_per_e; ++ii) {
          const int it = item_of(ii);
          if (!A.canted) {
            store_elem(A, it, p * kap + L, q * kap + Lp, v, f);
            store_elem(A, it, q * kap + L, p * kap + Lp, vt, ft);
          } else {
            for (int s = 0; s < 2; ++s) {
              store_elem(A, it, p * kap + s * nL + L, q * kap + s * nL + Lp, v, f);
              store_elem(A, it, p * kap + s * nL + L, q * kap + (1 - s) * nL + Lp, z0, f0);
              store_elem(A, it, q * kap + s * nL + L, p * kap + s * nL + Lp, vt, ft);
              store_elem(A, it, q * kap + s * nL + L, p * kap + (1 - s) * nL + Lp, z0, f0);
            }
          }
        }
      }
      __syncwarp();
      if (A.rowmax && lane < nL) {
        // row L of block (p, q) and row L of its transpose (q, p) have the same entries up to sign
        const int m = rmx[warp][lane];
        if (m > 0)
          for (int ii = 0; ii < A.items_per_e; ++ii) {
            int* rm = A.rowmax + size_t(item_of(ii)) * A.n;
            for (int s = 0; s < (A.canted ? 2 : 1); ++s) {
              atomicMax(rm + p * kap + s * nL + lane, m);
              atomicMax(rm + q * kap + s * nL + lane, m);
            }
          }
      }
      __syncwarp();
    }
    return;
  }
  const int unit = Lz.n_pairs + (int(blockIdx.x) - pb) * 8 + warp;
  if (unit >= Lz.n_pairs + Lz.N + Lz.pad) return;
  if (unit < Lz.n_pairs + Lz.N) {
    const int ps = unit - Lz.n_pairs;      // site in the LIZ's permuted order
    const int p = ps + off;                // block in the chunk matrix
    const int sp = Lz.species[ps];
    for (int ii = 0; ii < A.items_per_e; ++ii) {
      const int it = item_of(ii);
      for (int ent = lane; ent < kap * kap; ent += 32) {
        const int a = ent % kap, b = ent / kap;
        cd v = mk(0.0, 0.0);
        if (!A.canted) {
          if (a == b) {
            const double2 t = A.tinv[((size_t(ii) * A.n_species + sp) * A.nE + e) * (A.lmax + 1) + l_of(a)];
            v = mk(t.x, t.y);
          }
        } else {
          const int sa = a / nL, La = a % nL, sb = b / nL, Lb = b % nL;
          if (La == Lb) {
            const int l = l_of(La);
            const double2 u = A.tinv[((size_t(0) * A.n_species + sp) * A.nE + e) * (A.lmax + 1) + l];
            const double2 dn = A.tinv[((size_t(1) * A.n_species + sp) * A.nE + e) * (A.lmax + 1) + l];
            const cd av = mk(u.x, u.y), bv = mk(dn.x, dn.y);
            const cd hs = 0.5 * (av + bv), hd = 0.5 * (av - bv);
            const double ex = Lz.dirs[3 * ps], ey = Lz.dirs[3 * ps + 1], ez = Lz.dirs[3 * ps + 2];
            // sigma.e = [[ez, ex - i ey], [ex + i ey, -ez]]
            cd sig;
            if (sa == 0 && sb == 0) sig = mk(ez, 0.0);
            else if (sa == 0 && sb == 1) sig = mk(ex, -ey);
            else if (sa == 1 && sb == 0) sig = mk(ex, ey);
            else sig = mk(-ez, 0.0);
            v = hd * sig;
            if (sa == sb) v = v + hs;
          }
        }
        if (A.rowmax && a != b && A.canted) {   // spin-coupling entries of the site block
          const int m = absmax_bits(split_cd(v));
          if (m > 0) atomicMax(A.rowmax + size_t(it) * A.n + p * kap + a, m);
        }
        store_elem(A, it, p * kap + a, p * kap + b, v);
      }
    }
  } else {
    const int p = unit - Lz.n_pairs - Lz.N;   // padding site: identity block
    for (int ii = 0; ii < A.items_per_e; ++ii) {
      const int it = item_of(ii);
      for (int ent = lane; ent < kap * kap; ent += 32) {
        const int a = ent % kap, b = ent / kap;
        store_elem(A, it, p * kap + a, p * kap + b, mk(a == b ? 1.0 : 0.0, 0.0));
      }
    }
  }
}

// ------------------------------------------------------------------------
// Host launchers
void launch_geom(int N, int lmax, const double* pos_perm, const int2* pq, int n_pairs, double* d, double* Y,
                 cudaStream_t st) {
  const int l2max = 2 * lmax, nL2 = (l2max + 1) * (l2max + 1);
  if (n_pairs > 0) {
    geom_kernel<<<(n_pairs + 127) / 128, 128, 0, st>>>(N, nL2, l2max, pos_perm, pq, n_pairs, d, Y);
    prof_launched(PH_OTHER, 1);
  }
}

void launch_tinv(int nE, const double2* E, int n_pot, const double* V, double a, int lmax, double2* out,
                 cudaStream_t st) {
  const int t = nE * n_pot;
  if (t > 0) {
    tinv_kernel<<<(t + 127) / 128, 128, 0, st>>>(nE, E, n_pot, V, a, lmax, out);
    prof_launched(PH_OTHER, 1);
  }
}

void launch_assemble(const AsmArgs& A, int max_units, cudaStream_t st) {
  ProfScope ps(PH_ASSEMBLE, st);
  const int n_items = A.items_per_e * A.nEc * A.n_lz;
  if (A.M32 || A.scale64) {
    dim3 g((A.n + 255) / 256, n_items);
    scale_kernel<<<g, 256, 0, st>>>(A, const_cast<double*>(A.scale), const_cast<float*>(A.scale32));
    prof_launched(PH_ASSEMBLE, 1);
  }
  dim3 grid((max_units + 7) / 8, A.nEc, A.n_lz);
  const size_t smem = gaunt_cf_offset(A.g_nnz, A.nL) + size_t(A.g_nnz) * 8;
  // the Gaunt table of lmax = 4 (29 KB) plus the static buffers pass the
  // 48 KB that a launch gets without opting in
  static size_t smem_set = 0;
  if (smem > smem_set) {
    cudaFuncSetAttribute(assemble_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    smem_set = smem;
  }
  assemble_kernel<<<grid, 256, smem, st>>>(A);
  prof_launched(PH_ASSEMBLE, 1, n_items);
}

void launch_assemble_chunk(const AsmChunk& c, cudaStream_t st) {
  const must_liz* z0 = c.lz[0];
  AsmArgs A;
  A.nL = z0->nL; A.nL2 = z0->nL2; A.lmax = z0->lmax; A.kap = z0->kap; A.n = c.n; A.canted = z0->canted;
  A.n_lz = c.n_lz;
  int max_units = 0, any_pad = 0;
  for (int j = 0; j < c.n_lz; ++j) {
    const must_liz* z = c.lz[j];
    LizDev& d = A.L[j];
    d.N = z->N; d.n_pairs = z->n_pairs; d.pad = c.pad[j];
    d.species = z->d_species_perm; d.dirs = z->d_dirs_perm; d.pair_pq = z->d_pair_pq; d.pair_d = z->d_pair_d;
    d.pair_Y = z->d_pair_Y;
    max_units = std::max(max_units, asm_pair_blocks(d.n_pairs) * 8 + d.N + d.pad);
    any_pad |= (d.pad > 0);
  }
  A.g_nnz = z0->g_nnz;
  A.g_start = z0->d_g_start; A.g_L2 = z0->d_g_L2; A.g_c = z0->d_g_c;
  A.e0 = c.e0; A.nEc = c.nEc; A.nE = c.nE; A.nspin = c.nspin; A.n_species = c.n_species;
  A.E = c.E; A.tinv = c.tinv; A.M64 = c.M64; A.M32 = c.M32; A.ld = c.ld; A.stride = c.stride; A.scale = c.scale;
  A.scale32 = c.scale32;
  A.items_per_e = z0->canted ? 1 : c.nspin;
  A.scale64 = c.scale64;
  A.m64_df = c.m64_df;
  A.rowmax = (c.rowmax && (c.M32 || c.m64_df)) ? c.rowmax : nullptr;
  if (any_pad) {   // padding sites: zero their coupling blocks first
    const size_t items = size_t(A.items_per_e) * c.nEc * c.n_lz;
    if (c.M64) cudaMemsetAsync(c.M64, 0, items * c.stride * 16, st);
    if (c.M32) cudaMemsetAsync(c.M32, 0, items * c.stride * 8, st);
  }
  launch_assemble(A, max_units, st);
}
