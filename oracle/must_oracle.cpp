// CPU oracle for the LSMS tau_00 hot path.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
// reference against which the CUDA library is checked.  Only the tests, the
// smoke check and the benchmark's CPU-baseline / reference arm may load it.
// It shares no code, header, table or constant generator with the CUDA path.
//
// Everything is complex double (the paper's element type, Sec. 4.1), written
// as textbook loops with std::complex<double>; no BLAS, no blocking.
//
// Paper: "High Performance GPU Accelerated MuST Software" (arXiv 2308.16317).
//   Eq. (4)  tau(E) = [t^{-1}(E) - g0(E)]^{-1},  M = t^{-1} - g0, where g0 is
//            the free propagator between two *different* sites (Sec. 2.1).
//   Sec. 2.1 rank of M is N (lmax+1)^2, or 2 N (lmax+1)^2 with spin canting.
//   Sec. 2.2 LSMS: M is built over the local interaction zone (LIZ) of each
//            atom, and only the first (central) diagonal block of M^{-1} is
//            needed.
//   Sec. 3.2 the inverse is obtained by LU factorisation followed by a solve.
//
// The paper prints no formula for g0 or t; the readings used here are the
// standard Rydberg-unit KKR ones (hbar = 1, 2m = 1, E = kappa^2):
//   g0(x,x') = -exp(i kappa |x-x'|) / (4 pi |x-x'|)
//   G^{ij}_{LL'} = -4 pi i kappa sum_L'' i^{l-l'+l''} C(L,L',L'')
//                   h_l''(kappa |R_ij|) Y_L''(R_ij^),   R_ij = R_i - R_j
//   square-well single-site t_l from log-derivative matching at r = a.
// Each function below states which of these it implements.

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef std::complex<double> cplx;
static const double kPi = 3.14159265358979323846264338327950288;

// --------------------------------------------------------------------------
// Spherical Bessel functions of complex argument (Abramowitz & Stegun 10.1).
// j_l: power series for small |z|, else Miller's downward recurrence
//      normalised to the closed form j0 = sin z / z (or j1 near zeros of j0).
// y_l: upward recurrence from y0 = -cos z / z, y1 = -cos z / z^2 - sin z / z.
// h_l = j_l + i y_l  (outgoing spherical Hankel function, h0 = -i e^{iz}/z),
//      evaluated from its finite closed form (sph_h below).
// --------------------------------------------------------------------------
static void sph_j(int lmax, cplx z, cplx* j) {
  const double az = std::abs(z);
  if (az < 0.5) {
    // j_l(z) = z^l / (2l+1)!! * sum_k (-z^2/2)^k / (k! prod_{i=1..k} (2l+2i+1))
    cplx zl = 1.0;
    double dfact = 1.0;  // (2l+1)!!
    for (int l = 0; l <= lmax; ++l) {
      if (l > 0) { zl *= z; dfact *= (2.0 * l + 1.0); }
      cplx term = 1.0, sum = 1.0;
      const cplx mz2 = -0.5 * z * z;
      for (int k = 1; k < 60; ++k) {
        term *= mz2 / (double(k) * (2.0 * l + 2.0 * k + 1.0));
        sum += term;
        if (std::abs(term) < 1e-18 * std::abs(sum)) break;
      }
      j[l] = zl / dfact * sum;
    }
    return;
  }
  const int lstart = lmax + 40 + int(2.0 * az);
  std::vector<cplx> f(lstart + 2, cplx(0.0));
  f[lstart + 1] = 0.0;
  f[lstart] = 1e-30;
  for (int l = lstart; l >= 1; --l) {
    f[l - 1] = (2.0 * l + 1.0) / z * f[l] - f[l + 1];
    if (std::abs(f[l - 1]) > 1e200) {  // rescale to avoid overflow
      for (int m = l - 1; m <= lstart + 1; ++m) f[m] *= 1e-200;
    }
  }
  const cplx j0 = std::sin(z) / z;
  const cplx j1 = std::sin(z) / (z * z) - std::cos(z) / z;
  const cplx scale = (std::abs(j0) >= std::abs(j1)) ? j0 / f[0] : j1 / f[1];
  for (int l = 0; l <= lmax; ++l) j[l] = f[l] * scale;
}

static void sph_y(int lmax, cplx z, cplx* y) {
  y[0] = -std::cos(z) / z;
  if (lmax >= 1) y[1] = -std::cos(z) / (z * z) - std::sin(z) / z;
  for (int l = 1; l < lmax; ++l) y[l + 1] = (2.0 * l + 1.0) / z * y[l] - y[l - 1];
}

// h_l(z) = j_l + i y_l.  For Im z > 1, j_l and y_l grow like e^{Im z} while
// h_l decays like e^{-Im z}, so their sum cancels; there h_l is taken from its
// finite closed form (A&S 10.1.16)
//   h_l(z) = (-i)^{l+1} (e^{iz}/z) sum_{k=0..l} i^k (l+k)! / (k! (l-k)! (2z)^k).
// For Im z <= 1 the sum j_l + i y_l is used (the closed form would lose the
// small real part j_l near the real axis at small |z|).
static void sph_h(int lmax, cplx z, cplx* h) {
  if (z.imag() <= 1.0) {
    std::vector<cplx> j(lmax + 1), y(lmax + 1);
    sph_j(lmax, z, j.data());
    sph_y(lmax, z, y.data());
    for (int l = 0; l <= lmax; ++l) h[l] = j[l] + cplx(0, 1) * y[l];
    return;
  }
  const cplx ez = std::exp(cplx(0, 1) * z) / z;
  for (int l = 0; l <= lmax; ++l) {
    cplx sum = 0.0, ik = 1.0, tz = 1.0;
    for (int k = 0; k <= l; ++k) {
      if (k > 0) { ik *= cplx(0, 1); tz *= 2.0 * z; }
      double c = 1.0;   // (l+k)! / (k! (l-k)!)
      for (int q = l - k + 1; q <= l + k; ++q) c *= q;
      for (int q = 2; q <= k; ++q) c /= q;
      sum += ik * c / tz;
    }
    cplx ph = 1.0;
    for (int q = 0; q <= l; ++q) ph *= cplx(0, -1);
    h[l] = ph * ez * sum;
  }
}

// f_l'(z) = f_{l-1}(z) - (l+1)/z f_l(z);  f_0' = -f_1.  f must hold lmax+2 values.
static cplx sph_deriv(int l, cplx z, const cplx* f) {
  if (l == 0) return -f[1];
  return f[l - 1] - (l + 1.0) / z * f[l];
}

// --------------------------------------------------------------------------
// Real spherical harmonics, index L = l*l + l + m.
//   Y_lm = N_lm P_l^|m|(cos th) * { sqrt2 cos(m phi), m>0 ; 1, m=0 ;
//                                   sqrt2 sin(|m| phi), m<0 }
//   N_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!), P_l^m without the
//   Condon-Shortley phase, so Y_1,-1 ~ y, Y_1,0 ~ z, Y_1,1 ~ x.
// --------------------------------------------------------------------------
static double factorial(int n) { double f = 1.0; for (int i = 2; i <= n; ++i) f *= i; return f; }

static void real_ylm(int lmax, double x, double y, double z, double* out) {
  const double r = std::sqrt(x * x + y * y + z * z);
  const double rho = std::sqrt(x * x + y * y);
  const double ct = z / r, st = rho / r;
  const double phi = (rho > 0.0) ? std::atan2(y, x) : 0.0;
  for (int m = 0; m <= lmax; ++m) {
    // associated Legendre P_l^m(ct), l = m..lmax, upward in l
    std::vector<double> P(lmax + 1, 0.0);
    double pmm = 1.0;
    for (int i = 1; i <= m; ++i) pmm *= (2.0 * i - 1.0) * st;
    P[m] = pmm;
    if (m + 1 <= lmax) P[m + 1] = ct * (2.0 * m + 1.0) * pmm;
    for (int l = m + 2; l <= lmax; ++l)
      P[l] = ((2.0 * l - 1.0) * ct * P[l - 1] - (l + m - 1.0) * P[l - 2]) / double(l - m);
    for (int l = m; l <= lmax; ++l) {
      const double N = std::sqrt((2.0 * l + 1.0) / (4.0 * kPi) * factorial(l - m) / factorial(l + m));
      if (m == 0) {
        out[l * l + l] = N * P[l];
      } else {
        out[l * l + l + m] = std::sqrt(2.0) * N * P[l] * std::cos(m * phi);
        out[l * l + l - m] = std::sqrt(2.0) * N * P[l] * std::sin(m * phi);
      }
    }
  }
}

// --------------------------------------------------------------------------
// Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on P_n.
// --------------------------------------------------------------------------
static void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double t = std::cos(kPi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) { double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
      // p1 = P_n(t), p0 = P_{n-1}(t)
      const double dp = n * (t * p1 - p0) / (t * t - 1.0);
      const double dt = p1 / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double p0 = 1.0, p1 = t;
    for (int k = 2; k <= n; ++k) { double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
    const double dp = n * (t * p1 - p0) / (t * t - 1.0);
    x[i] = t;
    w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

// --------------------------------------------------------------------------
// Gaunt coefficients C(L1,L2,L3) = int Y_L1 Y_L2 Y_L3 dOmega, by a product
// quadrature (Gauss-Legendre in cos th, uniform in phi) that is exact for the
// integrand's total degree l1+l2+l3.  Values |C| < 1e-14 are set to zero.
// --------------------------------------------------------------------------
static void gaunt_table(int l1max, int l2max, int l3max, double* C) {
  const int n1 = (l1max + 1) * (l1max + 1), n2 = (l2max + 1) * (l2max + 1), n3 = (l3max + 1) * (l3max + 1);
  const int deg = l1max + l2max + l3max;
  const int nth = deg / 2 + 2, nph = deg + 2;
  std::vector<double> xt(nth), wt(nth);
  gauss_legendre(nth, xt.data(), wt.data());
  const int lm = std::max(l1max, std::max(l2max, l3max));
  const int nl = (lm + 1) * (lm + 1);
  std::vector<double> Y(nl);
  std::memset(C, 0, sizeof(double) * size_t(n1) * n2 * n3);
  for (int a = 0; a < nth; ++a) {
    const double ct = xt[a], st = std::sqrt(1.0 - ct * ct);
    for (int b = 0; b < nph; ++b) {
      const double phi = 2.0 * kPi * b / nph;
      const double wgt = wt[a] * 2.0 * kPi / nph;
      real_ylm(lm, st * std::cos(phi), st * std::sin(phi), ct, Y.data());
      for (int i = 0; i < n1; ++i)
        for (int j = 0; j < n2; ++j)
          for (int k = 0; k < n3; ++k)
            C[(size_t(i) * n2 + j) * n3 + k] += wgt * Y[i] * Y[j] * Y[k];
    }
  }
  for (size_t q = 0; q < size_t(n1) * n2 * n3; ++q)
    if (std::fabs(C[q]) < 1e-14) C[q] = 0.0;
}

static cplx ipow(int p) {  // i^p for any integer p
  switch (((p % 4) + 4) % 4) { case 0: return cplx(1, 0); case 1: return cplx(0, 1); case 2: return cplx(-1, 0); default: return cplx(0, -1); }
}

// kappa = sqrt(E), principal branch (Im kappa > 0 for Im E > 0: outgoing waves).
static cplx kappa_of(cplx E) { return std::sqrt(E); }

// --------------------------------------------------------------------------
// Structure constants (g0 of Eq. 4 between two different sites, Sec. 2.1):
//   G_{LL'}(R) = -4 pi i kappa sum_L'' i^{l-l'+l''} C(L,L',L'')
//                 h_l''(kappa |R|) Y_L''(R^),  R = R_i - R_j (row site i).
// gaunt: dense table for (lmax, lmax, 2 lmax).
// --------------------------------------------------------------------------
static void struct_const_block(int lmax, cplx E, const double* R, const double* gaunt, cplx* G) {
  const int nL = (lmax + 1) * (lmax + 1);
  const int l2max = 2 * lmax, nL2 = (l2max + 1) * (l2max + 1);
  const cplx kap = kappa_of(E);
  const double d = std::sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
  std::vector<cplx> h(l2max + 2);
  sph_h(l2max + 1, kap * d, h.data());
  std::vector<double> Y(nL2);
  real_ylm(l2max, R[0], R[1], R[2], Y.data());
  for (int L = 0; L < nL; ++L) {
    const int l = int(std::sqrt(double(L)) + 1e-9);
    for (int Lp = 0; Lp < nL; ++Lp) {
      const int lp = int(std::sqrt(double(Lp)) + 1e-9);
      cplx s = 0.0;
      for (int L2 = 0; L2 < nL2; ++L2) {
        const double c = gaunt[(size_t(L) * nL + Lp) * nL2 + L2];
        if (c == 0.0) continue;
        const int l2 = int(std::sqrt(double(L2)) + 1e-9);
        s += ipow(l - lp + l2) * c * h[l2] * Y[L2];
      }
      G[L * nL + Lp] = -4.0 * kPi * cplx(0, 1) * kap * s;
    }
  }
}

// --------------------------------------------------------------------------
// Square-well single-site scattering (V inside r < a, 0 outside), matching the
// logarithmic derivative of the interior regular solution j_l(q r),
// q = sqrt(E - V), to the exterior j_l - i kappa t_l h_l at r = a:
//   t_l = [k j'(ka) j(qa) - q j'(qa) j(ka)] / { i k [k h'(ka) j(qa) - q j'(qa) h(ka)] }
// (equivalently t_l = -(1/k) sin(delta_l) e^{i delta_l}).
// --------------------------------------------------------------------------
static void square_well_t(int lmax, cplx E, double V, double a, cplx* t, cplx* tinv) {
  const cplx k = kappa_of(E);
  const cplx q = std::sqrt(E - V);
  std::vector<cplx> jk(lmax + 2), hk(lmax + 2), jq(lmax + 2);
  sph_j(lmax + 1, k * a, jk.data());
  sph_h(lmax + 1, k * a, hk.data());
  sph_j(lmax + 1, q * a, jq.data());
  for (int l = 0; l <= lmax; ++l) {
    const cplx djk = sph_deriv(l, k * a, jk.data());
    const cplx dhk = sph_deriv(l, k * a, hk.data());
    const cplx djq = sph_deriv(l, q * a, jq.data());
    const cplx num = k * djk * jq[l] - q * djq * jk[l];
    const cplx den = cplx(0, 1) * k * (k * dhk * jq[l] - q * djq * hk[l]);
    if (t) t[l] = num / den;
    if (tinv) tinv[l] = den / num;
  }
}

// --------------------------------------------------------------------------
// KKR matrix M = t^{-1} - g0 over a LIZ (Eq. 4, Sec. 2.2), row-major, centre
// (site 0) first.  Collinear: index (site, L), n = N (lmax+1)^2.
// tinv_sites: [N][lmax+1] complex (t^{-1}_l of each site).
// --------------------------------------------------------------------------
static void assemble_collinear(int N, const double* pos, int lmax, cplx E, const cplx* tinv_sites,
                               const double* gaunt, cplx* M) {
  const int nL = (lmax + 1) * (lmax + 1);
  const size_t n = size_t(N) * nL;
  std::fill(M, M + n * n, cplx(0.0));
  std::vector<cplx> G(nL * nL);
  for (int i = 0; i < N; ++i) {
    for (int L = 0; L < nL; ++L) {
      const int l = int(std::sqrt(double(L)) + 1e-9);
      M[(size_t(i) * nL + L) * n + size_t(i) * nL + L] = tinv_sites[i * (lmax + 1) + l];
    }
    for (int j = 0; j < N; ++j) {
      if (j == i) continue;
      const double R[3] = {pos[3 * i] - pos[3 * j], pos[3 * i + 1] - pos[3 * j + 1], pos[3 * i + 2] - pos[3 * j + 2]};
      struct_const_block(lmax, E, R, gaunt, G.data());
      for (int L = 0; L < nL; ++L)
        for (int Lp = 0; Lp < nL; ++Lp)
          M[(size_t(i) * nL + L) * n + size_t(j) * nL + Lp] = -G[L * nL + Lp];
    }
  }
}

// Spin-canted KKR matrix (Sec. 2.1: rank 2 N (lmax+1)^2).  Index (site, spin, L),
// spin up first.  Site i has local moment direction e_i; in the global frame
//   t_i^{-1} = (a+b)/2 1 + (a-b)/2 (sigma . e_i),  a = t_up^{-1}, b = t_dn^{-1},
// and the free propagator is spin-diagonal: g0 (x) 1_2.
static void assemble_canted(int N, const double* pos, int lmax, cplx E, const cplx* tinv_up, const cplx* tinv_dn,
                            const double* dirs, const double* gaunt, cplx* M) {
  const int nL = (lmax + 1) * (lmax + 1);
  const size_t n = size_t(2) * N * nL;
  std::fill(M, M + n * n, cplx(0.0));
  std::vector<cplx> G(nL * nL);
  auto idx = [&](int site, int s, int L) { return (size_t(site) * 2 + s) * nL + L; };
  for (int i = 0; i < N; ++i) {
    const double ex = dirs[3 * i], ey = dirs[3 * i + 1], ez = dirs[3 * i + 2];
    // sigma . e = [[ez, ex - i ey], [ex + i ey, -ez]]
    const cplx sig[2][2] = {{cplx(ez, 0), cplx(ex, -ey)}, {cplx(ex, ey), cplx(-ez, 0)}};
    for (int L = 0; L < nL; ++L) {
      const int l = int(std::sqrt(double(L)) + 1e-9);
      const cplx a = tinv_up[i * (lmax + 1) + l], b = tinv_dn[i * (lmax + 1) + l];
      for (int s = 0; s < 2; ++s)
        for (int sp = 0; sp < 2; ++sp)
          M[idx(i, s, L) * n + idx(i, sp, L)] = (s == sp ? 0.5 * (a + b) : cplx(0.0)) + 0.5 * (a - b) * sig[s][sp];
    }
    for (int j = 0; j < N; ++j) {
      if (j == i) continue;
      const double R[3] = {pos[3 * i] - pos[3 * j], pos[3 * i + 1] - pos[3 * j + 1], pos[3 * i + 2] - pos[3 * j + 2]};
      struct_const_block(lmax, E, R, gaunt, G.data());
      for (int s = 0; s < 2; ++s)
        for (int L = 0; L < nL; ++L)
          for (int Lp = 0; Lp < nL; ++Lp)
            M[idx(i, s, L) * n + idx(j, s, Lp)] = -G[L * nL + Lp];
    }
  }
}

// --------------------------------------------------------------------------
// Dense LU with partial pivoting (Sec. 3.2: factorise, then solve), row-major,
// in place.  Pivot = largest modulus in the column, ties to the lowest row.
// Returns 0, or 1 if a zero pivot was met.
// --------------------------------------------------------------------------
static int lu_factor(size_t n, cplx* A, int* piv) {
  int singular = 0;
  for (size_t k = 0; k < n; ++k) {
    size_t p = k;
    double best = std::abs(A[k * n + k]);
    for (size_t i = k + 1; i < n; ++i) {
      const double v = std::abs(A[i * n + k]);
      if (v > best) { best = v; p = i; }
    }
    piv[k] = int(p);
    if (p != k)
      for (size_t j = 0; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]);
    if (best == 0.0) { singular = 1; continue; }
    const cplx inv = 1.0 / A[k * n + k];
    for (size_t i = k + 1; i < n; ++i) {
      const cplx f = A[i * n + k] * inv;
      A[i * n + k] = f;
      if (f == 0.0) continue;
      cplx* ri = A + i * n;
      const cplx* rk = A + k * n;
      for (size_t j = k + 1; j < n; ++j) ri[j] -= f * rk[j];
    }
  }
  return singular;
}

// Solve A X = B using the factors from lu_factor; B is n x m row-major, overwritten.
static void lu_solve(size_t n, const cplx* LU, const int* piv, size_t m, cplx* B) {
  for (size_t k = 0; k < n; ++k)
    if (size_t(piv[k]) != k)
      for (size_t c = 0; c < m; ++c) std::swap(B[k * m + c], B[size_t(piv[k]) * m + c]);
  for (size_t i = 0; i < n; ++i)            // forward: L unit lower
    for (size_t k = 0; k < i; ++k) {
      const cplx l = LU[i * n + k];
      if (l == 0.0) continue;
      for (size_t c = 0; c < m; ++c) B[i * m + c] -= l * B[k * m + c];
    }
  for (size_t ii = n; ii-- > 0;) {          // backward: U upper
    for (size_t k = ii + 1; k < n; ++k) {
      const cplx u = LU[ii * n + k];
      for (size_t c = 0; c < m; ++c) B[ii * m + c] -= u * B[k * m + c];
    }
    const cplx d = LU[ii * n + ii];
    for (size_t c = 0; c < m; ++c) B[ii * m + c] /= d;
  }
}

// --------------------------------------------------------------------------
// Double-double arithmetic for the refinement residual: Knuth's TwoSum and
// Dekker's TwoProduct (via fused multiply-add).  Compiled without FP
// contraction so the error-free transforms stay exact.
// --------------------------------------------------------------------------
struct dd { double hi, lo; };
static inline void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
static inline void two_prod(double a, double b, double& p, double& e) {
  p = a * b;
  e = std::fma(a, b, -p);
}
static inline void dd_add_double(dd& x, double v) {
  double s, e;
  two_sum(x.hi, v, s, e);
  e += x.lo;
  two_sum(s, e, x.hi, x.lo);
}
static inline void dd_add_prod(dd& x, double a, double b) {
  double p, e;
  two_prod(a, b, p, e);
  dd_add_double(x, p);
  dd_add_double(x, e);
}

// R = B - A X, with every product and sum carried in double-double.
static void residual_dd(size_t n, const cplx* A, size_t m, const cplx* X, const cplx* B, cplx* R) {
  for (size_t i = 0; i < n; ++i)
    for (size_t c = 0; c < m; ++c) {
      dd re = {B[i * m + c].real(), 0.0}, im = {B[i * m + c].imag(), 0.0};
      for (size_t k = 0; k < n; ++k) {
        const double ar = A[i * n + k].real(), ai = A[i * n + k].imag();
        const double xr = X[k * m + c].real(), xi = X[k * m + c].imag();
        dd_add_prod(re, -ar, xr);
        dd_add_prod(re, ai, xi);
        dd_add_prod(im, -ar, xi);
        dd_add_prod(im, -ai, xr);
      }
      R[i * m + c] = cplx(re.hi + re.lo, im.hi + im.lo);
    }
}

// --------------------------------------------------------------------------
// tau_00 = first kappa x kappa block of M^{-1} (Eq. 4, Sec. 2.2): solve
// M X = E0 (E0 = first kappa columns of I) by LU + iterative refinement with a
// double-double residual, until the correction is below 1e-16 relative.
// Returns the last relative correction (the oracle's own error estimate).
// --------------------------------------------------------------------------
static double solve_first_block(size_t n, const cplx* M, size_t kap, cplx* tau, int* status) {
  std::vector<cplx> LU(M, M + n * n);
  std::vector<int> piv(n);
  *status = lu_factor(n, LU.data(), piv.data());
  std::vector<cplx> E0(n * kap, cplx(0.0)), X(n * kap), R(n * kap);
  for (size_t c = 0; c < kap; ++c) E0[c * kap + c] = 1.0;
  X = E0;
  lu_solve(n, LU.data(), piv.data(), kap, X.data());
  double rel = 1.0;
  for (int it = 0; it < 12; ++it) {
    residual_dd(n, M, kap, X.data(), E0.data(), R.data());
    lu_solve(n, LU.data(), piv.data(), kap, R.data());
    double dn = 0.0, xn = 0.0;
    for (size_t q = 0; q < n * kap; ++q) {
      X[q] += R[q];
      dn += std::norm(R[q]);
      xn += std::norm(X[q]);
    }
    rel = std::sqrt(dn / xn);
    if (rel <= 1e-16) break;
  }
  for (size_t r = 0; r < kap; ++r)
    for (size_t c = 0; c < kap; ++c) tau[r * kap + c] = X[r * kap + c];
  return rel;
}

// Full inverse by Gauss-Jordan elimination with partial pivoting (tiny cases).
static int gauss_jordan(size_t n, const cplx* A, cplx* Ainv) {
  std::vector<cplx> W(n * 2 * n, cplx(0.0));
  for (size_t i = 0; i < n; ++i) {
    for (size_t j = 0; j < n; ++j) W[i * 2 * n + j] = A[i * n + j];
    W[i * 2 * n + n + i] = 1.0;
  }
  const size_t w = 2 * n;
  for (size_t k = 0; k < n; ++k) {
    size_t p = k;
    double best = std::abs(W[k * w + k]);
    for (size_t i = k + 1; i < n; ++i)
      if (std::abs(W[i * w + k]) > best) { best = std::abs(W[i * w + k]); p = i; }
    if (best == 0.0) return 1;
    if (p != k) for (size_t j = 0; j < w; ++j) std::swap(W[k * w + j], W[p * w + j]);
    const cplx inv = 1.0 / W[k * w + k];
    for (size_t j = 0; j < w; ++j) W[k * w + j] *= inv;
    for (size_t i = 0; i < n; ++i) {
      if (i == k) continue;
      const cplx f = W[i * w + k];
      if (f == 0.0) continue;
      for (size_t j = 0; j < w; ++j) W[i * w + j] -= f * W[k * w + j];
    }
  }
  for (size_t i = 0; i < n; ++i)
    for (size_t j = 0; j < n; ++j) Ainv[i * n + j] = W[i * w + n + j];
  return 0;
}

// ==========================================================================
// Full KKR (Sec. 5: the same matrix inverse for a periodic crystal instead of
// a LIZ).  With N_b sites b_s per cell of the lattice {R} and the real-space
// blocks G(rho) above, the Bloch-summed structure constants are
//   G^{st}_{LL'}(k) = sum_{R : rho != 0} e^{i k.R} G_{LL'}(rho),  rho = b_s - b_t - R,
// the KKR matrix of Eq. (4) becomes M(k) = t^{-1} - G(k) (order N_b (lmax+1)^2,
// Sec. 2.1), and the site-diagonal scattering-path block is the Brillouin-zone
// average  tau^{ss} = (1/N_k) sum_k [M(k)^{-1}]^{ss}  on a uniform k mesh.
//
// The lattice sum converges only for Im kappa > 0 and slowly near the real
// axis, so it is split (Ewald).  With D^{st}_L(k) = sum_R e^{ik.R}
// h_l(kappa|rho|) Y_L(rho^), and since h_l(kappa r) Y_L(r^) = (-kappa)^{-l}
// Y_L(grad) h_0(kappa r) (Hobson's theorem with the Rayleigh formula for h_l),
// h_0(kappa r) = -i e^{i kappa r}/(kappa r), and
//   e^{i kappa r}/r = (2/sqrt(pi)) int_0^inf exp(-r^2 xi^2 + E/(4 xi^2)) d xi,
// cut at xi0 = sqrt(eta)/2: the part below xi0 is summed in reciprocal space
// (Poisson; its Fourier transform is 4 pi e^{(E - q^2)/eta}/(q^2 - E)), the part
// above xi0 in real space, and the R = 0 term of the reciprocal sum is removed
// when s = t:
//   D_L = (-kappa)^{-l} (-i/kappa) [A_L + B_L + C_L]
//   A_L = (4 pi/Omega) i^l sum_K e^{i q.x} |q|^l Y_L(q^) e^{(E-q^2)/eta}/(q^2-E),
//         q = k + K, x = b_s - b_t
//   B_L = (2/sqrt(pi)) (-2)^l sum_{R: rho != 0} e^{ik.R} |rho|^l Y_L(rho^)
//         int_{xi0}^inf xi^{2l} exp(-rho^2 xi^2 + E/(4 xi^2)) d xi
//   C_0 = -(1/sqrt(4 pi)) [i kappa - sqrt(eta/pi) sum_{n>=0} (E/eta)^n/(n! (2n-1))]
//         for s = t (C_L = 0 otherwise)
// and G^{st}_{LL'}(k) = -4 pi i kappa sum_L'' i^{l-l'+l''} C(L,L',L'') D^{st}_L''.
// Both sums are truncated where their Gaussian factor falls below e^{-cut}.
// ==========================================================================

struct Lattice {
  double a[3][3];  // primitive vectors (rows), bohr
  double b[3][3];  // reciprocal vectors, a_i . b_j = 2 pi delta_ij
  double omega;    // cell volume
};

static Lattice make_lattice(const double* A) {
  Lattice L;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) L.a[i][j] = A[3 * i + j];
  auto cross = [](const double* u, const double* v, double* w) {
    w[0] = u[1] * v[2] - u[2] * v[1];
    w[1] = u[2] * v[0] - u[0] * v[2];
    w[2] = u[0] * v[1] - u[1] * v[0];
  };
  double c[3][3];
  cross(L.a[1], L.a[2], c[0]);
  cross(L.a[2], L.a[0], c[1]);
  cross(L.a[0], L.a[1], c[2]);
  const double vol = L.a[0][0] * c[0][0] + L.a[0][1] * c[0][1] + L.a[0][2] * c[0][2];
  L.omega = std::fabs(vol);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) L.b[i][j] = 2.0 * kPi * c[i][j] / vol;
  return L;
}

static double norm3(const double* v) { return std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

// All integer combinations n1 v1 + n2 v2 + n3 v3 (v = rows of V) within
// distance rmax of the point -c, i.e. |c + n.V| <= rmax.  dual = the rows of
// the dual basis divided by 2 pi, used to bound each |n_i|.
static void lattice_points(const double V[3][3], const double W[3][3], const double* c, double rmax,
                           std::vector<double>& out) {
  int nmax[3];
  const double cn = norm3(c);
  for (int i = 0; i < 3; ++i) nmax[i] = int(std::ceil((rmax + cn) * norm3(W[i]) / (2.0 * kPi))) + 1;
  out.clear();
  for (int n1 = -nmax[0]; n1 <= nmax[0]; ++n1)
    for (int n2 = -nmax[1]; n2 <= nmax[1]; ++n2)
      for (int n3 = -nmax[2]; n3 <= nmax[2]; ++n3) {
        double v[3];
        for (int d = 0; d < 3; ++d) v[d] = n1 * V[0][d] + n2 * V[1][d] + n3 * V[2][d];
        const double w[3] = {c[0] + v[0], c[1] + v[1], c[2] + v[2]};
        if (norm3(w) <= rmax) out.insert(out.end(), v, v + 3);
      }
}

// int_{xi0}^{inf} xi^{2l} exp(-rho^2 xi^2 + E/(4 xi^2)) d xi for l = 0..lmax,
// by composite 16-point Gauss-Legendre over [xi0, xi_hi], where
// rho^2 (xi_hi^2 - xi0^2) = 90 (the rest is below e^{-90} of the first node).
static void ewald_real_integrals(int lmax, double rho, double xi0, cplx E, cplx* I) {
  static thread_local std::vector<double> gx, gw;
  if (gx.empty()) { gx.resize(16); gw.resize(16); gauss_legendre(16, gx.data(), gw.data()); }
  const double xhi = std::sqrt(xi0 * xi0 + 90.0 / (rho * rho));
  const int panels = 48;
  const double h = (xhi - xi0) / panels;
  for (int l = 0; l <= lmax; ++l) I[l] = 0.0;
  for (int p = 0; p < panels; ++p) {
    const double lo = xi0 + p * h;
    for (int q = 0; q < 16; ++q) {
      const double xi = lo + 0.5 * h * (gx[q] + 1.0);
      const cplx f = std::exp(-rho * rho * xi * xi + E / (4.0 * xi * xi)) * (0.5 * h * gw[q]);
      double pw = 1.0;
      for (int l = 0; l <= lmax; ++l) { I[l] += pw * f; pw *= xi * xi; }
    }
  }
}

// Real-space terms of the Ewald sum for one displacement x = b_s - b_t:
// every lattice vector R with 0 < |x - R| <= sqrt(4 cut / eta), and for each
// the k-independent factor (2/sqrt(pi)) (-2)^l |rho|^l Y_L(rho^) I_l(|rho|).
struct EwaldRealTerms {
  std::vector<double> R;  // 3 per point
  std::vector<cplx> T;    // (l2max+1)^2 per point
};

static void ewald_real_terms(int l2max, cplx E, const Lattice& Lt, const double* x, double eta, double cut,
                             EwaldRealTerms& out) {
  const int nL2 = (l2max + 1) * (l2max + 1);
  const double xi0 = 0.5 * std::sqrt(eta);
  const double rmax = std::sqrt(4.0 * cut / eta);
  const double mx[3] = {-x[0], -x[1], -x[2]};
  std::vector<double> pts;
  lattice_points(Lt.a, Lt.b, mx, rmax, pts);
  std::vector<cplx> I(l2max + 1);
  std::vector<double> Y(nL2);
  out.R.clear();
  out.T.clear();
  for (size_t p = 0; p < pts.size(); p += 3) {
    const double rho[3] = {x[0] - pts[p], x[1] - pts[p + 1], x[2] - pts[p + 2]};
    const double rn = norm3(rho);
    if (rn < 1e-10) continue;  // the site itself
    ewald_real_integrals(l2max, rn, xi0, E, I.data());
    real_ylm(l2max, rho[0], rho[1], rho[2], Y.data());
    out.R.insert(out.R.end(), pts.begin() + p, pts.begin() + p + 3);
    for (int l = 0; l <= l2max; ++l) {
      const cplx f = (2.0 / std::sqrt(kPi)) * std::pow(-2.0, l) * std::pow(rn, l) * I[l];
      for (int m = -l; m <= l; ++m) out.T.push_back(f * Y[l * l + l + m]);
    }
  }
}

// Lattice sums D_L(k), L < (l2max+1)^2, for the displacement x = b_s - b_t
// whose real-space terms are `real` (self term included when x = 0).
// cut: truncation exponent of the reciprocal sum.
static void kkr_lattice_sum(int l2max, cplx E, const Lattice& Lt, const double* x, const double* k, double eta,
                            double cut, const EwaldRealTerms& real, cplx* D) {
  const int nL2 = (l2max + 1) * (l2max + 1);
  const cplx kap = kappa_of(E);
  std::vector<cplx> acc(nL2, cplx(0.0));
  std::vector<double> Y(nL2);
  // reciprocal space: all K with |k + K|^2 <= eta * cut + max(Re E, 0)
  std::vector<double> pts;
  const double qmax = std::sqrt(eta * cut + std::max(E.real(), 0.0));
  lattice_points(Lt.b, Lt.a, k, qmax, pts);
  for (size_t p = 0; p < pts.size(); p += 3) {
    const double q[3] = {k[0] + pts[p], k[1] + pts[p + 1], k[2] + pts[p + 2]};
    const double q2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
    const double qn = std::sqrt(q2);
    const cplx w = (4.0 * kPi / Lt.omega) * std::exp((E - q2) / eta) / (q2 - E) *
                   std::exp(cplx(0.0, q[0] * x[0] + q[1] * x[1] + q[2] * x[2]));
    if (qn > 0.0) {
      real_ylm(l2max, q[0], q[1], q[2], Y.data());
    } else {
      std::fill(Y.begin(), Y.end(), 0.0);
      Y[0] = 1.0 / std::sqrt(4.0 * kPi);
    }
    for (int l = 0; l <= l2max; ++l) {
      const cplx f = ipow(l) * std::pow(qn, l) * w;
      for (int m = -l; m <= l; ++m) acc[l * l + l + m] += f * Y[l * l + l + m];
    }
  }
  // real space
  const size_t npt = real.R.size() / 3;
  for (size_t p = 0; p < npt; ++p) {
    const double* R = &real.R[3 * p];
    const cplx ph = std::exp(cplx(0.0, k[0] * R[0] + k[1] * R[1] + k[2] * R[2]));
    for (int L = 0; L < nL2; ++L) acc[L] += ph * real.T[p * nL2 + L];
  }
  // the removed R = 0 term of the reciprocal sum
  if (norm3(x) < 1e-10) {
    cplx s = 0.0, term = 1.0;  // term = (E/eta)^n / n!
    for (int n = 0; n < 200; ++n) {
      const cplx add = term / double(2 * n - 1);
      s += add;
      if (n > 4 && std::abs(add) < 1e-18 * std::abs(s)) break;
      term *= (E / eta) / double(n + 1);
    }
    acc[0] -= (cplx(0.0, 1.0) * kap - std::sqrt(eta / kPi) * s) / std::sqrt(4.0 * kPi);
  }
  for (int l = 0; l <= l2max; ++l) {
    const cplx f = std::pow(-kap, -l) * (cplx(0.0, -1.0) / kap);
    for (int m = -l; m <= l; ++m) D[l * l + l + m] = f * acc[l * l + l + m];
  }
}

// The real-space terms of every site pair (s, t), index s * nb + t.
static std::vector<EwaldRealTerms> kkr_real_tables(int lmax, cplx E, const Lattice& Lt, int nb, const double* basis,
                                                   double eta, double cut) {
  std::vector<EwaldRealTerms> real(size_t(nb) * nb);
  for (int s = 0; s < nb; ++s)
    for (int t = 0; t < nb; ++t) {
      const double x[3] = {basis[3 * s] - basis[3 * t], basis[3 * s + 1] - basis[3 * t + 1],
                           basis[3 * s + 2] - basis[3 * t + 2]};
      ewald_real_terms(2 * lmax, E, Lt, x, eta, cut, real[size_t(s) * nb + t]);
    }
  return real;
}

// G^{st}(k) of every site pair, row-major n x n with n = N_b (lmax+1)^2,
// index (site, L).  gaunt: dense table for (lmax, lmax, 2 lmax).
static void kkr_struct_const_k(int lmax, cplx E, const Lattice& Lt, int nb, const double* basis, const double* k,
                               double eta, double cut, const std::vector<EwaldRealTerms>& real, const double* gaunt,
                               cplx* G) {
  const int nL = (lmax + 1) * (lmax + 1);
  const int l2max = 2 * lmax, nL2 = (l2max + 1) * (l2max + 1);
  const int n = nb * nL;
  const cplx kap = kappa_of(E);
  std::vector<cplx> D(nL2);
  for (int s = 0; s < nb; ++s)
    for (int t = 0; t < nb; ++t) {
      const double x[3] = {basis[3 * s] - basis[3 * t], basis[3 * s + 1] - basis[3 * t + 1],
                           basis[3 * s + 2] - basis[3 * t + 2]};
      kkr_lattice_sum(l2max, E, Lt, x, k, eta, cut, real[size_t(s) * nb + t], D.data());
      for (int L = 0; L < nL; ++L) {
        const int l = int(std::sqrt(double(L)) + 1e-9);
        for (int Lp = 0; Lp < nL; ++Lp) {
          const int lp = int(std::sqrt(double(Lp)) + 1e-9);
          cplx acc = 0.0;
          for (int L2 = 0; L2 < nL2; ++L2) {
            const double c = gaunt[(size_t(L) * nL + Lp) * nL2 + L2];
            if (c == 0.0) continue;
            const int l2 = int(std::sqrt(double(L2)) + 1e-9);
            acc += ipow(l - lp + l2) * c * D[L2];
          }
          G[size_t(s * nL + L) * n + t * nL + Lp] = -4.0 * kPi * cplx(0.0, 1.0) * kap * acc;
        }
      }
    }
}

// tau^{ss}(E) = (1/N_k) sum_k [M(k)^{-1}]^{ss}, M(k) = t^{-1} - G(k), on the
// Gamma-centred mesh k = sum_i (m_i / n_k) b_i, m_i = 0..n_k-1.
// tinv: [N_b][lmax+1]; tau: [N_b][kap][kap] row-major.  Returns 0, or 1 on a
// singular M(k).
static int kkr_tau(int lmax, cplx E, const Lattice& Lt, int nb, const double* basis, const cplx* tinv, int nk,
                   double eta, double cut, cplx* tau) {
  const int nL = (lmax + 1) * (lmax + 1);
  const int n = nb * nL;
  std::vector<double> C(size_t(nL) * nL * (2 * lmax + 1) * (2 * lmax + 1));
  gaunt_table(lmax, lmax, 2 * lmax, C.data());
  std::vector<cplx> G(size_t(n) * n), M(size_t(n) * n), Minv(size_t(n) * n);
  std::vector<cplx> sum(size_t(nb) * nL * nL, cplx(0.0));
  const std::vector<EwaldRealTerms> real = kkr_real_tables(lmax, E, Lt, nb, basis, eta, cut);
  for (int m1 = 0; m1 < nk; ++m1)
    for (int m2 = 0; m2 < nk; ++m2)
      for (int m3 = 0; m3 < nk; ++m3) {
        double k[3];
        for (int d = 0; d < 3; ++d) k[d] = (m1 * Lt.b[0][d] + m2 * Lt.b[1][d] + m3 * Lt.b[2][d]) / nk;
        kkr_struct_const_k(lmax, E, Lt, nb, basis, k, eta, cut, real, C.data(), G.data());
        for (int i = 0; i < n; ++i)
          for (int j = 0; j < n; ++j) M[size_t(i) * n + j] = -G[size_t(i) * n + j];
        for (int s = 0; s < nb; ++s)
          for (int L = 0; L < nL; ++L) {
            const int l = int(std::sqrt(double(L)) + 1e-9);
            M[size_t(s * nL + L) * n + s * nL + L] += tinv[s * (lmax + 1) + l];
          }
        if (gauss_jordan(n, M.data(), Minv.data())) return 1;
        for (int s = 0; s < nb; ++s)
          for (int L = 0; L < nL; ++L)
            for (int Lp = 0; Lp < nL; ++Lp)
              sum[(size_t(s) * nL + L) * nL + Lp] += Minv[size_t(s * nL + L) * n + s * nL + Lp];
      }
  const double w = 1.0 / (double(nk) * nk * nk);
  for (size_t q = 0; q < sum.size(); ++q) tau[q] = sum[q] * w;
  return 0;
}

// ==========================================================================
// C entry points (ctypes).  Complex arrays are interleaved (re, im) doubles.
// ==========================================================================
extern "C" {

void orc_sph_jyh(int lmax, double zr, double zi, double* j, double* y, double* h) {
  std::vector<cplx> jv(lmax + 1), yv(lmax + 1), hv(lmax + 1);
  sph_j(lmax, cplx(zr, zi), jv.data());
  sph_y(lmax, cplx(zr, zi), yv.data());
  sph_h(lmax, cplx(zr, zi), hv.data());
  std::memcpy(j, jv.data(), sizeof(cplx) * (lmax + 1));
  std::memcpy(y, yv.data(), sizeof(cplx) * (lmax + 1));
  if (h) std::memcpy(h, hv.data(), sizeof(cplx) * (lmax + 1));
}

void orc_real_ylm(int lmax, double x, double y, double z, double* out) { real_ylm(lmax, x, y, z, out); }

void orc_gauss_legendre(int n, double* x, double* w) { gauss_legendre(n, x, w); }

void orc_gaunt(int l1max, int l2max, int l3max, double* C) { gaunt_table(l1max, l2max, l3max, C); }

void orc_struct_const(int lmax, double er, double ei, const double* R, double* G) {
  const int nL = (lmax + 1) * (lmax + 1);
  std::vector<double> C(size_t(nL) * nL * (2 * lmax + 1) * (2 * lmax + 1));
  gaunt_table(lmax, lmax, 2 * lmax, C.data());
  struct_const_block(lmax, cplx(er, ei), R, C.data(), reinterpret_cast<cplx*>(G));
}

void orc_square_well(int lmax, double er, double ei, double V, double a, double* t, double* tinv) {
  square_well_t(lmax, cplx(er, ei), V, a, reinterpret_cast<cplx*>(t), reinterpret_cast<cplx*>(tinv));
}

// M (row-major, n x n) for one energy.  dirs == NULL: collinear, tinv_a = t^{-1}
// per site; else canted with tinv_a = up, tinv_b = down.
void orc_assemble(int N, const double* pos, int lmax, double er, double ei, const double* tinv_a,
                  const double* tinv_b, const double* dirs, double* M) {
  const int nL = (lmax + 1) * (lmax + 1);
  std::vector<double> C(size_t(nL) * nL * (2 * lmax + 1) * (2 * lmax + 1));
  gaunt_table(lmax, lmax, 2 * lmax, C.data());
  if (!dirs)
    assemble_collinear(N, pos, lmax, cplx(er, ei), reinterpret_cast<const cplx*>(tinv_a), C.data(),
                       reinterpret_cast<cplx*>(M));
  else
    assemble_canted(N, pos, lmax, cplx(er, ei), reinterpret_cast<const cplx*>(tinv_a),
                    reinterpret_cast<const cplx*>(tinv_b), dirs, C.data(), reinterpret_cast<cplx*>(M));
}

// Plain LU solve of A X = B (row-major), for checks against a library solver.
int orc_lu_solve(int n, const double* A, int m, double* B) {
  std::vector<cplx> LU(reinterpret_cast<const cplx*>(A), reinterpret_cast<const cplx*>(A) + size_t(n) * n);
  std::vector<int> piv(n);
  const int s = lu_factor(n, LU.data(), piv.data());
  lu_solve(n, LU.data(), piv.data(), m, reinterpret_cast<cplx*>(B));
  return s;
}

// tau_00 of a given matrix (row-major n x n), first kap x kap block.
double orc_first_block(int n, const double* M, int kap, double* tau, int* status) {
  return solve_first_block(n, reinterpret_cast<const cplx*>(M), kap, reinterpret_cast<cplx*>(tau), status);
}

int orc_inverse(int n, const double* A, double* Ainv) {
  return gauss_jordan(n, reinterpret_cast<const cplx*>(A), reinterpret_cast<cplx*>(Ainv));
}

// Many independent tau_00 solves over one LIZ geometry (OpenMP across items,
// one item per thread, mirroring the paper's one-thread-per-rank runs, Sec. 4.2).
//   collinear: tinv_a [n_items][N][lmax+1], dirs == NULL, tau [n_items][kap][kap]
//   canted   : tinv_a = up, tinv_b = down, dirs [N][3], tau [n_items][2kap][2kap]
// Returns the number of threads used.
int orc_tau00_batch(int N, const double* pos, int lmax, int n_items, const double* E, const double* tinv_a,
                    const double* tinv_b, const double* dirs, int nthreads, double* tau, double* err,
                    int* status) {
  const int nL = (lmax + 1) * (lmax + 1);
  const int spins = dirs ? 2 : 1;
  const size_t n = size_t(spins) * N * nL, kap = size_t(spins) * nL;
  std::vector<double> C(size_t(nL) * nL * (2 * lmax + 1) * (2 * lmax + 1));
  gaunt_table(lmax, lmax, 2 * lmax, C.data());
  int used = 1;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
  for (int it = 0; it < n_items; ++it) {
#ifdef _OPENMP
    if (omp_get_thread_num() == 0) used = omp_get_num_threads();
#endif
    std::vector<cplx> M(n * n);
    const cplx e(E[2 * it], E[2 * it + 1]);
    const size_t tstride = size_t(N) * (lmax + 1) * 2;
    if (!dirs)
      assemble_collinear(N, pos, lmax, e, reinterpret_cast<const cplx*>(tinv_a + it * tstride), C.data(), M.data());
    else
      assemble_canted(N, pos, lmax, e, reinterpret_cast<const cplx*>(tinv_a + it * tstride),
                      reinterpret_cast<const cplx*>(tinv_b + it * tstride), dirs, C.data(), M.data());
    err[it] = solve_first_block(n, M.data(), kap, reinterpret_cast<cplx*>(tau + size_t(it) * kap * kap * 2),
                                status + it);
  }
  return used;
}

// Lattice sums D_L(k), L < (l2max+1)^2 (Ewald; see the full-KKR section).
void orc_kkr_lattice_sum(int l2max, double er, double ei, const double* lattice, const double* x, const double* k,
                         double eta, double cut, double* D) {
  const Lattice Lt = make_lattice(lattice);
  EwaldRealTerms real;
  ewald_real_terms(l2max, cplx(er, ei), Lt, x, eta, cut, real);
  kkr_lattice_sum(l2max, cplx(er, ei), Lt, x, k, eta, cut, real, reinterpret_cast<cplx*>(D));
}

// G(k), row-major n x n, n = nb (lmax+1)^2.
void orc_kkr_struct_const(int lmax, double er, double ei, const double* lattice, int nb, const double* basis,
                          const double* k, double eta, double cut, double* G) {
  const int nL = (lmax + 1) * (lmax + 1);
  std::vector<double> C(size_t(nL) * nL * (2 * lmax + 1) * (2 * lmax + 1));
  gaunt_table(lmax, lmax, 2 * lmax, C.data());
  const Lattice Lt = make_lattice(lattice);
  const std::vector<EwaldRealTerms> real = kkr_real_tables(lmax, cplx(er, ei), Lt, nb, basis, eta, cut);
  kkr_struct_const_k(lmax, cplx(er, ei), Lt, nb, basis, k, eta, cut, real, C.data(), reinterpret_cast<cplx*>(G));
}

// Site-diagonal tau blocks of the crystal for many independent items (OpenMP
// across items).  E [n_items], tinv [n_items][nb][lmax+1], tau
// [n_items][nb][kap][kap] row-major.  Returns the threads used, or -1 if some
// M(k) was singular.
int orc_kkr_tau(int lmax, const double* lattice, int nb, const double* basis, int n_items, const double* E,
                const double* tinv, int nk, double eta, double cut, int nthreads, double* tau) {
  const Lattice Lt = make_lattice(lattice);
  const int nL = (lmax + 1) * (lmax + 1);
  int used = 1, bad = 0;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
  if (nthreads > n_items) nthreads = n_items > 0 ? n_items : 1;
#pragma omp parallel num_threads(nthreads) reduction(| : bad)
  {
#pragma omp single
    used = omp_get_num_threads();
#pragma omp for schedule(dynamic, 1)
#endif
    for (int it = 0; it < n_items; ++it) {
      const cplx e(E[2 * it], E[2 * it + 1]);
      bad |= kkr_tau(lmax, e, Lt, nb, basis, reinterpret_cast<const cplx*>(tinv) + size_t(it) * nb * (lmax + 1),
                     nk, eta, cut, reinterpret_cast<cplx*>(tau) + size_t(it) * nb * nL * nL);
    }
#ifdef _OPENMP
  }
#endif
  return bad ? -1 : used;
}

}  // extern "C"
