// Real-harmonic Gaunt coefficients for the structure-constant contraction,
// computed once per handle on the host from closed forms:
//   complex Gaunt  int Y_l1m1 Y_l2m2 Y_l3m3 dOmega
//       = sqrt((2l1+1)(2l2+1)(2l3+1)/(4 pi)) (l1 l2 l3; 0 0 0)(l1 l2 l3; m1 m2 m3)
//   Wigner 3j symbols by Racah's single-sum formula,
// then transformed to the real basis Y_lm (no Condon-Shortley phase):
//   m > 0: (1/sqrt2) ((-1)^m Y_l^m + Y_l^-m);  m < 0: (1/(i sqrt2)) ((-1)^|m| Y_l^|m| - Y_l^-|m|).
// The table feeds g0 of Eq. (4): G_{LL'} = -4 pi i kappa sum_L'' c_{LL'L''} h_l'' Y_L''
// with c = i^{l-l'+l''} C(L,L',L''), which is real since l+l'+l'' is even.
#include <cmath>
#include <complex>
#include <vector>

namespace {

double fact(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

double wigner3j(int j1, int j2, int j3, int m1, int m2, int m3) {
  if (m1 + m2 + m3 != 0) return 0.0;
  if (j3 < std::abs(j1 - j2) || j3 > j1 + j2) return 0.0;
  if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(m3) > j3) return 0.0;
  const double tri = fact(j1 + j2 - j3) * fact(j1 - j2 + j3) * fact(-j1 + j2 + j3) / fact(j1 + j2 + j3 + 1);
  const double pre = std::sqrt(tri * fact(j1 + m1) * fact(j1 - m1) * fact(j2 + m2) * fact(j2 - m2) *
                               fact(j3 + m3) * fact(j3 - m3));
  double sum = 0.0;
  for (int k = 0; k <= j1 + j2 + j3; ++k) {
    const int a = j3 - j2 + k + m1, b = j3 - j1 + k - m2, c = j1 + j2 - j3 - k, d = j1 - k - m1, e = j2 - k + m2;
    if (a < 0 || b < 0 || c < 0 || d < 0 || e < 0) continue;
    const double term = 1.0 / (fact(k) * fact(a) * fact(b) * fact(c) * fact(d) * fact(e));
    sum += (k % 2 ? -term : term);
  }
  const int ph = j1 - j2 - m3;
  return ((ph % 2 + 2) % 2 ? -1.0 : 1.0) * pre * sum;
}

double complex_gaunt(int l1, int m1, int l2, int m2, int l3, int m3) {
  const double pi = 3.14159265358979323846;
  const double w0 = wigner3j(l1, l2, l3, 0, 0, 0);
  if (w0 == 0.0) return 0.0;
  return std::sqrt((2.0 * l1 + 1.0) * (2.0 * l2 + 1.0) * (2.0 * l3 + 1.0) / (4.0 * pi)) * w0 *
         wigner3j(l1, l2, l3, m1, m2, m3);
}

// Coefficients of real Y_lm in the complex (Condon-Shortley) basis: (mu, weight) pairs.
void real_from_complex(int m, std::complex<double> w[2], int mu[2], int& cnt) {
  const double s = 1.0 / std::sqrt(2.0);
  if (m == 0) { mu[0] = 0; w[0] = 1.0; cnt = 1; return; }
  const int am = std::abs(m);
  const double sg = (am % 2) ? -1.0 : 1.0;
  if (m > 0) {
    mu[0] = am; w[0] = sg * s;
    mu[1] = -am; w[1] = s;
  } else {
    const std::complex<double> inv_i(0.0, -1.0);   // 1/i
    mu[0] = am; w[0] = inv_i * (sg * s);
    mu[1] = -am; w[1] = inv_i * (-s);
  }
  cnt = 2;
}

}  // namespace

// Real Gaunt C(L1, L2, L3) for l1, l2 <= lmax and l3 <= 2 lmax, dense [nL][nL][nL2].
void must_real_gaunt(int lmax, std::vector<double>& C) {
  const int nL = (lmax + 1) * (lmax + 1), l3max = 2 * lmax, nL2 = (l3max + 1) * (l3max + 1);
  C.assign(size_t(nL) * nL * nL2, 0.0);
  for (int l1 = 0; l1 <= lmax; ++l1)
    for (int m1 = -l1; m1 <= l1; ++m1)
      for (int l2 = 0; l2 <= lmax; ++l2)
        for (int m2 = -l2; m2 <= l2; ++m2)
          for (int l3 = 0; l3 <= l3max; ++l3)
            for (int m3 = -l3; m3 <= l3; ++m3) {
              std::complex<double> w1[2], w2[2], w3[2];
              int u1[2], u2[2], u3[2], c1, c2, c3;
              real_from_complex(m1, w1, u1, c1);
              real_from_complex(m2, w2, u2, c2);
              real_from_complex(m3, w3, u3, c3);
              std::complex<double> s = 0.0;
              for (int a = 0; a < c1; ++a)
                for (int b = 0; b < c2; ++b)
                  for (int c = 0; c < c3; ++c) {
                    const double g = complex_gaunt(l1, u1[a], l2, u2[b], l3, u3[c]);
                    if (g != 0.0) s += w1[a] * w2[b] * w3[c] * g;
                  }
              const double v = s.real();
              const int L1 = l1 * l1 + l1 + m1, L2 = l2 * l2 + l2 + m2, L3 = l3 * l3 + l3 + m3;
              C[(size_t(L1) * nL + L2) * nL2 + L3] = (std::fabs(v) < 1e-14) ? 0.0 : v;
            }
}

// Sparse contraction table: for every (L, L') the list of (L'', i^{l-l'+l''} C).
void must_gaunt_csr(int lmax, std::vector<int>& start, std::vector<int>& L2s, std::vector<double>& coef) {
  std::vector<double> C;
  must_real_gaunt(lmax, C);
  const int nL = (lmax + 1) * (lmax + 1), nL2 = (2 * lmax + 1) * (2 * lmax + 1);
  start.assign(size_t(nL) * nL + 1, 0);
  L2s.clear();
  coef.clear();
  for (int L = 0; L < nL; ++L) {
    const int l = int(std::sqrt(double(L)) + 1e-9);
    for (int Lp = 0; Lp < nL; ++Lp) {
      const int lp = int(std::sqrt(double(Lp)) + 1e-9);
      start[size_t(L) * nL + Lp] = int(L2s.size());
      for (int L3 = 0; L3 < nL2; ++L3) {
        const double c = C[(size_t(L) * nL + Lp) * nL2 + L3];
        if (c == 0.0) continue;
        const int l3 = int(std::sqrt(double(L3)) + 1e-9);
        const int p = ((l - lp + l3) % 4 + 4) % 4;   // even: 0 -> +1, 2 -> -1
        L2s.push_back(L3);
        coef.push_back(p == 0 ? c : -c);
      }
    }
  }
  start[size_t(nL) * nL] = int(L2s.size());
}
