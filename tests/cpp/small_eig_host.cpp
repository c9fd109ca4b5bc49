// Host driver for the library's small dense eigensolver (paper_2201_02250_gb300/csrc/small_eig.cuh):
// reads "m" and an m x m matrix from stdin, prints the return code, the eigenvalues ordered by
// decreasing modulus and, for the leading ones, the residual of the computed eigenvectors.
#include <cmath>
#include <cstdio>
#include <vector>

#include "../../paper_2201_02250_gb300/csrc/small_eig.cuh"

using namespace a2ls::se;

int main() {
  int m;
  if (std::scanf("%d", &m) != 1) return 1;
  const int ld = m + 1;
  std::vector<double> H(m * ld), Q(m * ld, 0.0), v(m), wr(m), wi(m), x(m), y(m), mod(m);
  std::vector<int> perm(m);
  for (int r = 0; r < m; ++r)
    for (int c = 0; c < m; ++c)
      if (std::scanf("%lf", &H[r * ld + c]) != 1) return 1;
  for (int r = 0; r < m; ++r) Q[r * ld + r] = 1.0;
  const std::vector<double> H0 = H;
  double hn = 0.0;
  for (int e = 0; e < m * m; ++e) hn = std::fmax(hn, std::fabs(H[(e / m) * ld + e % m]));
  const Team t{0, 1};
  hessenberg(H.data(), ld, Q.data(), ld, m, v.data(), t);
  const int rc = schur(H.data(), ld, Q.data(), ld, m, hn, t);
  schur_eigenvalues(H.data(), ld, m, wr.data(), wi.data());
  order_by_modulus(wr.data(), wi.data(), m, perm.data(), mod.data());
  std::printf("%d\n", rc);
  for (int j = 0; j < m; ++j) std::printf("%.17g %.17g\n", wr[perm[j]], wi[perm[j]]);
  double snorm = 0.0;
  for (int e = 0; e < m * m; ++e) snorm = std::fmax(snorm, std::fabs(H[(e / m) * ld + e % m]));
  const int nvec = m < 8 ? m : 8;
  for (int j = 0; j < nvec; ++j) {
    const int p = perm[j];
    if (wi[p] < 0) continue;
    schur_vector(H.data(), ld, m, p, wr[p], wi[p] > 0 ? wi[p] : 0.0, x.data(), y.data(), snorm);
    std::vector<double> zr(m), zi(m);
    for (int a = 0; a < m; ++a) {
      double sr = 0, si = 0;
      for (int c = 0; c < m; ++c) {
        sr += Q[a * ld + c] * x[c];
        si += Q[a * ld + c] * y[c];
      }
      zr[a] = sr;
      zi[a] = si;
    }
    double res = 0, nz = 0;
    for (int a = 0; a < m; ++a) {
      double hr = 0, hi = 0;
      for (int c = 0; c < m; ++c) {
        hr += H0[a * ld + c] * zr[c];
        hi += H0[a * ld + c] * zi[c];
      }
      const double rr = hr - (wr[p] * zr[a] - wi[p] * zi[a]);
      const double ri = hi - (wr[p] * zi[a] + wi[p] * zr[a]);
      res += rr * rr + ri * ri;
      nz += zr[a] * zr[a] + zi[a] * zi[a];
    }
    std::printf("res %.6e\n", std::sqrt(res / nz));
  }
  return 0;
}
