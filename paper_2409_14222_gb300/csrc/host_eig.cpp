// Eigenvalues of a small real upper-Hessenberg matrix by the shifted QR algorithm in complex
// arithmetic (Wilkinson shifts, Givens rotations, deflation from the bottom; Golub and Van Loan,
// "Matrix Computations", Sec. 7.5).  Used for the Ritz values of the Arnoldi process that estimates
// the largest eigenvalue of the Vanka-preconditioned operator (Chebyshev interval, Sec. 3).
#include <cmath>
#include <complex>
#include <vector>

#include "vk_internal.h"

namespace vk {

int hessenberg_eigenvalues(int m, const double* Hin, double* re, double* im) {
  using cd = std::complex<double>;
  if (m <= 0) return 0;
  std::vector<cd> H(size_t(m) * m);
  for (int i = 0; i < m * m; ++i) H[i] = Hin[i];
  auto at = [&](int i, int j) -> cd& { return H[size_t(i) * m + j]; };
  double hnorm = 0.0;
  for (int i = 0; i < m * m; ++i) hnorm = std::max(hnorm, std::abs(H[i]));
  const double eps = 2.220446049250313e-16;
  int n = m, iter = 0, total = 0;
  while (n > 0) {
    if (n == 1) {
      re[0] = at(0, 0).real();
      im[0] = at(0, 0).imag();
      break;
    }
    int l = n - 1;
    for (; l > 0; --l) {
      double s = std::abs(at(l, l)) + std::abs(at(l - 1, l - 1));
      if (s == 0.0) s = hnorm;
      if (std::abs(at(l, l - 1)) <= eps * s) break;
    }
    if (l == n - 1) {
      re[n - 1] = at(n - 1, n - 1).real();
      im[n - 1] = at(n - 1, n - 1).imag();
      --n;
      iter = 0;
      continue;
    }
    if (++total > 60 * m) return -1;
    // Wilkinson shift: eigenvalue of the trailing 2x2 block nearer to its last diagonal entry
    cd a = at(n - 2, n - 2), b = at(n - 2, n - 1), c = at(n - 1, n - 2), d = at(n - 1, n - 1);
    cd half = 0.5 * (a + d), disc = std::sqrt(0.25 * (a - d) * (a - d) + b * c);
    cd mu1 = half + disc, mu2 = half - disc;
    cd mu = std::abs(mu1 - d) < std::abs(mu2 - d) ? mu1 : mu2;
    if (iter == 10 || iter == 20) mu = d + 1.5 * std::abs(c);  // exceptional shift
    ++iter;
    // one QR step on the active block l..n-1: H - mu I = Q R, H <- R Q + mu I
    for (int i = l; i < n; ++i) at(i, i) -= mu;
    std::vector<cd> cs(n), sn(n);
    for (int i = l; i < n - 1; ++i) {
      cd x = at(i, i), y = at(i + 1, i);
      double r = std::hypot(std::abs(x), std::abs(y));
      cd cc = r == 0.0 ? cd(1.0) : x / r, ss = r == 0.0 ? cd(0.0) : y / r;
      cs[i] = cc;
      sn[i] = ss;
      for (int j = i; j < n; ++j) {  // rows i, i+1 <- [conj(c) conj(s); -s c] [row_i; row_i+1]
        cd u = at(i, j), v = at(i + 1, j);
        at(i, j) = std::conj(cc) * u + std::conj(ss) * v;
        at(i + 1, j) = -ss * u + cc * v;
      }
    }
    for (int i = l; i < n - 1; ++i) {  // columns i, i+1 <- [col_i, col_i+1] [c -conj(s); s conj(c)]
      cd cc = cs[i], ss = sn[i];
      for (int r = l; r <= std::min(i + 1, n - 1); ++r) {
        cd u = at(r, i), v = at(r, i + 1);
        at(r, i) = u * cc + v * ss;
        at(r, i + 1) = -u * std::conj(ss) + v * std::conj(cc);
      }
    }
    for (int i = l; i < n; ++i) at(i, i) += mu;
  }
  return 0;
}

}  // namespace vk
