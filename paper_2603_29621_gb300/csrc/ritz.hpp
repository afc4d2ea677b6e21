// Host helpers for the smoother bounds: eigenvalues (Ritz values) of the small Hessenberg matrix
// of an Arnoldi run, and the relaxation weight they imply.
#pragma once
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace mfns {

// Eigenvalues of an m x m upper Hessenberg matrix (row-major; entries below the subdiagonal are
// ignored) by the shifted QR algorithm in complex arithmetic: Givens rotations reduce H - mu I
// to triangular form and are applied back from the right (H <- R Q + mu I), with the shift
// taken from the trailing 2 x 2 block (the eigenvalue closer to its last diagonal entry) and
// deflation whenever a subdiagonal entry becomes negligible.
inline std::vector<std::complex<double>> hessenberg_eigenvalues(const std::vector<double>& Hr, int m) {
  using C = std::complex<double>;
  std::vector<C> H((size_t)m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) H[(size_t)i * m + j] = (j >= i - 1) ? C(Hr[(size_t)i * m + j], 0.0) : C(0.0, 0.0);
  auto at = [&](int i, int j) -> C& { return H[(size_t)i * m + j]; };
  std::vector<C> eig;
  std::vector<double> cs(m);
  std::vector<C> sn(m);
  int hi = m - 1, iter = 0, total = 0;
  const double eps = 1e-14;
  while (hi >= 0 && total < 100 * m + 1000) {
    if (hi == 0) {
      eig.push_back(at(0, 0));
      --hi;
      continue;
    }
    int l = hi;
    while (l > 0 && std::abs(at(l, l - 1)) > eps * (std::abs(at(l, l)) + std::abs(at(l - 1, l - 1)))) --l;
    if (l == hi) {  // the last diagonal entry has split off
      eig.push_back(at(hi, hi));
      --hi;
      iter = 0;
      continue;
    }
    // shift: eigenvalue of the trailing 2 x 2 block closer to its last diagonal entry
    const C a = at(hi - 1, hi - 1), b = at(hi - 1, hi), c = at(hi, hi - 1), d = at(hi, hi);
    const C half = 0.5 * (a + d), disc = std::sqrt(0.25 * (a - d) * (a - d) + b * c);
    C mu = std::abs(half + disc - d) < std::abs(half - disc - d) ? half + disc : half - disc;
    if (iter > 0 && iter % 10 == 0) mu = d + C(std::abs(c), 0.0);  // exceptional shift against cycling
    for (int k = l; k <= hi; ++k) at(k, k) -= mu;
    // H - mu I = Q R on the active block (rows l..hi), rotations G_k zero H(k+1, k)
    for (int k = l; k < hi; ++k) {
      const C x = at(k, k), y = at(k + 1, k);
      const double ax = std::abs(x), nrm = std::hypot(ax, std::abs(y));
      double ck;
      C sk;
      if (nrm == 0.0) {
        ck = 1.0;
        sk = 0.0;
      } else if (ax == 0.0) {
        ck = 0.0;
        sk = std::conj(y) / std::abs(y);
      } else {
        ck = ax / nrm;
        sk = (x / ax) * std::conj(y) / nrm;
      }
      cs[k] = ck;
      sn[k] = sk;
      for (int j = k; j <= hi; ++j) {
        const C t1 = at(k, j), t2 = at(k + 1, j);
        at(k, j) = ck * t1 + sk * t2;
        at(k + 1, j) = -std::conj(sk) * t1 + ck * t2;
      }
    }
    // R Q: the conjugate transposes of the rotations from the right (columns k, k+1)
    for (int k = l; k < hi; ++k) {
      const double ck = cs[k];
      const C sk = sn[k];
      for (int i = l; i <= std::min(k + 1, hi); ++i) {
        const C t1 = at(i, k), t2 = at(i, k + 1);
        at(i, k) = t1 * ck + t2 * std::conj(sk);
        at(i, k + 1) = -t1 * sk + t2 * ck;
      }
    }
    for (int k = l; k <= hi; ++k) at(k, k) += mu;
    ++iter;
    ++total;
  }
  return eig;  // fewer than m values only if the iteration limit was reached
}

// Relaxation weight omega > 0 minimising max |1 - omega theta| over the eigenvalue estimates
// theta in the upper half of the spectrum (|theta| >= rho / 2), the modes the smoother must damp.
// The maximum of the convex functions |1 - omega theta| is convex in omega: golden-section search
// on (0, 2 / min |theta|].  Returns 0 when no estimate is usable.
inline double relaxation_weight(const std::vector<std::complex<double>>& theta) {
  double rho = 0.0;
  for (const auto& t : theta) rho = std::max(rho, std::abs(t));
  if (!(rho > 0.0) || !std::isfinite(rho)) return 0.0;
  std::vector<std::complex<double>> S;
  double amin = rho;
  for (const auto& t : theta)
    if (std::abs(t) >= 0.5 * rho) {
      S.push_back(t);
      amin = std::min(amin, std::abs(t));
    }
  auto f = [&](double w) {
    double m = 0.0;
    for (const auto& t : S) m = std::max(m, std::abs(1.0 - w * t));
    return m;
  };
  double lo = 0.0, hi = 2.0 / amin;
  const double g = 0.5 * (std::sqrt(5.0) - 1.0);
  double x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo), f1 = f(x1), f2 = f(x2);
  for (int it = 0; it < 200; ++it) {
    if (f1 <= f2) {
      hi = x2;
      x2 = x1;
      f2 = f1;
      x1 = hi - g * (hi - lo);
      f1 = f(x1);
    } else {
      lo = x1;
      x1 = x2;
      f1 = f2;
      x2 = lo + g * (hi - lo);
      f2 = f(x2);
    }
  }
  return 0.5 * (lo + hi);
}

}  // namespace mfns
