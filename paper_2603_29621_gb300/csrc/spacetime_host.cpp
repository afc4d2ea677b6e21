// Temporal matrices of DG(r) on right Gauss--Radau points (see spacetime.hpp).
#include <cmath>

#include "mesh.hpp"
#include "spacetime.hpp"

namespace mfns {

namespace {

// P_n(x) by the three-term recurrence.
double legendre_value(int n, double x) {
  if (n == 0) return 1.0;
  double p0 = 1.0, p1 = x;
  for (int m = 2; m <= n; ++m) {
    const double p2 = ((2.0 * m - 1.0) * x * p1 - (m - 1.0) * p0) / m;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

// Solves the dense system A X = B (A n x n, B n x m, row-major) in place by Gaussian elimination
// with partial pivoting; false if A is singular.
bool solve_dense(std::vector<double> A, std::vector<double>& B, int n, int m) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[p * n + c])) p = r;
    if (std::fabs(A[p * n + c]) < 1e-300) return false;
    if (p != c) {
      for (int j = 0; j < n; ++j) std::swap(A[c * n + j], A[p * n + j]);
      for (int j = 0; j < m; ++j) std::swap(B[c * m + j], B[p * m + j]);
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[r * n + c] / A[c * n + c];
      if (f == 0.0) continue;
      for (int j = c; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
      for (int j = 0; j < m; ++j) B[r * m + j] -= f * B[c * m + j];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int j = 0; j < m; ++j) B[r * m + j] /= A[r * n + r];
  return true;
}

}  // namespace

std::vector<double> radau_right(int Q) {
  std::vector<double> t;
  if (Q <= 0) return t;
  // the right Radau points on [-1, 1] are the roots of P_Q - P_{Q-1}; x = 1 is one of them, the
  // Q - 1 others are simple roots in (-1, 1): bracket them on a fine grid, then bisect
  auto f = [Q](double x) { return legendre_value(Q, x) - legendre_value(Q - 1, x); };
  const int grid = 64 * Q * Q;
  const double hi_end = 1.0 - 1.0 / (4.0 * grid);
  double a = -1.0, fa = f(a);
  for (int i = 1; i <= grid && (int)t.size() < Q - 1; ++i) {
    const double b = -1.0 + (hi_end + 1.0) * i / grid, fb = f(b);
    if ((fa < 0) != (fb < 0)) {
      double lo = a, hi = b, flo = fa;
      for (int it = 0; it < 200 && hi - lo > 1e-17; ++it) {
        const double mid = 0.5 * (lo + hi), fm = f(mid);
        if ((fm < 0) == (flo < 0)) {
          lo = mid;
          flo = fm;
        } else {
          hi = mid;
        }
      }
      t.push_back(0.5 * (0.5 * (lo + hi) + 1.0));
    }
    a = b;
    fa = fb;
  }
  t.push_back(1.0);
  return t;
}

bool temporal_matrices(int r, TemporalMatrices& out, std::string* err) {
  if (r < 0 || r > 7) {
    if (err) *err = "temporal degree must lie in 0..7";
    return false;
  }
  const int Q = r + 1;
  out = TemporalMatrices();
  out.Q = Q;
  out.t = radau_right(Q);
  if ((int)out.t.size() != Q) {
    if (err) *err = "Radau points not found";
    return false;
  }
  std::vector<double> xg, wg;
  gauss_rule(Q + 1, xg, wg);  // exact for the degree-2Q polynomials integrated here
  out.M.assign(Q * Q, 0.0);
  out.A.assign(Q * Q, 0.0);
  out.m.assign(Q, 0.0);
  for (int j = 0; j < Q; ++j) {
    out.m[j] = lagrange(out.t, j, 0.0);
    for (int i = 0; i < Q; ++i) {
      double mij = 0.0, aij = 0.0;
      for (size_t g = 0; g < xg.size(); ++g) {
        const double pj = lagrange(out.t, j, xg[g]);
        mij += wg[g] * lagrange(out.t, i, xg[g]) * pj;
        aij += wg[g] * lagrange_deriv(out.t, i, xg[g]) * pj;
      }
      out.M[j * Q + i] = mij;
      out.A[j * Q + i] = aij + lagrange(out.t, i, 0.0) * out.m[j];
    }
  }
  out.G = out.A;
  if (!solve_dense(out.M, out.G, Q, Q)) {
    if (err) *err = "singular temporal mass matrix";
    return false;
  }
  return true;
}

std::vector<double> time_prolongation(int rc, int rf) {
  const std::vector<double> tc = radau_right(rc + 1), tf = radau_right(rf + 1);
  std::vector<double> P((size_t)(rf + 1) * (rc + 1));
  for (int i = 0; i <= rf; ++i)
    for (int j = 0; j <= rc; ++j) P[(size_t)i * (rc + 1) + j] = lagrange(tc, j, tf[i]);
  return P;
}

}  // namespace mfns
