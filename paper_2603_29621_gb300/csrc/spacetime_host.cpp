// Temporal matrices of DG(r) on right Gauss--Radau points (see spacetime.hpp).
#include <algorithm>
#include <array>
#include <cmath>
#include <map>

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

std::vector<StLevelSpec> stmg_sequence(int k, int r, int n_forests, bool time_steps) {
  std::vector<StLevelSpec> seq;
  StLevelSpec s;
  s.k = k;
  s.r = r;
  s.forest = 0;
  seq.push_back(s);
  while (seq.back().k > 2) {
    s = seq.back();
    s.k = std::max(2, s.k / 2);
    seq.push_back(s);
  }
  for (int i = 1; i < n_forests; ++i) {
    s = seq.back();
    s.forest = i;
    seq.push_back(s);
  }
  while (time_steps && seq.back().r > 0) {
    s = seq.back();
    s.r = s.r / 2;
    seq.push_back(s);
  }
  return seq;
}

bool vertex_star_covers_all(const Forest& f) {
  const int dim = f.dim;
  const int L = f.max_level();
  std::map<std::array<int64_t, 3>, int64_t> count;
  int64_t best = 0;
  for (size_t c = 0; c < f.n_cells(); ++c) {
    const int64_t s = int64_t(1) << (L - f.lev[c]);
    for (int a = 0; a < (1 << dim); ++a) {
      std::array<int64_t, 3> key = {0, 0, 0};
      for (int d = 0; d < dim; ++d) key[d] = (f.crd[3 * c + d] + ((a >> d) & 1)) * s;
      best = std::max(best, ++count[key]);
    }
  }
  return best == (int64_t)f.n_cells();
}

std::vector<std::vector<int32_t>> vertex_star_patches(const Forest& f, const NodeSpace& nu, const NodeSpace& np) {
  const int dim = f.dim;
  const size_t nc = f.n_cells();
  const int L = f.max_level();
  const int64_t n_main = nu.n_nodes * dim;
  // holding cells of every node (compressed rows), one table per field
  auto holders = [&](const NodeSpace& ns, std::vector<int64_t>& ptr, std::vector<int32_t>& idx) {
    ptr.assign(ns.n_nodes + 1, 0);
    for (size_t c = 0; c < nc; ++c)
      for (int b = 0; b < ns.nb; ++b) ptr[ns.cell_nodes[c * ns.nb + b] + 1]++;
    for (int64_t g = 0; g < ns.n_nodes; ++g) ptr[g + 1] += ptr[g];
    idx.assign(ptr[ns.n_nodes], 0);
    std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
    for (size_t c = 0; c < nc; ++c)
      for (int b = 0; b < ns.nb; ++b) idx[fill[ns.cell_nodes[c * ns.nb + b]]++] = (int32_t)c;
  };
  std::vector<int64_t> pu, pp;
  std::vector<int32_t> iu, ip;
  holders(nu, pu, iu);
  holders(np, pp, ip);
  std::vector<char> hang_u(nu.n_nodes, 0), hang_p(np.n_nodes, 0);
  for (int32_t g : nu.hang_node) hang_u[g] = 1;
  for (int32_t g : np.hang_node) hang_p[g] = 1;
  // stars: corner position (finest-lattice units) -> cells
  std::map<std::array<int64_t, 3>, std::vector<int32_t>> stars;
  for (size_t c = 0; c < nc; ++c) {
    const int64_t s = int64_t(1) << (L - f.lev[c]);
    for (int a = 0; a < (1 << dim); ++a) {
      std::array<int64_t, 3> key = {0, 0, 0};
      for (int d = 0; d < dim; ++d) key[d] = (f.crd[3 * c + d] + ((a >> d) & 1)) * s;
      stars[key].push_back((int32_t)c);
    }
  }
  std::vector<std::vector<int32_t>> out;
  std::vector<char> in_star(nc, 0);
  for (auto& kv : stars) {
    const std::vector<int32_t>& cells = kv.second;
    for (int32_t c : cells) in_star[c] = 1;
    std::vector<int32_t> patch;
    auto inside = [&](const std::vector<int64_t>& ptr, const std::vector<int32_t>& idx, int32_t g) {
      for (int64_t j = ptr[g]; j < ptr[g + 1]; ++j)
        if (!in_star[idx[j]]) return false;
      return true;
    };
    std::vector<int32_t> nodes_u, nodes_p;
    for (int32_t c : cells) {
      for (int b = 0; b < nu.nb; ++b) nodes_u.push_back(nu.cell_nodes[(size_t)c * nu.nb + b]);
      for (int b = 0; b < np.nb; ++b) nodes_p.push_back(np.cell_nodes[(size_t)c * np.nb + b]);
    }
    std::sort(nodes_u.begin(), nodes_u.end());
    nodes_u.erase(std::unique(nodes_u.begin(), nodes_u.end()), nodes_u.end());
    std::sort(nodes_p.begin(), nodes_p.end());
    nodes_p.erase(std::unique(nodes_p.begin(), nodes_p.end()), nodes_p.end());
    for (int32_t g : nodes_u)
      if (!nu.boundary[g] && !hang_u[g] && inside(pu, iu, g))
        for (int c = 0; c < dim; ++c) patch.push_back((int32_t)(g * dim + c));
    for (int32_t g : nodes_p)
      if (!hang_p[g] && inside(pp, ip, g)) patch.push_back((int32_t)(n_main + g));
    for (int32_t c : cells) in_star[c] = 0;
    if (!patch.empty()) {
      std::sort(patch.begin(), patch.end());
      out.push_back(std::move(patch));
    }
  }
  return out;
}

bool invert_dense_rel(std::vector<double>& A, int64_t n, double rel_tol) {
  double amax = 0.0;
  for (double v : A) amax = std::max(amax, std::fabs(v));
  if (amax == 0.0) return false;
  std::vector<double> I((size_t)n * n, 0.0);
  for (int64_t i = 0; i < n; ++i) I[i * n + i] = 1.0;
  for (int64_t c = 0; c < n; ++c) {
    int64_t piv = c;
    for (int64_t r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (std::fabs(A[piv * n + c]) <= rel_tol * amax) return false;
    if (piv != c)
      for (int64_t j = 0; j < n; ++j) {
        std::swap(A[c * n + j], A[piv * n + j]);
        std::swap(I[c * n + j], I[piv * n + j]);
      }
    const double inv = 1.0 / A[c * n + c];
    for (int64_t j = 0; j < n; ++j) {
      A[c * n + j] *= inv;
      I[c * n + j] *= inv;
    }
    for (int64_t r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[r * n + c];
      if (f == 0.0) continue;
      for (int64_t j = 0; j < n; ++j) {
        A[r * n + j] -= f * A[c * n + j];
        I[r * n + j] -= f * I[c * n + j];
      }
    }
  }
  A.swap(I);
  return true;
}

int colour_patches_for_probing(const Forest& f, const NodeSpace& nu, const NodeSpace& np,
                               const std::vector<std::vector<int32_t>>& patches, std::vector<int32_t>& colour) {
  const int dim = f.dim;
  const size_t nc = f.n_cells();
  const int64_t n_main = nu.n_nodes * dim;
  // cells reached by a node of a field: cells holding it, and cells holding a hanging node of
  // which it is a master (compressed rows)
  auto reach_table = [&](const NodeSpace& ns, std::vector<int64_t>& ptr, std::vector<int32_t>& idx) {
    std::vector<std::vector<int32_t>> hang_of(ns.n_nodes);  // master -> hanging nodes
    for (size_t i = 0; i < ns.hang_node.size(); ++i)
      for (int32_t j = ns.hang_ptr[i]; j < ns.hang_ptr[i + 1]; ++j) hang_of[ns.hang_master[j]].push_back(ns.hang_node[i]);
    std::vector<std::vector<int32_t>> held(ns.n_nodes);
    for (size_t c = 0; c < nc; ++c)
      for (int b = 0; b < ns.nb; ++b) held[ns.cell_nodes[c * ns.nb + b]].push_back((int32_t)c);
    ptr.assign(ns.n_nodes + 1, 0);
    idx.clear();
    for (int64_t g = 0; g < ns.n_nodes; ++g) {
      std::vector<int32_t> cs = held[g];
      for (int32_t h : hang_of[g]) cs.insert(cs.end(), held[h].begin(), held[h].end());
      std::sort(cs.begin(), cs.end());
      cs.erase(std::unique(cs.begin(), cs.end()), cs.end());
      idx.insert(idx.end(), cs.begin(), cs.end());
      ptr[g + 1] = (int64_t)idx.size();
    }
  };
  std::vector<int64_t> pu, pp;
  std::vector<int32_t> iu, ip;
  reach_table(nu, pu, iu);
  reach_table(np, pp, ip);
  // cells reached by every patch
  std::vector<std::vector<int32_t>> reach(patches.size());
  for (size_t p = 0; p < patches.size(); ++p) {
    std::vector<int32_t>& R = reach[p];
    for (int32_t e : patches[p]) {
      if (e < n_main) {
        const int32_t g = e / dim;
        R.insert(R.end(), iu.begin() + pu[g], iu.begin() + pu[g + 1]);
      } else {
        const int32_t g = (int32_t)(e - n_main);
        R.insert(R.end(), ip.begin() + pp[g], ip.begin() + pp[g + 1]);
      }
    }
    std::sort(R.begin(), R.end());
    R.erase(std::unique(R.begin(), R.end()), R.end());
  }
  // greedy: a patch takes the lowest colour not used by a patch reaching one of its cells (two
  // patches couple an entry pair only through a cell both reach)
  std::vector<std::vector<int32_t>> cell_colours(nc);
  colour.assign(patches.size(), -1);
  int ncol = 0;
  std::vector<char> used;
  for (size_t p = 0; p < patches.size(); ++p) {
    used.assign(ncol + 1, 0);
    for (int32_t c : reach[p])
      for (int32_t col : cell_colours[c]) used[col] = 1;
    int col = 0;
    while (used[col]) ++col;
    colour[p] = col;
    ncol = std::max(ncol, col + 1);
    for (int32_t c : reach[p]) cell_colours[c].push_back(col);
  }
  return ncol;
}

}  // namespace mfns
