// Host-side geometry (see mesh.hpp).
#include "mesh.hpp"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <stdexcept>

namespace mfns {

// ---------------------------------------------------------------- 1D helpers
static void legendre(int n, double x, double& p, double& dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { p = 1.0; dp = 0.0; return; }
  for (int m = 1; m < n; ++m) {
    double p2 = ((2.0 * m + 1.0) * x * p1 - m * p0) / (m + 1.0);
    p0 = p1;
    p1 = p2;
  }
  p = p1;
  dp = n * (x * p1 - p0) / (x * x - 1.0);
}

std::vector<double> gll_nodes(int k) {
  std::vector<double> t(k + 1);
  t[0] = -1.0;
  t[k] = 1.0;
  for (int j = 1; j < k; ++j) {
    double x = -std::cos(M_PI * j / k);
    for (int it = 0; it < 100; ++it) {  // Newton on P_k'(x) using the Legendre ODE for P_k''
      double p, dp;
      legendre(k, x, p, dp);
      double d2p = (2.0 * x * dp - k * (k + 1.0) * p) / (1.0 - x * x);
      double dx = dp / d2p;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    t[j] = x;
  }
  std::vector<double> out(k + 1);
  for (int j = 0; j <= k; ++j) out[j] = 0.5 * (t[j] + 1.0);
  for (int j = 0; j <= k; ++j) out[j] = 0.5 * (out[j] + (1.0 - out[k - j]));  // exact symmetry
  if (k % 2 == 0) out[k / 2] = 0.5;
  out[0] = 0.0;
  out[k] = 1.0;
  return out;
}

void gauss_rule(int q, std::vector<double>& x, std::vector<double>& w) {
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  for (int i = 0; i < q; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (q + 0.5));
    double p = 0, dp = 1;
    for (int it = 0; it < 100; ++it) {
      legendre(q, t, p, dp);
      double dt = p / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    legendre(q, t, p, dp);
    x[q - 1 - i] = 0.5 * (t + 1.0);
    w[q - 1 - i] = 1.0 / ((1.0 - t * t) * dp * dp);  // 2/((1-t^2) P'^2) halved for [0,1]
  }
  for (int i = 0; i < q; ++i) {  // symmetrise
    double xs = 0.5 * (x[i] + 1.0 - x[q - 1 - i]);
    double ws = 0.5 * (w[i] + w[q - 1 - i]);
    x[i] = xs;
    w[i] = ws;
  }
  for (int i = 0; i < q; ++i) x[q - 1 - i] = 1.0 - x[i];
  if (q % 2 == 1) x[q / 2] = 0.5;
}

double lagrange(const std::vector<double>& nodes, int a, double x) {
  double v = 1.0;
  for (size_t m = 0; m < nodes.size(); ++m)
    if ((int)m != a) v *= (x - nodes[m]) / (nodes[a] - nodes[m]);
  return v;
}

double lagrange_deriv(const std::vector<double>& nodes, int a, double x) {
  double s = 0.0;
  for (size_t m = 0; m < nodes.size(); ++m) {
    if ((int)m == a) continue;
    double t = 1.0 / (nodes[a] - nodes[m]);
    for (size_t n = 0; n < nodes.size(); ++n)
      if ((int)n != a && n != m) t *= (x - nodes[n]) / (nodes[a] - nodes[n]);
    s += t;
  }
  return s;
}

// ---------------------------------------------------------------- forests
int Forest::max_level() const {
  int L = 0;
  for (int l : lev) L = std::max(L, l);
  return L;
}

double Forest::h(size_t c) const { return 1.0 / (double(n) * double(1u << lev[c])); }

void Forest::sort() {
  std::vector<size_t> idx(lev.size());
  std::iota(idx.begin(), idx.end(), 0);
  std::sort(idx.begin(), idx.end(), [&](size_t a, size_t b) {
    if (lev[a] != lev[b]) return lev[a] < lev[b];
    for (int d = 2; d >= 0; --d)
      if (crd[3 * a + d] != crd[3 * b + d]) return crd[3 * a + d] < crd[3 * b + d];
    return false;
  });
  std::vector<int32_t> l2(lev.size()), c2(crd.size());
  for (size_t i = 0; i < idx.size(); ++i) {
    l2[i] = lev[idx[i]];
    for (int d = 0; d < 3; ++d) c2[3 * i + d] = crd[3 * idx[i] + d];
  }
  lev.swap(l2);
  crd.swap(c2);
}

Forest forest_uniform(int dim, int n) {
  Forest f;
  f.dim = dim;
  f.n = n;
  int nz = dim == 3 ? n : 1;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        f.lev.push_back(0);
        f.crd.push_back(i);
        f.crd.push_back(j);
        f.crd.push_back(k);
      }
  return f;
}

Forest forest_refine(const Forest& f, const std::vector<char>& mask) {
  Forest g;
  g.dim = f.dim;
  g.n = f.n;
  int nk = 1 << f.dim;
  for (size_t c = 0; c < f.n_cells(); ++c) {
    if (!mask[c]) {
      g.lev.push_back(f.lev[c]);
      for (int d = 0; d < 3; ++d) g.crd.push_back(f.crd[3 * c + d]);
      continue;
    }
    for (int ch = 0; ch < nk; ++ch) {
      g.lev.push_back(f.lev[c] + 1);
      for (int d = 0; d < 3; ++d) g.crd.push_back(d < f.dim ? 2 * f.crd[3 * c + d] + ((ch >> d) & 1) : 0);
    }
  }
  g.sort();
  return g;
}

Lattice make_lattice(const Forest& f) {
  Lattice lat;
  lat.dim = f.dim;
  int L = f.max_level();
  lat.N = f.n << L;
  size_t N = lat.N;
  size_t nz = f.dim == 3 ? N : 1;
  lat.cell.assign(N * N * nz, -1);
  for (size_t c = 0; c < f.n_cells(); ++c) {
    int s = 1 << (L - f.lev[c]);
    int x0 = f.crd[3 * c] * s, y0 = f.crd[3 * c + 1] * s, z0 = f.dim == 3 ? f.crd[3 * c + 2] * s : 0;
    int sz = f.dim == 3 ? s : 1;
    for (int k = 0; k < sz; ++k)
      for (int j = 0; j < s; ++j)
        for (int i = 0; i < s; ++i)
          lat.cell[(size_t)(x0 + i) + N * ((size_t)(y0 + j) + N * (size_t)(z0 + k))] = (int32_t)c;
  }
  if (!f.partial)
    for (int32_t v : lat.cell)
      if (v < 0) throw std::runtime_error("forest does not cover the domain");
  return lat;
}

Forest forest_level(const Forest& f, int l) {
  Forest out;
  out.dim = f.dim;
  out.n = f.n;
  out.partial = true;
  std::vector<std::array<int32_t, 3>> cells;
  for (size_t c = 0; c < f.n_cells(); ++c) {
    const int sh = f.lev[c] - l;
    if (sh < 0) continue;
    cells.push_back({f.crd[3 * c] >> sh, f.crd[3 * c + 1] >> sh, f.crd[3 * c + 2] >> sh});
  }
  std::sort(cells.begin(), cells.end());
  cells.erase(std::unique(cells.begin(), cells.end()), cells.end());
  for (auto& c : cells) {
    out.lev.push_back(l);
    for (int d = 0; d < 3; ++d) out.crd.push_back(c[d]);
  }
  out.sort();
  return out;
}

bool ls_owned_nodes(const Forest& fine, const NodeSpace& fns, const Forest& lf, const NodeSpace& lns,
                    const std::vector<uint8_t>& edge, int l, std::vector<int32_t>& owner,
                    std::vector<int32_t>& cf, std::vector<int32_t>& cl, std::string* err, bool own_boundary) {
  const int nb = fns.nb;
  if (lns.nb != nb || (int64_t)owner.size() != fns.n_nodes || (int64_t)edge.size() != lns.n_nodes) {
    if (err) *err = "inconsistent node spaces";
    return false;
  }
  std::vector<char> hang(fns.n_nodes, 0);
  for (int32_t g : fns.hang_node) hang[g] = 1;
  std::vector<std::pair<std::array<int32_t, 3>, int32_t>> at(lf.n_cells());
  for (size_t c = 0; c < lf.n_cells(); ++c) at[c] = {{lf.crd[3 * c], lf.crd[3 * c + 1], lf.crd[3 * c + 2]}, (int32_t)c};
  std::sort(at.begin(), at.end());
  for (size_t c = 0; c < fine.n_cells(); ++c) {
    if (fine.lev[c] != l) continue;
    const std::array<int32_t, 3> key = {fine.crd[3 * c], fine.crd[3 * c + 1], fine.crd[3 * c + 2]};
    auto it = std::lower_bound(at.begin(), at.end(), std::make_pair(key, int32_t(-1)));
    if (it == at.end() || it->first != key) {
      if (err) *err = "active cell missing from its level";
      return false;
    }
    for (int b = 0; b < nb; ++b) {
      const int32_t gf = fns.cell_nodes[c * nb + b];
      if (fns.cell_master[c * nb + b] != gf || hang[gf]) continue;  // hanging
      if (fns.boundary[gf] && !own_boundary) continue;               // every component Dirichlet
      const int32_t gl = lns.cell_nodes[(size_t)it->second * nb + b];
      if (edge[gl]) continue;
      if (owner[gf] == l) continue;  // already listed from a neighbouring cell of this level
      if (owner[gf] >= 0) {
        if (err) *err = "a fine DoF owned by two levels";
        return false;
      }
      owner[gf] = l;
      cf.push_back(gf);
      cl.push_back(gl);
    }
  }
  return true;
}

bool ls_all_owned(const NodeSpace& fns, const std::vector<int32_t>& owner, bool own_boundary) {
  std::vector<char> hang(fns.n_nodes, 0);
  for (int32_t g : fns.hang_node) hang[g] = 1;
  for (int64_t g = 0; g < fns.n_nodes; ++g)
    if (!hang[g] && (own_boundary || !fns.boundary[g]) && owner[g] < 0) return false;
  return true;
}

std::vector<uint8_t> refinement_edge(const Forest& f, const NodeSpace& ns) {
  std::vector<uint8_t> edge(ns.n_nodes, 0);
  const size_t nc = f.n_cells();
  if (nc == 0) return edge;
  const int dim = f.dim, k = ns.k, np = k + 1, l = f.lev[0];
  const int64_t N = (int64_t)f.n << l;
  auto key = [&](const int64_t c[3]) { return c[0] + N * (c[1] + N * c[2]); };
  std::vector<int64_t> present(nc);
  for (size_t c = 0; c < nc; ++c) {
    if (f.lev[c] != l) throw std::runtime_error("refinement_edge: cells of different levels");
    const int64_t cc[3] = {f.crd[3 * c], f.crd[3 * c + 1], f.crd[3 * c + 2]};
    present[c] = key(cc);
  }
  std::sort(present.begin(), present.end());
  auto has = [&](const int64_t c[3]) { return std::binary_search(present.begin(), present.end(), key(c)); };
  for (size_t c = 0; c < nc; ++c)
    for (int b = 0; b < ns.nb; ++b) {
      const int s[3] = {b % np, (b / np) % np, dim == 3 ? b / (np * np) : 0};
      // the level cells whose closure holds the node: one or two per direction
      int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
      for (int d = 0; d < dim; ++d) {
        const int64_t cd = f.crd[3 * c + d];
        lo[d] = s[d] == 0 ? cd - 1 : cd;
        hi[d] = s[d] == k ? cd + 1 : cd;
      }
      bool on_edge = false;
      for (int64_t z = lo[2]; z <= hi[2] && !on_edge; ++z)
        for (int64_t y = lo[1]; y <= hi[1] && !on_edge; ++y)
          for (int64_t x = lo[0]; x <= hi[0] && !on_edge; ++x) {
            const int64_t cand[3] = {x, y, z};
            bool inside = true;
            for (int d = 0; d < dim; ++d) inside = inside && cand[d] >= 0 && cand[d] < N;
            if (inside && !has(cand)) on_edge = true;
          }
      if (on_edge) edge[ns.cell_nodes[c * ns.nb + b]] = 1;
    }
  return edge;
}

Forest forest_balance(Forest f) {
  while (true) {
    Lattice lat = make_lattice(f);
    int N = lat.N;
    int nz = f.dim == 3 ? N : 1;
    std::vector<char> need(f.n_cells(), 0);
    bool any = false;
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
          int32_t c = lat.at(i, j, k);
          int lc = f.lev[c];
          if (need[c]) continue;
          int kz0 = f.dim == 3 ? std::max(k - 1, 0) : 0, kz1 = f.dim == 3 ? std::min(k + 1, N - 1) : 0;
          for (int kk = kz0; kk <= kz1 && !need[c]; ++kk)
            for (int jj = std::max(j - 1, 0); jj <= std::min(j + 1, N - 1) && !need[c]; ++jj)
              for (int ii = std::max(i - 1, 0); ii <= std::min(i + 1, N - 1); ++ii)
                if (f.lev[lat.at(ii, jj, kk)] >= lc + 2) {
                  need[c] = 1;
                  any = true;
                  break;
                }
        }
    if (!any) return f;
    f = forest_refine(f, need);
  }
}

Forest forest_refine_ball(Forest f, const double centre[3], double radius, int levels) {
  for (int l = 0; l < levels; ++l) {
    std::vector<char> mask(f.n_cells(), 0);
    for (size_t c = 0; c < f.n_cells(); ++c) {
      if (f.lev[c] != l) continue;
      double h = f.h(c), r2 = 0.0;
      for (int d = 0; d < f.dim; ++d) {
        double x = (f.crd[3 * c + d] + 0.5) * h - centre[d];
        r2 += x * x;
      }
      mask[c] = std::sqrt(r2) < radius;
    }
    f = forest_refine(f, mask);
  }
  return forest_balance(f);
}

bool forest_can_coarsen(const Forest& f, int stop_n) {
  if (f.max_level() > 0) return true;
  return f.n > stop_n;
}

Forest forest_coarsen(const Forest& f) {
  int L = f.max_level();
  if (L == 0) return forest_uniform(f.dim, (f.n + 1) / 2);  // non-nested when n is odd
  Forest g;
  g.dim = f.dim;
  g.n = f.n;
  std::vector<std::array<int32_t, 3>> parents;
  for (size_t c = 0; c < f.n_cells(); ++c) {
    if (f.lev[c] == L) {
      parents.push_back({f.crd[3 * c] >> 1, f.crd[3 * c + 1] >> 1, f.crd[3 * c + 2] >> 1});
    } else {
      g.lev.push_back(f.lev[c]);
      for (int d = 0; d < 3; ++d) g.crd.push_back(f.crd[3 * c + d]);
    }
  }
  std::sort(parents.begin(), parents.end());
  parents.erase(std::unique(parents.begin(), parents.end()), parents.end());
  for (auto& p : parents) {
    g.lev.push_back(L - 1);
    for (int d = 0; d < 3; ++d) g.crd.push_back(p[d]);
  }
  g.sort();
  return g;
}

// ---------------------------------------------------------------- constraints
std::vector<uint32_t> constraint_masks(const Forest& f, const Lattice& lat) {
  int L = f.max_level(), N = lat.N, dim = f.dim;
  std::vector<uint32_t> mask(f.n_cells(), 0);
  for (size_t c = 0; c < f.n_cells(); ++c) {
    int l = f.lev[c];
    if (l == 0) continue;
    int s = 1 << (L - l);
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
      lo[d] = d < dim ? f.crd[3 * c + d] * s : 0;
      hi[d] = d < dim ? (f.crd[3 * c + d] + 1) * s : 1;
    }
    auto level_at = [&](const int p[3]) -> int {
      for (int d = 0; d < dim; ++d)
        if (p[d] < 0 || p[d] >= N) return 1 << 20;
      const int32_t id = lat.at(p[0], p[1], dim == 3 ? p[2] : 0);
      return id < 0 ? 1 << 20 : f.lev[id];  // a hole of a partial forest has no cell to hang from
    };
    uint32_t m = 0;
    for (int d = 0; d < dim; ++d)
      for (int side = 0; side < 2; ++side) {
        int p[3] = {lo[0], lo[1], lo[2]};
        p[d] = side ? hi[d] : lo[d] - 1;
        if (level_at(p) < l) m |= 1u << (2 * d + side);
      }
    if (dim == 3) {
      for (int d = 0; d < 3; ++d) {
        int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
        if (d1 > d2) std::swap(d1, d2);
        for (int s2 = 0; s2 < 2; ++s2)
          for (int s1 = 0; s1 < 2; ++s1) {
            int p[3] = {lo[0], lo[1], lo[2]};
            p[d1] = s1 ? hi[d1] : lo[d1] - 1;
            p[d2] = s2 ? hi[d2] : lo[d2] - 1;
            if (level_at(p) < l) m |= 1u << (6 + 4 * d + 2 * s2 + s1);
          }
      }
    }
    if (m)
      for (int d = 0; d < dim; ++d) m |= uint32_t(f.crd[3 * c + d] & 1) << (kChildShift + d);
    mask[c] = m;
  }
  return mask;
}

// Directions in which slot (s0,s1,s2) of a cell with mask m is interpolated.
static int slot_dirs(int dim, int k, uint32_t m, const int s[3]) {
  int dirs = 0;
  for (int d = 0; d < dim; ++d)
    for (int side = 0; side < 2; ++side)
      if ((m >> (2 * d + side)) & 1u)
        if (s[d] == (side ? k : 0)) dirs |= ((1 << dim) - 1) & ~(1 << d);
  if (dim == 3)
    for (int d = 0; d < 3; ++d) {
      int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
      if (d1 > d2) std::swap(d1, d2);
      for (int s2 = 0; s2 < 2; ++s2)
        for (int s1 = 0; s1 < 2; ++s1)
          if ((m >> (6 + 4 * d + 2 * s2 + s1)) & 1u)
            if (s[d1] == (s1 ? k : 0) && s[d2] == (s2 ? k : 0)) dirs |= 1 << d;
    }
  return dirs;
}

namespace {
struct Key {
  int64_t v[3];
  bool operator<(const Key& o) const {
    for (int d = 2; d >= 0; --d)
      if (v[d] != o.v[d]) return v[d] < o.v[d];
    return false;
  }
  bool operator==(const Key& o) const { return v[0] == o.v[0] && v[1] == o.v[1] && v[2] == o.v[2]; }
};
}  // namespace

NodeSpace make_nodes(const Forest& f, const Lattice& lat, const std::vector<uint32_t>& masks, int k,
                     std::string* err) {
  NodeSpace ns;
  int dim = f.dim;
  ns.dim = dim;
  ns.k = k;
  int np = k + 1;
  ns.nb = dim == 3 ? np * np * np : np * np;
  std::vector<double> xi = gll_nodes(k);
  size_t nc = f.n_cells();
  ns.cell_nodes.resize(nc * ns.nb);
  auto slot = [&](int b, int s[3]) {
    s[0] = b % np;
    s[1] = (b / np) % np;
    s[2] = dim == 3 ? b / (np * np) : 0;
  };
  if (f.uniform()) {
    ns.lexicographic = true;
    int64_t M = (int64_t)k * f.n + 1;
    int64_t Mz = dim == 3 ? M : 1;
    ns.n_nodes = M * M * Mz;
    ns.x.resize(ns.n_nodes * dim);
    ns.boundary.assign(ns.n_nodes, 0);
    for (int64_t g = 0; g < ns.n_nodes; ++g) {
      int64_t gi[3] = {g % M, (g / M) % M, g / (M * M)};
      bool bnd = false;
      for (int d = 0; d < dim; ++d) {
        int64_t c = gi[d] / k, a = gi[d] % k;
        if (c == f.n) { c = f.n - 1; a = k; }
        ns.x[g * dim + d] = (double(c) + xi[a]) / f.n;
        bnd |= gi[d] == 0 || gi[d] == M - 1;
      }
      ns.boundary[g] = bnd;
    }
    for (size_t c = 0; c < nc; ++c)
      for (int b = 0; b < ns.nb; ++b) {
        int s[3];
        slot(b, s);
        int64_t gi[3] = {0, 0, 0};
        for (int d = 0; d < dim; ++d) gi[d] = (int64_t)k * f.crd[3 * c + d] + s[d];
        ns.cell_nodes[c * ns.nb + b] = (int32_t)(gi[0] + M * (gi[1] + M * gi[2]));
      }
    ns.cell_master = ns.cell_nodes;
    ns.hang_ptr.assign(1, 0);
    return ns;
  }
  // general forest: identify nodes by exact keys
  int L = f.max_level();
  int64_t N = lat.N;
  std::vector<char> rational(np);
  for (int a = 0; a < np; ++a)
    rational[a] = std::fabs(xi[a]) < 1e-14 || std::fabs(xi[a] - 1.0) < 1e-14 || std::fabs(xi[a] - 0.5) < 1e-14;
  auto key1 = [&](int l, int64_t c, int a) -> int64_t {
    int64_t s = int64_t(1) << (L - l);
    if (rational[a]) return 2 * c * s + (int64_t)std::llround(2.0 * xi[a] * double(s));
    return -1 - (((int64_t)l * (N + 1) + c) * np + a);
  };
  auto cell_key = [&](int l, const int64_t c[3], const int s[3]) {
    Key key{{0, 0, 0}};
    for (int d = 0; d < dim; ++d) key.v[d] = key1(l, c[d], s[d]);
    return key;
  };
  std::vector<std::pair<Key, int64_t>> all(nc * ns.nb);
  for (size_t c = 0; c < nc; ++c) {
    int64_t cc[3] = {f.crd[3 * c], f.crd[3 * c + 1], f.crd[3 * c + 2]};
    for (int b = 0; b < ns.nb; ++b) {
      int s[3];
      slot(b, s);
      all[c * ns.nb + b] = {cell_key(f.lev[c], cc, s), (int64_t)(c * ns.nb + b)};
    }
  }
  std::sort(all.begin(), all.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  std::vector<Key> uniq;
  uniq.reserve(all.size() / 4);
  for (size_t i = 0; i < all.size(); ++i) {
    if (i == 0 || !(all[i].first == all[i - 1].first)) uniq.push_back(all[i].first);
    ns.cell_nodes[all[i].second] = (int32_t)(uniq.size() - 1);
  }
  ns.n_nodes = uniq.size();
  ns.x.assign(ns.n_nodes * dim, 0.0);
  ns.boundary.assign(ns.n_nodes, 0);
  for (size_t c = 0; c < nc; ++c) {
    double h = f.h(c);
    for (int b = 0; b < ns.nb; ++b) {
      int s[3];
      slot(b, s);
      int32_t g = ns.cell_nodes[c * ns.nb + b];
      for (int d = 0; d < dim; ++d) ns.x[(size_t)g * dim + d] = (f.crd[3 * c + d] + xi[s[d]]) * h;
    }
  }
  for (int64_t g = 0; g < ns.n_nodes; ++g)
    for (int d = 0; d < dim; ++d)
      if (uniq[g].v[d] == 0 || uniq[g].v[d] == 2 * N) ns.boundary[g] = 1;
  auto find = [&](const Key& key) -> int32_t {
    auto it = std::lower_bound(uniq.begin(), uniq.end(), key);
    if (it == uniq.end() || !(*it == key)) return -1;
    return (int32_t)(it - uniq.begin());
  };
  // 1D interpolation from a coarse edge to the child half h: P[h][s][m] = l_m((h + xi_s)/2)
  std::vector<double> P(2 * np * np);
  for (int h = 0; h < 2; ++h)
    for (int s = 0; s < np; ++s)
      for (int m = 0; m < np; ++m) P[(h * np + s) * np + m] = lagrange(xi, m, 0.5 * (h + xi[s]));
  ns.cell_master = ns.cell_nodes;
  std::vector<int32_t> hang_first(ns.n_nodes, -1);
  std::vector<std::vector<std::pair<int32_t, double>>> hang_list;
  std::vector<int32_t> hang_ids;
  for (size_t c = 0; c < nc; ++c) {
    uint32_t m = masks[c];
    if (!(m & 0x3FFFFu)) continue;
    int l = f.lev[c];
    int64_t pc[3] = {f.crd[3 * c] >> 1, f.crd[3 * c + 1] >> 1, f.crd[3 * c + 2] >> 1};
    int half[3] = {int((m >> kChildShift) & 1u), int((m >> (kChildShift + 1)) & 1u),
                   int((m >> (kChildShift + 2)) & 1u)};
    for (int b = 0; b < ns.nb; ++b) {
      int s[3];
      slot(b, s);
      int dirs = slot_dirs(dim, k, m, s);
      if (!dirs) continue;
      int ms[3] = {0, 0, 0};
      for (int d = 0; d < dim; ++d) {
        if ((dirs >> d) & 1) {
          ms[d] = s[d];
        } else {
          if (s[d] != 0 && s[d] != k) {
            if (err) *err = "constrained slot not on the cell boundary";
            return NodeSpace();
          }
          ms[d] = s[d];
        }
      }
      int32_t master = find(cell_key(l - 1, pc, ms));
      if (master < 0) {
        if (err) *err = "hanging-node master not found";
        return NodeSpace();
      }
      ns.cell_master[c * ns.nb + b] = master;
      // weights of the parent's face/edge nodes for this slot's own node
      std::vector<std::pair<int32_t, double>> w;
      int ext[3] = {1, 1, 1};
      for (int d = 0; d < dim; ++d) ext[d] = ((dirs >> d) & 1) ? np : 1;
      for (int t2 = 0; t2 < ext[2]; ++t2)
        for (int t1 = 0; t1 < ext[1]; ++t1)
          for (int t0 = 0; t0 < ext[0]; ++t0) {
            int t[3] = {t0, t1, t2};
            int mm[3] = {ms[0], ms[1], ms[2]};
            double wt = 1.0;
            for (int d = 0; d < dim; ++d)
              if ((dirs >> d) & 1) {
                mm[d] = t[d];
                wt *= P[(half[d] * np + s[d]) * np + t[d]];
              }
            if (std::fabs(wt) < 1e-14) continue;
            int32_t g = find(cell_key(l - 1, pc, mm));
            if (g < 0) {
              if (err) *err = "hanging-node weight master not found";
              return NodeSpace();
            }
            w.push_back({g, wt});
          }
      int32_t own = ns.cell_nodes[c * ns.nb + b];
      if (w.size() == 1 && w[0].first == own && std::fabs(w[0].second - 1.0) < 1e-12) continue;
      if (hang_first[own] < 0) {
        hang_first[own] = (int32_t)hang_list.size();
        hang_list.push_back(w);
        hang_ids.push_back(own);
      }
    }
  }
  // order hanging nodes by id; chains are not expected on 2:1-balanced forests
  std::vector<size_t> order(hang_ids.size());
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](size_t a, size_t b) { return hang_ids[a] < hang_ids[b]; });
  ns.hang_ptr.assign(1, 0);
  for (size_t o : order) {
    ns.hang_node.push_back(hang_ids[o]);
    for (auto& mw : hang_list[o]) {
      if (hang_first[mw.first] >= 0) {
        if (err) *err = "hanging-node chain (mesh not 2:1 balanced)";
        return NodeSpace();
      }
      ns.hang_master.push_back(mw.first);
      ns.hang_w.push_back(mw.second);
    }
    ns.hang_ptr.push_back((int32_t)ns.hang_master.size());
  }
  return ns;
}

int color_cells(const Forest& f, const std::vector<const NodeSpace*>& spaces, std::vector<int32_t>& color) {
  size_t nc = f.n_cells();
  color.assign(nc, -1);
  if (f.uniform()) {
    for (size_t c = 0; c < nc; ++c) {
      int col = 0;
      for (int d = 0; d < f.dim; ++d) col |= (f.crd[3 * c + d] & 1) << d;
      color[c] = col;
    }
    return 1 << f.dim;
  }
  // node -> cells (over master ids of every space)
  std::vector<std::vector<int32_t>> ptr(spaces.size()), cells(spaces.size());
  for (size_t s = 0; s < spaces.size(); ++s) {
    const NodeSpace& ns = *spaces[s];
    ptr[s].assign(ns.n_nodes + 1, 0);
    for (size_t i = 0; i < nc * ns.nb; ++i) ptr[s][ns.cell_master[i] + 1]++;
    for (int64_t g = 0; g < ns.n_nodes; ++g) ptr[s][g + 1] += ptr[s][g];
    cells[s].resize(nc * ns.nb);
    std::vector<int32_t> fill(ptr[s].begin(), ptr[s].end() - 1);
    for (size_t c = 0; c < nc; ++c)
      for (int b = 0; b < ns.nb; ++b) cells[s][fill[ns.cell_master[c * ns.nb + b]]++] = (int32_t)c;
  }
  std::vector<int64_t> seen(4096, -1);
  int ncol = 0;
  for (size_t c = 0; c < nc; ++c) {
    for (size_t s = 0; s < spaces.size(); ++s) {
      const NodeSpace& ns = *spaces[s];
      for (int b = 0; b < ns.nb; ++b) {
        int32_t g = ns.cell_master[c * ns.nb + b];
        for (int32_t i = ptr[s][g]; i < ptr[s][g + 1]; ++i) {
          int32_t o = cells[s][i];
          if (color[o] >= 0) seen[color[o]] = (int64_t)c;
        }
      }
    }
    int col = 0;
    while (seen[col] == (int64_t)c) ++col;
    color[c] = col;
    ncol = std::max(ncol, col + 1);
  }
  return ncol;
}

}  // namespace mfns
