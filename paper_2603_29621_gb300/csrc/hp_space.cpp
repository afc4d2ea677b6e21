// hp-adaptive node spaces on the host (see hp_space.hpp).
#include "hp_space.hpp"

#include <algorithm>
#include <array>
#include <cmath>
#include <utility>

namespace mfns {

namespace {
using Key = std::array<int64_t, 3>;

bool is_rational(double t) { return std::fabs(t) < 1e-14 || std::fabs(t - 1.0) < 1e-14 || std::fabs(t - 0.5) < 1e-14; }
}  // namespace

bool make_hp_space(const Forest& f, const std::vector<int32_t>& degree, HpSpace& out, std::string* err) {
  auto fail = [&](const char* m) {
    if (err) *err = m;
    return false;
  };
  const int dim = f.dim;
  const size_t nc = f.n_cells();
  if (degree.size() != nc) return fail("one degree per cell expected");
  int kmax = 1;
  for (int32_t k : degree) {
    if (k < 1 || k > 8) return fail("degrees must lie in 1..8");
    kmax = std::max<int>(kmax, k);
  }
  const int L = f.max_level();
  const int64_t N = (int64_t)f.n << L;
  out = HpSpace();
  out.dim = dim;
  out.degree = degree;
  std::vector<std::vector<double>> gll(kmax + 1);
  for (int k = 1; k <= kmax; ++k) gll[k] = gll_nodes(k);
  // slots of every cell with exact keys: half-lattice units at rational positions, a code unique
  // to (level, cell coordinate, degree, slot) at irrational ones
  out.cell_ptr.assign(nc + 1, 0);
  for (size_t c = 0; c < nc; ++c) {
    const int64_t np = degree[c] + 1;
    out.cell_ptr[c + 1] = out.cell_ptr[c] + (dim == 3 ? np * np * np : np * np);
  }
  const int64_t nslots = out.cell_ptr[nc];
  std::vector<std::pair<Key, int64_t>> all(nslots);
  std::vector<double> lat_slot(nslots * dim);
  std::vector<int32_t> slot_cell(nslots);
  for (size_t c = 0; c < nc; ++c) {
    const int k = degree[c], np = k + 1, l = f.lev[c];
    const int64_t s = int64_t(1) << (L - l);
    for (int64_t i = 0; i < out.cell_ptr[c + 1] - out.cell_ptr[c]; ++i) {
      const int a[3] = {int(i % np), int((i / np) % np), dim == 3 ? int(i / (np * np)) : 0};
      Key key = {0, 0, 0};
      const int64_t g = out.cell_ptr[c] + i;
      for (int d = 0; d < dim; ++d) {
        const int64_t cd = f.crd[3 * c + d];
        const double xi = gll[k][a[d]];
        key[d] = is_rational(xi) ? 2 * cd * s + (int64_t)std::llround(2.0 * xi * double(s))
                                 : -1 - ((((int64_t)l * (N + 1) + cd) * (kmax + 1) + k) * (kmax + 1) + a[d]);
        lat_slot[g * dim + d] = (double(cd) + xi) * double(s);
      }
      all[g] = {key, g};
      slot_cell[g] = (int32_t)c;
    }
  }
  std::sort(all.begin(), all.end());
  out.cell_nodes.assign(nslots, -1);
  std::vector<double> lat;  // per node, finest-lattice units
  for (int64_t i = 0; i < nslots; ++i) {
    if (i == 0 || all[i].first != all[i - 1].first) {
      for (int d = 0; d < dim; ++d) lat.push_back(lat_slot[all[i].second * dim + d]);
      ++out.n_nodes;
    }
    out.cell_nodes[all[i].second] = (int32_t)(out.n_nodes - 1);
  }
  const int64_t nn = out.n_nodes;
  out.x.resize(nn * dim);
  out.boundary.assign(nn, 0);
  for (int64_t g = 0; g < nn; ++g)
    for (int d = 0; d < dim; ++d) {
      out.x[g * dim + d] = lat[g * dim + d] / double(N);
      if (lat[g * dim + d] <= 1e-12 || lat[g * dim + d] >= double(N) - 1e-12) out.boundary[g] = 1;
    }
  // owners of every node (compressed rows) and the dominating (level, degree) among them
  std::vector<int64_t> own_ptr(nn + 1, 0);
  for (int64_t j = 0; j < nslots; ++j) own_ptr[out.cell_nodes[j] + 1]++;
  for (int64_t g = 0; g < nn; ++g) own_ptr[g + 1] += own_ptr[g];
  std::vector<int32_t> own(nslots);
  {
    std::vector<int64_t> fill(own_ptr.begin(), own_ptr.end() - 1);
    for (int64_t j = 0; j < nslots; ++j) own[fill[out.cell_nodes[j]]++] = slot_cell[j];
  }
  auto dom_key = [&](int32_t c) { return std::make_pair((int)f.lev[c], (int)degree[c]); };
  const Lattice latt = make_lattice(f);
  // direct constraints, in ascending node order: index of the node's row (-1: free)
  std::vector<int32_t> row_of(nn, -1);
  std::vector<int32_t> d_node, d_ptr(1, 0), d_master;
  std::vector<double> d_w;
  for (int64_t g = 0; g < nn; ++g) {
    const int32_t* ob = own.data() + own_ptr[g];
    const int32_t* oe = own.data() + own_ptr[g + 1];
    std::pair<int, int> dom = {1 << 30, 1 << 30};
    int kmin_owner = 1 << 30;
    for (const int32_t* o = ob; o != oe; ++o) {
      dom = std::min(dom, dom_key(*o));
      kmin_owner = std::min<int>(kmin_owner, degree[*o]);
    }
    int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) {
      const double t = lat[g * dim + d];
      lo[d] = std::min<int64_t>(std::max<int64_t>((int64_t)std::floor(t - 1e-9), 0), N - 1);
      hi[d] = std::min<int64_t>(std::max<int64_t>((int64_t)std::floor(t + 1e-9), 0), N - 1);
    }
    std::pair<int, int> best_key = {1 << 30, 1 << 30};
    int32_t best = -1;
    for (int64_t z = lo[2]; z <= hi[2]; ++z)
      for (int64_t y = lo[1]; y <= hi[1]; ++y)
        for (int64_t xx = lo[0]; xx <= hi[0]; ++xx) {
          const int32_t c = latt.at((int)xx, (int)y, (int)z);
          if (std::find(ob, oe, c) != oe) continue;
          const std::pair<int, int> key = dom_key(c);
          if (key < dom && (best < 0 || key < best_key || (key == best_key && c < best))) {
            best_key = key;
            best = c;
          }
        }
    if (best < 0) continue;
    // hanging on a coarser cell: no fine owner of lower degree
    if (best_key.first < dom.first && best_key.second > kmin_owner)
      return fail("unsupported: a hanging face whose coarse cell has a higher degree than a fine cell");
    // the dominating cell's finite-element function at the node
    const int k = degree[best], np = k + 1;
    const double s = double(int64_t(1) << (L - f.lev[best]));
    double xi[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) xi[d] = std::min(1.0, std::max(0.0, (lat[g * dim + d] - f.crd[3 * best + d] * s) / s));
    double l1[3][9];
    for (int d = 0; d < dim; ++d)
      for (int a = 0; a < np; ++a) l1[d][a] = lagrange(gll[k], a, xi[d]);
    row_of[g] = (int32_t)d_node.size();
    d_node.push_back((int32_t)g);
    for (int64_t i = 0; i < out.cell_ptr[best + 1] - out.cell_ptr[best]; ++i) {
      const int a[3] = {int(i % np), int((i / np) % np), dim == 3 ? int(i / (np * np)) : 0};
      double v = 1.0;
      for (int d = 0; d < dim; ++d) v *= l1[d][a[d]];
      if (std::fabs(v) > 1e-13) {
        d_master.push_back(out.cell_nodes[out.cell_ptr[best] + i]);
        d_w.push_back(v);
      }
    }
    d_ptr.push_back((int32_t)d_master.size());
  }
  // resolve chains to free masters (rows in ascending node order; a row's masters may be rows)
  std::vector<char> state(d_node.size(), 0);  // 0 open, 1 in progress, 2 resolved
  std::vector<std::vector<std::pair<int32_t, double>>> res(d_node.size());
  std::vector<std::pair<int32_t, int>> stack;
  for (size_t r0 = 0; r0 < d_node.size(); ++r0) {
    if (state[r0] == 2) continue;
    stack.assign(1, {(int32_t)r0, 0});
    state[r0] = 1;
    while (!stack.empty()) {
      const int32_t r = stack.back().first;
      bool pushed = false;
      for (int32_t j = d_ptr[r]; j < d_ptr[r + 1] && !pushed; ++j) {
        const int32_t q = row_of[d_master[j]];
        if (q < 0 || state[q] == 2) continue;
        if (state[q] == 1) return fail("constraint cycle");
        state[q] = 1;
        stack.push_back({q, 0});
        pushed = true;
      }
      if (pushed) continue;
      std::vector<std::pair<int32_t, double>> acc;
      for (int32_t j = d_ptr[r]; j < d_ptr[r + 1]; ++j) {
        const int32_t m = d_master[j], q = row_of[m];
        if (q < 0) {
          acc.push_back({m, d_w[j]});
        } else {
          for (auto& mw : res[q]) acc.push_back({mw.first, d_w[j] * mw.second});
        }
      }
      std::sort(acc.begin(), acc.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
      auto& out_r = res[r];
      for (auto& mw : acc) {
        if (!out_r.empty() && out_r.back().first == mw.first)
          out_r.back().second += mw.second;
        else
          out_r.push_back(mw);
      }
      state[r] = 2;
      stack.pop_back();
    }
  }
  out.hang_ptr.assign(1, 0);
  for (size_t r = 0; r < d_node.size(); ++r) {
    out.hang_node.push_back(d_node[r]);
    for (auto& mw : res[r]) {
      out.hang_master.push_back(mw.first);
      out.hang_w.push_back(mw.second);
    }
    out.hang_ptr.push_back((int32_t)out.hang_master.size());
  }
  return true;
}

int hp_color_cells(const HpSpace& sp, const std::vector<int32_t>& cells, std::vector<int32_t>& color) {
  // node -> subset positions (compressed rows)
  std::vector<int64_t> ptr(sp.n_nodes + 1, 0);
  for (int32_t c : cells)
    for (int64_t j = sp.cell_ptr[c]; j < sp.cell_ptr[c + 1]; ++j) ptr[sp.cell_nodes[j] + 1]++;
  for (int64_t g = 0; g < sp.n_nodes; ++g) ptr[g + 1] += ptr[g];
  std::vector<int32_t> idx(ptr[sp.n_nodes]);
  {
    std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
    for (int32_t i = 0; i < (int32_t)cells.size(); ++i)
      for (int64_t j = sp.cell_ptr[cells[i]]; j < sp.cell_ptr[cells[i] + 1]; ++j) idx[fill[sp.cell_nodes[j]]++] = i;
  }
  color.assign(cells.size(), -1);
  std::vector<int32_t> stamp;  // stamp[col] == i: colour col is taken by a neighbour of cell i
  int ncol = 0;
  for (int32_t i = 0; i < (int32_t)cells.size(); ++i) {
    for (int64_t j = sp.cell_ptr[cells[i]]; j < sp.cell_ptr[cells[i] + 1]; ++j) {
      const int32_t g = sp.cell_nodes[j];
      for (int64_t q = ptr[g]; q < ptr[g + 1]; ++q) {
        const int32_t o = idx[q];
        if (color[o] >= 0) {
          if ((size_t)color[o] >= stamp.size()) stamp.resize(color[o] + 1, -1);
          stamp[color[o]] = i;
        }
      }
    }
    int col = 0;
    while ((size_t)col < stamp.size() && stamp[col] == i) ++col;
    color[i] = col;
    ncol = std::max(ncol, col + 1);
  }
  return ncol;
}

int hp_probe_groups(const HpSpace& sp, const std::vector<char>& free_node, std::vector<int32_t>& group) {
  const int64_t nn = sp.n_nodes;
  const size_t nc = sp.cell_ptr.size() - 1;
  // free masters reached by every node: itself when free, its free masters when constrained
  std::vector<int64_t> mptr(nn + 1, 0);
  std::vector<int32_t> hrow(nn, -1);
  for (size_t i = 0; i < sp.hang_node.size(); ++i) hrow[sp.hang_node[i]] = (int32_t)i;
  auto for_masters = [&](int32_t g, auto&& fn) {
    if (free_node[g]) {
      fn(g);
    } else if (hrow[g] >= 0 && !sp.boundary[g]) {  // Dirichlet entries do not couple
      for (int32_t j = sp.hang_ptr[hrow[g]]; j < sp.hang_ptr[hrow[g] + 1]; ++j)
        if (free_node[sp.hang_master[j]]) fn(sp.hang_master[j]);
    }
  };
  // cell -> its free masters (compressed, duplicates removed)
  std::vector<int64_t> cptr(nc + 1, 0);
  std::vector<int32_t> cidx;
  for (size_t c = 0; c < nc; ++c) {
    const size_t start = cidx.size();
    for (int64_t j = sp.cell_ptr[c]; j < sp.cell_ptr[c + 1]; ++j) for_masters(sp.cell_nodes[j], [&](int32_t m) { cidx.push_back(m); });
    std::sort(cidx.begin() + start, cidx.end());
    cidx.erase(std::unique(cidx.begin() + start, cidx.end()), cidx.end());
    cptr[c + 1] = (int64_t)cidx.size();
  }
  // master -> cells (compressed)
  std::vector<int64_t> optr(nn + 1, 0);
  for (int32_t m : cidx) optr[m + 1]++;
  for (int64_t g = 0; g < nn; ++g) optr[g + 1] += optr[g];
  std::vector<int32_t> oidx(optr[nn]);
  {
    std::vector<int64_t> fill(optr.begin(), optr.end() - 1);
    for (size_t c = 0; c < nc; ++c)
      for (int64_t q = cptr[c]; q < cptr[c + 1]; ++q) oidx[fill[cidx[q]]++] = (int32_t)c;
  }
  group.assign(nn, -1);
  std::vector<int64_t> stamp;
  int ng = 0;
  for (int64_t m = 0; m < nn; ++m) {
    if (!free_node[m]) continue;
    for (int64_t q = optr[m]; q < optr[m + 1]; ++q) {
      const int32_t c = oidx[q];
      for (int64_t r = cptr[c]; r < cptr[c + 1]; ++r) {
        const int32_t o = group[cidx[r]];
        if (o >= 0) {
          if ((size_t)o >= stamp.size()) stamp.resize(o + 1, -1);
          stamp[o] = m;
        }
      }
    }
    int col = 0;
    while ((size_t)col < stamp.size() && stamp[col] == m) ++col;
    group[m] = col;
    ng = std::max(ng, col + 1);
  }
  return ng;
}

}  // namespace mfns
