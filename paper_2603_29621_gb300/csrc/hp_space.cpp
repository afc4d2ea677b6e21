// hp-adaptive node spaces on the host (see hp_space.hpp).
#include "hp_space.hpp"

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <stdexcept>
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
  // owners of every node and the dominating (level, degree) among them
  std::vector<std::vector<int32_t>> owners(nn);
  for (int64_t g = 0; g < nslots; ++g) {
    auto& o = owners[out.cell_nodes[g]];
    if (o.empty() || o.back() != slot_cell[g]) o.push_back(slot_cell[g]);
  }
  std::vector<std::pair<int, int>> dom(nn, {1 << 30, 1 << 30});
  for (int64_t g = 0; g < nn; ++g)
    for (int32_t c : owners[g]) dom[g] = std::min(dom[g], std::make_pair((int)f.lev[c], (int)degree[c]));
  const Lattice latt = make_lattice(f);
  // direct constraints
  std::map<int32_t, std::vector<std::pair<int32_t, double>>> direct;
  for (int64_t g = 0; g < nn; ++g) {
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
          if (std::find(owners[g].begin(), owners[g].end(), c) != owners[g].end()) continue;
          const std::pair<int, int> key = {f.lev[c], degree[c]};
          if (key < dom[g] && (best < 0 || key < best_key || (key == best_key && c < best))) {
            best_key = key;
            best = c;
          }
        }
    if (best < 0) continue;
    if (best_key.first < dom[g].first) {  // hanging on a coarser cell: no fine owner of lower degree
      int kmin = 1 << 30;
      for (int32_t c : owners[g]) kmin = std::min<int>(kmin, degree[c]);
      if (best_key.second > kmin) return fail("unsupported: a hanging face whose coarse cell has a higher degree than a fine cell");
    }
    // the dominating cell's finite-element function at the node
    const int k = degree[best], np = k + 1;
    const double s = double(int64_t(1) << (L - f.lev[best]));
    double xi[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) xi[d] = std::min(1.0, std::max(0.0, (lat[g * dim + d] - f.crd[3 * best + d] * s) / s));
    std::vector<std::pair<int32_t, double>> w;
    for (int64_t i = 0; i < out.cell_ptr[best + 1] - out.cell_ptr[best]; ++i) {
      const int a[3] = {int(i % np), int((i / np) % np), dim == 3 ? int(i / (np * np)) : 0};
      double v = 1.0;
      for (int d = 0; d < dim; ++d) v *= lagrange(gll[k], a[d], xi[d]);
      if (std::fabs(v) > 1e-13) w.push_back({out.cell_nodes[out.cell_ptr[best] + i], v});
    }
    direct[(int32_t)g] = std::move(w);
  }
  // resolve chains to free masters
  std::map<int32_t, std::vector<std::pair<int32_t, double>>> resolved;
  auto resolve = [&](int32_t g, auto&& self, int depth) -> const std::vector<std::pair<int32_t, double>>& {
    auto it = resolved.find(g);
    if (it != resolved.end()) return it->second;
    if (depth > 64) throw std::runtime_error("constraint cycle");
    std::map<int32_t, double> acc;
    for (auto& mw : direct[g]) {
      if (direct.count(mw.first)) {
        for (auto& mm : self(mw.first, self, depth + 1)) acc[mm.first] += mw.second * mm.second;
      } else {
        acc[mw.first] += mw.second;
      }
    }
    auto& r = resolved[g];
    for (auto& kv : acc) r.push_back(kv);
    return r;
  };
  out.hang_ptr.assign(1, 0);
  try {
    for (auto& kv : direct) {
      const auto& r = resolve(kv.first, resolve, 0);
      out.hang_node.push_back(kv.first);
      for (auto& mw : r) {
        out.hang_master.push_back(mw.first);
        out.hang_w.push_back(mw.second);
      }
      out.hang_ptr.push_back((int32_t)out.hang_master.size());
    }
  } catch (const std::exception& e) {
    return fail(e.what());
  }
  return true;
}

}  // namespace mfns
