// hp-adaptive node spaces on the host (see hp_space.hpp).
#include "hp_space.hpp"

#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <utility>

namespace mfns {

namespace {
using Key = std::array<int64_t, 3>;

bool is_rational(double t) { return std::fabs(t) < 1e-14 || std::fabs(t - 1.0) < 1e-14 || std::fabs(t - 0.5) < 1e-14; }

// The local rule (header comment): direct constraints from the dominating cell, chains resolved.
// Returns 0 on success, 1 when a hanging face has a coarse cell of higher degree than a fine one
// (the rule does not apply; err names it), -1 on another error.
int dominance_constraints(const Forest& f, const std::vector<int32_t>& degree,
                          const std::vector<std::vector<double>>& gll, const std::vector<double>& lat,
                          const std::vector<int64_t>& own_ptr, const std::vector<int32_t>& own,
                          const std::vector<std::pair<int, int>>& dom_of, const Lattice& latt, HpSpace& out,
                          std::string* err) {
  auto fail = [&](int code, const char* m) {
    if (err) *err = m;
    return code;
  };
  const int dim = f.dim;
  const int L = f.max_level();
  const int64_t N = (int64_t)f.n << L;
  const int64_t nn = out.n_nodes;
  auto dom_key = [&](int32_t c) { return std::make_pair((int)f.lev[c], (int)degree[c]); };
  // direct constraints, in ascending node order: index of the node's row (-1: free)
  std::vector<int32_t> row_of(nn, -1);
  std::vector<int32_t> d_node, d_ptr(1, 0), d_master;
  std::vector<double> d_w;
  for (int64_t g = 0; g < nn; ++g) {
    const int32_t* ob = own.data() + own_ptr[g];
    const int32_t* oe = own.data() + own_ptr[g + 1];
    const std::pair<int, int> dom = dom_of[g];
    int kmin_owner = 1 << 30;
    for (const int32_t* o = ob; o != oe; ++o) kmin_owner = std::min<int>(kmin_owner, degree[*o]);
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
      return fail(1, "unsupported: a hanging face whose coarse cell has a higher degree than a fine cell");
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
        if (state[q] == 1) return fail(-1, "constraint cycle");
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
  out.hang_node.clear();
  out.hang_master.clear();
  out.hang_w.clear();
  out.hang_ptr.assign(1, 0);
  for (size_t r = 0; r < d_node.size(); ++r) {
    out.hang_node.push_back(d_node[r]);
    for (auto& mw : res[r]) {
      out.hang_master.push_back(mw.first);
      out.hang_w.push_back(mw.second);
    }
    out.hang_ptr.push_back((int32_t)out.hang_master.size());
  }
  return 0;
}

// Constraints by elimination (header comment).  Continuity of the traces on every face piece
// shared by two cells whose traces are not identical by construction (different level or
// degree): the difference of the two traces vanishes at the tensor GLL points of degree
// max(k_a, k_b) on the piece, one linear condition per point in the unknown node values.  The
// conditions are brought to reduced row echelon form by Gauss--Jordan elimination on sparse rows,
// with the columns ordered from the least to the most preferred node (preference: coarser
// dominating cell, then lower degree, then the lower dimension of the entity the node is interior
// to in that cell -- vertex, edge, face, cell -- then lower node id) and the largest entry of the
// column as pivot.  The entity order keeps vertices and edges of a combined face as masters, so
// every slave is expressed in nodes of its own face or edge.  The reduced form depends only on the row space and the column order, so every pivot
// column (slave) and its expression in the free columns (masters) are those of any other sample
// of the same conditions.
bool eliminate_constraints(const Forest& f, const std::vector<int32_t>& degree,
                           const std::vector<std::vector<double>>& gll,
                           const std::vector<std::pair<int, int>>& dom, const std::vector<int8_t>& entity,
                           const Lattice& latt, bool dirichlet, HpSpace& out, std::string* err) {
  using Row = std::vector<std::pair<int32_t, double>>;  // (column, value), columns ascending
  const int dim = f.dim;
  const int L = f.max_level();
  const int64_t N = (int64_t)f.n << L;
  const int64_t nn = out.n_nodes;
  const size_t nc = f.n_cells();
  // columns: the unknown node values, least preferred first
  std::vector<int32_t> var;
  for (int64_t g = 0; g < nn; ++g)
    if (!(dirichlet && out.boundary[g])) var.push_back((int32_t)g);
  std::sort(var.begin(), var.end(), [&](int32_t a, int32_t b) {
    if (dom[a] != dom[b]) return dom[a] > dom[b];
    if (entity[a] != entity[b]) return entity[a] > entity[b];
    return a > b;
  });
  const int32_t nv = (int32_t)var.size();
  std::vector<int32_t> col_of(nn, -1);
  for (int32_t j = 0; j < nv; ++j) col_of[var[j]] = j;
  // the conditions
  std::vector<Row> rows;
  Row row;
  for (size_t a = 0; a < nc; ++a) {
    const int la = f.lev[a];
    const int64_t sa = int64_t(1) << (L - la);
    for (int d = 0; d < dim; ++d)
      for (int side = 0; side < 2; ++side) {
        const int64_t q = (f.crd[3 * a + d] + side) * sa;
        if (q == 0 || q == N) continue;  // domain boundary
        int64_t pos[3] = {0, 0, 0};
        for (int j = 0; j < dim; ++j) pos[j] = f.crd[3 * a + j] * sa;
        pos[d] = side ? q : q - 1;
        const int32_t b = latt.at((int)pos[0], (int)pos[1], (int)pos[2]);
        if (b < 0) continue;
        const int lb = f.lev[b];
        // each piece once, from its finer side (a coarser or same-level neighbour covers the face)
        if (lb > la || (lb == la && b < (int32_t)a)) continue;
        if (lb == la && degree[b] == degree[a]) continue;  // the same nodes on both sides
        const int m = std::max(degree[a], degree[b]);
        int tang[2] = {0, 0}, nt = 0;
        for (int j = 0; j < dim; ++j)
          if (j != d) tang[nt++] = j;
        const int np = m + 1, npts = nt == 2 ? np * np : np;
        for (int p = 0; p < npts; ++p) {
          double pt[3] = {0, 0, 0};  // finest-lattice units
          pt[d] = double(q);
          pt[tang[0]] = double(f.crd[3 * a + tang[0]] * sa) + double(sa) * gll[m][p % np];
          if (nt == 2) pt[tang[1]] = double(f.crd[3 * a + tang[1]] * sa) + double(sa) * gll[m][p / np];
          row.clear();
          for (int sd = 0; sd < 2; ++sd) {
            const int32_t c = sd == 0 ? (int32_t)a : b;
            const double sgn = sd == 0 ? 1.0 : -1.0;
            const int k = degree[c], kp = k + 1;
            const double sc = double(int64_t(1) << (L - f.lev[c]));
            // slot index of the face in the normal direction: a's face at `side`, b's opposite
            const int an = (sd == 0) == (side == 1) ? k : 0;
            double l1[2][9];
            for (int t = 0; t < nt; ++t) {
              const double xi = std::min(1.0, std::max(0.0, (pt[tang[t]] - double(f.crd[3 * c + tang[t]]) * sc) / sc));
              for (int i = 0; i < kp; ++i) l1[t][i] = lagrange(gll[k], i, xi);
            }
            for (int i1 = 0; i1 < (nt == 2 ? kp : 1); ++i1)
              for (int i0 = 0; i0 < kp; ++i0) {
                int ai[3] = {0, 0, 0};
                ai[d] = an;
                ai[tang[0]] = i0;
                if (nt == 2) ai[tang[1]] = i1;
                const int64_t slot = ai[0] + kp * (ai[1] + kp * ai[2]);
                const int32_t g = out.cell_nodes[out.cell_ptr[c] + slot];
                if (col_of[g] < 0) continue;
                const double v = sgn * l1[0][i0] * (nt == 2 ? l1[1][i1] : 1.0);
                row.push_back({col_of[g], v});
              }
          }
          std::sort(row.begin(), row.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
          Row merged;
          for (auto& e : row) {
            if (!merged.empty() && merged.back().first == e.first)
              merged.back().second += e.second;
            else
              merged.push_back(e);
          }
          Row kept;
          for (auto& e : merged)
            if (std::fabs(e.second) > 1e-14) kept.push_back(e);
          if (!kept.empty()) rows.push_back(std::move(kept));
        }
      }
  }
  // Gauss--Jordan elimination, column by column in preference order
  const int32_t nr = (int32_t)rows.size();
  std::vector<std::vector<int32_t>> col_rows(nv);  // rows that may hold the column (stale allowed)
  for (int32_t i = 0; i < nr; ++i)
    for (auto& e : rows[i]) col_rows[e.first].push_back(i);
  auto entry = [](const Row& r, int32_t c) {
    auto it = std::lower_bound(r.begin(), r.end(), c, [](const auto& e, int32_t v) { return e.first < v; });
    return it != r.end() && it->first == c ? it->second : 0.0;
  };
  std::vector<int32_t> piv_col(nr, -1), stamp(nr, -1);
  std::vector<char> is_piv(nv, 0);
  Row tmp;
  for (int32_t c = 0; c < nv; ++c) {
    std::vector<int32_t>& cand = col_rows[c];
    if (cand.empty()) continue;
    int32_t best = -1;
    double bv = 1e-10;
    for (int32_t i : cand)
      if (piv_col[i] < 0) {
        const double v = std::fabs(entry(rows[i], c));
        if (v > bv) {
          bv = v;
          best = i;
        }
      }
    if (best < 0) {
      std::vector<int32_t>().swap(cand);
      continue;
    }
    piv_col[best] = c;
    is_piv[c] = 1;
    Row& P = rows[best];
    const double pv = entry(P, c);
    for (auto& e : P) e.second = e.first == c ? 1.0 : e.second / pv;
    for (int32_t i : cand) {
      if (i == best || stamp[i] == c) continue;
      stamp[i] = c;
      Row& R = rows[i];
      const double v = entry(R, c);
      if (v == 0.0) continue;
      tmp.clear();
      size_t x = 0, y = 0;
      while (x < R.size() || y < P.size()) {
        const int32_t cx = x < R.size() ? R[x].first : INT32_MAX, cy = y < P.size() ? P[y].first : INT32_MAX;
        if (cx < cy) {
          tmp.push_back(R[x++]);
        } else if (cy < cx) {
          const double w = -v * P[y].second;
          if (cy != c && std::fabs(w) > 1e-14) {
            tmp.push_back({cy, w});
            col_rows[cy].push_back(i);
          }
          ++y;
        } else {
          const double w = R[x].second - v * P[y].second;
          if (cx != c && std::fabs(w) > 1e-14) tmp.push_back({cx, w});
          ++x;
          ++y;
        }
      }
      R.swap(tmp);
    }
    std::vector<int32_t>().swap(cand);
  }
  // slaves and their masters, by node id
  std::vector<std::pair<int32_t, int32_t>> slaves;  // (node, row)
  for (int32_t i = 0; i < nr; ++i)
    if (piv_col[i] >= 0) slaves.push_back({var[piv_col[i]], i});
  std::sort(slaves.begin(), slaves.end());
  out.hang_node.clear();
  out.hang_master.clear();
  out.hang_w.clear();
  out.hang_ptr.assign(1, 0);
  std::vector<std::pair<int32_t, double>> ms;
  for (auto& sr : slaves) {
    ms.clear();
    for (auto& e : rows[sr.second]) {
      if (e.first == piv_col[sr.second]) continue;
      if (is_piv[e.first]) {
        if (err) *err = "elimination left a pivot column in a reduced row";
        return false;
      }
      if (std::fabs(e.second) >= 1e-13) ms.push_back({var[e.first], -e.second});
    }
    std::sort(ms.begin(), ms.end());
    out.hang_node.push_back(sr.first);
    for (auto& mw : ms) {
      out.hang_master.push_back(mw.first);
      out.hang_w.push_back(mw.second);
    }
    out.hang_ptr.push_back((int32_t)out.hang_master.size());
  }
  return true;
}
}  // namespace

// Some face of a cell has finer neighbours across it of lower degree than the cell (found from the
// finer side: the cell just across each interior face of every cell).
static bool has_combined_face(const Forest& f, const std::vector<int32_t>& degree, const Lattice& latt) {
  const int dim = f.dim;
  const int64_t N = (int64_t)f.n << f.max_level();
  for (size_t a = 0; a < f.n_cells(); ++a) {
    const int64_t sa = int64_t(1) << (f.max_level() - f.lev[a]);
    for (int d = 0; d < dim; ++d)
      for (int side = 0; side < 2; ++side) {
        const int64_t q = (f.crd[3 * a + d] + side) * sa;
        if (q == 0 || q == N) continue;
        int64_t pos[3] = {0, 0, 0};
        for (int j = 0; j < dim; ++j) pos[j] = f.crd[3 * a + j] * sa;
        pos[d] = side ? q : q - 1;
        const int32_t b = latt.at((int)pos[0], (int)pos[1], (int)pos[2]);
        if (b >= 0 && f.lev[b] < f.lev[a] && degree[b] > degree[a]) return true;
      }
  }
  return false;
}

bool make_hp_space(const Forest& f, const std::vector<int32_t>& degree, HpSpace& out, std::string* err,
                   HpRule rule, bool dirichlet) {
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
  // the dominating (level, degree) among every node's owners: the preference of the node
  std::vector<std::pair<int, int>> dom(nn, {1 << 30, 1 << 30});
  for (int64_t g = 0; g < nn; ++g)
    for (int64_t j = own_ptr[g]; j < own_ptr[g + 1]; ++j) dom[g] = std::min(dom[g], dom_key(own[j]));
  // entity dimension of every node in a dominating owner (coordinates strictly inside (0, k))
  std::vector<int8_t> entity(nn, -1);
  for (size_t c = 0; c < nc; ++c) {
    const int k = degree[c], np = k + 1;
    for (int64_t i = 0; i < out.cell_ptr[c + 1] - out.cell_ptr[c]; ++i) {
      const int32_t g = out.cell_nodes[out.cell_ptr[c] + i];
      if (entity[g] >= 0 || dom_key((int32_t)c) != dom[g]) continue;
      const int a[3] = {int(i % np), int((i / np) % np), dim == 3 ? int(i / (np * np)) : 0};
      int8_t e = 0;
      for (int d = 0; d < dim; ++d) e += (a[d] > 0 && a[d] < k) ? 1 : 0;
      entity[g] = e;
    }
  }
  const Lattice latt = make_lattice(f);
  // A combined face -- a face of a coarse cell whose neighbours across it are finer and of lower
  // degree -- makes the local rule inapplicable even where no node of the finer cells hangs (coarse
  // degree 2 against fine degree 1: every fine node is a coarse node, yet the coarse quadratic
  // trace is not piecewise linear).  The automatic rule then eliminates from the start; an
  // edge-only contact of that kind is caught by the local rule itself (a fine node hanging on a
  // coarse cell of higher degree).
  if (rule == HpRule::kAuto && has_combined_face(f, degree, latt)) {
    if (!eliminate_constraints(f, degree, gll, dom, entity, latt, dirichlet, out, err)) return false;
    return true;
  }
  if (rule != HpRule::kElimination) {
    const int st = dominance_constraints(f, degree, gll, lat, own_ptr, own, dom, latt, out, err);
    if (st == 0) return true;
    if (st < 0 || rule == HpRule::kDominance) return false;
  }
  return eliminate_constraints(f, degree, gll, dom, entity, latt, dirichlet, out, err);
}

std::vector<std::vector<int32_t>> hp_asm_blocks(const Forest& f, const HpSpace& sp, int ncomp) {
  const int dim = f.dim;
  const int L = f.max_level();
  const int64_t N = (int64_t)f.n << L;
  const Lattice latt = make_lattice(f);
  std::vector<char> hang(sp.n_nodes, 0);
  for (int32_t g : sp.hang_node) hang[g] = 1;
  // combined faces, found from their finer side: (coarse cell, direction, side of the coarse cell)
  std::vector<std::array<int64_t, 3>> faces;
  for (size_t a = 0; a < f.n_cells(); ++a) {
    const int64_t sa = int64_t(1) << (L - f.lev[a]);
    for (int d = 0; d < dim; ++d)
      for (int side = 0; side < 2; ++side) {
        const int64_t q = (f.crd[3 * a + d] + side) * sa;
        if (q == 0 || q == N) continue;
        int64_t pos[3] = {0, 0, 0};
        for (int j = 0; j < dim; ++j) pos[j] = f.crd[3 * a + j] * sa;
        pos[d] = side ? q : q - 1;
        const int32_t b = latt.at((int)pos[0], (int)pos[1], (int)pos[2]);
        if (b < 0 || f.lev[b] >= f.lev[a] || sp.degree[b] <= sp.degree[a]) continue;
        faces.push_back({b, d, 1 - side});
      }
  }
  std::sort(faces.begin(), faces.end());
  faces.erase(std::unique(faces.begin(), faces.end()), faces.end());
  std::vector<std::vector<int32_t>> out;
  for (const auto& fc : faces) {
    const int32_t c = (int32_t)fc[0];
    const int d = (int)fc[1], side = (int)fc[2];
    const int64_t sc = int64_t(1) << (L - f.lev[c]);
    const double plane = double((f.crd[3 * c + d] + side) * sc) / double(N);
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int j = 0; j < dim; ++j) {
      lo[j] = double(f.crd[3 * c + j] * sc) / double(N);
      hi[j] = double((f.crd[3 * c + j] + 1) * sc) / double(N);
    }
    // cells holding nodes of the face: the coarse cell and the cells just across it
    std::vector<int32_t> cells{c};
    const int64_t q = (f.crd[3 * c + d] + side) * sc;
    const int64_t across = side ? q : q - 1;
    int64_t r0[3] = {0, 0, 0}, r1[3] = {1, 1, 1};
    for (int j = 0; j < dim; ++j) {
      r0[j] = f.crd[3 * c + j] * sc;
      r1[j] = (f.crd[3 * c + j] + 1) * sc;
    }
    r0[d] = across;
    r1[d] = across + 1;
    if (across >= 0 && across < N)
      for (int64_t z = r0[2]; z < (dim == 3 ? r1[2] : 1); ++z)
        for (int64_t y = r0[1]; y < r1[1]; ++y)
          for (int64_t x = r0[0]; x < r1[0]; ++x) cells.push_back(latt.at((int)x, (int)y, (int)z));
    std::sort(cells.begin(), cells.end());
    cells.erase(std::unique(cells.begin(), cells.end()), cells.end());
    std::vector<int32_t> nodes;
    for (int32_t cc : cells) {
      if (cc < 0) continue;
      for (int64_t j = sp.cell_ptr[cc]; j < sp.cell_ptr[cc + 1]; ++j) {
        const int32_t g = sp.cell_nodes[j];
        if (sp.boundary[g] || hang[g]) continue;
        bool on = std::fabs(sp.x[g * dim + d] - plane) <= 1e-12;
        for (int jj = 0; jj < dim && on; ++jj)
          if (sp.x[g * dim + jj] < lo[jj] - 1e-12 || sp.x[g * dim + jj] > hi[jj] + 1e-12) on = false;
        if (on) nodes.push_back(g);
      }
    }
    std::sort(nodes.begin(), nodes.end());
    nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
    std::vector<int32_t> blk;
    for (int32_t g : nodes)
      for (int comp = 0; comp < ncomp; ++comp) blk.push_back((int32_t)(g * ncomp + comp));
    std::sort(blk.begin(), blk.end());
    if (!blk.empty()) out.push_back(std::move(blk));
  }
  return out;
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

}  // namespace mfns
