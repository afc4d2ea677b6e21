// hp levels (Section 3): the operator of a mesh whose cells carry different degrees.
//
// The cells of each degree form a group that the degree's cell kernel applies on its own node ids
// (no constraint masks).  The constraints of h- and p-adaptivity act around the cell kernels: the
// input is copied and its constrained entries completed from their masters, every group adds its
// products, the products on constrained entries are folded into their masters with the same
// weights (C^T), and constrained rows are identity rows: A = C^T K C on the free DoFs.  The exact
// diagonal is formed on the host at set-up (hp_exact_diagonal below).
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>

#include "problem.hpp"
#include "vec.hpp"

namespace mfns {

template <typename T>
static DevBuf upload_as(Budget* bud, const std::vector<double>& v) {
  std::vector<T> t(v.begin(), v.end());
  return upload(bud, t);
}

// Exact diagonal of C^T K C for one field of an hp level, accumulated into diag (FP64, host).
// The cell forms of hp levels are tensor products of 1D reference matrices on axis-aligned cubes:
// the vector Laplacian nu (grad u, grad v) acts on every component as the scalar form
// nu h^(d-2) sum_dir (K1 or M1 per axis), the mass (p, q) as h^d M1 x M1 (x M1), with M1, K1 the
// degree's 1D mass and stiffness matrices on [0, 1] under the kernels' Gauss rule.  For a free node
// i and a cell, v_i is i's weight at every slot of the cell (1 at its own slot, its constraint
// weight at the slots of nodes hanging on it; Dirichlet nodes are zero); the cell adds
// v_i^T K_cell v_i.  Every component of node i gets the same value.
static void hp_exact_diagonal(const Forest& f, const HpSpace& S, int ncomp, bool dirichlet, int64_t offset,
                              bool laplacian, double nu, std::vector<double>& diag) {
  const int dim = S.dim;
  std::vector<int32_t> hang_row(S.n_nodes, -1);  // row of a hanging node in the constraint lists
  for (size_t r = 0; r < S.hang_node.size(); ++r) hang_row[S.hang_node[r]] = (int32_t)r;
  auto zero = [&](int32_t g) { return dirichlet && S.boundary[g]; };
  std::map<int, std::pair<std::vector<double>, std::vector<double>>> mats;  // degree -> (M1, K1)
  auto tables = [&](int k) -> const std::pair<std::vector<double>, std::vector<double>>& {
    auto it = mats.find(k);
    if (it != mats.end()) return it->second;
    OpLaunch L;
    L.dim = dim;
    L.k = k;
    L.op = OP_STOKES_A;
    fill_tables(L);
    const int q = L.Q, n = L.N;
    std::vector<double> dS((size_t)q * n, 0.0);  // basis derivatives at the Gauss points
    for (int i = 0; i < q; ++i)
      for (int a = 0; a < n; ++a) {
        double v = 0.0;
        for (int r = 0; r < q; ++r) v += L.D[i * q + r] * L.S[r * n + a];
        dS[(size_t)i * n + a] = v;
      }
    std::vector<double> M1((size_t)n * n, 0.0), K1((size_t)n * n, 0.0);
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b)
        for (int i = 0; i < q; ++i) {
          M1[(size_t)a * n + b] += L.W[i] * L.S[i * n + a] * L.S[i * n + b];
          K1[(size_t)a * n + b] += L.W[i] * dS[(size_t)i * n + a] * dS[(size_t)i * n + b];
        }
    return mats.emplace(k, std::make_pair(std::move(M1), std::move(K1))).first->second;
  };
  struct Ent {
    int32_t node;  // free node
    int slot;
    double w;
  };
  std::vector<Ent> vloc;  // (free node, slot, weight) of the cell, grouped by node
  for (size_t c = 0; c < f.n_cells(); ++c) {
    const int k = S.degree[c], n = k + 1;
    const auto& mk = tables(k);
    const std::vector<double>& M1 = mk.first;
    const std::vector<double>& K1 = mk.second;
    const double h = f.h(c);
    const double scale = laplacian ? nu * std::pow(h, dim - 2) : std::pow(h, dim);
    const int64_t base = S.cell_ptr[c];
    const int nb = (int)(S.cell_ptr[c + 1] - base);
    vloc.clear();
    for (int s = 0; s < nb; ++s) {
      const int32_t g = S.cell_nodes[base + s];
      if (zero(g)) continue;
      const int32_t r = hang_row[g];
      if (r < 0) {
        vloc.push_back({g, s, 1.0});
        continue;
      }
      for (int32_t j = S.hang_ptr[r]; j < S.hang_ptr[r + 1]; ++j)
        if (!zero(S.hang_master[j])) vloc.push_back({S.hang_master[j], s, S.hang_w[j]});
    }
    std::stable_sort(vloc.begin(), vloc.end(), [](const Ent& a, const Ent& b) { return a.node < b.node; });
    auto entry = [&](int s, int t) {  // K_cell[s][t] / scale
      int as[3] = {s % n, (s / n) % n, dim == 3 ? s / (n * n) : 0};
      int at[3] = {t % n, (t / n) % n, dim == 3 ? t / (n * n) : 0};
      if (!laplacian) {
        double v = 1.0;
        for (int ax = 0; ax < dim; ++ax) v *= M1[(size_t)as[ax] * n + at[ax]];
        return v;
      }
      double v = 0.0;
      for (int dir = 0; dir < dim; ++dir) {
        double p = 1.0;
        for (int ax = 0; ax < dim; ++ax) p *= (ax == dir ? K1 : M1)[(size_t)as[ax] * n + at[ax]];
        v += p;
      }
      return v;
    };
    for (size_t b0 = 0; b0 < vloc.size();) {
      size_t b1 = b0 + 1;
      while (b1 < vloc.size() && vloc[b1].node == vloc[b0].node) ++b1;
      double acc = 0.0;
      for (size_t a = b0; a < b1; ++a)
        for (size_t b = b0; b < b1; ++b) acc += vloc[a].w * vloc[b].w * entry(vloc[a].slot, vloc[b].slot);
      for (int comp = 0; comp < ncomp; ++comp)
        diag[(size_t)(offset + (int64_t)vloc[b0].node * ncomp + comp)] += scale * acc;
      b0 = b1;
    }
  }
}

void build_hp_oplevel(OpLevel& lv, const Forest& f, const std::vector<int32_t>& degree, const Physics& ph,
                      Budget* bud, int op) {
  if (op != OP_STOKES_A && op != OP_STOKES && op != OP_PMASS) throw Error(kErrUnsupported, "hp level of this operator");
  const int dim = f.dim;
  auto hp = std::make_unique<HpData>();
  std::string err;
  // constraints: the local rule, elimination where a combined h+p face needs it; the main field has
  // Dirichlet conditions unless it is the pressure mass's
  if (!make_hp_space(f, degree, hp->space, &err, HpRule::kAuto, op != OP_PMASS))
    throw Error(err.rfind("unsupported", 0) == 0 ? kErrUnsupported : kErrArg, err);
  const HpSpace& sp = hp->space;
  // Taylor--Hood: the pressure space has degree k - 1 on every cell
  HpSpace psp;
  if (op == OP_STOKES) {
    std::vector<int32_t> dp(degree);
    for (auto& k : dp) {
      if (k < 2) throw Error(kErrUnsupported, "Taylor--Hood needs velocity degrees >= 2");
      k -= 1;
    }
    if (!make_hp_space(f, dp, psp, &err, HpRule::kAuto, false)) throw Error(err.rfind("unsupported", 0) == 0 ? kErrUnsupported : kErrArg, err);
  }
  const bool dirichlet = op != OP_PMASS;
  lv.op = op;
  lv.dim = dim;
  lv.k = *std::max_element(degree.begin(), degree.end());
  lv.forest = f;
  lv.NU = op == OP_PMASS ? 1 : dim;
  lv.nu = NodeSpace();
  lv.nu.dim = dim;
  lv.nu.n_nodes = sp.n_nodes;
  lv.nu.x = sp.x;
  lv.nu.boundary = sp.boundary;
  lv.n_main_dofs = sp.n_nodes * lv.NU;
  lv.n_dofs = lv.n_main_dofs + (op == OP_STOKES ? psp.n_nodes : 0);
  if (op == OP_STOKES) {
    lv.np = NodeSpace();
    lv.np.dim = dim;
    lv.np.n_nodes = psp.n_nodes;
    lv.np.x = psp.x;
    lv.np.boundary = psp.boundary;
  }
  if (lv.n_dofs >= (int64_t(1) << 31) - 1) throw Error(kErrUnsupported, "more than 2^31 DoFs per level");
  // groups of one degree: colour-sorted cell tables with node ids and the Dirichlet bit (two
  // cells sharing a pressure node share a velocity node too: the velocity colouring suffices)
  for (int k = 1; k <= lv.k; ++k) {
    std::vector<int32_t> cells;
    for (size_t c = 0; c < f.n_cells(); ++c)
      if (degree[c] == k) cells.push_back((int32_t)c);
    if (cells.empty()) continue;
    auto g = std::make_unique<HpGroup>();
    g->k = k;
    std::vector<int32_t> color;
    const int ncol = hp_color_cells(sp, cells, color);
    std::vector<int32_t> order(cells.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return color[a] < color[b]; });
    const int nb = (int)(sp.cell_ptr[cells[0] + 1] - sp.cell_ptr[cells[0]]);
    const int nbp = op == OP_STOKES ? (int)(psp.cell_ptr[cells[0] + 1] - psp.cell_ptr[cells[0]]) : 0;
    std::vector<int32_t> cu(cells.size() * nb), cp(cells.size() * nbp);
    std::vector<uint32_t> mk(cells.size(), 0u);
    std::vector<double> hc(cells.size());
    OpLaunch& L = g->L;
    L.dim = dim;
    L.k = k;
    L.op = op;
    L.structured = false;
    L.n = f.n;
    L.h = 1.0 / f.n;
    L.n_cells = (int64_t)cells.size();
    L.n_colors = ncol;
    L.color_ptr.assign(ncol + 1, 0);
    for (size_t i = 0; i < cells.size(); ++i) {
      const int32_t c = cells[order[i]];
      g->cells.push_back(c);
      L.color_ptr[color[order[i]] + 1]++;
      hc[i] = f.h(c);
      for (int b = 0; b < nb; ++b) {
        const int32_t node = sp.cell_nodes[sp.cell_ptr[c] + b];
        cu[i * nb + b] = node | (dirichlet && sp.boundary[node] ? int32_t(0x80000000u) : 0);
      }
      for (int b = 0; b < nbp; ++b) cp[i * nbp + b] = psp.cell_nodes[psp.cell_ptr[c] + b];
    }
    for (int c = 0; c < ncol; ++c) L.color_ptr[c + 1] += L.color_ptr[c];
    L.nu = ph.nu;
    L.dt = ph.dt;
    L.div_sign = ph.div_sign;
    L.terms = ph.terms;
    fill_tables(L);
    g->cell_u = upload(bud, cu);
    g->cell_p = upload(bud, cp);
    g->mask = upload(bud, mk);
    g->hcell[0] = upload_as<double>(bud, hc);
    g->hcell[1] = upload_as<float>(bud, hc);
    L.cell_u = g->cell_u.as<int32_t>();
    L.cell_p = op == OP_STOKES ? g->cell_p.as<int32_t>() : nullptr;
    L.mask = g->mask.as<uint32_t>();
    L.hcell[0] = g->hcell[0].get();
    L.hcell[1] = g->hcell[1].get();
    L.p_offset = lv.n_main_dofs;
    L.timer = g->timer.get();
    hp->groups.push_back(std::move(g));
  }
  // the level's own launch description stays empty: hp levels run through their groups
  lv.L = OpLaunch();
  lv.L.dim = dim;
  lv.L.k = lv.k;
  lv.L.op = op;
  // constrained rows and constraint lists (no Dirichlet slaves or masters in a Dirichlet field);
  // fields: the main one (NU components per node), then for Taylor--Hood the pressure block
  struct Field {
    const HpSpace* sp;
    int ncomp;
    bool dirichlet;
    int64_t offset;
  };
  std::vector<Field> fields = {{&sp, lv.NU, dirichlet, 0}};
  if (op == OP_STOKES) fields.push_back({&psp, 1, false, lv.n_main_dofs});
  std::vector<int32_t> hd, hptr(1, 0), hs;
  std::vector<double> hw;
  std::map<int32_t, std::vector<std::pair<int32_t, double>>> transpose;  // master dof -> (slave dof, w)
  std::vector<std::vector<char>> hangs;
  for (const Field& F : fields) {
    const HpSpace& S = *F.sp;
    std::vector<char> hang(S.n_nodes, 0);
    for (int32_t g : S.hang_node) hang[g] = 1;
    for (int64_t g = 0; g < S.n_nodes; ++g)
      if ((F.dirichlet && S.boundary[g]) || hang[g])
        for (int c = 0; c < F.ncomp; ++c) lv.constrained_host.push_back((int32_t)(F.offset + g * F.ncomp + c));
    for (size_t i = 0; i < S.hang_node.size(); ++i) {
      const int32_t g = S.hang_node[i];
      if (F.dirichlet && S.boundary[g]) continue;
      for (int c = 0; c < F.ncomp; ++c) {
        const int32_t sd = (int32_t)(F.offset + g * F.ncomp + c);
        hd.push_back(sd);
        for (int32_t j = S.hang_ptr[i]; j < S.hang_ptr[i + 1]; ++j) {
          const int32_t m = S.hang_master[j];
          if (F.dirichlet && S.boundary[m]) continue;
          const int32_t md = (int32_t)(F.offset + m * F.ncomp + c);
          hs.push_back(md);
          hw.push_back(S.hang_w[j]);
          transpose[md].push_back({sd, S.hang_w[j]});
        }
        hptr.push_back((int32_t)hs.size());
      }
    }
    hangs.push_back(std::move(hang));
  }
  std::sort(lv.constrained_host.begin(), lv.constrained_host.end());
  lv.constrained = upload(bud, lv.constrained_host);
  lv.n_hang = (int64_t)hd.size();
  lv.hang_dof = upload(bud, hd);
  lv.hang_ptr = upload(bud, hptr);
  lv.hang_src = upload(bud, hs);
  lv.hang_w[0] = upload_as<double>(bud, hw);
  lv.hang_w[1] = upload_as<float>(bud, hw);
  if (op == OP_STOKES) {  // free pressure entries: the constant-pressure null space
    for (int64_t g = 0; g < psp.n_nodes; ++g)
      if (!hangs[1][g]) lv.pres_host.push_back((int32_t)(lv.n_main_dofs + g));
    lv.n_pres = (int64_t)lv.pres_host.size();
    lv.pres = upload(bud, lv.pres_host);
  }
  std::vector<int32_t> cm, cpt(1, 0), cs;
  std::vector<double> cw;
  for (auto& kv : transpose) {
    cm.push_back(kv.first);
    for (auto& sw : kv.second) {
      cs.push_back(sw.first);
      cw.push_back(sw.second);
    }
    cpt.push_back((int32_t)cs.size());
  }
  hp->n_ct = (int64_t)cm.size();
  hp->ct_master = upload(bud, cm);
  hp->ct_ptr = upload(bud, cpt);
  hp->ct_slave = upload(bud, cs);
  hp->ct_w[0] = upload_as<double>(bud, cw);
  hp->ct_w[1] = upload_as<float>(bud, cw);
  // the exact diagonal: the main field's form (the Taylor--Hood pressure rows have no diagonal
  // block: zero), constrained rows identity
  {
    std::vector<double> dg((size_t)lv.n_dofs, 0.0);
    hp_exact_diagonal(f, sp, lv.NU, dirichlet, 0, op != OP_PMASS, ph.nu, dg);
    for (int32_t i : lv.constrained_host) dg[(size_t)i] = 1.0;
    hp->diag[0] = upload_as<double>(bud, dg);
    hp->diag[1] = upload_as<float>(bud, dg);
  }
  for (int prec = 0; prec < 2; ++prec) hp->tmp[prec].alloc(bud, lv.n_dofs * esize(prec));
  if (op == OP_STOKES) hp->pspace = std::move(psp);
  lv.hp = std::move(hp);
}

void hp_distribute(const OpLevel& lv, int prec, void* x, cudaStream_t s) { oplevel_distribute(lv, prec, x, s); }

void hp_condense(const OpLevel& lv, int prec, void* y, cudaStream_t s) {
  const HpData& H = *lv.hp;
  if (prec == 0)
    vcondense<double>((double*)y, H.ct_master.as<int32_t>(), H.ct_ptr.as<int32_t>(), H.ct_slave.as<int32_t>(),
                      H.ct_w[0].as<double>(), H.n_ct, s);
  else
    vcondense<float>((float*)y, H.ct_master.as<int32_t>(), H.ct_ptr.as<int32_t>(), H.ct_slave.as<int32_t>(),
                     H.ct_w[1].as<float>(), H.n_ct, s);
}

void hp_vmult(const OpLevel& lv, int prec, const void* src, void* dst, cudaStream_t s) {
  const HpData& H = *lv.hp;
  const int64_t n = lv.n_dofs;
  void* t = H.tmp[prec].get();
  MFNS_CUDA(cudaMemcpyAsync(t, src, n * esize(prec), cudaMemcpyDeviceToDevice, s));
  hp_distribute(lv, prec, t, s);
  MFNS_CUDA(cudaMemsetAsync(dst, 0, n * esize(prec), s));
  for (auto& g : H.groups) op_apply(g->L, prec, t, dst, false, s);
  hp_condense(lv, prec, dst, s);
  const int64_t nc = (int64_t)lv.constrained_host.size();
  if (prec == 0)
    vcopy_idx<double>((double*)dst, (const double*)src, lv.constrained.as<int32_t>(), nc, s);
  else
    vcopy_idx<float>((float*)dst, (const float*)src, lv.constrained.as<int32_t>(), nc, s);
}

void hp_diag(const OpLevel& lv, int prec, void* diag, cudaStream_t s) {
  MFNS_CUDA(cudaMemcpyAsync(diag, lv.hp->diag[prec].get(), lv.n_dofs * esize(prec), cudaMemcpyDeviceToDevice, s));
}

}  // namespace mfns
