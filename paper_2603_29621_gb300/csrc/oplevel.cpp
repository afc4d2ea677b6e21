// Operator levels: upload of cell tables, constrained rows, hanging-node
// distribution lists and the frozen state; vmult / diagonal drivers.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <unordered_map>

#include "problem.hpp"
#include "vec.hpp"

namespace mfns {

// uniform 3D stabilised / vector-Laplacian / pressure-mass levels of at most this many cells take
// deferred products
#ifndef MFNS_DEFER_MAX_CELLS
#define MFNS_DEFER_MAX_CELLS 4096
#endif
constexpr int64_t kDeferMaxCells = MFNS_DEFER_MAX_CELLS;

size_t OpLevel::bytes() const {
  size_t b = fq[0].bytes() + fq[1].bytes() + cell_u.bytes() + cell_p.bytes() + cell_f.bytes() + mask.bytes() + constrained.bytes() +
             hang_dof.bytes() + hang_ptr.bytes() + hang_src.bytes() + pres.bytes() + tnodes.bytes() +
             tpnodes.bytes();
  for (int i = 0; i < 2; ++i) b += hcell[i].bytes() + frozen[i].bytes() + hang_w[i].bytes() + dinv[i].bytes();
  return b;
}

static void taylor_green(int dim, const double* x, double* out) {
  const double tp = 2.0 * M_PI;
  if (dim == 3) {
    out[0] = std::sin(tp * x[0]) * std::cos(tp * x[1]) * std::cos(tp * x[2]);
    out[1] = -std::cos(tp * x[0]) * std::sin(tp * x[1]) * std::cos(tp * x[2]);
    out[2] = 0.0;
    out[3] = (std::cos(2 * tp * x[0]) + std::cos(2 * tp * x[1])) * (std::cos(2 * tp * x[2]) + 2.0) / 16.0;
  } else {
    out[0] = std::sin(tp * x[0]) * std::cos(tp * x[1]);
    out[1] = -std::cos(tp * x[0]) * std::sin(tp * x[1]);
    out[2] = (std::cos(2 * tp * x[0]) + std::cos(2 * tp * x[1])) / 16.0;
  }
}

template <typename T>
static DevBuf upload_as(Budget* bud, const std::vector<double>& v) {
  std::vector<T> t(v.begin(), v.end());
  return upload(bud, t);
}

void build_oplevel(OpLevel& lv, const Forest& f, int op, int k, const Physics& ph, Budget* bud, bool edge_dirichlet) {
  lv.op = op;
  lv.dim = f.dim;
  lv.k = k;
  lv.forest = f;
  const int dim = f.dim;
  lv.NU = (op == OP_STOKES_A || op == OP_VMASS) ? dim : op == OP_PMASS ? 1 : op == OP_STOKES ? dim : dim + 1;
  Lattice lat = make_lattice(f);
  std::vector<uint32_t> masks = constraint_masks(f, lat);
  std::string err;
  lv.nu = make_nodes(f, lat, masks, k, &err);
  if (!err.empty()) throw Error(kErrArg, err);
  if (op == OP_STOKES) {
    lv.np = make_nodes(f, lat, masks, k - 1, &err);
    if (!err.empty()) throw Error(kErrArg, err);
  }
  // local smoothing: homogeneous Dirichlet conditions on the refinement edge, for the velocity
  // (the boundary flag) and, for the stabilised operator, the pressure too (constrained rows)
  std::vector<uint8_t> edge_p;
  if (edge_dirichlet) {
    if (!f.partial || (op != OP_STOKES_A && op != OP_STAB_NS))
      throw Error(kErrUnsupported, "refinement-edge conditions need a level forest of the vector Laplacian or stabilised NS");
    const std::vector<uint8_t> e = refinement_edge(f, lv.nu);
    for (int64_t g = 0; g < lv.nu.n_nodes; ++g)
      if (e[g]) lv.nu.boundary[g] = 1;
    if (op == OP_STAB_NS) edge_p = e;
  }
  lv.n_main_dofs = lv.nu.n_nodes * lv.NU;
  lv.n_dofs = lv.n_main_dofs + (op == OP_STOKES ? lv.np.n_nodes : 0);
  if (lv.n_dofs >= (int64_t(1) << 31) - 1) throw Error(kErrUnsupported, "more than 2^31 DoFs per level");

  // colours and the colour-sorted cell order
  std::vector<const NodeSpace*> spaces = {&lv.nu};
  if (op == OP_STOKES) spaces.push_back(&lv.np);
  std::vector<int32_t> color;
  int ncol = color_cells(f, spaces, color);
  size_t nc = f.n_cells();
  lv.perm.resize(nc);
  std::iota(lv.perm.begin(), lv.perm.end(), 0);
  std::stable_sort(lv.perm.begin(), lv.perm.end(), [&](int32_t a, int32_t b) { return color[a] < color[b]; });
  OpLaunch& L = lv.L;
  L.dim = dim;
  L.k = k;
  L.op = op;
  L.n_cells = nc;
  L.n_colors = ncol;
  L.color_ptr.assign(ncol + 1, 0);
  for (size_t c = 0; c < nc; ++c) L.color_ptr[color[c] + 1]++;
  for (int c = 0; c < ncol; ++c) L.color_ptr[c + 1] += L.color_ptr[c];
  L.structured = f.uniform();
  L.n = f.n;
  L.h = 1.0 / f.n;
  L.nu = ph.nu;
  L.dt = ph.dt;
  L.div_sign = ph.div_sign;
  L.terms = ph.terms;
  fill_tables(L);
  L.timer = lv.timer.get();

  // cell tables in colour order
  const int nb = lv.nu.nb;
  std::vector<int32_t> cu(nc * nb), cf, cp;
  std::vector<uint32_t> mk(nc);
  std::vector<double> hc(nc);
  const bool need_f = op == OP_STAB_NS && !f.uniform();
  if (need_f) cf.resize(nc * nb);
  for (size_t i = 0; i < nc; ++i) {
    const int32_t c = lv.perm[i];
    mk[i] = masks[c];
    hc[i] = f.h(c);
    for (int b = 0; b < nb; ++b) {
      const int32_t g = lv.nu.cell_master[(size_t)c * nb + b];
      const bool bnd = op != OP_PMASS && lv.nu.boundary[g];
      cu[i * nb + b] = g | (bnd ? int32_t(0x80000000u) : 0);
      if (need_f) cf[i * nb + b] = lv.nu.cell_nodes[(size_t)c * nb + b];
    }
  }
  if (op == OP_STOKES) {
    const int nbp = lv.np.nb;
    cp.resize(nc * nbp);
    for (size_t i = 0; i < nc; ++i)
      for (int b = 0; b < nbp; ++b) cp[i * nbp + b] = lv.np.cell_master[(size_t)lv.perm[i] * nbp + b];
  }
  // last colour touching each main node (fused smoother / residual epilogue): colours run in
  // index order, so it is the largest colour index among the cells whose slots name the node
  if (op != OP_STOKES) {
    std::vector<uint8_t> lc(lv.nu.n_nodes, 0);
    if (L.structured) {  // the structured launch's colour = parity bits of the cell coordinates
      const int n = f.n;
      const int64_t M = (int64_t)k * n + 1;
      for (int64_t g = 0; g < lv.nu.n_nodes; ++g) {
        int64_t idx[3] = {g % M, (g / M) % M, dim == 3 ? g / (M * M) : 0};
        int col = 0;
        for (int d = 0; d < dim; ++d) {
          // cells touching the node along d: i/k, and i/k - 1 when the node lies on a cell face
          const int64_t i = idx[d];
          int bit = 0;
          const int64_t c0 = i / k;
          if (c0 < n && (c0 & 1)) bit = 1;
          if (i % k == 0 && c0 - 1 >= 0 && ((c0 - 1) & 1)) bit = 1;
          col |= bit << d;
        }
        lc[g] = (uint8_t)col;
      }
    } else {
      if (ncol > 255) throw Error(kErrUnsupported, "more than 255 cell colours");
      for (int c = 0; c < ncol; ++c)
        for (int32_t i = L.color_ptr[c]; i < L.color_ptr[c + 1]; ++i)
          for (int b = 0; b < nb; ++b) lc[cu[(size_t)i * nb + b] & 0x7fffffff] = (uint8_t)c;
    }
    lv.lastc = upload(bud, lc);
    L.lastc = lv.lastc.as<uint8_t>();
  }
  lv.cell_u = upload(bud, cu);
  lv.cell_p = upload(bud, cp);
  lv.cell_f = upload(bud, cf);
  lv.mask = upload(bud, mk);
  lv.hcell[0] = upload_as<double>(bud, hc);
  lv.hcell[1] = upload_as<float>(bud, hc);
  L.cell_u = lv.cell_u.as<int32_t>();
  L.cell_p = lv.cell_p.as<int32_t>();
  L.cell_f = lv.cell_f.as<int32_t>();
  L.mask = lv.mask.as<uint32_t>();
  L.hcell[0] = lv.hcell[0].get();
  L.hcell[1] = lv.hcell[1].get();
  L.p_offset = lv.n_main_dofs;

  // frozen state (stabilised NS): nodal interpolant of the Taylor--Green field
  if (op == OP_STAB_NS) {
    std::vector<double> fz(lv.n_main_dofs);
    double xyz[3] = {0, 0, 0}, v[4];
    for (int64_t g = 0; g < lv.nu.n_nodes; ++g) {
      for (int d = 0; d < dim; ++d) xyz[d] = lv.nu.x[g * dim + d];
      taylor_green(dim, xyz, v);
      for (int c = 0; c <= dim; ++c) fz[g * lv.NU + c] = v[c];
    }
    lv.frozen[0] = upload_as<double>(bud, fz);
    lv.frozen[1] = upload_as<float>(bud, fz);
    L.frozen[0] = lv.frozen[0].get();
    L.frozen[1] = lv.frozen[1].get();
    if (ph.precompute_frozen) {
      // point values of the frozen state (u, grad u, Rbar, tau), computed once by the cell kernel
      const int64_t per_cell = frozen_point_values_per_cell(dim, k);
      for (int prec = 0; prec < 2; ++prec) {
        lv.fq[prec].alloc(bud, (size_t)nc * per_cell * esize(prec));
        L.fq[prec] = lv.fq[prec].get();
        op_precompute_frozen(L, prec, 0);
      }
      MFNS_CUDA(cudaStreamSynchronize(0));
    }
  }

  // constrained rows, hanging distribution, pressure entries
  std::vector<char> hang(lv.nu.n_nodes, 0);
  for (int32_t g : lv.nu.hang_node) hang[g] = 1;
  const bool has_dir = op != OP_PMASS;
  const int nvel = op == OP_STAB_NS ? dim : (op == OP_PMASS ? 0 : dim);
  std::vector<int32_t> hd, hp(1, 0), hs;
  std::vector<double> hw;
  for (int64_t g = 0; g < lv.nu.n_nodes; ++g) {
    const bool bnd = has_dir && lv.nu.boundary[g];
    const bool pedge = !edge_p.empty() && edge_p[g];
    for (int c = 0; c < lv.NU; ++c) {
      const bool dir = (bnd && c < nvel) || (pedge && c == dim);
      if (dir || hang[g]) lv.constrained_host.push_back((int32_t)(g * lv.NU + c));
    }
  }
  for (size_t i = 0; i < lv.nu.hang_node.size(); ++i) {
    const int32_t g = lv.nu.hang_node[i];
    const bool bnd = has_dir && lv.nu.boundary[g];
    for (int c = 0; c < lv.NU; ++c) {
      if (bnd && c < nvel) continue;
      hd.push_back((int32_t)(g * lv.NU + c));
      for (int32_t j = lv.nu.hang_ptr[i]; j < lv.nu.hang_ptr[i + 1]; ++j) {
        hs.push_back((int32_t)(lv.nu.hang_master[j] * lv.NU + c));
        hw.push_back(lv.nu.hang_w[j]);
      }
      hp.push_back((int32_t)hs.size());
    }
  }
  if (op == OP_STOKES) {
    std::vector<char> hangp(lv.np.n_nodes, 0);
    for (int32_t g : lv.np.hang_node) hangp[g] = 1;
    for (int64_t g = 0; g < lv.np.n_nodes; ++g)
      if (hangp[g]) lv.constrained_host.push_back((int32_t)(lv.n_main_dofs + g));
    for (size_t i = 0; i < lv.np.hang_node.size(); ++i) {
      hd.push_back((int32_t)(lv.n_main_dofs + lv.np.hang_node[i]));
      for (int32_t j = lv.np.hang_ptr[i]; j < lv.np.hang_ptr[i + 1]; ++j) {
        hs.push_back((int32_t)(lv.n_main_dofs + lv.np.hang_master[j]));
        hw.push_back(lv.np.hang_w[j]);
      }
      hp.push_back((int32_t)hs.size());
    }
    for (int64_t g = 0; g < lv.np.n_nodes; ++g)
      if (!hangp[g]) lv.pres_host.push_back((int32_t)(lv.n_main_dofs + g));
  } else if (op == OP_STAB_NS) {
    for (int64_t g = 0; g < lv.nu.n_nodes; ++g)
      if (!hang[g] && (edge_p.empty() || !edge_p[g])) lv.pres_host.push_back((int32_t)(g * lv.NU + dim));
  }
  std::sort(lv.constrained_host.begin(), lv.constrained_host.end());
  lv.constrained = upload(bud, lv.constrained_host);
  // uniform meshes: the constrained rows are the velocity rows of boundary nodes, which the
  // structured cell kernels never write; the clearing kernel of a product sets them from its mask
  if (lv.L.structured && lv.n_dofs > 0) {
    std::vector<uint32_t> km((size_t)((lv.n_dofs + 31) / 32), 0u);
    for (int32_t i : lv.constrained_host) km[(size_t)i >> 5] |= 1u << (i & 31);
    lv.keep_mask = upload(bud, km);
  }
  // small uniform 3D stabilised, vector-Laplacian and pressure-mass levels: products as one launch
  // over all colours plus a gather pass (their eight colour launches are latency, not work)
  if (lv.L.structured && (op == OP_STAB_NS || op == OP_STOKES_A || op == OP_PMASS) && dim == 3 &&
      (int64_t)lv.L.n_cells <= kDeferMaxCells) {
    const size_t entries = (size_t)lv.L.n_cells * (size_t)((k + 1) * (k + 1) * (k + 1)) * lv.NU;
    for (int prec = 0; prec < 2; ++prec) lv.defer[prec].alloc(bud, entries * esize(prec));
  }
  lv.n_hang = (int64_t)hd.size();
  lv.hang_dof = upload(bud, hd);
  lv.hang_ptr = upload(bud, hp);
  lv.hang_src = upload(bud, hs);
  lv.hang_w[0] = upload_as<double>(bud, hw);
  lv.hang_w[1] = upload_as<float>(bud, hw);
  lv.n_pres = (int64_t)lv.pres_host.size();
  lv.pres = upload(bud, lv.pres_host);
}

void oplevel_vmult(const OpLevel& lv, int prec, const void* src, void* dst, cudaStream_t s) {
  if (lv.hp) return hp_vmult(lv, prec, src, dst, s);
  // clearing kernel, then the colour launches (each may start before its predecessor drains);
  // on uniform meshes the clearing kernel also writes the identity rows, which no colour touches
  if (lv.defer[prec].get()) {  // small uniform levels: one launch over all colours, one gather pass
    op_apply_deferred(lv.L, prec, src, dst, lv.defer[prec].get(), s);
    return;
  }
  if (lv.keep_mask.get()) {
    op_apply_cleared(lv.L, prec, src, dst, lv.n_dofs, s, lv.keep_mask.as<uint32_t>());
    return;
  }
  op_apply_cleared(lv.L, prec, src, dst, lv.n_dofs, s);
  const int64_t nc = (int64_t)lv.constrained_host.size();
  if (prec == 0)
    vcopy_idx<double>((double*)dst, (const double*)src, lv.constrained.as<int32_t>(), nc, s);
  else
    vcopy_idx<float>((float*)dst, (const float*)src, lv.constrained.as<int32_t>(), nc, s);
}

void oplevel_vmult_cols(const OpLevel& lv, int prec, const void* X, void* Y, int ncols, cudaStream_t s) {
  if (lv.hp) throw Error(kErrUnsupported, "multi-column products of hp levels");
  const int64_t n = lv.n_dofs;
  MFNS_CUDA(cudaMemsetAsync(Y, 0, (size_t)ncols * n * esize(prec), s));
  op_apply_cols(lv.L, prec, X, Y, ncols, n, s);
  const int64_t nc = (int64_t)lv.constrained_host.size();
  if (prec == 0)
    vcopy_idx_cols<double>((double*)Y, (const double*)X, lv.constrained.as<int32_t>(), nc, n, ncols, s);
  else
    vcopy_idx_cols<float>((float*)Y, (const float*)X, lv.constrained.as<int32_t>(), nc, n, ncols, s);
}

void oplevel_smooth_step(const OpLevel& lv, int prec, const void* x, void* xout, void* d, const void* b,
                         const void* dinv, void* t, double c1, double c2, cudaStream_t s) {
  MFNS_CUDA(cudaMemsetAsync(t, 0, lv.n_dofs * esize(prec), s));
  OpEpilogue e;
  e.mode = 1;
  e.b = b;
  e.dinv = dinv;
  e.d = d;
  e.xout = xout;
  e.c1 = c1;
  e.c2 = c2;
  op_apply_epi(lv.L, prec, x, t, e, s);
  const int64_t nc = (int64_t)lv.constrained_host.size();
  if (prec == 0)
    vcheby_idx<double>((const double*)x, (double*)xout, (double*)d, (const double*)b, (const double*)dinv, c1, c2,
                       lv.constrained.as<int32_t>(), nc, s);
  else
    vcheby_idx<float>((const float*)x, (float*)xout, (float*)d, (const float*)b, (const float*)dinv, (float)c1,
                      (float)c2, lv.constrained.as<int32_t>(), nc, s);
}

void oplevel_residual_fused(const OpLevel& lv, int prec, const void* x, const void* b, void* r, void* t,
                            cudaStream_t s) {
  MFNS_CUDA(cudaMemsetAsync(t, 0, lv.n_dofs * esize(prec), s));
  OpEpilogue e;
  e.mode = 2;
  e.b = b;
  e.xout = r;
  op_apply_epi(lv.L, prec, x, t, e, s);
  const int64_t nc = (int64_t)lv.constrained_host.size();
  if (prec == 0)
    vsub_idx<double>((double*)r, (const double*)b, (const double*)x, lv.constrained.as<int32_t>(), nc, s);
  else
    vsub_idx<float>((float*)r, (const float*)b, (const float*)x, lv.constrained.as<int32_t>(), nc, s);
}

void oplevel_diag(const OpLevel& lv, int prec, void* diag, cudaStream_t s) {
  if (lv.hp) return hp_diag(lv, prec, diag, s);
  MFNS_CUDA(cudaMemsetAsync(diag, 0, lv.n_dofs * esize(prec), s));
  op_apply(lv.L, prec, nullptr, diag, true, s);
  const int64_t nc = (int64_t)lv.constrained_host.size();
  if (prec == 0)
    vset_idx<double>((double*)diag, 1.0, lv.constrained.as<int32_t>(), nc, s);
  else
    vset_idx<float>((float*)diag, 1.0f, lv.constrained.as<int32_t>(), nc, s);
}

void oplevel_distribute(const OpLevel& lv, int prec, void* x, cudaStream_t s) {
  if (prec == 0)
    vdistribute<double>((double*)x, lv.hang_dof.as<int32_t>(), lv.hang_ptr.as<int32_t>(), lv.hang_src.as<int32_t>(),
                        lv.hang_w[0].as<double>(), lv.n_hang, s);
  else
    vdistribute<float>((float*)x, lv.hang_dof.as<int32_t>(), lv.hang_ptr.as<int32_t>(), lv.hang_src.as<int32_t>(),
                       lv.hang_w[1].as<float>(), lv.n_hang, s);
}

void oplevel_support(const OpLevel& lv, double* xyz, int* field) {
  const int dim = lv.dim;
  for (int64_t g = 0; g < lv.nu.n_nodes; ++g)
    for (int c = 0; c < lv.NU; ++c) {
      const int64_t i = g * lv.NU + c;
      for (int d = 0; d < 3; ++d) xyz[3 * i + d] = d < dim ? lv.nu.x[g * dim + d] : 0.0;
      field[i] = lv.op == OP_PMASS ? dim : c;
    }
  if (lv.op == OP_STOKES)
    for (int64_t g = 0; g < lv.np.n_nodes; ++g) {
      const int64_t i = lv.n_main_dofs + g;
      for (int d = 0; d < 3; ++d) xyz[3 * i + d] = d < dim ? lv.np.x[g * dim + d] : 0.0;
      field[i] = dim;
    }
}

}  // namespace mfns
