// Hierarchy set-up, smoothers, V-cycle, coarse solver and FGMRES.
//
// Section 3: A^{-1} is approximated by one V-cycle of global-coarsening
// multigrid (p-coarsening to linear elements first, then h); Section 5: the
// stabilised system uses a monolithic hierarchy with h-coarsening first.
// Smoothers: Chebyshev iteration around point Jacobi (Saad, Alg. 12.1 on
// D^{-1} A, lmin = lmax / 20) or Jacobi relaxation with w = 2 / (lmin + lmax).
// Coarse level: dense inverse (host LU), or Chebyshev of degree 30 when the
// coarse system is larger than 4096 unknowns.  FGMRES(m) with classical
// Gram--Schmidt applied twice (Section 3 "We solve the Stokes system with FGMRES").
#include <algorithm>
#include <array>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <chrono>
#include <cmath>
#include <cstring>
#include <random>

#include "problem.hpp"
#include "ritz.hpp"
#include "vec.hpp"

namespace mfns {

static int mg_op_of(int kind) {
  switch (kind) {
    case 0: return OP_STOKES_A;  // Stokes: multigrid on the A block
    case 1: return OP_STOKES_A;
    case 2: return OP_STAB_NS;
    default: return OP_PMASS;
  }
}
static int sys_op_of(int kind) {
  switch (kind) {
    case 0: return OP_STOKES;
    case 1: return OP_STOKES_A;
    case 2: return OP_STAB_NS;
    default: return OP_PMASS;
  }
}

Problem::~Problem() {
  invalidate_graphs(*this);
  if (cap_stream) cudaStreamDestroy(cap_stream);
  if (hh_host) cudaFreeHost(hh_host);
  if (ev_step) cudaEventDestroy(ev_step);
}

static std::atomic<uint64_t> g_problem_uid{0};
static int64_t sys_of_n(const Problem& p) { return p.system ? p.system->n_dofs : p.levels[0]->n_dofs; }

static void build_local_smoothing(Problem& p, const Forest& f, int k, const Physics& ph, int mg_order,
                                  int coarse_stop_n, Budget* bud);

std::unique_ptr<Problem> build_problem(const Forest& f, int kind, int k, const Physics& ph, int mg_order,
                                       int coarse_stop_n, Budget* bud, int hierarchy) {
  auto p = std::make_unique<Problem>();
  p->uid = ++g_problem_uid;
  p->kind = kind;
  p->dim = f.dim;
  p->k = k;
  p->phys = ph;
  p->bud = bud;
  const int mop = mg_op_of(kind);
  if (mg_order == 0) mg_order = kind == 2 ? 2 : 1;
  // (forest, degree) sequence of the hierarchy, finest first
  std::vector<std::pair<Forest, int>> seq;
  const bool local = hierarchy == 1 && f.max_level() > 0;
  if (hierarchy == 1 && mop != OP_STOKES_A && mop != OP_STAB_NS)
    throw Error(kErrUnsupported, "local smoothing is built for the vector Laplacian, the Stokes A block and stabilised NS");
  if (kind == 3 || local) {
    seq.push_back({f, k});  // local smoothing: the fine operator only; the levels live in p->ls
  } else {
    std::vector<Forest> fs{f};
    while (forest_can_coarsen(fs.back(), coarse_stop_n)) fs.push_back(forest_coarsen(fs.back()));
    if (mg_order == 1) {
      for (int kk = k; kk >= 1; --kk) seq.push_back({f, kk});
      for (size_t i = 1; i < fs.size(); ++i) seq.push_back({fs[i], 1});
    } else {
      for (auto& ff : fs) seq.push_back({ff, k});
      for (int kk = k - 1; kk >= 1; --kk) seq.push_back({fs.back(), kk});
    }
  }
  if (seq.size() > 32) throw Error(kErrUnsupported, "more than 32 multigrid levels");
  for (auto& s : seq) {
    auto lv = std::make_unique<OpLevel>();
    build_oplevel(*lv, s.first, mop, s.second, ph, bud);
    p->levels.push_back(std::move(lv));
  }
  for (size_t l = 0; l + 1 < p->levels.size(); ++l) {
    auto t = std::make_unique<Transfer>();
    build_transfer(*t, *p->levels[l], *p->levels[l + 1], bud);
    p->transfers.push_back(std::move(t));
  }
  if (kind == 0) {
    p->system = std::make_unique<OpLevel>();
    build_oplevel(*p->system, f, OP_STOKES, k, ph, bud);
    p->pmass = std::make_unique<OpLevel>();
    build_oplevel(*p->pmass, f, OP_PMASS, k - 1, ph, bud);
  }
  if (local) build_local_smoothing(*p, f, k, ph, mg_order, coarse_stop_n, bud);
  return p;
}

static void level_copy_list(const OpLevel& fine, const OpLevel& lvl, int l, const std::vector<uint8_t>& edge,
                            std::vector<int32_t>& owner, std::vector<int32_t>& cf, std::vector<int32_t>& cl) {
  std::string err;
  // the stabilised system's pressure has no boundary condition: its boundary nodes need owners
  const bool own_boundary = fine.op == OP_STAB_NS;
  if (!ls_owned_nodes(fine.forest, fine.nu, lvl.forest, lvl.nu, edge, l, owner, cf, cl, &err, own_boundary))
    throw Error(kErrArg, "local smoothing: " + err);
}

static void build_local_smoothing(Problem& p, const Forest& f, int k, const Physics& ph, int mg_order,
                                  int coarse_stop_n, Budget* bud) {
  auto S = std::make_unique<LocalSmoothing>();
  const OpLevel& fine = *p.levels[0];
  const int L = f.max_level();
  // level 0 and below: the base mesh with its own global-coarsening hierarchy (vector Laplacian)
  Forest base = forest_uniform(f.dim, f.n);
  const int mop = fine.op;  // OP_STOKES_A (vector Laplacian, Stokes A block) or OP_STAB_NS
  S->base = build_problem(base, mop == OP_STAB_NS ? 2 : 1, k, ph, mg_order, coarse_stop_n, bud, 0);
  std::vector<int32_t> owner(fine.nu.n_nodes, -1);
  std::vector<int32_t> cf, cl;
  {
    const OpLevel& b0 = *S->base->levels[0];
    level_copy_list(fine, b0, 0, std::vector<uint8_t>(b0.nu.n_nodes, 0), owner, cf, cl);
    S->n_copy = (int64_t)cf.size();
    S->copy_fine = upload(bud, cf);
    S->copy_lvl = upload(bud, cl);
  }
  const int64_t cap = sys_of_n(p);
  for (int l = 1; l <= L; ++l) {
    auto lv = std::make_unique<LsLevel>();
    const Forest lf = forest_level(f, l);
    lv->op = std::make_unique<OpLevel>();
    build_oplevel(*lv->op, lf, mop, k, ph, bud, true);
    lv->full = std::make_unique<OpLevel>();
    build_oplevel(*lv->full, lf, mop, k, ph, bud, false);
    if (lv->op->n_dofs != lv->full->n_dofs || lv->op->perm != lv->full->perm)
      throw Error(kErrArg, "local smoothing: level operators disagree on the numbering");
    if (lv->op->n_dofs > cap) throw Error(kErrUnsupported, "local smoothing: level larger than the fine system");
    const OpLevel& coarse = l == 1 ? *S->base->levels[0] : *S->lv.back()->full;
    build_transfer(lv->down, *lv->full, coarse, bud, true);
    const std::vector<uint8_t> edge = refinement_edge(lf, lv->full->nu);
    cf.clear();
    cl.clear();
    level_copy_list(fine, *lv->full, l, edge, owner, cf, cl);
    lv->n_copy = (int64_t)cf.size();
    lv->copy_fine = upload(bud, cf);
    lv->copy_lvl = upload(bud, cl);
    for (int prec = 0; prec < 2; ++prec) {
      const size_t b = lv->op->n_dofs * esize(prec);
      Workspace& w = lv->ws[prec];
      w.r.alloc(bud, b);
      w.d.alloc(bud, b);
      w.t.alloc(bud, b);
      w.b.alloc(bud, b);
      w.x.alloc(bud, b);
      lv->z[prec].alloc(bud, b);
      lv->c[prec].alloc(bud, b);
      for (DevBuf* v : {&w.r, &w.d, &w.t, &w.b, &w.x, &lv->z[prec], &lv->c[prec]}) MFNS_CUDA(cudaMemset(v->get(), 0, b));
    }
    S->lv.push_back(std::move(lv));
  }
  // every free fine node has exactly one owner
  if (!ls_all_owned(fine.nu, owner, fine.op == OP_STAB_NS))
    throw Error(kErrArg, "local smoothing: a free fine DoF is owned by no level");
  for (int prec = 0; prec < 2; ++prec) {
    const size_t b = S->base->levels[0]->n_dofs * esize(prec);
    S->b[prec].alloc(bud, b);
    S->x[prec].alloc(bud, b);
    S->c[prec].alloc(bud, b);
  }
  alloc_level_workspaces(*S->base);
  p.ls = std::move(S);
}

std::unique_ptr<Problem> build_problem_hp(const Forest& f, const std::vector<int32_t>& degree, const Physics& ph,
                                          int coarse_stop_n, Budget* bud, int kind) {
  if (degree.size() != f.n_cells()) throw Error(kErrArg, "one degree per cell expected");
  if (kind != 0 && kind != 1) throw Error(kErrUnsupported, "hp problems: Stokes or its A block");
  auto uniform = [](const std::vector<int32_t>& d) {
    return std::all_of(d.begin(), d.end(), [&](int32_t k) { return k == d[0]; });
  };
  if (uniform(degree)) return build_problem(f, kind, degree[0], ph, 1, coarse_stop_n, bud, 0);
  auto p = std::make_unique<Problem>();
  p->uid = ++g_problem_uid;
  p->kind = kind;
  p->dim = f.dim;
  p->k = *std::max_element(degree.begin(), degree.end());
  p->phys = ph;
  p->bud = bud;
  // Section 3: every cell's degree lowered by one per level until all cells are linear ...
  std::vector<int32_t> d = degree;
  while (!uniform(d)) {
    auto lv = std::make_unique<OpLevel>();
    build_hp_oplevel(*lv, f, d, ph, bud);
    p->levels.push_back(std::move(lv));
    for (auto& k : d) k = std::max(k - 1, 1);
  }
  for (int kk = d[0]; kk >= 1; --kk) {  // (all linear after the loop; kept general)
    auto lv = std::make_unique<OpLevel>();
    build_oplevel(*lv, f, OP_STOKES_A, kk, ph, bud);
    p->levels.push_back(std::move(lv));
  }
  // ... then global coarsening with linear elements
  Forest fc = f;
  while (forest_can_coarsen(fc, coarse_stop_n)) {
    fc = forest_coarsen(fc);
    auto lv = std::make_unique<OpLevel>();
    build_oplevel(*lv, fc, OP_STOKES_A, 1, ph, bud);
    p->levels.push_back(std::move(lv));
  }
  if (p->levels.size() > 32) throw Error(kErrUnsupported, "more than 32 multigrid levels");
  for (size_t l = 0; l + 1 < p->levels.size(); ++l) {
    auto t = std::make_unique<Transfer>();
    if (p->levels[l]->hp)
      build_hp_transfer(*t, *p->levels[l], *p->levels[l + 1], bud);
    else
      build_transfer(*t, *p->levels[l], *p->levels[l + 1], bud);
    p->transfers.push_back(std::move(t));
  }
  if (kind == 0) {  // Taylor--Hood system and the pressure mass of the Schur complement (Eq. 5)
    p->system = std::make_unique<OpLevel>();
    build_hp_oplevel(*p->system, f, degree, ph, bud, OP_STOKES);
    std::vector<int32_t> dp(degree);
    for (auto& k : dp) k -= 1;
    p->pmass = std::make_unique<OpLevel>();
    build_hp_oplevel(*p->pmass, f, dp, ph, bud, OP_PMASS);
  }
  return p;
}

int mg_level_count(const Problem& p) {
  if (!p.ls) return (int)p.levels.size();
  return (int)(p.ls->lv.size() + p.ls->base->levels.size());
}

OpLevel& mg_level(Problem& p, int i) {
  if (!p.ls) return *p.levels.at(i);
  const int nl = (int)p.ls->lv.size();
  if (i < nl) return *p.ls->lv[nl - 1 - i]->op;
  return *p.ls->base->levels.at(i - nl);
}

static OpLevel& sys_of(Problem& p) { return p.system ? *p.system : *p.levels[0]; }
static double host_dot(Problem& p, const double* a, const double* b, int64_t n, cudaStream_t s);
double arnoldi_spectral_radius(Problem& p, OpLevel& lv, cudaStream_t s,
                               std::vector<std::complex<double>>* ritz = nullptr);

// Timers record events on the launching stream; they are paused while a graph is captured.
struct TimerPause {
  std::vector<std::pair<KernelTimer*, bool>> saved;
  explicit TimerPause(Problem& p) {
    for (auto& lv : p.levels) keep(lv->timer.get());
    if (p.system) keep(p.system->timer.get());
    if (p.pmass) keep(p.pmass->timer.get());
  }
  void keep(KernelTimer* t) {
    saved.push_back({t, t->enabled});
    t->enabled = false;
  }
  ~TimerPause() {
    for (auto& s : saved) s.first->enabled = s.second;
  }
};

void alloc_level_workspaces(Problem& p) {
  Budget* bud = p.bud;
  for (int prec = 0; prec < 2; ++prec) {
    p.ws[prec].clear();
    p.ws[prec].resize(p.levels.size());
    for (size_t l = 0; l < p.levels.size(); ++l) {
      const size_t b = p.levels[l]->n_dofs * esize(prec);
      Workspace& w = p.ws[prec][l];
      w.r.alloc(bud, b);
      w.d.alloc(bud, b);
      w.t.alloc(bud, b);
      w.b.alloc(bud, b);
      w.x.alloc(bud, b);
      // defined contents: a smoothing step with coefficient 0 on the previous direction (the fused
      // epilogue multiplies it) must not meet NaN bit patterns left in recycled device memory
      for (DevBuf* v : {&w.r, &w.d, &w.t, &w.b, &w.x}) MFNS_CUDA(cudaMemset(v->get(), 0, b));
    }
  }
}

void alloc_workspaces(Problem& p) {
  Budget* bud = p.bud;
  alloc_level_workspaces(p);
  OpLevel& S = sys_of(p);
  const int64_t n = S.n_dofs;
  const int m = p.restart;
  p.V.alloc(bud, (size_t)(m + 1) * n * 8);
  p.Z.alloc(bud, (size_t)m * n * 8);
  p.w.alloc(bud, n * 8);
  p.tmp.alloc(bud, n * 8);
  p.sys_r.alloc(bud, n * 8);
  p.sys_z.alloc(bud, n * 8);
  p.hvec.alloc(bud, 2 * kMaxDots * 8);
  p.yvec.alloc(bud, kMaxDots * 8);
  p.part.alloc(bud, (size_t)kRedBlocks * kMaxDots * 8);
  p.scal.alloc(bud, 16 * 8);
  std::vector<const double*> pv(m + 1), pz(m);
  for (int j = 0; j <= m; ++j) pv[j] = p.V.as<double>() + (size_t)j * n;
  for (int j = 0; j < m; ++j) pz[j] = p.Z.as<double>() + (size_t)j * n;
  p.ptrV = upload(bud, pv);
  p.ptrZ = upload(bud, pz);
  if (!p.hh_host) MFNS_CUDA(cudaMallocHost(&p.hh_host, (2 * kMaxDots + 2) * sizeof(double)));
  p.mg_b32.alloc(bud, n * 4);
  p.mg_x32.alloc(bud, n * 4);
  p.pc_in.alloc(bud, n * 8);
  p.pc_out.alloc(bud, n * 8);
  for (int prec = 0; prec < 2; ++prec) {
    p.vc_in[prec].alloc(bud, p.levels[0]->n_dofs * esize(prec));
    p.vc_out[prec].alloc(bud, p.levels[0]->n_dofs * esize(prec));
  }
  if (p.kind == 0) {
    const int64_t np = p.pmass->n_dofs;
    const size_t es = 8;  // the Stokes preconditioner keeps fp64 and fp32 copies in separate buffers
    p.cg_r.alloc(bud, np * es);
    p.cg_z.alloc(bud, np * es);
    p.cg_p.alloc(bud, np * es);
    p.cg_q.alloc(bud, np * es);
    p.cg_x.alloc(bud, np * es);
    p.stokes_u_rhs.alloc(bud, n * es);
    p.stokes_u_sol.alloc(bud, n * es);
    p.pmass->dinv[0].alloc(bud, np * 8);
    p.pmass->dinv[1].alloc(bud, np * 4);
  }
}

// fp32: evaluate the diagonal in FP32 whatever the multigrid precision (Newton refreshes: the
// diagonal only scales the smoother's correction, and FP64 cell kernels run at 1/60 the rate)
static void level_dinv(Problem& p, OpLevel& lv, cudaStream_t s, bool fp32 = false) {
  const int64_t n = lv.n_dofs;
  // kept across refreshes (captured graphs hold these pointers)
  if (lv.dinv[0].bytes() != (size_t)n * 8) lv.dinv[0].alloc(p.bud, n * 8);
  if (lv.dinv[1].bytes() != (size_t)n * 4) lv.dinv[1].alloc(p.bud, n * 4);
  // the diagonal in the multigrid precision (fp32 mode never evaluates fp64 cell kernels here)
  if (p.mg_precision == 1 || fp32) {
    oplevel_diag(lv, 1, lv.dinv[1].get(), s);
    vrecip<float>(lv.dinv[1].as<float>(), lv.dinv[1].as<float>(), n, s);
    vcast_f2d(lv.dinv[0].as<double>(), lv.dinv[1].as<float>(), n, s);
  } else {
    oplevel_diag(lv, 0, lv.dinv[0].get(), s);
    vrecip<double>(lv.dinv[0].as<double>(), lv.dinv[0].as<double>(), n, s);
    vcast_d2f(lv.dinv[1].as<float>(), lv.dinv[0].as<double>(), n, s);
  }
}

void autotune(Problem& p, cudaStream_t s) {
  // scratch: the level workspaces (contents are overwritten before any use)
  for (int prec = 0; prec < 2; ++prec)
    for (size_t l = 0; l < p.levels.size(); ++l) {
      Workspace& w = p.ws[prec][l];
      OpLevel& lv = *p.levels[l];
      MFNS_CUDA(cudaMemsetAsync(w.x.get(), 0, lv.n_dofs * esize(prec), s));
      if (lv.hp) {  // hp levels: every degree group on its own
        for (auto& g : lv.hp->groups) autotune_warps(g->L, prec, w.x.get(), w.t.get(), lv.n_dofs, s);
      } else {
        autotune_warps(lv.L, prec, w.x.get(), w.t.get(), lv.n_dofs, s);
      }
    }
  if (p.ls) {
    for (auto& lv : p.ls->lv)
      for (int prec = 0; prec < 2; ++prec) {
        Workspace& w = lv->ws[prec];
        MFNS_CUDA(cudaMemsetAsync(w.x.get(), 0, lv->op->n_dofs * esize(prec), s));
        autotune_warps(lv->op->L, prec, w.x.get(), w.t.get(), lv->op->n_dofs, s);
        autotune_warps(lv->full->L, prec, w.x.get(), w.t.get(), lv->full->n_dofs, s);
      }
    autotune(*p.ls->base, s);
  }
  for (OpLevel* lv : {p.system.get(), p.pmass.get()}) {
    if (!lv) continue;
    for (int prec = 0; prec < 2; ++prec) {
      void* a = prec == 0 ? p.w.get() : p.mg_b32.get();
      void* b = prec == 0 ? p.tmp.get() : p.mg_x32.get();
      if ((int64_t)lv->n_dofs > (int64_t)sys_of(p).n_dofs) continue;
      MFNS_CUDA(cudaMemsetAsync(a, 0, lv->n_dofs * esize(prec), s));
      if (lv->hp) {  // hp operators: every degree group on its own (the level's own launch is empty)
        for (auto& g : lv->hp->groups) autotune_warps(g->L, prec, a, b, lv->n_dofs, s);
      } else {
        autotune_warps(lv->L, prec, a, b, lv->n_dofs, s);
      }
    }
  }
}

static void sync_ls_settings(Problem& p) {
  Problem& B = *p.ls->base;
  B.smoother = p.smoother;
  B.smoother_degree = p.smoother_degree;
  B.mg_precision = p.mg_precision;
  B.fused_smoother = p.fused_smoother;
  B.coarse_cheby_degree = p.coarse_cheby_degree;
}

void estimate_lambda(Problem& p, cudaStream_t s) {
  if (p.kind == 0) {  // Stokes: the pressure mass diagonal of the Schur-complement CG
    OpLevel& pm = *p.pmass;
    oplevel_diag(pm, 0, pm.dinv[0].get(), s);
    vrecip<double>(pm.dinv[0].as<double>(), pm.dinv[0].as<double>(), pm.n_dofs, s);
    vcast_d2f(pm.dinv[1].as<float>(), pm.dinv[0].as<double>(), pm.n_dofs, s);
  }
  if (p.ls) {  // the levels the cycle smooths on: refined levels and the base hierarchy
    sync_ls_settings(p);
    const int nl = mg_level_count(p);
    for (int i = 0; i < nl; ++i) level_dinv(p, mg_level(p, i), s);
    for (int i = 0; i < nl; ++i) {
      OpLevel& lv = mg_level(p, i);
      if (lv.lmax > 0) continue;
      if (lv.n_dofs > sys_of(p).n_dofs) throw Error(kErrUnsupported, "multigrid level larger than the system");
      std::vector<std::complex<double>> ritz;
      const double rho = arnoldi_spectral_radius(p, lv, s, &ritz);
      const double w = p.smoother == 1 ? relaxation_weight(ritz) : 0.0;
      lv.lmax = p.smoother != 1 ? 1.2 * rho : (w > 0.0 && std::isfinite(w)) ? 2.0 / (1.05 * w) : 2.0 * rho;
    }
    return;
  }
  // diagonals, then the Arnoldi estimate of lambda_max(D^{-1} A) per level
  for (auto& lv : p.levels) level_dinv(p, *lv, s);
  // Section 3's blended smoother: Schwarz blocks on the combined faces of hp levels (the estimate
  // below is then of lambda_max(P^{-1} A))
  if (p.smoother == 2)
    for (auto& lv : p.levels)
      if (lv->hp && !lv->hp->asm_) build_hp_asm(*lv, p.bud, s);
  // lambda_max of D^{-1} A per level: Arnoldi (classical Gram--Schmidt twice) in FP64 from a
  // seeded random start; the estimate is the spectral radius rho of the m x m Hessenberg matrix
  // (the modulus of its largest Ritz value), times 1.2 for the Chebyshev smoother.  The
  // relaxation smoother's weight omega minimises max |1 - omega theta| over the Ritz values
  // theta in the upper half of the spectrum (|theta| >= rho / 2): the stabilised operator's
  // D^{-1} A has complex eigenvalues there, and a weight from rho alone over-relaxed them (Q1Q1
  // with viscosity-dominated tau stagnated, in the oracle as on the GPU).  lmax is stored so that
  // the smoother's omega = 2 / (lmax / 20 + lmax) equals that weight.
  for (size_t l = 0; l < p.levels.size(); ++l) {
    OpLevel& lv = *p.levels[l];
    if (lv.lmax > 0) continue;
    std::vector<std::complex<double>> ritz;
    const double rho = arnoldi_spectral_radius(p, lv, s, &ritz);
    if (p.smoother == 1) {
      const double w = relaxation_weight(ritz);
      lv.lmax = (w > 0.0 && std::isfinite(w)) ? 2.0 / (1.05 * w) : 2.0 * rho;
    } else {
      lv.lmax = 1.2 * rho;
    }
  }
}

// Spectral radius of a small dense matrix H (m x m, row-major) by power iteration with
// renormalisation: rho = lim (||H^k v|| / ||v||)^(1/k).
static double small_spectral_radius(const std::vector<double>& H, int m) {
  std::vector<double> v(m, 1.0), w(m);
  for (int i = 0; i < m; ++i) v[i] = 1.0 + 0.01 * i;
  double logsum = 0.0;
  const int warm = 200, iters = 2000;
  for (int it = 0; it < warm + iters; ++it) {
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) {
      double t = 0.0;
      for (int j = 0; j < m; ++j) t += H[i * m + j] * v[j];
      w[i] = t;
      nrm += t * t;
    }
    nrm = std::sqrt(nrm);
    if (nrm == 0.0 || !std::isfinite(nrm)) return 0.0;
    if (it >= warm) logsum += std::log(nrm);
    for (int i = 0; i < m; ++i) v[i] = w[i] / nrm;
  }
  return std::exp(logsum / iters);
}

double arnoldi_spectral_radius(Problem& p, OpLevel& lv, cudaStream_t s,
                               std::vector<std::complex<double>>* ritz) {
  const int64_t n = lv.n_dofs;
  const int m = (int)std::min<int64_t>(std::min(p.restart, 30), std::max<int64_t>(n - 1, 1));
  double* V = p.V.as<double>();
  const int64_t stride = sys_of(p).n_dofs;  // V holds restart+1 vectors of the system length
  const double** Vp = (const double**)p.ptrV.as<const double*>();
  double* w = p.w.as<double>();
  const double* dinv = lv.dinv[0].as<double>();
  std::mt19937_64 rng(1);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  std::vector<double> v0(n);
  for (auto& v : v0) v = U(rng);
  MFNS_CUDA(cudaMemcpyAsync(V, v0.data(), n * 8, cudaMemcpyHostToDevice, s));
  const double n0 = std::sqrt(host_dot(p, V, V, n, s));
  vscale<double>(V, 1.0 / n0, n, s);
  std::vector<double> H((size_t)(m + 1) * m, 0.0);
  int mm = 0;
  for (int j = 0; j < m; ++j) {
    oplevel_vmult(lv, 0, V + (size_t)j * stride, p.tmp.get(), s);
    if (lv.hp && lv.hp->asm_)
      hp_asm_apply(lv, 0, p.tmp.get(), w, s);
    else
      vmul<double>(w, dinv, p.tmp.as<double>(), n, s);
    double* hd = p.hvec.as<double>();
    multidot(hd, nullptr, w, j + 1, n, p.part.as<double>(), Vp, s);
    multi_axpy(w, Vp, hd, j + 1, n, s);
    multidot(hd + kMaxDots, nullptr, w, j + 1, n, p.part.as<double>(), Vp, s);
    multi_axpy(w, Vp, hd + kMaxDots, j + 1, n, s);
    std::vector<double> hh(2 * kMaxDots);
    MFNS_CUDA(cudaMemcpyAsync(hh.data(), hd, 2 * kMaxDots * 8, cudaMemcpyDeviceToHost, s));
    const double hn = std::sqrt(host_dot(p, w, w, n, s));
    for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hh[i] + hh[kMaxDots + i];
    mm = j + 1;
    if (!(hn > 1e-14) || j + 1 == m) break;
    H[(size_t)(j + 1) * m + j] = hn;
    vcopy<double>(V + (size_t)(j + 1) * stride, w, n, s);
    vscale<double>(V + (size_t)(j + 1) * stride, 1.0 / hn, n, s);
  }
  std::vector<double> Hm((size_t)mm * mm);
  for (int i = 0; i < mm; ++i)
    for (int j = 0; j < mm; ++j) Hm[(size_t)i * mm + j] = H[(size_t)i * m + j];
  if (ritz) *ritz = hessenberg_eigenvalues(Hm, mm);
  return small_spectral_radius(Hm, mm);
}

// Dense LU inverse with partial pivoting (host, in place).
static bool invert_dense(std::vector<double>& A, int64_t n) {
  std::vector<double> I(n * n, 0.0);
  for (int64_t i = 0; i < n; ++i) I[i * n + i] = 1.0;
  for (int64_t c = 0; c < n; ++c) {
    int64_t piv = c;
    for (int64_t r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return false;
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

void setup_coarse(Problem& p, cudaStream_t s) {
  if (p.ls) return setup_coarse(*p.ls->base, s);
  OpLevel& cl = *p.levels.back();
  const int64_t n = cl.n_dofs;
  p.coarse_n = n;
  p.coarse_dense = n <= 4096;
  if (!p.coarse_dense) return;
  // assemble the coarse matrix with the fp64 operator: blocks of kCols unit vectors, each block
  // applied in one multi-column launch per colour
  constexpr int64_t kCols = 128;
  std::vector<double> A(n * n), cols(n * kCols);
  const int64_t blk = std::min<int64_t>(kCols, n);
  if (p.coarse_cols.bytes() != (size_t)(2 * n * blk * 8)) p.coarse_cols.alloc(p.bud, 2 * n * blk * 8);
  double* X = p.coarse_cols.as<double>();
  double* Y = X + n * blk;
  for (int64_t j0 = 0; j0 < n; j0 += kCols) {
    const int64_t nb = std::min<int64_t>(kCols, n - j0);
    vunit_cols(X, n, j0, nb, s);
    oplevel_vmult_cols(cl, 0, X, Y, (int)nb, s);
    MFNS_CUDA(cudaMemcpyAsync(cols.data(), Y, nb * n * 8, cudaMemcpyDeviceToHost, s));
    MFNS_CUDA(cudaStreamSynchronize(s));
    for (int64_t j = 0; j < nb; ++j)
      for (int64_t i = 0; i < n; ++i) A[i * n + j0 + j] = cols[j * n + i];
  }
  // constant-pressure null space: add e e^T over the free pressure entries
  if (cl.n_pres > 0 && (cl.op == OP_STAB_NS || cl.op == OP_STOKES)) {
    const double v = 1.0 / (double)cl.n_pres;
    for (int32_t i : cl.pres_host)
      for (int32_t j : cl.pres_host) A[(int64_t)i * n + j] += v;
  }
  if (!invert_dense(A, n)) throw Error(kErrArg, "singular coarse matrix");
  std::vector<float> Af(A.begin(), A.end());
  if (p.coarse_inv[0].bytes() == (size_t)n * n * 8) {  // refresh in place (graphs hold the pointers)
    MFNS_CUDA(cudaMemcpyAsync(p.coarse_inv[0].get(), A.data(), n * n * 8, cudaMemcpyHostToDevice, s));
    MFNS_CUDA(cudaMemcpyAsync(p.coarse_inv[1].get(), Af.data(), n * n * 4, cudaMemcpyHostToDevice, s));
    MFNS_CUDA(cudaStreamSynchronize(s));
  } else {
    p.coarse_inv[0] = upload(p.bud, A);
    p.coarse_inv[1] = upload(p.bud, Af);
  }
}

// ---------------------------------------------------------------------- smoothing
template <typename T>
static void smooth_op(const Problem& p, OpLevel& lv, Workspace& w, int prec, const T* b, T* x, bool x_is_zero,
                      int degree, cudaStream_t s) {
  const int64_t n = lv.n_dofs;
  const T* dinv = lv.dinv[prec].as<T>();
  T* d = w.d.as<T>();
  T* t = w.t.as<T>();
  // with p.fused_smoother on a uniform level, steps with an operator application fuse the update
  // into the cell kernel's last-colour scatter; the new iterate then goes to the other of two
  // buffers (x and the level's residual vector, free while smoothing).  Otherwise the product
  // is written out and a streaming kernel applies the update.
  const bool fused = p.fused_smoother && lv.L.structured && lv.L.lastc;
  T* cur = x;
  auto step = [&](double c1, double c2) {
    if (!fused) {
      oplevel_vmult(lv, prec, x, t, s);
      vcheby<T>(x, d, b, t, dinv, (T)c1, (T)c2, n, s);
      return;
    }
    T* out = cur == x ? w.r.as<T>() : x;
    oplevel_smooth_step(lv, prec, cur, out, d, b, dinv, t, c1, c2, s);
    cur = out;
  };
  const double lmax = lv.lmax, lmin = lmax / 20.0;
  if (lv.hp && lv.hp->asm_) {  // Chebyshev around the blended preconditioner (Section 3)
    T* r = w.r.as<T>();
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
    double rho_old = 1.0 / sigma;
    for (int j = 0; j < degree; ++j) {
      if (j == 0 && x_is_zero) {
        vzero<T>(x, n, s);
        hp_asm_apply(lv, prec, b, t, s);
      } else {
        oplevel_vmult(lv, prec, x, t, s);
        vsub<T>(r, b, t, n, s);
        hp_asm_apply(lv, prec, r, t, s);
      }
      if (j == 0) {
        vcheby_pre<T>(x, d, t, (T)0, (T)(1.0 / theta), n, s);
      } else {
        const double rho = 1.0 / (2.0 * sigma - rho_old);
        vcheby_pre<T>(x, d, t, (T)(rho * rho_old), (T)(2.0 * rho / delta), n, s);
        rho_old = rho;
      }
    }
    return;
  }
  if (p.smoother == 1) {  // Jacobi relaxation
    const T omega = (T)(2.0 / (lmin + lmax));
    for (int it = 0; it < degree; ++it) {
      if (it == 0 && x_is_zero)
        vcheby0<T>(x, d, b, dinv, omega, n, s);
      else
        step(0.0, (double)omega);
    }
  } else {
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
    double rho_old = 1.0 / sigma;
    if (x_is_zero)
      vcheby0<T>(x, d, b, dinv, (T)(1.0 / theta), n, s);
    else
      step(0.0, 1.0 / theta);
    for (int j = 1; j < degree; ++j) {
      const double rho = 1.0 / (2.0 * sigma - rho_old);
      step(rho * rho_old, 2.0 * rho / delta);
      rho_old = rho;
    }
  }
  if (cur != x) vcopy<T>(x, cur, n, s);
}

template <typename T>
static void smooth_t(Problem& p, int level, int prec, const T* b, T* x, bool x_is_zero, int degree, cudaStream_t s) {
  smooth_op<T>(p, *p.levels[level], p.ws[prec][level], prec, b, x, x_is_zero, degree, s);
}

void smooth(Problem& p, int level, int prec, const void* b, void* x, bool x_is_zero, cudaStream_t s) {
  if (prec == 0)
    smooth_t<double>(p, level, 0, (const double*)b, (double*)x, x_is_zero, p.smoother_degree, s);
  else
    smooth_t<float>(p, level, 1, (const float*)b, (float*)x, x_is_zero, p.smoother_degree, s);
}

template <typename T>
static void coarse_solve(Problem& p, int prec, const T* b, T* x, cudaStream_t s) {
  const int L = (int)p.levels.size() - 1;
  if (p.coarse_dense) {
    vgemv<T>(x, p.coarse_inv[prec].as<T>(), b, p.coarse_n, s);
  } else {
    smooth_t<T>(p, L, prec, b, x, true, p.coarse_cheby_degree, s);
  }
}

template <typename T>
static void vcycle_level(Problem& p, int prec, int l, const T* b, T* x, cudaStream_t s) {
  const int L = (int)p.levels.size() - 1;
  if (l == L) {
    coarse_solve<T>(p, prec, b, x, s);
    return;
  }
  OpLevel& lv = *p.levels[l];
  Workspace& w = p.ws[prec][l];
  Workspace& wc = p.ws[prec][l + 1];
  const int64_t n = lv.n_dofs;
  smooth_t<T>(p, l, prec, b, x, true, p.smoother_degree, s);
  if (p.fused_smoother && lv.L.structured && lv.L.lastc) {
    oplevel_residual_fused(lv, prec, x, b, w.r.get(), w.t.get(), s);  // r = b - A x, fused
  } else {
    oplevel_vmult(lv, prec, x, w.t.get(), s);
    vsub<T>(w.r.as<T>(), b, w.t.as<T>(), n, s);
  }
  transfer_restrict(*p.transfers[l], lv, *p.levels[l + 1], prec, w.r.get(), wc.b.get(), s);
  vcycle_level<T>(p, prec, l + 1, wc.b.as<T>(), wc.x.as<T>(), s);
  transfer_prolongate_add(*p.transfers[l], lv, *p.levels[l + 1], prec, wc.x.get(), x, s);
  smooth_t<T>(p, l, prec, b, x, false, p.smoother_degree, s);
}

// Local-smoothing cycle (Section 2).  The fine defect b is copied to the level that owns each
// DoF.  Down the levels: smooth from zero on the level's cells with the refinement edge held at
// zero, form the level residual with the unconstrained-edge operator (its edge rows carry the
// correction's effect on the coarser level), restrict it and add it to the coarser defect.  Level 0
// runs the base hierarchy's V-cycle.  Up the levels: prolongate the coarser iterate (which sets
// the edge values), form the residual with those edge values, smooth the correction from zero and
// add it.  The fine result is copied back from the owning levels; constrained entries stay zero.
template <typename T>
static void ls_vcycle(Problem& p, int prec, const T* b, T* x, cudaStream_t s) {
  LocalSmoothing& S = *p.ls;
  sync_ls_settings(p);
  const int nc = p.levels[0]->NU;
  const int L = (int)S.lv.size();
  Problem& B = *S.base;
  const OpLevel& b0 = *B.levels[0];
  T* bl0 = S.b[prec].as<T>();
  MFNS_CUDA(cudaMemsetAsync(bl0, 0, b0.n_dofs * sizeof(T), s));
  vcopy_map<T>(bl0, S.copy_lvl.as<int32_t>(), b, S.copy_fine.as<int32_t>(), S.n_copy, nc, s);
  for (auto& lv : S.lv) {
    T* bl = lv->ws[prec].b.as<T>();
    MFNS_CUDA(cudaMemsetAsync(bl, 0, lv->op->n_dofs * sizeof(T), s));
    vcopy_map<T>(bl, lv->copy_lvl.as<int32_t>(), b, lv->copy_fine.as<int32_t>(), lv->n_copy, nc, s);
  }
  for (int l = L; l >= 1; --l) {
    LsLevel& lv = *S.lv[l - 1];
    Workspace& w = lv.ws[prec];
    const int64_t n = lv.op->n_dofs;
    T* z = lv.z[prec].as<T>();
    vcopy<T>(z, w.b.as<T>(), n, s);
    vset_idx<T>(z, T(0), lv.op->constrained.as<int32_t>(), (int64_t)lv.op->constrained_host.size(), s);
    smooth_op<T>(p, *lv.op, w, prec, z, w.x.as<T>(), true, p.smoother_degree, s);
    oplevel_vmult(*lv.full, prec, w.x.get(), w.t.get(), s);
    vsub<T>(w.r.as<T>(), w.b.as<T>(), w.t.as<T>(), n, s);
    const OpLevel& coarse = l == 1 ? b0 : *S.lv[l - 2]->full;
    T* cb = l == 1 ? bl0 : S.lv[l - 2]->ws[prec].b.as<T>();
    T* cc = l == 1 ? S.c[prec].as<T>() : S.lv[l - 2]->c[prec].as<T>();
    transfer_restrict(lv.down, *lv.full, coarse, prec, w.r.get(), cc, s);
    vaxpy<T>(cb, T(1), cc, coarse.n_dofs, s);
  }
  vcycle_level<T>(B, prec, 0, bl0, S.x[prec].as<T>(), s);
  for (int l = 1; l <= L; ++l) {
    LsLevel& lv = *S.lv[l - 1];
    Workspace& w = lv.ws[prec];
    const int64_t n = lv.op->n_dofs;
    const OpLevel& coarse = l == 1 ? b0 : *S.lv[l - 2]->full;
    const void* xc = l == 1 ? S.x[prec].get() : S.lv[l - 2]->ws[prec].x.get();
    transfer_prolongate_add(lv.down, *lv.full, coarse, prec, xc, w.x.get(), s);
    oplevel_vmult(*lv.full, prec, w.x.get(), w.t.get(), s);
    vsub<T>(w.r.as<T>(), w.b.as<T>(), w.t.as<T>(), n, s);
    vset_idx<T>(w.r.as<T>(), T(0), lv.op->constrained.as<int32_t>(), (int64_t)lv.op->constrained_host.size(), s);
    T* dlt = lv.c[prec].as<T>();
    smooth_op<T>(p, *lv.op, w, prec, w.r.as<T>(), dlt, true, p.smoother_degree, s);
    vaxpy<T>(w.x.as<T>(), T(1), dlt, n, s);
  }
  MFNS_CUDA(cudaMemsetAsync(x, 0, p.levels[0]->n_dofs * sizeof(T), s));
  vcopy_map<T>(x, S.copy_fine.as<int32_t>(), S.x[prec].as<T>(), S.copy_lvl.as<int32_t>(), S.n_copy, nc, s);
  for (auto& lv : S.lv)
    vcopy_map<T>(x, lv->copy_fine.as<int32_t>(), lv->ws[prec].x.as<T>(), lv->copy_lvl.as<int32_t>(), lv->n_copy, nc, s);
  // the constrained (Dirichlet, hanging) rows are identity rows outside every level: inverted exactly
  const OpLevel& f0 = *p.levels[0];
  vcopy_idx<T>(x, b, f0.constrained.as<int32_t>(), (int64_t)f0.constrained_host.size(), s);
}

// one multigrid cycle on the problem's hierarchy (global coarsening or local smoothing)
template <typename T>
static void mg_cycle(Problem& p, int prec, const T* b, T* x, cudaStream_t s) {
  if (p.ls)
    ls_vcycle<T>(p, prec, b, x, s);
  else
    vcycle_level<T>(p, prec, 0, b, x, s);
}

void vcycle(Problem& p, int prec, const void* b, void* x, cudaStream_t s) {
  if (prec == 0)
    mg_cycle<double>(p, 0, (const double*)b, (double*)x, s);
  else
    mg_cycle<float>(p, 1, (const float*)b, (float*)x, s);
}

// ---------------------------------------------------------------------- FGMRES
static double host_dot(Problem& p, const double* a, const double* b, int64_t n, cudaStream_t s) {
  double* d = p.scal.as<double>();
  dot<double>(d, a, b, n, p.part.as<double>(), s);
  double h;
  MFNS_CUDA(cudaMemcpyAsync(&h, d, 8, cudaMemcpyDeviceToHost, s));
  MFNS_CUDA(cudaStreamSynchronize(s));
  return h;
}

template <typename T>
static void project_pressure(OpLevel& S, T* x, double* scal, double* part, cudaStream_t s) {
  if (S.n_pres == 0) return;
  sum_idx<T>(scal + 8, x, S.pres.as<int32_t>(), S.n_pres, part, s);
  sub_mean_idx<T>(x, S.pres.as<int32_t>(), S.n_pres, scal + 8, s);
}

// Stokes block preconditioner (Eq. 5) in precision T: in/out are T vectors of system length.
template <typename T>
static void stokes_block(Problem& p, int prec, const T* r, T* z, cudaStream_t s) {
  OpLevel& S = *p.system;
  OpLevel& M = *p.pmass;
  const int64_t nu = S.n_main_dofs, np = M.n_dofs, n = S.n_dofs;
  T* cx = p.cg_x.as<T>();
  T* cr = p.cg_r.as<T>();
  T* cz = p.cg_z.as<T>();
  T* cp = p.cg_p.as<T>();
  T* cq = p.cg_q.as<T>();
  const T* dinv = M.dinv[prec].as<T>();
  double* sc = p.scal.as<double>();
  // z_p = -nu M_p^{-1} r_p by a fixed number of Jacobi-preconditioned CG steps from zero; the CG
  // scalars stay on the device (sc[2 + (it & 1)] = r.z of the current and next step, sc[4] = p.q)
  vzero<T>(cx, np, s);
  vcopy<T>(cr, r + nu, np, s);
  vmul<T>(cz, dinv, cr, np, s);
  vcopy<T>(cp, cz, np, s);
  dot<T>(sc + 2, cr, cz, np, p.part.as<double>(), s);
  for (int it = 0; it < p.cg_iterations; ++it) {
    double* rz = sc + 2 + (it & 1);
    double* rz_new = sc + 2 + ((it + 1) & 1);
    oplevel_vmult(M, prec, cp, cq, s);
    dot<T>(sc + 4, cp, cq, np, p.part.as<double>(), s);
    cg_step_xr<T>(cx, cr, cp, cq, rz, sc + 4, np, s);
    vmul<T>(cz, dinv, cr, np, s);
    dot<T>(rz_new, cr, cz, np, p.part.as<double>(), s);
    cg_step_p<T>(cp, cz, rz_new, rz, np, s);
  }
  // full = [0, z_p]; B z_p = velocity part of the Stokes operator applied to it
  T* full = p.stokes_u_rhs.as<T>();
  T* Bz = p.stokes_u_sol.as<T>();
  vzero<T>(full, n, s);
  vcopy<T>(full + nu, cx, np, s);
  vscale<T>(full + nu, (T)(-p.phys.nu), np, s);
  vcopy<T>(z + nu, full + nu, np, s);
  oplevel_vmult(S, prec, full, Bz, s);
  // velocity rhs r_u - B z_p, then one V-cycle on the A block
  vsub<T>(Bz, r, Bz, nu, s);
  mg_cycle<T>(p, prec, Bz, z, s);
}

static void precondition_body(Problem& p, const double* v, double* z, cudaStream_t s);

// The preconditioner is a fixed sequence of kernels on fixed buffers: it is captured once into
// a CUDA graph (input p.pc_in, output p.pc_out) and replayed.
static void precondition(Problem& p, const double* v, double* z, cudaStream_t s) {
  OpLevel& S = p.system ? *p.system : *p.levels[0];
  const int64_t n = S.n_dofs;
  if (!p.use_graphs) return precondition_body(p, v, z, s);
  if (!p.pc_graph) {
    if (!p.cap_stream) MFNS_CUDA(cudaStreamCreateWithFlags(&p.cap_stream, cudaStreamNonBlocking));
    TimerPause pause(p);
    MFNS_CUDA(cudaStreamBeginCapture(p.cap_stream, cudaStreamCaptureModeThreadLocal));
    precondition_body(p, p.pc_in.as<double>(), p.pc_out.as<double>(), p.cap_stream);
    cudaGraph_t g;
    MFNS_CUDA(cudaStreamEndCapture(p.cap_stream, &g));
    MFNS_CUDA(cudaGraphInstantiate(&p.pc_graph, g, 0));
    MFNS_CUDA(cudaGraphDestroy(g));
  }
  MFNS_CUDA(cudaMemcpyAsync(p.pc_in.get(), v, n * 8, cudaMemcpyDeviceToDevice, s));
  MFNS_CUDA(cudaGraphLaunch(p.pc_graph, s));
  MFNS_CUDA(cudaMemcpyAsync(z, p.pc_out.get(), n * 8, cudaMemcpyDeviceToDevice, s));
}

void invalidate_graphs(Problem& p) {
  ++p.graph_epoch;
  if (p.pc_graph) cudaGraphExecDestroy(p.pc_graph);
  p.pc_graph = nullptr;
  for (int i = 0; i < 2; ++i) {
    if (p.vc_graph[i]) cudaGraphExecDestroy(p.vc_graph[i]);
    p.vc_graph[i] = nullptr;
  }
}

void vcycle_graph(Problem& p, int prec, const void* b, void* x, cudaStream_t s) {
  Workspace& w = p.ws[prec][0];
  const size_t bytes = p.levels[0]->n_dofs * esize(prec);
  if (!p.vc_graph[prec]) {
    if (!p.cap_stream) MFNS_CUDA(cudaStreamCreateWithFlags(&p.cap_stream, cudaStreamNonBlocking));
    TimerPause pause(p);
    MFNS_CUDA(cudaStreamBeginCapture(p.cap_stream, cudaStreamCaptureModeThreadLocal));
    vcycle(p, prec, p.vc_in[prec].get(), p.vc_out[prec].get(), p.cap_stream);
    cudaGraph_t g;
    MFNS_CUDA(cudaStreamEndCapture(p.cap_stream, &g));
    MFNS_CUDA(cudaGraphInstantiate(&p.vc_graph[prec], g, 0));
    MFNS_CUDA(cudaGraphDestroy(g));
  }
  (void)w;
  MFNS_CUDA(cudaMemcpyAsync(p.vc_in[prec].get(), b, bytes, cudaMemcpyDeviceToDevice, s));
  MFNS_CUDA(cudaGraphLaunch(p.vc_graph[prec], s));
  MFNS_CUDA(cudaMemcpyAsync(x, p.vc_out[prec].get(), bytes, cudaMemcpyDeviceToDevice, s));
}

static void precondition_body(Problem& p, const double* v, double* z, cudaStream_t s) {
  OpLevel& S = sys_of(p);
  const int64_t n = S.n_dofs;
  if (p.mg_precision == 0) {
    if (p.kind == 0)
      stokes_block<double>(p, 0, v, z, s);
    else
      mg_cycle<double>(p, 0, v, z, s);
  } else {
    vcast_d2f(p.mg_b32.as<float>(), v, n, s);
    if (p.kind == 0)
      stokes_block<float>(p, 1, p.mg_b32.as<float>(), p.mg_x32.as<float>(), s);
    else
      mg_cycle<float>(p, 1, p.mg_b32.as<float>(), p.mg_x32.as<float>(), s);
    vcast_f2d(z, p.mg_x32.as<float>(), n, s);
  }
}

// ---------------------------------------------------------------------- FGMRES as a state machine
// One call of krylov_enqueue + krylov_complete performs one Arnoldi step (preconditioner, operator,
// CGS2, Givens); a restart cycle ends with the update of x and a true residual.  Batched rounds
// enqueue the device work of many problems (each on its own stream) before completing any.

static void start_cycle(Problem& p, double beta) {
  OpLevel& S = sys_of(p);
  Krylov& K = p.kry;
  const int m = p.restart;
  vcopy<double>(p.V.as<double>(), p.tmp.as<double>(), S.n_dofs, K.stream);
  vscale<double>(p.V.as<double>(), 1.0 / beta, S.n_dofs, K.stream);
  std::fill(K.g.begin(), K.g.end(), 0.0);
  K.g[0] = beta;
  K.j = 0;
  (void)m;
}

void krylov_begin(Problem& p, const double* b_in, double* x, cudaStream_t s) {
  OpLevel& S = sys_of(p);
  Krylov& K = p.kry;
  const int64_t n = S.n_dofs;
  const int m = p.restart;
  K = Krylov();
  K.stream = s;
  K.x = x;
  K.H.assign((size_t)(m + 1) * m, 0.0);
  K.cs.assign(m, 0.0);
  K.sn.assign(m, 0.0);
  K.g.assign(m + 1, 0.0);
  double* b = p.sys_r.as<double>();  // projected right-hand side
  vcopy<double>(b, b_in, n, s);
  project_pressure<double>(S, b, p.scal.as<double>(), p.part.as<double>(), s);
  vzero<double>(x, n, s);
  vcopy<double>(p.tmp.as<double>(), b, n, s);  // r = b - A 0
  K.bnorm = std::sqrt(host_dot(p, b, b, n, s));
  K.relres = 0.0;
  K.active = true;
  if (K.bnorm == 0.0) {
    K.active = false;
    K.converged = true;
    return;
  }
  K.relres = 1.0;
  start_cycle(p, K.bnorm);
}

// Device work of one Arnoldi step split around the preconditioner (batched rounds).
void krylov_enqueue_pre(Problem& p) {
  Krylov& K = p.kry;
  if (!K.active) return;
  const int64_t n = sys_of(p).n_dofs;
  MFNS_CUDA(cudaMemcpyAsync(p.pc_in.get(), p.V.as<double>() + (size_t)K.j * n, n * 8, cudaMemcpyDeviceToDevice,
                            K.stream));
  if (!p.ev_step) MFNS_CUDA(cudaEventCreateWithFlags(&p.ev_step, cudaEventDisableTiming));
  MFNS_CUDA(cudaEventRecord(p.ev_step, K.stream));
}

static void krylov_after_precondition(Problem& p, double* zj);

void krylov_enqueue_post(Problem& p, cudaEvent_t ready) {
  Krylov& K = p.kry;
  if (!K.active) return;
  const int64_t n = sys_of(p).n_dofs;
  double* zj = p.Z.as<double>() + (size_t)K.j * n;
  MFNS_CUDA(cudaStreamWaitEvent(K.stream, ready, 0));
  MFNS_CUDA(cudaMemcpyAsync(zj, p.pc_out.get(), n * 8, cudaMemcpyDeviceToDevice, K.stream));
  krylov_after_precondition(p, zj);
}

// Device work of one Arnoldi step (asynchronous on the problem's stream).
void krylov_enqueue(Problem& p) {
  Krylov& K = p.kry;
  if (!K.active) return;
  OpLevel& S = sys_of(p);
  const int64_t n = S.n_dofs;
  cudaStream_t s = K.stream;
  const int j = K.j;
  double* V = p.V.as<double>();
  double* zj = p.Z.as<double>() + (size_t)j * n;
  precondition(p, V + (size_t)j * n, zj, s);
  krylov_after_precondition(p, zj);
}

static void krylov_after_precondition(Problem& p, double* zj) {
  Krylov& K = p.kry;
  OpLevel& S = sys_of(p);
  const int64_t n = S.n_dofs;
  cudaStream_t s = K.stream;
  const int j = K.j;
  const double** Vp = (const double**)p.ptrV.as<const double*>();
  double* w = p.w.as<double>();
  project_pressure<double>(S, zj, p.scal.as<double>(), p.part.as<double>(), s);
  oplevel_vmult(S, 0, zj, w, s);
  double* hd = p.hvec.as<double>();
  multidot(hd, nullptr, w, j + 1, n, p.part.as<double>(), Vp, s);
  multi_axpy(w, Vp, hd, j + 1, n, s);
  multidot(hd + kMaxDots, nullptr, w, j + 1, n, p.part.as<double>(), Vp, s);
  multi_axpy(w, Vp, hd + kMaxDots, j + 1, n, s);
  dot<double>(p.scal.as<double>() + 12, w, w, n, p.part.as<double>(), s);
  MFNS_CUDA(cudaMemcpyAsync(p.hh_host, hd, 2 * kMaxDots * 8, cudaMemcpyDeviceToHost, s));
  MFNS_CUDA(cudaMemcpyAsync(p.hh_host + 2 * kMaxDots, p.scal.as<double>() + 12, 8, cudaMemcpyDeviceToHost, s));
}

// Host part of the step (after the problem's stream has been synchronised); ends the restart
// cycle when needed.  Returns true while the solve is still running.
bool krylov_complete(Problem& p) {
  Krylov& K = p.kry;
  if (!K.active) return false;
  OpLevel& S = sys_of(p);
  const int64_t n = S.n_dofs;
  const int m = p.restart;
  cudaStream_t s = K.stream;
  const int j = K.j;
  double* V = p.V.as<double>();
  std::vector<double>& H = K.H;
  const double* hh = p.hh_host;
  const double hn = std::sqrt(std::max(hh[2 * kMaxDots], 0.0));
  for (int i = 0; i <= j; ++i) H[i * m + j] = hh[i] + hh[kMaxDots + i];
  H[(j + 1) * m + j] = hn;
  if (hn > 0) {
    vcopy<double>(V + (size_t)(j + 1) * n, p.w.as<double>(), n, s);
    vscale<double>(V + (size_t)(j + 1) * n, 1.0 / hn, n, s);
  }
  for (int i = 0; i < j; ++i) {
    const double t = K.cs[i] * H[i * m + j] + K.sn[i] * H[(i + 1) * m + j];
    H[(i + 1) * m + j] = -K.sn[i] * H[i * m + j] + K.cs[i] * H[(i + 1) * m + j];
    H[i * m + j] = t;
  }
  const double den = std::hypot(H[j * m + j], H[(j + 1) * m + j]);
  K.cs[j] = H[j * m + j] / den;
  K.sn[j] = H[(j + 1) * m + j] / den;
  H[j * m + j] = den;
  H[(j + 1) * m + j] = 0.0;
  K.g[j + 1] = -K.sn[j] * K.g[j];
  K.g[j] = K.cs[j] * K.g[j];
  ++K.it;
  K.j = j + 1;
  const bool cycle_end = std::fabs(K.g[j + 1]) <= p.tol * K.bnorm || K.it >= p.maxit || K.j == m;
  if (!cycle_end) return true;
  // end of the restart cycle: x += Z y, true residual r = b - A x
  const int jd = K.j;
  std::vector<double> y(jd);
  for (int i = jd - 1; i >= 0; --i) {
    double acc = K.g[i];
    for (int k2 = i + 1; k2 < jd; ++k2) acc -= H[i * m + k2] * y[k2];
    y[i] = acc / H[i * m + i];
  }
  MFNS_CUDA(cudaMemcpyAsync(p.yvec.get(), y.data(), jd * 8, cudaMemcpyHostToDevice, s));
  multi_axpy_add(K.x, (const double**)p.ptrZ.as<const double*>(), p.yvec.as<double>(), jd, n, s);
  oplevel_vmult(S, 0, K.x, p.w.get(), s);
  vsub<double>(p.tmp.as<double>(), p.sys_r.as<double>(), p.w.as<double>(), n, s);
  const double beta = std::sqrt(host_dot(p, p.tmp.as<double>(), p.tmp.as<double>(), n, s));
  K.relres = beta / K.bnorm;
  std::fill(H.begin(), H.end(), 0.0);
  if (beta <= p.tol * K.bnorm) {
    K.active = false;
    K.converged = true;
    return false;
  }
  if (K.it >= p.maxit) {
    K.active = false;
    K.converged = false;
    return false;
  }
  start_cycle(p, beta);
  return true;
}

int fgmres_solve(Problem& p, const double* b_in, double* x, double* relres, bool* converged, cudaStream_t s) {
  krylov_begin(p, b_in, x, s);
  while (p.kry.active) {
    krylov_enqueue(p);
    MFNS_CUDA(cudaStreamSynchronize(s));
    krylov_complete(p);
  }
  *relres = p.kry.relres;
  *converged = p.kry.converged;
  return p.kry.it;
}

// ---------------------------------------------------------------------- Newton / BDF (Section 5)
void set_state_fine(Problem& p, double dt, double alpha, const double* U, const double* g, cudaStream_t s) {
  if (p.kind != 2) throw Error(kErrUnsupported, "set_state: stabilised NS problems only");
  if (!(dt > 0.0) || !(alpha > 0.0)) throw Error(kErrArg, "set_state: dt and alpha must be positive");
  const bool has_g = g != nullptr;
  for (auto& lvp : p.levels) {
    OpLevel& lv = *lvp;
    lv.L.dt = dt;
    lv.L.alpha = alpha;
    if (has_g && !lv.gexp[0].get()) {
      lv.gexp[0].alloc(p.bud, lv.n_main_dofs * 8);
      lv.gexp[1].alloc(p.bud, lv.n_main_dofs * 4);
    }
    lv.L.gexp[0] = has_g ? lv.gexp[0].get() : nullptr;
    lv.L.gexp[1] = has_g ? lv.gexp[1].get() : nullptr;
  }
  // captured graphs hold dt, alpha and the explicit-field pointer as launch parameters
  if (dt != p.st_dt || alpha != p.st_alpha || has_g != p.st_g) invalidate_graphs(p);
  p.st_dt = dt;
  p.st_alpha = alpha;
  p.st_g = has_g;
  p.phys.dt = dt;
  OpLevel& f0 = *p.levels[0];
  // hanging-node entries of the state follow their masters (the kernels read the state at the true
  // nodes of every cell)
  MFNS_CUDA(cudaMemcpyAsync(f0.frozen[0].get(), U, f0.n_main_dofs * 8, cudaMemcpyDeviceToDevice, s));
  oplevel_distribute(f0, 0, f0.frozen[0].get(), s);
  vcast_d2f(f0.frozen[1].as<float>(), f0.frozen[0].as<double>(), f0.n_main_dofs, s);
  if (has_g) {
    MFNS_CUDA(cudaMemcpyAsync(f0.gexp[0].get(), g, f0.n_main_dofs * 8, cudaMemcpyDeviceToDevice, s));
    oplevel_distribute(f0, 0, f0.gexp[0].get(), s);
    vcast_d2f(f0.gexp[1].as<float>(), f0.gexp[0].as<double>(), f0.n_main_dofs, s);
  }
  for (int prec = 0; prec < 2; ++prec) op_precompute_frozen(f0.L, prec, s);
}

void refresh_preconditioner(Problem& p, cudaStream_t s) {
  if (p.ls) throw Error(kErrUnsupported, "Newton states are carried to global-coarsening levels only");
  // the finest state (and g) interpolated level by level down the hierarchy
  const bool has_g = p.st_g;
  for (size_t l = 0; l + 1 < p.levels.size(); ++l) {
    Transfer& t = *p.transfers[l];
    OpLevel& f = *p.levels[l];
    OpLevel& c = *p.levels[l + 1];
    cell_interpolate(t, f, c, f.frozen[0].as<double>(), c.frozen[0].as<double>(), p.bud, s);
    oplevel_distribute(c, 0, c.frozen[0].get(), s);
    vcast_d2f(c.frozen[1].as<float>(), c.frozen[0].as<double>(), c.n_main_dofs, s);
    if (has_g) {
      cell_interpolate(t, f, c, f.gexp[0].as<double>(), c.gexp[0].as<double>(), p.bud, s);
      oplevel_distribute(c, 0, c.gexp[0].get(), s);
      vcast_d2f(c.gexp[1].as<float>(), c.gexp[0].as<double>(), c.n_main_dofs, s);
    }
    for (int prec = 0; prec < 2; ++prec) op_precompute_frozen(c.L, prec, s);
  }
  for (auto& lvp : p.levels) level_dinv(p, *lvp, s, true);
  setup_coarse(p, s);  // synchronises
}

void set_state(Problem& p, double dt, double alpha, const double* U, const double* g, cudaStream_t s) {
  set_state_fine(p, dt, alpha, U, g, s);
  refresh_preconditioner(p, s);
}

void residual(Problem& p, int prec, void* dst, cudaStream_t s) {
  if (p.kind != 2) throw Error(kErrUnsupported, "residual: stabilised NS problems only");
  OpLevel& lv = *p.levels[0];
  MFNS_CUDA(cudaMemsetAsync(dst, 0, lv.n_dofs * esize(prec), s));
  op_residual(lv.L, prec, dst, s);
  const int64_t nc = (int64_t)lv.constrained_host.size();
  if (prec == 0)
    vset_idx<double>((double*)dst, 0.0, lv.constrained.as<int32_t>(), nc, s);
  else
    vset_idx<float>((float*)dst, 0.0f, lv.constrained.as<int32_t>(), nc, s);
}

double max_velocity(Problem& p, const double* u, cudaStream_t s) {
  OpLevel& lv = *p.levels[0];
  if (p.kind != 2) throw Error(kErrUnsupported, "max_velocity: stabilised NS problems only");
  unsigned long long* d = reinterpret_cast<unsigned long long*>(p.scal.as<double>() + 14);
  max_node_norm2(d, u, lv.nu.n_nodes, lv.NU, lv.dim, s);
  unsigned long long bits = 0;
  MFNS_CUDA(cudaMemcpyAsync(&bits, d, 8, cudaMemcpyDeviceToHost, s));
  MFNS_CUDA(cudaStreamSynchronize(s));
  double m2;
  std::memcpy(&m2, &bits, 8);
  return std::sqrt(m2);
}

NewtonResult bdf_step(Problem& p, const NewtonParams& np, const double* u_n, const double* u_nm1,
                      const double* forcing, double* u, cudaStream_t s) {
  if (p.kind != 2) throw Error(kErrUnsupported, "bdf_step: stabilised NS problems only");
  if (!(np.dt > 0.0) || np.omega < 0.0) throw Error(kErrArg, "bdf_step: dt > 0 and omega >= 0 required");
  if (np.omega > 0.0 && !u_nm1) throw Error(kErrArg, "bdf_step: BDF2 needs u^{n-1}");
  OpLevel& lv = *p.levels[0];
  const int64_t n = lv.n_dofs;
  if (p.nt_g.bytes() != (size_t)n * 8) {
    p.nt_g.alloc(p.bud, n * 8);
    p.nt_F.alloc(p.bud, n * 8);
    p.nt_d.alloc(p.bud, n * 8);
  }
  double* g = p.nt_g.as<double>();
  double* F = p.nt_F.as<double>();
  double* d = p.nt_d.as<double>();
  // variable-step BDF2: alpha u^{n+1} + beta_n u^n + beta_nm1 u^{n-1}, omega = dt_n / dt_{n-1}
  const double w = np.omega;
  const double alpha = w == 0.0 ? 1.0 : (1.0 + 2.0 * w) / (1.0 + w);
  const double bn = w == 0.0 ? -1.0 : -(1.0 + w);
  const double bnm1 = w == 0.0 ? 0.0 : w * w / (1.0 + w);
  vlincomb3(g, bn / np.dt, u_n, bnm1 / np.dt, w == 0.0 ? nullptr : u_nm1, -1.0, forcing, n, s);
  const int64_t ncon = (int64_t)lv.constrained_host.size();
  if (np.extrapolate) {  // free entries from (1 + w) u^n - w u^{n-1}; constrained entries kept from u
    vlincomb3(d, 1.0 + w, u_n, -w, w == 0.0 ? nullptr : u_nm1, 0.0, nullptr, n, s);
    vcopy_idx<double>(d, u, lv.constrained.as<int32_t>(), ncon, s);
    MFNS_CUDA(cudaMemcpyAsync(u, d, n * 8, cudaMemcpyDeviceToDevice, s));
  }
  oplevel_distribute(lv, 0, u, s);  // hanging entries of the start follow their masters
  NewtonResult res;
  const double tol_saved = p.tol;
  for (int it = 0;; ++it) {
    // the finest level's state suffices for the residual and the Jacobian; the multigrid levels,
    // diagonals and the coarse inverse are refreshed only before a linear solve
    set_state_fine(p, np.dt, alpha, u, g, s);
    residual(p, 0, F, s);
    const double r = std::sqrt(host_dot(p, F, F, n, s));
    if (it == 0) res.residual0 = r;
    res.residual = r;
    res.newton_iterations = it;
    if (r <= std::max(np.atol, np.rtol * res.residual0)) {
      res.converged = true;
      break;
    }
    if (it == np.max_newton || !std::isfinite(r)) break;
    // J(u) d = -F by FGMRES with the multigrid preconditioner at the current state
    refresh_preconditioner(p, s);
    vscale<double>(F, -1.0, n, s);
    p.tol = np.lin_tol;
    double rel = 0.0;
    bool conv = false;
    try {
      res.linear_iterations += fgmres_solve(p, F, d, &rel, &conv, s);
    } catch (...) {
      p.tol = tol_saved;
      throw;
    }
    p.tol = tol_saved;
    vaxpy<double>(u, 1.0, d, n, s);
    oplevel_distribute(lv, 0, u, s);  // hanging entries follow their masters
  }
  return res;
}

// ---------------------------------------------------------------------- batched V-cycles (D6)
bool batchable(const Problem& p) {
  if ((p.kind != 1 && p.kind != 2) || p.fused_smoother || !p.use_graphs || p.ls) return false;
  for (auto& l : p.levels)
    if (!l->L.structured) return false;
  return true;
}

struct BatchGroup {
  std::vector<int> mem;  // problem indices
  MultiOpPtr op;         // x -> t at this level for every member
};

struct BatchVcycle {
  int prec = 1;
  std::vector<Problem*> ps;
  std::vector<const void*> b0;
  std::vector<void*> x0;
  int steps = 0;                               // max levels over the problems
  std::vector<std::vector<BatchGroup>> groups;  // [level][group]
};

void BatchVcycleDel::operator()(BatchVcycle* b) const { delete b; }

BatchVcyclePtr make_batch_vcycle(const std::vector<Problem*>& ps, int prec, const std::vector<const void*>& b,
                                 const std::vector<void*>& x, Budget* bud) {
  BatchVcyclePtr B(new BatchVcycle);
  B->prec = prec;
  B->ps = ps;
  B->b0 = b;
  B->x0 = x;
  for (Problem* p : ps) {
    if (!batchable(*p)) throw Error(kErrArg, "batched V-cycle: unsupported problem");
    B->steps = std::max<int>(B->steps, (int)p->levels.size());
  }
  B->groups.resize(B->steps);
  for (int t = 0; t < B->steps; ++t) {
    // members: problems for which level t is not the coarse level; grouped by what one launch shares
    std::map<std::tuple<int, int, int, bool, int, int, int>, std::vector<int>> key;
    for (int i = 0; i < (int)ps.size(); ++i) {
      const Problem& p = *ps[i];
      if (t >= (int)p.levels.size() - 1) continue;
      const OpLaunch& L = p.levels[t]->L;
      key[{L.dim, L.k, L.op, L.fq[prec] != nullptr, L.warps[prec], p.smoother, p.smoother_degree}].push_back(i);
    }
    for (auto& kv : key) {
      BatchGroup g;
      g.mem = kv.second;
      std::vector<const OpLevel*> lv;
      std::vector<const void*> src;
      std::vector<void*> dst;
      for (int i : g.mem) {
        Problem& p = *ps[i];
        lv.push_back(p.levels[t].get());
        src.push_back(t == 0 ? x[i] : p.ws[prec][t].x.get());
        dst.push_back(p.ws[prec][t].t.get());
      }
      g.op = MultiOpPtr(multi_op_create(lv, src, dst, prec, bud));
      B->groups[t].push_back(std::move(g));
    }
  }
  return B;
}

// One smoothing sweep of every member of a group: the same steps as smooth_t (without fusion),
// the operator applications of all members in one multi-problem launch per colour.
template <typename T>
static void batch_smooth(BatchVcycle& B, int t, BatchGroup& G, bool x_is_zero, cudaStream_t s) {
  const int prec = B.prec;
  const Problem& p0 = *B.ps[G.mem[0]];
  const int degree = p0.smoother_degree;
  struct M {
    T *x, *d, *t;
    const T *b, *dinv;
    int64_t n;
    double theta, delta, sigma, rho_old;
    T omega;
  };
  std::vector<M> ms;
  for (int i : G.mem) {
    Problem& p = *B.ps[i];
    OpLevel& lv = *p.levels[t];
    Workspace& w = p.ws[prec][t];
    M m;
    m.x = t == 0 ? (T*)B.x0[i] : w.x.as<T>();
    m.b = t == 0 ? (const T*)B.b0[i] : w.b.as<T>();
    m.d = w.d.as<T>();
    m.t = w.t.as<T>();
    m.dinv = lv.dinv[prec].as<T>();
    m.n = lv.n_dofs;
    const double lmax = lv.lmax, lmin = lmax / 20.0;
    m.omega = (T)(2.0 / (lmin + lmax));
    m.theta = 0.5 * (lmax + lmin);
    m.delta = 0.5 * (lmax - lmin);
    m.sigma = m.theta / m.delta;
    m.rho_old = 1.0 / m.sigma;
    ms.push_back(m);
  }
  if (p0.smoother == 1) {  // Jacobi relaxation
    for (int it = 0; it < degree; ++it) {
      if (it == 0 && x_is_zero) {
        for (M& m : ms) vcheby0<T>(m.x, m.d, m.b, m.dinv, m.omega, m.n, s);
      } else {
        multi_vmult(*G.op, s);
        for (M& m : ms) vcheby<T>(m.x, m.d, m.b, m.t, m.dinv, T(0), (T)(double)m.omega, m.n, s);
      }
    }
    return;
  }
  if (x_is_zero) {
    for (M& m : ms) vcheby0<T>(m.x, m.d, m.b, m.dinv, (T)(1.0 / m.theta), m.n, s);
  } else {
    multi_vmult(*G.op, s);
    for (M& m : ms) vcheby<T>(m.x, m.d, m.b, m.t, m.dinv, T(0), (T)(1.0 / m.theta), m.n, s);
  }
  for (int j = 1; j < degree; ++j) {
    multi_vmult(*G.op, s);
    for (M& m : ms) {
      const double rho = 1.0 / (2.0 * m.sigma - m.rho_old);
      vcheby<T>(m.x, m.d, m.b, m.t, m.dinv, (T)(rho * m.rho_old), (T)(2.0 * rho / m.delta), m.n, s);
      m.rho_old = rho;
    }
  }
}

template <typename T>
static void batch_vcycle_t(BatchVcycle& B, cudaStream_t s) {
  const int prec = B.prec;
  const int np = (int)B.ps.size();
  auto bv = [&](int i, int l) -> T* { return l == 0 ? (T*)B.b0[i] : B.ps[i]->ws[prec][l].b.as<T>(); };
  auto xv = [&](int i, int l) -> T* { return l == 0 ? (T*)B.x0[i] : B.ps[i]->ws[prec][l].x.as<T>(); };
  auto nl = [&](int i) { return (int)B.ps[i]->levels.size(); };
  // descent: pre-smoothing, residual and restriction per level; coarse solves where a hierarchy ends
  for (int t = 0; t < B.steps; ++t) {
    for (int i = 0; i < np; ++i)
      if (t == nl(i) - 1) coarse_solve<T>(*B.ps[i], prec, bv(i, t), xv(i, t), s);
    for (BatchGroup& g : B.groups[t]) batch_smooth<T>(B, t, g, true, s);
    for (BatchGroup& g : B.groups[t]) {
      multi_vmult(*g.op, s);
      for (int i : g.mem) {
        Problem& p = *B.ps[i];
        Workspace& w = p.ws[prec][t];
        vsub<T>(w.r.as<T>(), bv(i, t), w.t.as<T>(), p.levels[t]->n_dofs, s);
        transfer_restrict(*p.transfers[t], *p.levels[t], *p.levels[t + 1], prec, w.r.get(),
                          p.ws[prec][t + 1].b.get(), s);
      }
    }
  }
  // ascent: prolongation and post-smoothing
  for (int t = B.steps - 2; t >= 0; --t) {
    for (BatchGroup& g : B.groups[t]) {
      for (int i : g.mem) {
        Problem& p = *B.ps[i];
        transfer_prolongate_add(*p.transfers[t], *p.levels[t], *p.levels[t + 1], prec, p.ws[prec][t + 1].x.get(),
                                xv(i, t), s);
      }
      batch_smooth<T>(B, t, g, false, s);
    }
  }
}

void batch_vcycle(BatchVcycle& B, cudaStream_t s) {
  if (B.prec == 0)
    batch_vcycle_t<double>(B, s);
  else
    batch_vcycle_t<float>(B, s);
}

struct BatchPrecond {
  std::vector<Problem*> ps;
  BatchVcyclePtr vc[2];
  cudaStream_t cap = nullptr;
  cudaGraphExec_t graph = nullptr;
  ~BatchPrecond() {
    if (graph) cudaGraphExecDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
  }
};

void BatchPrecondDel::operator()(BatchPrecond* b) const { delete b; }

// the preconditioners of precondition_body for every member, the V-cycles batched per precision
static void batch_precond_body(BatchPrecond& B, cudaStream_t s) {
  for (Problem* p : B.ps)
    if (p->mg_precision == 1) vcast_d2f(p->mg_b32.as<float>(), p->pc_in.as<double>(), sys_of(*p).n_dofs, s);
  for (int prec = 0; prec < 2; ++prec)
    if (B.vc[prec]) batch_vcycle(*B.vc[prec], s);
  for (Problem* p : B.ps)
    if (p->mg_precision == 1) vcast_f2d(p->pc_out.as<double>(), p->mg_x32.as<float>(), sys_of(*p).n_dofs, s);
}

BatchPrecondPtr make_batch_precond(const std::vector<Problem*>& ps) {
  BatchPrecondPtr B(new BatchPrecond);
  B->ps = ps;
  for (int prec = 0; prec < 2; ++prec) {
    std::vector<Problem*> mem;
    std::vector<const void*> b;
    std::vector<void*> x;
    for (Problem* p : ps) {
      if (p->mg_precision != prec) continue;
      mem.push_back(p);
      b.push_back(prec == 1 ? p->mg_b32.get() : p->pc_in.get());
      x.push_back(prec == 1 ? p->mg_x32.get() : p->pc_out.get());
    }
    if (!mem.empty()) B->vc[prec] = make_batch_vcycle(mem, prec, b, x, nullptr);
  }
  MFNS_CUDA(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
  std::vector<std::unique_ptr<TimerPause>> pause;
  for (Problem* p : ps) pause.push_back(std::make_unique<TimerPause>(*p));
  MFNS_CUDA(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
  batch_precond_body(*B, B->cap);
  cudaGraph_t g;
  MFNS_CUDA(cudaStreamEndCapture(B->cap, &g));
  MFNS_CUDA(cudaGraphInstantiate(&B->graph, g, 0));
  MFNS_CUDA(cudaGraphDestroy(g));
  return B;
}

void batch_precond_launch(BatchPrecond& B, cudaStream_t s) { MFNS_CUDA(cudaGraphLaunch(B.graph, s)); }

}  // namespace mfns
