// C ABI (include/mfns.h): argument checking, error translation, dispatch.
#include "../../include/mfns.h"

#include <algorithm>
#include <chrono>
#include <cstring>
#include <string>

#include "capi_types.hpp"
#include "problem.hpp"
#include "vec.hpp"

namespace mfns {
bool op_supported(int dim, int k, int op);
}
using namespace mfns;
static bool op_supported_kind(int dim, int kind, int k);

static thread_local std::string g_err;

// Every failure also consumes the runtime's pending error, if any: a failed library call (say a
// memset or launch-configuration error caught by MFNS_CUDA) must not leave an error behind that
// the caller's next, unrelated CUDA call (PyTorch's, for instance) would report as its own.
static int fail(int code, const std::string& msg) {
  (void)cudaGetLastError();
  g_err = msg;
  return code;
}

// A vector argument's length (elements) against the length the call expects.
static bool len_ok(int64_t got, int64_t want, const char* what) {
  if (got == want) return true;
  fail(MFNS_ERR_ARG, std::string(what) + " has " + std::to_string(got) + " entries, expected " +
                         std::to_string(want));
  return false;
}
#define CHECK_LEN(got, want, what) \
  if (!len_ok((got), (want), (what))) return MFNS_ERR_ARG

namespace mfns {
int capi_fail(int code, const char* msg) { return fail(code, msg); }
}  // namespace mfns

// Every entry first consumes a runtime error left pending in this thread by another component of
// the process (the runtime is shared, e.g. with PyTorch): the library checks each of its own calls
// when it fails, and the post-launch checks must not report someone else's error.
#define API_BEGIN \
  try {           \
    (void)cudaGetLastError();
#define API_END                                                      \
  }                                                                  \
  catch (const Error& e) { return fail(e.code, e.what()); }          \
  catch (const std::bad_alloc&) { return fail(kErrOom, "host allocation failed"); } \
  catch (const std::exception& e) { return fail(kErrArg, e.what()); } \
  return MFNS_OK;

static cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

BatchRound* batch_round(mfns_ctx* ctx, const std::vector<Problem*>& ps) {
  std::vector<std::pair<uint64_t, uint64_t>> key;
  for (Problem* p : ps) key.push_back({p->uid, p->graph_epoch});
  if (!ctx->round) {
    ctx->round = std::make_unique<BatchRound>();
    MFNS_CUDA(cudaStreamCreateWithFlags(&ctx->round->stream, cudaStreamNonBlocking));
    MFNS_CUDA(cudaEventCreateWithFlags(&ctx->round->done, cudaEventDisableTiming));
  }
  BatchRound& r = *ctx->round;
  if (!r.plan || r.key != key) {
    MFNS_CUDA(cudaStreamSynchronize(r.stream));
    r.plan.reset();
    r.plan = make_batch_precond(ps);
    r.key = key;
  }
  return &r;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

extern "C" {

const char* mfns_last_error(void) { return g_err.c_str(); }

int mfns_ctx_create(int device, size_t hbm_budget_bytes, mfns_ctx** out) {
  API_BEGIN
  if (!out) return fail(MFNS_ERR_ARG, "out is null");
  int n = 0;
  MFNS_CUDA(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return fail(MFNS_ERR_ARG, "invalid device");
  MFNS_CUDA(cudaSetDevice(device));
  auto* c = new mfns_ctx;
  c->device = device;
  c->budget.limit = hbm_budget_bytes;
  *out = c;
  API_END
}

int mfns_ctx_set_batching(mfns_ctx* ctx, int enable) {
  if (!ctx) return fail(MFNS_ERR_ARG, "ctx is null");
  ctx->batching = enable != 0;
  return MFNS_OK;
}

int mfns_ctx_destroy(mfns_ctx* ctx) {
  delete ctx;
  return MFNS_OK;
}

int mfns_ctx_memory(const mfns_ctx* ctx, size_t* used, size_t* peak) {
  if (!ctx) return fail(MFNS_ERR_ARG, "ctx is null");
  if (used) *used = ctx->budget.used;
  if (peak) *peak = ctx->budget.peak;
  return MFNS_OK;
}

int mfns_mesh_uniform(mfns_ctx* ctx, int dim, int n, mfns_mesh** out) {
  API_BEGIN
  if (!ctx || !out) return fail(MFNS_ERR_ARG, "null argument");
  if ((dim != 2 && dim != 3) || n < 1 || n > 1024) return fail(MFNS_ERR_ARG, "dim must be 2 or 3, 1 <= n <= 1024");
  auto* m = new mfns_mesh;
  m->ctx = ctx;
  m->forest = forest_uniform(dim, n);
  *out = m;
  API_END
}

int mfns_mesh_refine_ball(mfns_mesh* mesh, const double centre[3], double radius, int levels) {
  API_BEGIN
  if (!mesh || !centre || levels < 0 || levels > 6 || !(radius > 0)) return fail(MFNS_ERR_ARG, "bad refinement");
  mesh->forest = forest_refine_ball(mesh->forest, centre, radius, levels);
  API_END
}

int mfns_mesh_info(const mfns_mesh* mesh, int64_t* n_cells, int* max_level) {
  if (!mesh) return fail(MFNS_ERR_ARG, "mesh is null");
  if (n_cells) *n_cells = (int64_t)mesh->forest.n_cells();
  if (max_level) *max_level = mesh->forest.max_level();
  return MFNS_OK;
}

int mfns_mesh_destroy(mfns_mesh* mesh) {
  delete mesh;
  return MFNS_OK;
}

static int finish_problem(mfns_ctx* ctx, const mfns_problem_desc* desc, std::unique_ptr<Problem> p, size_t used0,
                          mfns_problem** out);

int mfns_problem_create(mfns_ctx* ctx, const mfns_mesh* mesh, const mfns_problem_desc* desc, mfns_problem** out) {
  API_BEGIN
  if (!ctx || !mesh || !desc || !out) return fail(MFNS_ERR_ARG, "null argument");
  if (desc->kind < 0 || desc->kind > 3) return fail(MFNS_ERR_ARG, "unknown kind");
  if (!(desc->nu > 0)) return fail(MFNS_ERR_ARG, "nu must be positive");
  if (desc->mg_precision != MFNS_FP64 && desc->mg_precision != MFNS_FP32) return fail(MFNS_ERR_ARG, "bad precision");
  const int dim = mesh->forest.dim, k = desc->degree;
  if (!op_supported_kind(dim, desc->kind, k)) return fail(MFNS_ERR_UNSUPPORTED, "unsupported (dim, kind, degree)");
  MFNS_CUDA(cudaSetDevice(ctx->device));
  Physics ph;
  ph.nu = desc->nu;
  ph.dt = desc->dt > 0 ? desc->dt : 0.0;
  ph.terms = desc->terms == 0 ? MFNS_TERMS_ALL : desc->terms;
  ph.div_sign = desc->div_sign != 0 ? desc->div_sign : (desc->kind == MFNS_STAB_NS ? 1.0 : -1.0);
  ph.precompute_frozen = desc->recompute_frozen == 0;
  const size_t used0 = ctx->budget.used;
  if (desc->hierarchy != 0 && desc->hierarchy != 1) return fail(MFNS_ERR_ARG, "hierarchy must be 0 or 1");
  if (desc->hierarchy == 1 && desc->kind == MFNS_PMASS)
    return fail(MFNS_ERR_UNSUPPORTED, "local smoothing is built for MFNS_STOKES, MFNS_STOKES_A and MFNS_STAB_NS");
  std::unique_ptr<Problem> p = build_problem(mesh->forest, desc->kind, k, ph, desc->mg_order,
                                             desc->coarse_stop_n > 0 ? desc->coarse_stop_n : 2, &ctx->budget,
                                             desc->hierarchy);
  return finish_problem(ctx, desc, std::move(p), used0, out);
  API_END
}

// settings, workspaces, autotuning, smoother bounds and the coarse solver of a built problem
static int finish_problem(mfns_ctx* ctx, const mfns_problem_desc* desc, std::unique_ptr<Problem> p, size_t used0,
                          mfns_problem** out) {
  if (desc->smoother < 0 || desc->smoother > 3) return fail(MFNS_ERR_ARG, "smoother must be 0, 1, 2 or 3");
  // internal: 0 = Chebyshev, 1 = Jacobi relaxation, 2 = Chebyshev around Jacobi + Schwarz blocks on
  // the combined faces of hp levels (Chebyshev around Jacobi on the other levels)
  p->smoother = desc->smoother == 0 ? (desc->kind == MFNS_STAB_NS ? 1 : 0) : desc->smoother - 1;
  p->smoother_degree = desc->smoother_degree > 0 ? desc->smoother_degree : 5;
  p->mg_precision = desc->mg_precision;
  p->restart = desc->fgmres_restart > 0 ? desc->fgmres_restart : 30;
  if (p->restart >= kMaxDots) return fail(MFNS_ERR_ARG, "fgmres_restart must be < 32");
  p->tol = desc->tol > 0 ? desc->tol : 1e-8;
  p->maxit = desc->maxit > 0 ? desc->maxit : 500;
  p->cg_iterations = desc->cg_iterations > 0 ? desc->cg_iterations : 10;
  p->fused_smoother = desc->fused_smoother != 0;
  if (desc->lambda_max > 0)
    for (int l = 0; l < mg_level_count(*p); ++l) mg_level(*p, l).lmax = desc->lambda_max;
  alloc_workspaces(*p);
  cudaStream_t s = 0;
  autotune(*p, s);
  estimate_lambda(*p, s);
  setup_coarse(*p, s);
  MFNS_CUDA(cudaStreamSynchronize(s));
  p->bytes = ctx->budget.used - used0;
  auto* w = new mfns_problem;
  w->ctx = ctx;
  w->p = std::move(p);
  *out = w;
  return MFNS_OK;
}

int mfns_problem_create_hp(mfns_ctx* ctx, const mfns_mesh* mesh, const mfns_problem_desc* desc,
                           const int32_t* cell_degree, int64_t n_cells, mfns_problem** out) {
  API_BEGIN
  if (!ctx || !mesh || !desc || !cell_degree || !out) return fail(MFNS_ERR_ARG, "null argument");
  if (n_cells != (int64_t)mesh->forest.n_cells()) return fail(MFNS_ERR_ARG, "one degree per mesh cell expected");
  if (desc->kind != MFNS_STOKES_A && desc->kind != MFNS_STOKES)
    return fail(MFNS_ERR_UNSUPPORTED, "hp problems are built for MFNS_STOKES_A and MFNS_STOKES");
  if (desc->hierarchy != 0) return fail(MFNS_ERR_UNSUPPORTED, "hp problems use global coarsening");
  if (!(desc->nu > 0)) return fail(MFNS_ERR_ARG, "nu must be positive");
  if (desc->mg_precision != MFNS_FP64 && desc->mg_precision != MFNS_FP32) return fail(MFNS_ERR_ARG, "bad precision");
  const int dim = mesh->forest.dim;
  std::vector<int32_t> degree(cell_degree, cell_degree + n_cells);
  for (int32_t k : degree)
    if (!op_supported_kind(dim, desc->kind, k)) return fail(MFNS_ERR_UNSUPPORTED, "unsupported cell degree");
  MFNS_CUDA(cudaSetDevice(ctx->device));
  Physics ph;
  ph.nu = desc->nu;
  ph.div_sign = -1.0;
  const size_t used0 = ctx->budget.used;
  std::unique_ptr<Problem> p = build_problem_hp(mesh->forest, degree, ph,
                                                desc->coarse_stop_n > 0 ? desc->coarse_stop_n : 2, &ctx->budget,
                                                desc->kind == MFNS_STOKES ? 0 : 1);
  return finish_problem(ctx, desc, std::move(p), used0, out);
  API_END
}

int mfns_mesh_cells(const mfns_mesh* mesh, int32_t* cells, int64_t cap, int64_t* n) {
  if (!mesh || !n) return fail(MFNS_ERR_ARG, "null argument");
  const Forest& f = mesh->forest;
  *n = (int64_t)f.n_cells();
  if (cells)
    for (int64_t c = 0; c < *n && c < cap; ++c) {
      cells[4 * c] = f.lev[c];
      for (int d = 0; d < 3; ++d) cells[4 * c + 1 + d] = f.crd[3 * c + d];
    }
  return MFNS_OK;
}

int mfns_problem_destroy(mfns_problem* p) {
  if (p && p->ctx) cudaSetDevice(p->ctx->device);
  delete p;
  return MFNS_OK;
}

static OpLevel* select_op(mfns_problem* p, int which) {
  Problem& P = *p->p;
  if (which == MFNS_OP_SYSTEM) return P.system ? P.system.get() : P.levels[0].get();
  if (which == MFNS_OP_PMASS) return P.pmass ? P.pmass.get() : nullptr;
  if (which >= 0 && which < mg_level_count(P)) return &mg_level(P, which);
  return nullptr;
}

int mfns_problem_info(const mfns_problem* pc, mfns_info* out) {
  if (!pc || !out) return fail(MFNS_ERR_ARG, "null argument");
  mfns_problem* p = const_cast<mfns_problem*>(pc);
  Problem& P = *p->p;
  std::memset(out, 0, sizeof(*out));
  OpLevel& S = *select_op(p, MFNS_OP_SYSTEM);
  out->dim = P.dim;
  out->degree = P.k;
  out->kind = P.kind;
  const int nl = mg_level_count(P);
  out->n_levels = nl;
  out->n_dofs = S.n_dofs;
  out->n_velocity_dofs = S.n_main_dofs;
  out->n_cells = (int64_t)S.forest.n_cells();
  out->n_colors = S.L.n_colors;
  for (int l = 0; l < nl && l < 32; ++l) {
    OpLevel& lv = mg_level(P, l);
    out->level_dofs[l] = lv.n_dofs;
    out->level_degree[l] = lv.k;
    out->level_cells[l] = (int64_t)lv.forest.n_cells();
    out->lambda_max[l] = lv.lmax;
  }
  out->device_bytes = P.bytes;
  out->cycle_dofs = P.levels[0]->n_dofs;
  return MFNS_OK;
}

int mfns_dof_support_points(const mfns_problem* pc, int which, double* xyz, int* field) {
  API_BEGIN
  OpLevel* lv = pc ? select_op(const_cast<mfns_problem*>(pc), which) : nullptr;
  if (!lv || !xyz || !field) return fail(MFNS_ERR_ARG, "bad operator selector or null output");
  oplevel_support(*lv, xyz, field);
  API_END
}

int mfns_constrained_dofs(const mfns_problem* pc, int which, int64_t* idx, int64_t cap, int64_t* n) {
  API_BEGIN
  OpLevel* lv = pc ? select_op(const_cast<mfns_problem*>(pc), which) : nullptr;
  if (!lv || !n) return fail(MFNS_ERR_ARG, "bad operator selector");
  *n = (int64_t)lv->constrained_host.size();
  if (idx)
    for (int64_t i = 0; i < *n && i < cap; ++i) idx[i] = lv->constrained_host[i];
  API_END
}

int mfns_set_lambda_max(mfns_problem* p, int level, double lmax) {
  if (!p || level < 0 || level >= mg_level_count(*p->p) || !(lmax > 0)) return fail(MFNS_ERR_ARG, "bad level");
  mg_level(*p->p, level).lmax = lmax;
  invalidate_graphs(*p->p);
  return MFNS_OK;
}

int mfns_vmult(mfns_problem* p, int which, int prec, const void* src, void* dst, int64_t n, void* stream) {
  API_BEGIN
  OpLevel* lv = p ? select_op(p, which) : nullptr;
  if (!lv || !src || !dst || src == dst) return fail(MFNS_ERR_ARG, "bad arguments");
  CHECK_LEN(n, lv->n_dofs, "src/dst");
  if (prec != 0 && prec != 1) return fail(MFNS_ERR_ARG, "bad precision");
  if (!aligned16(src) || !aligned16(dst)) return fail(MFNS_ERR_ARG, "vectors must be 16-byte aligned");
  MFNS_CUDA(cudaSetDevice(p->ctx->device));
  oplevel_vmult(*lv, prec, src, dst, S(stream));
  API_END
}

// staging of mfns_vmult_host for (which, prec, n), (re)built when the pair changes
static HostIO& host_io(mfns_problem* p, int which, int prec, int64_t n) {
  std::unique_ptr<HostIO>& h = p->hio;
  if (h && h->which == which && h->prec == prec && h->n == n) return *h;
  if (h) {
    MFNS_CUDA(cudaStreamSynchronize(h->s_in));
    MFNS_CUDA(cudaStreamSynchronize(h->s_out));
    h.reset();
  }
  auto nh = std::make_unique<HostIO>();
  nh->which = which;
  nh->prec = prec;
  nh->n = n;
  const size_t bytes = (size_t)n * esize(prec);
  for (int k = 0; k < 2; ++k) {
    nh->in[k].alloc(p->p->bud, bytes);
    nh->out[k].alloc(p->p->bud, bytes);
  }
  MFNS_CUDA(cudaStreamCreateWithFlags(&nh->s_in, cudaStreamNonBlocking));
  MFNS_CUDA(cudaStreamCreateWithFlags(&nh->s_out, cudaStreamNonBlocking));
  for (cudaEvent_t* e : {&nh->ev_start, &nh->ev_done, &nh->ev_in[0], &nh->ev_in[1], &nh->ev_ap[0], &nh->ev_ap[1],
                         &nh->ev_out[0], &nh->ev_out[1]})
    MFNS_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  h = std::move(nh);
  return *h;
}

int mfns_vmult_host(mfns_problem* p, int which, int prec, const void* const* src_host, void* const* dst_host,
                    int count, int64_t n, void* stream) {
  API_BEGIN
  OpLevel* lv = p ? select_op(p, which) : nullptr;
  if (!lv || !src_host || !dst_host || count < 1) return fail(MFNS_ERR_ARG, "bad arguments");
  CHECK_LEN(n, lv->n_dofs, "src_host/dst_host");
  if (prec != 0 && prec != 1) return fail(MFNS_ERR_ARG, "bad precision");
  for (int i = 0; i < count; ++i)
    if (!src_host[i] || !dst_host[i]) return fail(MFNS_ERR_ARG, "null host vector");
  MFNS_CUDA(cudaSetDevice(p->ctx->device));
  HostIO& h = host_io(p, which, prec, n);
  const cudaStream_t s = S(stream);
  const size_t bytes = (size_t)n * esize(prec);
  // the copy streams start after the work already in `stream` (and so after any earlier call)
  MFNS_CUDA(cudaEventRecord(h.ev_start, s));
  MFNS_CUDA(cudaStreamWaitEvent(h.s_in, h.ev_start, 0));
  MFNS_CUDA(cudaStreamWaitEvent(h.s_out, h.ev_start, 0));
  for (int i = 0; i < count; ++i) {
    const int k = i & 1;
    // staging set k: its previous product has read in[k], its previous read-back has read out[k]
    // (events not yet recorded count as complete)
    MFNS_CUDA(cudaStreamWaitEvent(h.s_in, h.ev_ap[k], 0));
    MFNS_CUDA(cudaMemcpyAsync(h.in[k].get(), src_host[i], bytes, cudaMemcpyHostToDevice, h.s_in));
    MFNS_CUDA(cudaEventRecord(h.ev_in[k], h.s_in));
    MFNS_CUDA(cudaStreamWaitEvent(s, h.ev_in[k], 0));
    MFNS_CUDA(cudaStreamWaitEvent(s, h.ev_out[k], 0));
    oplevel_vmult(*lv, prec, h.in[k].get(), h.out[k].get(), s);
    MFNS_CUDA(cudaEventRecord(h.ev_ap[k], s));
    MFNS_CUDA(cudaStreamWaitEvent(h.s_out, h.ev_ap[k], 0));
    MFNS_CUDA(cudaMemcpyAsync(dst_host[i], h.out[k].get(), bytes, cudaMemcpyDeviceToHost, h.s_out));
    MFNS_CUDA(cudaEventRecord(h.ev_out[k], h.s_out));
  }
  MFNS_CUDA(cudaEventRecord(h.ev_done, h.s_out));
  MFNS_CUDA(cudaStreamWaitEvent(s, h.ev_done, 0));
  API_END
}

int mfns_kernel_timing(mfns_problem* p, int which, int mode, double* total_ms, int64_t* launches) {
  API_BEGIN
  OpLevel* lv = p ? select_op(p, which) : nullptr;
  if (!lv || mode < 0 || mode > 2) return fail(MFNS_ERR_ARG, "bad arguments");
  MFNS_CUDA(cudaSetDevice(p->ctx->device));
  KernelTimer& t = *lv->timer;
  if (mode == 1) {
    t.read_ms(nullptr);
    t.enabled = true;
  } else if (mode == 0) {
    t.enabled = false;
  } else {
    const double ms = t.read_ms(launches);
    if (total_ms) *total_ms = ms;
  }
  API_END
}

int mfns_diagonal(mfns_problem* p, int which, int prec, void* diag, int64_t n, void* stream) {
  API_BEGIN
  OpLevel* lv = p ? select_op(p, which) : nullptr;
  if (!lv || !diag || (prec != 0 && prec != 1)) return fail(MFNS_ERR_ARG, "bad arguments");
  CHECK_LEN(n, lv->n_dofs, "diag");
  MFNS_CUDA(cudaSetDevice(p->ctx->device));
  oplevel_diag(*lv, prec, diag, S(stream));
  API_END
}

int mfns_apply_constraints(mfns_problem* p, int which, int prec, void* x, int64_t n, void* stream) {
  API_BEGIN
  OpLevel* lv = p ? select_op(p, which) : nullptr;
  if (!lv || !x || (prec != 0 && prec != 1)) return fail(MFNS_ERR_ARG, "bad arguments");
  CHECK_LEN(n, lv->n_dofs, "x");
  MFNS_CUDA(cudaSetDevice(p->ctx->device));
  oplevel_distribute(*lv, prec, x, S(stream));
  API_END
}

int mfns_smooth(mfns_problem* p, int level, int prec, const void* b, void* x, int64_t n, int x_is_zero,
                void* stream) {
  API_BEGIN
  if (!p || level < 0 || level >= (int)p->p->levels.size() || !b || !x || (prec != 0 && prec != 1))
    return fail(MFNS_ERR_ARG, "bad arguments");
  if (p->p->ls) return fail(MFNS_ERR_UNSUPPORTED, "single-level smoothing is not exposed for local smoothing");
  CHECK_LEN(n, p->p->levels[level]->n_dofs, "b/x");
  MFNS_CUDA(cudaSetDevice(p->ctx->device));
  smooth(*p->p, level, prec, b, x, x_is_zero != 0, S(stream));
  API_END
}

int mfns_prolongate_add(mfns_problem* p, int level, int prec, const void* coarse, int64_t n_coarse, void* fine,
                        int64_t n_fine, void* stream) {
  API_BEGIN
  if (!p || level < 0 || level + 1 >= (int)p->p->levels.size() || !coarse || !fine || (prec != 0 && prec != 1))
    return fail(MFNS_ERR_ARG, "bad arguments");
  Problem& P = *p->p;
  CHECK_LEN(n_coarse, P.levels[level + 1]->n_dofs, "coarse");
  CHECK_LEN(n_fine, P.levels[level]->n_dofs, "fine");
  MFNS_CUDA(cudaSetDevice(p->ctx->device));
  transfer_prolongate_add(*P.transfers[level], *P.levels[level], *P.levels[level + 1], prec, coarse, fine, S(stream));
  API_END
}

int mfns_restrict(mfns_problem* p, int level, int prec, const void* fine, int64_t n_fine, void* coarse,
                  int64_t n_coarse, void* stream) {
  API_BEGIN
  if (!p || level < 0 || level + 1 >= (int)p->p->levels.size() || !coarse || !fine || (prec != 0 && prec != 1))
    return fail(MFNS_ERR_ARG, "bad arguments");
  Problem& P = *p->p;
  CHECK_LEN(n_fine, P.levels[level]->n_dofs, "fine");
  CHECK_LEN(n_coarse, P.levels[level + 1]->n_dofs, "coarse");
  MFNS_CUDA(cudaSetDevice(p->ctx->device));
  transfer_restrict(*P.transfers[level], *P.levels[level], *P.levels[level + 1], prec, fine, coarse, S(stream));
  API_END
}

int mfns_vcycle(mfns_problem* p, int prec, const void* b, void* x, int64_t n, void* stream) {
  API_BEGIN
  if (!p || !b || !x || (prec != 0 && prec != 1)) return fail(MFNS_ERR_ARG, "bad arguments");
  CHECK_LEN(n, p->p->levels[0]->n_dofs, "b/x (cycle_dofs)");
  MFNS_CUDA(cudaSetDevice(p->ctx->device));
  if (p->p->use_graphs)
    vcycle_graph(*p->p, prec, b, x, S(stream));
  else
    vcycle(*p->p, prec, b, x, S(stream));
  API_END
}

int mfns_solve(mfns_problem* p, const void* b, void* x, int64_t n, mfns_solve_info* info, void* stream) {
  API_BEGIN
  if (!p || !b || !x) return fail(MFNS_ERR_ARG, "bad arguments");
  if (p->p->kind == MFNS_PMASS) return fail(MFNS_ERR_UNSUPPORTED, "no solver for the pressure mass problem");
  CHECK_LEN(n, select_op(p, MFNS_OP_SYSTEM)->n_dofs, "b/x");
  MFNS_CUDA(cudaSetDevice(p->ctx->device));
  auto t0 = std::chrono::steady_clock::now();
  double rel = 0;
  bool conv = false;
  int it = fgmres_solve(*p->p, (const double*)b, (double*)x, &rel, &conv, S(stream));
  MFNS_CUDA(cudaStreamSynchronize(S(stream)));
  auto t1 = std::chrono::steady_clock::now();
  if (info) {
    info->iterations = it;
    info->rel_residual = rel;
    info->seconds = std::chrono::duration<double>(t1 - t0).count();
    info->converged = conv ? 1 : 0;
  }
  if (!conv) return fail(MFNS_ERR_NOT_CONVERGED, "FGMRES reached maxit");
  API_END
}

int mfns_set_state(mfns_problem* p, double dt, double alpha, const void* state, const void* explicit_field,
                   int64_t n, void* stream) {
  API_BEGIN
  if (!p || !state) return fail(MFNS_ERR_ARG, "bad arguments");
  CHECK_LEN(n, select_op(p, MFNS_OP_SYSTEM)->n_dofs, "state/explicit_field");
  MFNS_CUDA(cudaSetDevice(p->ctx->device));
  set_state(*p->p, dt, alpha, (const double*)state, (const double*)explicit_field, S(stream));
  API_END
}

int mfns_residual(mfns_problem* p, int precision, void* dst, int64_t n, void* stream) {
  API_BEGIN
  if (!p || !dst || (precision != MFNS_FP64 && precision != MFNS_FP32)) return fail(MFNS_ERR_ARG, "bad arguments");
  CHECK_LEN(n, select_op(p, MFNS_OP_SYSTEM)->n_dofs, "dst");
  MFNS_CUDA(cudaSetDevice(p->ctx->device));
  residual(*p->p, precision, dst, S(stream));
  API_END
}

int mfns_bdf_step(mfns_problem* p, const mfns_newton_desc* desc, const void* u_n, const void* u_nm1,
                  const void* forcing, void* u, int64_t n, mfns_newton_info* info, void* stream) {
  API_BEGIN
  if (!p || !desc || !u_n || !u) return fail(MFNS_ERR_ARG, "bad arguments");
  CHECK_LEN(n, select_op(p, MFNS_OP_SYSTEM)->n_dofs, "u_n/u_nm1/forcing/u");
  MFNS_CUDA(cudaSetDevice(p->ctx->device));
  NewtonParams np;
  np.dt = desc->dt;
  np.omega = desc->omega;
  np.rtol = desc->rtol > 0 ? desc->rtol : 1e-8;
  np.atol = desc->atol > 0 ? desc->atol : 0.0;
  np.lin_tol = desc->lin_tol > 0 ? desc->lin_tol : 1e-4;
  np.max_newton = desc->max_newton > 0 ? desc->max_newton : 10;
  np.extrapolate = desc->extrapolate != 0;
  auto t0 = std::chrono::steady_clock::now();
  NewtonResult r = bdf_step(*p->p, np, (const double*)u_n, (const double*)u_nm1, (const double*)forcing,
                            (double*)u, S(stream));
  MFNS_CUDA(cudaStreamSynchronize(S(stream)));
  auto t1 = std::chrono::steady_clock::now();
  if (info) {
    info->newton_iterations = r.newton_iterations;
    info->linear_iterations = r.linear_iterations;
    info->residual0 = r.residual0;
    info->residual = r.residual;
    info->seconds = std::chrono::duration<double>(t1 - t0).count();
    info->converged = r.converged ? 1 : 0;
  }
  if (!r.converged) return fail(MFNS_ERR_NOT_CONVERGED, "Newton reached max_newton");
  API_END
}

int mfns_max_velocity(mfns_problem* p, const void* u, int64_t n, double* umax, void* stream) {
  API_BEGIN
  if (!p || !u || !umax) return fail(MFNS_ERR_ARG, "bad arguments");
  CHECK_LEN(n, select_op(p, MFNS_OP_SYSTEM)->n_dofs, "u");
  MFNS_CUDA(cudaSetDevice(p->ctx->device));
  *umax = max_velocity(*p->p, (const double*)u, S(stream));
  API_END
}

int mfns_solve_begin(mfns_problem* p, const void* b, void* x, int64_t n, void* stream) {
  API_BEGIN
  if (!p || !b || !x) return fail(MFNS_ERR_ARG, "bad arguments");
  if (p->p->kind == MFNS_PMASS) return fail(MFNS_ERR_UNSUPPORTED, "no solver for the pressure mass problem");
  CHECK_LEN(n, select_op(p, MFNS_OP_SYSTEM)->n_dofs, "b/x");
  MFNS_CUDA(cudaSetDevice(p->ctx->device));
  krylov_begin(*p->p, (const double*)b, (double*)x, S(stream));
  API_END
}

int mfns_batch_step(mfns_problem** ps, int n, int* running) {
  API_BEGIN
  if (!ps || n < 0) return fail(MFNS_ERR_ARG, "bad arguments");
  for (int i = 0; i < n; ++i)
    if (!ps[i]) return fail(MFNS_ERR_ARG, "null problem in batch");
  if (n > 0) MFNS_CUDA(cudaSetDevice(ps[0]->ctx->device));
  // the preconditioners of the active problems that use one V-cycle on uniform levels run as one
  // batched, graph-captured V-cycle (operator applications of all of them in shared launches per
  // level and colour); every other problem, and all the rest of each step, on its own stream
  std::vector<Problem*> bat;
  for (int i = 0; i < n; ++i) {
    Problem& P = *ps[i]->p;
    if (P.kry.active && batchable(P) && ps[i]->ctx == ps[0]->ctx) bat.push_back(&P);
  }
  if (bat.size() < 2 || !ps[0]->ctx->batching) bat.clear();
  BatchRound* br = bat.empty() ? nullptr : batch_round(ps[0]->ctx, bat);
  for (int i = 0; i < n; ++i) {
    Problem& P = *ps[i]->p;
    if (br && P.kry.active && std::find(bat.begin(), bat.end(), &P) != bat.end())
      krylov_enqueue_pre(P);
    else
      krylov_enqueue(P);
  }
  if (br) {
    for (Problem* P : bat) MFNS_CUDA(cudaStreamWaitEvent(br->stream, P->ev_step, 0));
    batch_precond_launch(*br->plan, br->stream);
    MFNS_CUDA(cudaEventRecord(br->done, br->stream));
    for (Problem* P : bat) krylov_enqueue_post(*P, br->done);
  }
  for (int i = 0; i < n; ++i) {
    Problem& P = *ps[i]->p;
    bool run = false;
    if (P.kry.active) {
      MFNS_CUDA(cudaStreamSynchronize(P.kry.stream));
      run = krylov_complete(P);
    }
    if (running) running[i] = run ? 1 : 0;
  }
  API_END
}

int mfns_batch_vcycle(mfns_problem** ps, int n, int precision, void* const* b, void* const* x,
                      const int64_t* lengths, void* stream) {
  API_BEGIN
  if (!ps || n <= 0 || !b || !x || !lengths || (precision != MFNS_FP64 && precision != MFNS_FP32))
    return fail(MFNS_ERR_ARG, "bad arguments");
  std::vector<Problem*> pp;
  std::vector<const void*> bb;
  std::vector<void*> xx;
  for (int i = 0; i < n; ++i) {
    if (!ps[i] || !b[i] || !x[i]) return fail(MFNS_ERR_ARG, "null problem or vector in batch");
    if (ps[i]->ctx != ps[0]->ctx) return fail(MFNS_ERR_ARG, "problems of different contexts");
    CHECK_LEN(lengths[i], ps[i]->p->levels[0]->n_dofs, "b[i]/x[i]");
    if (!batchable(*ps[i]->p))
      return fail(MFNS_ERR_UNSUPPORTED, "batched V-cycle: one-V-cycle problems on uniform levels only");
    pp.push_back(ps[i]->p.get());
    bb.push_back(b[i]);
    xx.push_back(x[i]);
  }
  MFNS_CUDA(cudaSetDevice(ps[0]->ctx->device));
  BatchVcyclePtr B = make_batch_vcycle(pp, precision, bb, xx, nullptr);
  batch_vcycle(*B, S(stream));
  MFNS_CUDA(cudaStreamSynchronize(S(stream)));  // the plan's tables are freed on return
  API_END
}

int mfns_solve_status(const mfns_problem* p, mfns_solve_info* info) {
  if (!p || !info) return fail(MFNS_ERR_ARG, "bad arguments");
  const Krylov& K = p->p->kry;
  info->iterations = K.it;
  info->rel_residual = K.relres;
  info->seconds = 0.0;
  info->converged = K.converged ? 1 : 0;
  return MFNS_OK;
}

}  // extern "C"

static bool op_supported_kind(int dim, int kind, int k) {
  switch (kind) {
    case MFNS_STOKES: return mfns::op_supported(dim, k, OP_STOKES) && mfns::op_supported(dim, k - 1, OP_PMASS);
    case MFNS_STOKES_A: return mfns::op_supported(dim, k, OP_STOKES_A);
    case MFNS_STAB_NS: return mfns::op_supported(dim, k, OP_STAB_NS);
    case MFNS_PMASS: return mfns::op_supported(dim, k, OP_PMASS);
  }
  return false;
}
