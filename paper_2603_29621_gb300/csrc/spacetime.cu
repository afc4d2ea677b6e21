// The space-time slab operator K = G_Q (x) M + tau I_Q (x) A of Section 4 (see spacetime.hpp) on
// the Taylor--Hood space of a Stokes problem, and its C-ABI entry points.
//
// One product: A on all Q stages (the Stokes cell kernel, one launch over Q columns, identity rows
// on constrained entries), M on all Q stages (the velocity-mass cell kernel over the same velocity
// nodes, constrained velocity rows cleared), then one streaming pass y_q = tau (A x)_q +
// sum_j G[q][j] (M x)_j.
#include <algorithm>
#include <memory>
#include <string>

#include "capi_types.hpp"
#include "op_launch.hpp"
#include "spacetime.hpp"
#include "vec.hpp"

namespace {

constexpr int kMaxStages = 8;
struct StageMatrix {
  double g[kMaxStages][kMaxStages];
};

template <typename T>
__global__ void k_stage_mix(T* __restrict__ y, const T* __restrict__ mx, StageMatrix G, int Q, int64_t n, T tau) {
  const int64_t total = (int64_t)Q * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx / n);
    const int64_t i = idx - (int64_t)q * n;
    T v = tau * y[idx];
    for (int j = 0; j < Q; ++j) v += (T)G.g[q][j] * mx[(int64_t)j * n + i];
    y[idx] = v;
  }
}

}  // namespace

struct mfns_spacetime {
  mfns_problem* problem = nullptr;  // not owned; outlives the slab
  int r = 0, Q = 1;
  double tau = 0.0;
  mfns::TemporalMatrices T;
  std::unique_ptr<mfns::OpLevel> mass;  // velocity mass on the problem's velocity nodes
  mfns::DevBuf mx[2];                   // Q x n: M applied to every stage (FP64, FP32)
  int64_t n = 0;                        // spatial vector length (the Stokes system's)
};

namespace mfns {

static void st_vmult(mfns_spacetime& st, int prec, const void* x, void* y, cudaStream_t s) {
  OpLevel& A = *st.problem->p->system;
  const int64_t n = st.n;
  const size_t es = esize(prec);
  // tau A on every stage (identity rows on constrained entries)
  oplevel_vmult_cols(A, prec, x, y, st.Q, s);
  // M on every stage: the velocity block of each stage (its first n_main entries); pressure rows
  // and constrained velocity rows of M are zero
  void* mx = st.mx[prec].get();
  MFNS_CUDA(cudaMemsetAsync(mx, 0, (size_t)st.Q * n * es, s));
  op_apply_cols(st.mass->L, prec, x, mx, st.Q, n, s);
  const int64_t nc = (int64_t)st.mass->constrained_host.size();
  for (int q = 0; q < st.Q; ++q) {
    if (prec == 0)
      vset_idx<double>((double*)mx + (int64_t)q * n, 0.0, st.mass->constrained.as<int32_t>(), nc, s);
    else
      vset_idx<float>((float*)mx + (int64_t)q * n, 0.0f, st.mass->constrained.as<int32_t>(), nc, s);
  }
  StageMatrix G{};
  for (int q = 0; q < st.Q; ++q)
    for (int j = 0; j < st.Q; ++j) G.g[q][j] = st.T.G[q * st.Q + j];
  const int64_t total = (int64_t)st.Q * n;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16));
  if (prec == 0)
    k_stage_mix<double><<<grid, 256, 0, s>>>((double*)y, (const double*)mx, G, st.Q, n, st.tau);
  else
    k_stage_mix<float><<<grid, 256, 0, s>>>((float*)y, (const float*)mx, G, st.Q, n, (float)st.tau);
  MFNS_CUDA(cudaGetLastError());
}

}  // namespace mfns

extern "C" int mfns_spacetime_create(mfns_problem* p, int r, double tau, mfns_spacetime** out) {
  using namespace mfns;
  try {
    (void)cudaGetLastError();
    if (!p || !out || !(tau > 0.0)) return capi_fail(kErrArg, "bad arguments");
    *out = nullptr;
    Problem& P = *p->p;
    if (P.kind != 0 || !P.system || P.system->op != OP_STOKES)
      return capi_fail(kErrUnsupported, "space-time slabs are built on Taylor--Hood Stokes problems (MFNS_STOKES)");
    if (P.system->hp) return capi_fail(kErrUnsupported, "space-time slabs on hp spaces are not built");
    if (r < 0 || r + 1 > kMaxStages) return capi_fail(kErrArg, "temporal degree must lie in 0..7");
    MFNS_CUDA(cudaSetDevice(p->ctx->device));
    auto st = std::make_unique<mfns_spacetime>();
    st->problem = p;
    st->r = r;
    st->Q = r + 1;
    st->tau = tau;
    std::string err;
    if (!temporal_matrices(r, st->T, &err)) return capi_fail(kErrArg, err.c_str());
    const OpLevel& A = *P.system;
    st->n = A.n_dofs;
    st->mass = std::make_unique<OpLevel>();
    build_oplevel(*st->mass, A.forest, OP_VMASS, A.k, P.phys, P.bud);
    if (st->mass->n_dofs != A.n_main_dofs) return capi_fail(kErrArg, "velocity mass and system disagree on the velocity nodes");
    for (int prec = 0; prec < 2; ++prec) st->mx[prec].alloc(P.bud, (size_t)st->Q * st->n * esize(prec));
    *out = st.release();
  } catch (const Error& e) {
    return capi_fail(e.code, e.what());
  } catch (const std::exception& e) {
    return capi_fail(kErrArg, e.what());
  }
  return MFNS_OK;
}

extern "C" int mfns_spacetime_info(const mfns_spacetime* st, int* stages, int64_t* n_stage, double* nodes_host,
                                   double* g_host) {
  if (!st) return mfns::capi_fail(mfns::kErrArg, "bad arguments");
  if (stages) *stages = st->Q;
  if (n_stage) *n_stage = st->n;
  if (nodes_host) std::copy(st->T.t.begin(), st->T.t.end(), nodes_host);
  if (g_host) std::copy(st->T.G.begin(), st->T.G.end(), g_host);
  return MFNS_OK;
}

extern "C" int mfns_spacetime_vmult(mfns_spacetime* st, int prec, const void* x, void* y, void* stream) {
  using namespace mfns;
  try {
    (void)cudaGetLastError();
    if (!st || !x || !y || x == y || (prec != 0 && prec != 1)) return capi_fail(kErrArg, "bad arguments");
    MFNS_CUDA(cudaSetDevice(st->problem->ctx->device));
    st_vmult(*st, prec, x, y, reinterpret_cast<cudaStream_t>(stream));
  } catch (const Error& e) {
    return capi_fail(e.code, e.what());
  } catch (const std::exception& e) {
    return capi_fail(kErrArg, e.what());
  }
  return MFNS_OK;
}

extern "C" int mfns_spacetime_destroy(mfns_spacetime* st) {
  delete st;
  return MFNS_OK;
}

extern "C" int mfns_spacetime_temporal(int r, double* nodes_host, double* m_host, double* mq_host, double* aq_host,
                                       double* g_host) {
  mfns::TemporalMatrices T;
  std::string err;
  if (!mfns::temporal_matrices(r, T, &err)) return mfns::capi_fail(mfns::kErrArg, err.c_str());
  if (nodes_host) std::copy(T.t.begin(), T.t.end(), nodes_host);
  if (m_host) std::copy(T.m.begin(), T.m.end(), m_host);
  if (mq_host) std::copy(T.M.begin(), T.M.end(), mq_host);
  if (aq_host) std::copy(T.A.begin(), T.A.end(), aq_host);
  if (g_host) std::copy(T.G.begin(), T.G.end(), g_host);
  return MFNS_OK;
}
