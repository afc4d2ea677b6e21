// The space-time slab operator K = G_Q (x) M + tau I_Q (x) A of Section 4 (see spacetime.hpp) on
// the Taylor--Hood space of a Stokes problem, and its C-ABI entry points.
//
// One product: A on all Q stages (the Stokes cell kernel, one launch over Q columns, identity rows
// on constrained entries), M on all Q stages (the velocity-mass cell kernel over the same velocity
// nodes, constrained velocity rows cleared), then one streaming pass y_q = tau (A x)_q +
// sum_j G[q][j] (M x)_j.
#include <algorithm>
#include <cmath>
#include <memory>
#include <string>

#include "capi_types.hpp"
#include "op_launch.hpp"
#include "pdisc.hpp"
#include "pdisc_dev.hpp"
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


// fine[q n + i] += sum_j P[q][j] coarse[j n + i]  (P: Qf x Qc)
__global__ void k_time_prolong_add(double* __restrict__ fine, const double* __restrict__ coarse, StageMatrix P,
                                   int Qf, int Qc, int64_t n) {
  const int64_t total = (int64_t)Qf * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx / n);
    const int64_t i = idx - (int64_t)q * n;
    double v = fine[idx];
    for (int j = 0; j < Qc; ++j) v += P.g[q][j] * coarse[(int64_t)j * n + i];
    fine[idx] = v;
  }
}

// coarse[j n + i] = sum_q P[q][j] fine[q n + i]
__global__ void k_time_restrict(double* __restrict__ coarse, const double* __restrict__ fine, StageMatrix P, int Qf,
                                int Qc, int64_t n) {
  const int64_t total = (int64_t)Qc * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx / n);
    const int64_t i = idx - (int64_t)j * n;
    double v = 0.0;
    for (int q = 0; q < Qf; ++q) v += P.g[q][j] * fine[(int64_t)q * n + i];
    coarse[idx] = v;
  }
}

// Patch solves of the Schwarz smoother, one block per patch: the patch's entries of all stages
// (stage-major, Q m values) gathered into shared memory, times the patch's inverse (stored column
// by column, so that the threads of a warp, one row each, read consecutive words), written to the
// patch's slice of zloc (offset Q * p_ptr[p]).  TK: the type the inverses are stored in and the
// products formed in (double, or float for the FP32 smoother: half the bytes); zloc is FP64.
template <typename TK>
__global__ void k_patch_solve(const double* __restrict__ r, double* __restrict__ zloc, const int64_t* __restrict__ p_ptr,
                              const int32_t* __restrict__ p_idx, const int64_t* __restrict__ k_ptr,
                              const TK* __restrict__ kinv, int Q, int64_t n) {
  extern __shared__ __align__(16) unsigned char rl_raw[];
  TK* rl = reinterpret_cast<TK*>(rl_raw);
  const int64_t p = blockIdx.x;
  const int64_t b0 = p_ptr[p];
  const int m = (int)(p_ptr[p + 1] - b0);
  const int mq = Q * m;
  for (int t = threadIdx.x; t < mq; t += blockDim.x) {
    const int q = t / m, a = t - q * m;
    rl[t] = (TK)r[(int64_t)q * n + p_idx[b0 + a]];
  }
  __syncthreads();
  const TK* Kp = kinv + k_ptr[p];
  double* out = zloc + (int64_t)Q * b0;
  for (int row = threadIdx.x; row < mq; row += blockDim.x) {
    // eight independent partial sums: eight loads of a row in flight instead of one dependent
    // chain of mq steps
    TK v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int j = 0;
    for (; j + 7 < mq; j += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] += Kp[(int64_t)(j + u) * mq + row] * rl[j + u];
    }
    for (; j < mq; ++j) v[0] += Kp[(int64_t)j * mq + row] * rl[j];
    out[row] = (double)(((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])));
  }
}

// z[q n + i] = w[i] sum over the patches holding i of their result for (q, i), in a fixed order
// (occurrence o: zloc index e_base[o] + q * e_np[o]).
__global__ void k_patch_gather(double* __restrict__ z, const double* __restrict__ zloc, const int64_t* __restrict__ e_ptr,
                               const int64_t* __restrict__ e_base, const int32_t* __restrict__ e_np,
                               const double* __restrict__ w, int Q, int64_t n) {
  const int64_t total = (int64_t)Q * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx / n);
    const int64_t i = idx - (int64_t)q * n;
    double v = 0.0;
    for (int64_t o = e_ptr[i]; o < e_ptr[i + 1]; ++o) v += zloc[e_base[o] + (int64_t)q * e_np[o]];
    z[idx] = w[i] * v;
  }
}

// constrained rows of the slab operator are tau times identity rows: z = r / tau there
__global__ void k_constrained_scale(double* __restrict__ z, const double* __restrict__ r, const int32_t* __restrict__ con,
                                    int64_t ncon, int Q, int64_t n, double inv_tau) {
  const int64_t total = (int64_t)Q * ncon;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(t / ncon);
    const int64_t i = (int64_t)q * n + con[t - (int64_t)q * ncon];
    z[i] = r[i] * inv_tau;
  }
}

unsigned stream_grid(int64_t total) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16));
}

}  // namespace

namespace mfns {

// One level of the space-time multigrid (finest first).
struct StmgLevel {
  int k = 2, r = 0, Q = 1;
  int64_t kinv_bytes = 0;  // bytes of the Schwarz patch inverses (read once per smoother application)
  // kind 0 (Taylor--Hood): A the Stokes system, P the pressure space (transfers); kind 1
  // (Q_k / P^disc_{k-1}, uniform meshes): A the velocity block (vector Laplacian), with the cell
  // block B of the pressure coupling and the pressure embedding Ep towards the next coarser level
  int kind = 0;
  std::unique_ptr<OpLevel> A, M, P;  // A, velocity mass, pressure space
  PdiscGeom pg;
  DevBuf Bcell, Ep;
  bool ep_hstep = false;
  TemporalMatrices T;
  int64_t n = 0;
  // transfer to the next coarser level: 0 none (coarsest), 1 temporal, 2 spatial
  int tkind = 0;
  StageMatrix Pt{};  // temporal: Q x Qc
  int Qc = 1;
  std::unique_ptr<Transfer> tv, tp;  // spatial: velocity, pressure
  // Schwarz smoother
  int64_t n_patch = 0, max_patch = 0;
  DevBuf p_ptr, p_idx, k_ptr, kinv, e_ptr, e_base, e_np, w, con;  // kinv: FP64, or FP32 (inv_prec 1)
  int inv_prec = 0;
  int64_t n_con = 0;
  // FP64 work vectors of Q n entries, and the patch results
  DevBuf vx, vb, vr, vt, vz, vmx, zloc;
};

struct Stmg {
  std::vector<std::unique_ptr<StmgLevel>> lv;
  // FGMRES on the finest level (allocated on first use): basis V (m + 1 vectors), Z (m), work,
  // the device table of the basis vectors and the Gram--Schmidt coefficients (two passes and
  // the norm) with their pinned host copy
  int restart = 30;
  DevBuf V, Z, w, bp, pres0, ptrV, hvec;
  double* hh_host = nullptr;
  // the V-cycle captured once into a CUDA graph (replayed by every preconditioner application)
  cudaGraphExec_t vc_graph = nullptr;
  cudaStream_t cap_stream = nullptr;
  ~Stmg() {
    if (vc_graph) cudaGraphExecDestroy(vc_graph);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (hh_host) cudaFreeHost(hh_host);
  }
  int64_t n_pres0 = 0;
  int nu_s = 4;
  int inv_prec = 0;  // precision of the Schwarz patch inverses: 0 FP64, 1 FP32
  double omega = 0.7, tau = 0.1;
  DevBuf cinv;      // coarsest: inverse of K + sum_q E_q E_q^T, (Q n)^2
  int64_t cn = 0;   // Q n of the coarsest level
  DevBuf pres;      // coarsest: free pressure entries (spatial)
  int64_t n_pres = 0;
  DevBuf part, scal;
};

}  // namespace mfns

struct mfns_spacetime {
  mfns_ctx* ctx = nullptr;
  mfns::Budget* bud = nullptr;
  mfns_problem* problem = nullptr;  // Taylor--Hood slabs: not owned, outlives the slab
  std::unique_ptr<mfns::StmgLevel> top;  // P^disc slabs: the slab's own space (FP64)
  double nu = 1.0;                       // P^disc slabs: viscosity
  int r = 0, Q = 1;
  double tau = 0.0;
  mfns::TemporalMatrices T;
  std::unique_ptr<mfns::OpLevel> mass;  // velocity mass on the problem's velocity nodes
  mfns::DevBuf mx[2];                   // Q x n: M applied to every stage (FP64, FP32)
  int64_t n = 0;                        // spatial vector length (the Stokes system's)
  std::unique_ptr<mfns::Stmg> mg;       // space-time multigrid (built on request)
};

namespace mfns {

// y = (G (x) M + tau I (x) A) x on Q stages of length n; mx: Q * n scratch of the precision.
static void slab_vmult(const OpLevel& A, const OpLevel& M, const std::vector<double>& Gq, int Q, double tau,
                       int64_t n, void* mx, int prec, const void* x, void* y, cudaStream_t s) {
  const size_t es = esize(prec);
  // A on every stage (identity rows on constrained entries)
  oplevel_vmult_cols(A, prec, x, y, Q, s);
  // M on every stage: the velocity block of each stage (its first n_main entries); pressure rows
  // and constrained velocity rows of M are zero
  MFNS_CUDA(cudaMemsetAsync(mx, 0, (size_t)Q * n * es, s));
  op_apply_cols(M.L, prec, x, mx, Q, n, s);
  const int64_t nc = (int64_t)M.constrained_host.size();
  for (int q = 0; q < Q; ++q) {
    if (prec == 0)
      vset_idx<double>((double*)mx + (int64_t)q * n, 0.0, M.constrained.as<int32_t>(), nc, s);
    else
      vset_idx<float>((float*)mx + (int64_t)q * n, 0.0f, M.constrained.as<int32_t>(), nc, s);
  }
  StageMatrix G{};
  for (int q = 0; q < Q; ++q)
    for (int j = 0; j < Q; ++j) G.g[q][j] = Gq[q * Q + j];
  const int64_t total = (int64_t)Q * n;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16));
  if (prec == 0)
    k_stage_mix<double><<<grid, 256, 0, s>>>((double*)y, (const double*)mx, G, Q, n, tau);
  else
    k_stage_mix<float><<<grid, 256, 0, s>>>((float*)y, (const float*)mx, G, Q, n, (float)tau);
  MFNS_CUDA(cudaGetLastError());
}

// spatial P^disc Stokes operator on one vector: y_u = A_uu x_u + B^T x_p (identity rows on Dirichlet
// velocity entries), y_p = B x_u
static void pdisc_spatial(const StmgLevel& L, const double* x, double* y, cudaStream_t s) {
  oplevel_vmult(*L.A, 0, x, y, s);
  pdisc_grad_add(L.pg, L.Bcell.as<double>(), x, y, s);
  pdisc_div(L.pg, L.Bcell.as<double>(), x, y, s);
}

// y = (G (x) M + tau I (x) A_pd) x on the Q stages of a P^disc level
static void slab_vmult_pdisc(const StmgLevel& L, double tau, void* mx, const double* x, double* y, cudaStream_t s) {
  const int64_t n = L.n;
  for (int q = 0; q < L.Q; ++q) pdisc_spatial(L, x + (int64_t)q * n, y + (int64_t)q * n, s);
  MFNS_CUDA(cudaMemsetAsync(mx, 0, (size_t)L.Q * n * 8, s));
  op_apply_cols(L.M->L, 0, x, mx, L.Q, n, s);
  const int64_t nc = (int64_t)L.M->constrained_host.size();
  for (int q = 0; q < L.Q; ++q)
    vset_idx<double>((double*)mx + (int64_t)q * n, 0.0, L.M->constrained.as<int32_t>(), nc, s);
  StageMatrix G{};
  for (int q = 0; q < L.Q; ++q)
    for (int j = 0; j < L.Q; ++j) G.g[q][j] = L.T.G[q * L.Q + j];
  const int64_t total = (int64_t)L.Q * n;
  k_stage_mix<double><<<stream_grid(total), 256, 0, s>>>(y, (const double*)mx, G, L.Q, n, tau);
  MFNS_CUDA(cudaGetLastError());
}

static void st_vmult(mfns_spacetime& st, int prec, const void* x, void* y, cudaStream_t s) {
  if (st.top) {
    if (prec != 0) throw Error(kErrUnsupported, "P^disc slabs: FP64 only");
    return slab_vmult_pdisc(*st.top, st.tau, st.top->vmx.get(), (const double*)x, (double*)y, s);
  }
  slab_vmult(*st.problem->p->system, *st.mass, st.T.G, st.Q, st.tau, st.n, st.mx[prec].get(), prec, x, y, s);
}

// the P^disc space of one level: velocity block, velocity mass, cell block
static void build_pdisc_level(StmgLevel& L, const Forest& f, int k, double nu, Budget* bud) {
  if (!f.uniform()) throw Error(kErrUnsupported, "P^disc spaces: uniform meshes only");
  if (k < 2 || k > 4) throw Error(kErrUnsupported, "P^disc spaces: velocity degree 2..4");
  Physics ph;
  ph.nu = nu;
  ph.div_sign = -1.0;
  L.kind = 1;
  L.A = std::make_unique<OpLevel>();
  build_oplevel(*L.A, f, OP_STOKES_A, k, ph, bud);
  L.M = std::make_unique<OpLevel>();
  build_oplevel(*L.M, f, OP_VMASS, k, ph, bud);
  L.pg.dim = f.dim;
  L.pg.k = k;
  L.pg.n = f.n;
  L.pg.npc = (int)pdisc_exponents(f.dim, k - 1).size();
  L.pg.n_main = L.A->n_main_dofs;
  const int64_t n_cells = (int64_t)f.n_cells();
  L.n = L.A->n_main_dofs + n_cells * L.pg.npc;
  L.Bcell = upload(bud, pdisc_cell_B(f.dim, k, 1.0 / f.n));
}

static void level_support(const StmgLevel& L, double* xyz, int* field) {
  oplevel_support(*L.A, xyz, field);  // Taylor--Hood: every entry; P^disc: the velocity entries
  if (L.kind == 0) return;
  const Forest& f = L.A->forest;
  const int dim = f.dim;
  for (size_t c = 0; c < f.n_cells(); ++c)
    for (int a = 0; a < L.pg.npc; ++a) {
      const int64_t i = L.pg.n_main + (int64_t)c * L.pg.npc + a;
      for (int d = 0; d < 3; ++d) xyz[3 * i + d] = d < dim ? (f.crd[3 * c + d] + 0.5) / f.n : 0.0;
      field[i] = dim + a;  // coefficient a of the cell's pressure
    }
}

// ---------------------------------------------------------------- space-time multigrid (FP64)
static void level_vmult(Stmg& mg, StmgLevel& L, const double* x, double* y, cudaStream_t s) {
  if (L.kind == 1) return slab_vmult_pdisc(L, mg.tau, L.vmx.get(), x, y, s);
  slab_vmult(*L.A, *L.M, L.T.G, L.Q, mg.tau, L.n, L.vmx.get(), 0, x, y, s);
}

// Schwarz patches of level L: spatial blocks of A and M by probing, the space-time block
// G (x) M_pp + tau I (x) A_pp of every patch inverted on the host.
static void build_schwarz(Stmg& mg, StmgLevel& L, Budget* bud, cudaStream_t s) {
  const OpLevel& A = *L.A;
  const int64_t n = L.n;
  const int Q = L.Q;
  // Taylor--Hood: vertex stars, coloured by the cells they reach; P^disc: one cell per patch, coloured
  // by the cell coordinates modulo 3 (the cells reached from two patches of a colour -- each cell
  // and its neighbours -- do not meet)
  std::vector<std::vector<int32_t>> patches;
  std::vector<int32_t> colour;
  int ncol = 0;
  if (L.kind == 0) {
    patches = vertex_star_patches(A.forest, A.nu, A.np);
    ncol = colour_patches_for_probing(A.forest, A.nu, A.np, patches, colour);
  } else {
    const int dim = L.pg.dim, nm = L.pg.n;
    patches = pdisc_cell_patches(dim, nm, L.pg.k);
    colour.resize(patches.size());
    for (size_t c = 0; c < patches.size(); ++c) {
      const int cx = (int)(c % nm), cy = (int)((c / nm) % nm), cz = dim == 3 ? (int)(c / ((size_t)nm * nm)) : 0;
      colour[c] = (cx % 3) + 3 * (cy % 3) + 9 * (cz % 3);
    }
    ncol = dim == 3 ? 27 : 9;
  }
  std::vector<std::vector<int32_t>> members(ncol);
  for (size_t p = 0; p < patches.size(); ++p) members[colour[p]].push_back((int32_t)p);
  std::vector<std::pair<int, int>> cols;  // (colour, local index)
  for (int c = 0; c < ncol; ++c) {
    size_t len = 0;
    for (int32_t p : members[c]) len = std::max(len, patches[p].size());
    for (size_t m = 0; m < len; ++m) cols.push_back({c, (int)m});
  }
  std::vector<std::vector<double>> App(patches.size()), Mpp(patches.size());
  for (size_t p = 0; p < patches.size(); ++p) {
    App[p].assign(patches[p].size() * patches[p].size(), 0.0);
    Mpp[p].assign(patches[p].size() * patches[p].size(), 0.0);
  }
  const int B = 32;
  DevBuf X, YA, YM;
  X.alloc(bud, (size_t)n * B * 8);
  YA.alloc(bud, (size_t)n * B * 8);
  YM.alloc(bud, (size_t)n * B * 8);
  std::vector<double> Xh((size_t)n * B), Ya((size_t)n * B), Ym((size_t)n * B);
  for (size_t c0 = 0; c0 < cols.size(); c0 += B) {
    const int nb = (int)std::min<size_t>(B, cols.size() - c0);
    std::fill(Xh.begin(), Xh.begin() + (size_t)n * nb, 0.0);
    for (int j = 0; j < nb; ++j) {
      const int c = cols[c0 + j].first, m = cols[c0 + j].second;
      for (int32_t p : members[c])
        if ((size_t)m < patches[p].size()) Xh[(size_t)j * n + patches[p][m]] = 1.0;
    }
    MFNS_CUDA(cudaMemcpyAsync(X.get(), Xh.data(), (size_t)n * nb * 8, cudaMemcpyHostToDevice, s));
    if (L.kind == 0) {
      oplevel_vmult_cols(A, 0, X.get(), YA.get(), nb, s);
    } else {
      for (int j = 0; j < nb; ++j) pdisc_spatial(L, X.as<double>() + (int64_t)j * n, YA.as<double>() + (int64_t)j * n, s);
    }
    MFNS_CUDA(cudaMemsetAsync(YM.get(), 0, (size_t)n * nb * 8, s));
    op_apply_cols(L.M->L, 0, X.get(), YM.get(), nb, n, s);
    MFNS_CUDA(cudaMemcpyAsync(Ya.data(), YA.get(), (size_t)n * nb * 8, cudaMemcpyDeviceToHost, s));
    MFNS_CUDA(cudaMemcpyAsync(Ym.data(), YM.get(), (size_t)n * nb * 8, cudaMemcpyDeviceToHost, s));
    MFNS_CUDA(cudaStreamSynchronize(s));
    for (int j = 0; j < nb; ++j) {
      const int c = cols[c0 + j].first, m = cols[c0 + j].second;
      for (int32_t p : members[c]) {
        const size_t np = patches[p].size();
        if ((size_t)m >= np) continue;
        for (size_t a = 0; a < np; ++a) {
          App[p][a * np + m] = Ya[(size_t)j * n + patches[p][a]];
          Mpp[p][a * np + m] = Ym[(size_t)j * n + patches[p][a]];
        }
      }
    }
  }
  // space-time blocks, inverted; flattened tables
  std::vector<int64_t> p_ptr(1, 0), k_ptr(1, 0);
  std::vector<int32_t> p_idx;
  std::vector<double> kinv;
  int64_t max_patch = 0;
  for (size_t p = 0; p < patches.size(); ++p) {
    const int64_t m = (int64_t)patches[p].size(), mq = Q * m;
    std::vector<double> K((size_t)mq * mq, 0.0);
    for (int q = 0; q < Q; ++q)
      for (int j = 0; j < Q; ++j) {
        const double g = L.T.G[q * Q + j];
        for (int64_t a = 0; a < m; ++a)
          for (int64_t b = 0; b < m; ++b) {
            double v = g * Mpp[p][a * m + b];
            if (q == j) v += mg.tau * App[p][a * m + b];
            K[(size_t)(q * m + a) * mq + (j * m + b)] = v;
          }
      }
    if (!invert_dense_rel(K, mq, 1e-14)) throw Error(kErrUnsupported, "space-time multigrid: singular Schwarz patch");
    p_idx.insert(p_idx.end(), patches[p].begin(), patches[p].end());
    p_ptr.push_back((int64_t)p_idx.size());
    for (int64_t j = 0; j < mq; ++j)  // column by column
      for (int64_t i = 0; i < mq; ++i) kinv.push_back(K[(size_t)i * mq + j]);
    k_ptr.push_back((int64_t)kinv.size());
    max_patch = std::max(max_patch, m);
  }
  const size_t tk = mg.inv_prec == 1 ? 4 : 8;
  if ((size_t)Q * max_patch * tk > 48 * 1024) throw Error(kErrUnsupported, "space-time multigrid: patch too large");
  // occurrences of every spatial entry (patch results to add) and the weights 1 / multiplicity
  std::vector<int64_t> cnt(n + 1, 0);
  for (auto& pt : patches)
    for (int32_t i : pt) cnt[i + 1]++;
  for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  std::vector<int64_t> e_base(cnt[n]);
  std::vector<int32_t> e_np(cnt[n]);
  {
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (size_t p = 0; p < patches.size(); ++p)
      for (size_t a = 0; a < patches[p].size(); ++a) {
        const int32_t i = patches[p][a];
        e_base[fill[i]] = (int64_t)Q * p_ptr[p] + (int64_t)a;
        e_np[fill[i]] = (int32_t)patches[p].size();
        fill[i]++;
      }
  }
  std::vector<double> w(n, 0.0);
  for (int64_t i = 0; i < n; ++i)
    if (cnt[i + 1] > cnt[i]) w[i] = 1.0 / double(cnt[i + 1] - cnt[i]);
  L.n_patch = (int64_t)patches.size();
  L.max_patch = max_patch;
  L.p_ptr = upload(bud, p_ptr);
  L.p_idx = upload(bud, p_idx);
  L.k_ptr = upload(bud, k_ptr);
  L.inv_prec = mg.inv_prec;
  if (L.inv_prec == 1) {
    std::vector<float> k32(kinv.begin(), kinv.end());  // rounded to nearest
    L.kinv = upload(bud, k32);
  } else {
    L.kinv = upload(bud, kinv);
  }
  L.kinv_bytes = (int64_t)kinv.size() * (int64_t)tk;
  L.e_ptr = upload(bud, cnt);
  L.e_base = upload(bud, e_base);
  L.e_np = upload(bud, e_np);
  L.w = upload(bud, w);
  L.con = upload(bud, A.constrained_host);
  L.n_con = (int64_t)A.constrained_host.size();
  L.zloc.alloc(bud, (size_t)std::max<int64_t>(1, (int64_t)Q * p_ptr.back()) * 8);
}

// z = S r on level L (weighted additive Schwarz; constrained rows solved exactly)
static void schwarz(Stmg& mg, StmgLevel& L, const double* r, double* z, cudaStream_t s) {
  const int64_t total = (int64_t)L.Q * L.n;
  // one thread per row of the largest patch (whole warps, at most 1024): every patch in one pass
  const unsigned threads = (unsigned)std::min<int64_t>(1024, std::max<int64_t>(32, (L.Q * L.max_patch + 31) / 32 * 32));
  if (L.n_patch > 0 && L.inv_prec == 1)
    k_patch_solve<float><<<(unsigned)L.n_patch, threads, (size_t)L.Q * L.max_patch * 4, s>>>(
        r, L.zloc.as<double>(), L.p_ptr.as<int64_t>(), L.p_idx.as<int32_t>(), L.k_ptr.as<int64_t>(),
        L.kinv.as<float>(), L.Q, L.n);
  else if (L.n_patch > 0)
    k_patch_solve<double><<<(unsigned)L.n_patch, threads, (size_t)L.Q * L.max_patch * 8, s>>>(
        r, L.zloc.as<double>(), L.p_ptr.as<int64_t>(), L.p_idx.as<int32_t>(), L.k_ptr.as<int64_t>(),
        L.kinv.as<double>(), L.Q, L.n);
  k_patch_gather<<<stream_grid(total), 256, 0, s>>>(z, L.zloc.as<double>(), L.e_ptr.as<int64_t>(),
                                                     L.e_base.as<int64_t>(), L.e_np.as<int32_t>(), L.w.as<double>(),
                                                     L.Q, L.n);
  if (L.n_con > 0)
    k_constrained_scale<<<stream_grid((int64_t)L.Q * L.n_con), 256, 0, s>>>(z, r, L.con.as<int32_t>(), L.n_con, L.Q,
                                                                              L.n, 1.0 / mg.tau);
  MFNS_CUDA(cudaGetLastError());
}

static void level_prolongate_add(StmgLevel& F, StmgLevel& C, const double* xc, double* xf, cudaStream_t s) {
  if (F.tkind == 1) {
    k_time_prolong_add<<<stream_grid((int64_t)F.Q * F.n), 256, 0, s>>>(xf, xc, F.Pt, F.Q, F.Qc, F.n);
    MFNS_CUDA(cudaGetLastError());
    return;
  }
  for (int q = 0; q < F.Q; ++q) {
    const double* c = xc + (int64_t)q * C.n;
    double* f = xf + (int64_t)q * F.n;
    transfer_prolongate_add(*F.tv, *F.A, *C.A, 0, c, f, s);
    if (F.kind == 1)
      pdisc_prolongate_add(F.pg.dim, F.pg.n, F.pg.npc, C.pg.npc, F.ep_hstep, F.Ep.as<double>(), c + C.pg.n_main,
                           f + F.pg.n_main, s);
    else
      transfer_prolongate_add(*F.tp, *F.P, *C.P, 0, c + C.A->n_main_dofs, f + F.A->n_main_dofs, s);
  }
}

static void level_restrict(StmgLevel& F, StmgLevel& C, const double* rf, double* rc, cudaStream_t s) {
  if (F.tkind == 1) {
    k_time_restrict<<<stream_grid((int64_t)F.Qc * F.n), 256, 0, s>>>(rc, rf, F.Pt, F.Q, F.Qc, F.n);
    MFNS_CUDA(cudaGetLastError());
    return;
  }
  for (int q = 0; q < F.Q; ++q) {
    const double* f = rf + (int64_t)q * F.n;
    double* c = rc + (int64_t)q * C.n;
    // velocity first: on Taylor--Hood levels it clears the whole coarse vector of the stage; the
    // pressure block follows
    transfer_restrict(*F.tv, *F.A, *C.A, 0, f, c, s);
    if (F.kind == 1)
      pdisc_restrict(F.pg.dim, F.pg.n, F.pg.npc, C.pg.npc, F.ep_hstep, F.Ep.as<double>(), f + F.pg.n_main,
                     c + C.pg.n_main, s);
    else
      transfer_restrict(*F.tp, *F.P, *C.P, 0, f + F.A->n_main_dofs, c + C.A->n_main_dofs, s);
  }
}

static void coarse_solve(Stmg& mg, StmgLevel& C, cudaStream_t s) {
  // x = (K + sum_q E_q E_q^T)^{-1} P b, P the projection removing every stage's constant pressure:
  // the pseudo-inverse solution (K and K^T have the constant pressures as their null space)
  double* t = C.vt.as<double>();
  MFNS_CUDA(cudaMemcpyAsync(t, C.vb.get(), (size_t)C.Q * C.n * 8, cudaMemcpyDeviceToDevice, s));
  for (int q = 0; q < C.Q; ++q) {
    double* tq = t + (int64_t)q * C.n;
    sum_idx<double>(mg.scal.as<double>(), tq, mg.pres.as<int32_t>(), mg.n_pres, mg.part.as<double>(), s);
    sub_mean_idx<double>(tq, mg.pres.as<int32_t>(), mg.n_pres, mg.scal.as<double>(), s);
  }
  vgemv<double>(C.vx.as<double>(), mg.cinv.as<double>(), t, mg.cn, s);
}

static void stmg_smooth(Stmg& mg, StmgLevel& L, cudaStream_t s) {
  const int64_t total = (int64_t)L.Q * L.n;
  for (int it = 0; it < mg.nu_s; ++it) {
    level_vmult(mg, L, L.vx.as<double>(), L.vt.as<double>(), s);
    vsub<double>(L.vr.as<double>(), L.vb.as<double>(), L.vt.as<double>(), total, s);
    schwarz(mg, L, L.vr.as<double>(), L.vz.as<double>(), s);
    vaxpy<double>(L.vx.as<double>(), mg.omega, L.vz.as<double>(), total, s);
  }
}

// L.vx = V-cycle(L.vb) from a zero start (Section 4: nu_s damped Schwarz steps before and after the
// coarse correction, a direct solve on the coarsest level)
static void stmg_cycle(Stmg& mg, size_t l, cudaStream_t s) {
  StmgLevel& L = *mg.lv[l];
  if (l + 1 == mg.lv.size()) return coarse_solve(mg, L, s);
  StmgLevel& C = *mg.lv[l + 1];
  const int64_t total = (int64_t)L.Q * L.n;
  vzero<double>(L.vx.as<double>(), total, s);
  stmg_smooth(mg, L, s);
  level_vmult(mg, L, L.vx.as<double>(), L.vt.as<double>(), s);
  vsub<double>(L.vr.as<double>(), L.vb.as<double>(), L.vt.as<double>(), total, s);
  level_restrict(L, C, L.vr.as<double>(), C.vb.as<double>(), s);
  stmg_cycle(mg, l + 1, s);
  level_prolongate_add(L, C, C.vx.as<double>(), L.vx.as<double>(), s);
  stmg_smooth(mg, L, s);
}

// every stage's constant pressure removed from a finest-level vector (its component along the
// null space of K and K^T)
static void project_constants(Stmg& mg, double* v, cudaStream_t s) {
  StmgLevel& L = *mg.lv[0];
  if (mg.n_pres0 == 0) return;
  for (int q = 0; q < L.Q; ++q) {
    double* vq = v + (int64_t)q * L.n;
    sum_idx<double>(mg.scal.as<double>(), vq, mg.pres0.as<int32_t>(), mg.n_pres0, mg.part.as<double>(), s);
    sub_mean_idx<double>(vq, mg.pres0.as<int32_t>(), mg.n_pres0, mg.scal.as<double>(), s);
  }
}

// L.vx = V-cycle(L.vb) on the finest level, replayed from a CUDA graph captured on first use (the
// cycle has no host synchronisation and works on the levels' own vectors)
static void stmg_vcycle(Stmg& mg, cudaStream_t s) {
  if (!mg.vc_graph) {
    if (!mg.cap_stream) MFNS_CUDA(cudaStreamCreateWithFlags(&mg.cap_stream, cudaStreamNonBlocking));
    MFNS_CUDA(cudaStreamBeginCapture(mg.cap_stream, cudaStreamCaptureModeThreadLocal));
    stmg_cycle(mg, 0, mg.cap_stream);
    cudaGraph_t g;
    MFNS_CUDA(cudaStreamEndCapture(mg.cap_stream, &g));
    const cudaError_t e = cudaGraphInstantiate(&mg.vc_graph, g, 0);
    cudaGraphDestroy(g);
    MFNS_CUDA(e);
  }
  MFNS_CUDA(cudaGraphLaunch(mg.vc_graph, s));
}

static double dev_dot(Stmg& mg, const double* a, const double* b, int64_t n, cudaStream_t s) {
  dot<double>(mg.scal.as<double>() + 1, a, b, n, mg.part.as<double>(), s);
  double h;
  MFNS_CUDA(cudaMemcpyAsync(&h, mg.scal.as<double>() + 1, 8, cudaMemcpyDeviceToHost, s));
  MFNS_CUDA(cudaStreamSynchronize(s));
  return h;
}

// FGMRES(m) in FP64 on the slab operator, right-preconditioned by one space-time V-cycle
// (classical Gram--Schmidt applied twice, Givens rotations); the constant pressures of every
// stage are removed from b and from every preconditioned vector, so x is the solution without
// them.  Returns the iterations; relres = ||b - K x|| / ||b|| of the projected b.
static int stmg_fgmres(mfns_spacetime& st, const double* b, double* x, double tol, int maxit, double* relres,
                       bool* converged, cudaStream_t s) {
  Stmg& mg = *st.mg;
  StmgLevel& L = *mg.lv[0];
  const int64_t N = (int64_t)L.Q * L.n;
  const int m = mg.restart;
  if (m + 1 > kMaxDots) throw Error(kErrUnsupported, "space-time FGMRES restart beyond the multi-dot width");
  if (!mg.V.get()) {
    Budget* bud = st.bud;
    mg.V.alloc(bud, (size_t)(m + 1) * N * 8);
    mg.Z.alloc(bud, (size_t)m * N * 8);
    mg.w.alloc(bud, (size_t)N * 8);
    mg.bp.alloc(bud, (size_t)N * 8);
    std::vector<const double*> pv(m + 1);
    for (int i = 0; i <= m; ++i) pv[i] = mg.V.as<double>() + (int64_t)i * N;
    mg.ptrV = upload(bud, pv);
    mg.hvec.alloc(bud, (size_t)(2 * kMaxDots + 1) * 8);
    MFNS_CUDA(cudaMallocHost(&mg.hh_host, (size_t)(2 * kMaxDots + 1) * 8));
  }
  double* V = mg.V.as<double>();
  double* Z = mg.Z.as<double>();
  double* w = mg.w.as<double>();
  double* bp = mg.bp.as<double>();
  MFNS_CUDA(cudaMemcpyAsync(bp, b, (size_t)N * 8, cudaMemcpyDeviceToDevice, s));
  project_constants(mg, bp, s);
  vzero<double>(x, N, s);
  const double bnorm = std::sqrt(dev_dot(mg, bp, bp, N, s));
  *converged = false;
  if (bnorm == 0.0) {
    *relres = 0.0;
    *converged = true;
    return 0;
  }
  int it = 0;
  double beta = bnorm;
  MFNS_CUDA(cudaMemcpyAsync(V, bp, (size_t)N * 8, cudaMemcpyDeviceToDevice, s));  // r = b (x = 0)
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m), h(m + 1), h2(m + 1);
  while (true) {
    if (beta <= tol * bnorm) {
      *converged = true;
      break;
    }
    if (it >= maxit) break;
    vscale<double>(V, 1.0 / beta, N, s);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j_done = 0;
    for (int j = 0; j < m && it < maxit; ++j) {
      double* Vj = V + (int64_t)j * N;
      double* Zj = Z + (int64_t)j * N;
      MFNS_CUDA(cudaMemcpyAsync(L.vb.get(), Vj, (size_t)N * 8, cudaMemcpyDeviceToDevice, s));
      stmg_vcycle(mg, s);
      MFNS_CUDA(cudaMemcpyAsync(Zj, L.vx.get(), (size_t)N * 8, cudaMemcpyDeviceToDevice, s));
      project_constants(mg, Zj, s);
      level_vmult(mg, L, Zj, w, s);
      // classical Gram--Schmidt twice: all coefficients of a pass in one multi-dot, the update in
      // one multi-axpy, and one host round trip per iteration for both passes and the norm
      const double** Vp = (const double**)mg.ptrV.as<const double*>();
      double* hd = mg.hvec.as<double>();
      multidot(hd, nullptr, w, j + 1, N, mg.part.as<double>(), Vp, s);
      multi_axpy(w, Vp, hd, j + 1, N, s);
      multidot(hd + kMaxDots, nullptr, w, j + 1, N, mg.part.as<double>(), Vp, s);
      multi_axpy(w, Vp, hd + kMaxDots, j + 1, N, s);
      dot<double>(hd + 2 * kMaxDots, w, w, N, mg.part.as<double>(), s);
      MFNS_CUDA(cudaMemcpyAsync(mg.hh_host, hd, (size_t)(2 * kMaxDots + 1) * 8, cudaMemcpyDeviceToHost, s));
      MFNS_CUDA(cudaStreamSynchronize(s));
      for (int i = 0; i <= j; ++i) {
        h[i] = mg.hh_host[i];
        h2[i] = mg.hh_host[kMaxDots + i];
      }
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h[i] + h2[i];
      const double hn = std::sqrt(std::max(mg.hh_host[2 * kMaxDots], 0.0));
      H[(size_t)(j + 1) * m + j] = hn;
      if (hn > 0.0) {
        MFNS_CUDA(cudaMemcpyAsync(V + (int64_t)(j + 1) * N, w, (size_t)N * 8, cudaMemcpyDeviceToDevice, s));
        vscale<double>(V + (int64_t)(j + 1) * N, 1.0 / hn, N, s);
      }
      for (int i = 0; i < j; ++i) {  // earlier rotations
        const double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      const double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
      const double rr = std::hypot(a, c);
      cs[j] = rr > 0.0 ? a / rr : 1.0;
      sn[j] = rr > 0.0 ? c / rr : 0.0;
      H[(size_t)j * m + j] = rr;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++it;
      j_done = j + 1;
      if (std::fabs(g[j + 1]) <= tol * bnorm || hn == 0.0) break;
    }
    for (int i = j_done - 1; i >= 0; --i) {  // H y = g (upper triangular)
      double v = g[i];
      for (int k = i + 1; k < j_done; ++k) v -= H[(size_t)i * m + k] * y[k];
      y[i] = v / H[(size_t)i * m + i];
    }
    for (int i = 0; i < j_done; ++i) vaxpy<double>(x, y[i], Z + (int64_t)i * N, N, s);
    level_vmult(mg, L, x, w, s);  // true residual, into the first basis vector
    vsub<double>(V, bp, w, N, s);
    beta = std::sqrt(dev_dot(mg, V, V, N, s));
  }
  *relres = beta / bnorm;
  return it;
}

static void build_stmg(mfns_spacetime& st, int nu_s, double omega, int coarse_n, int inv_prec, cudaStream_t s) {
  const bool pd = st.top != nullptr;  // P^disc slab (else Taylor--Hood on st.problem)
  Budget* bud = st.bud;
  const OpLevel& A0 = pd ? *st.top->A : *st.problem->p->system;
  const Physics phys = pd ? Physics() : st.problem->p->phys;
  const int k0 = pd ? st.top->k : A0.k;
  if (!A0.forest.uniform()) throw Error(kErrUnsupported, "space-time multigrid: uniform meshes only");
  if (nu_s < 1 || !(omega > 0.0) || coarse_n < 2)
    throw Error(kErrArg, "space-time multigrid: nu_s >= 1, omega > 0 and coarse_n >= 2");
  std::vector<Forest> fs{A0.forest};
  while (forest_can_coarsen(fs.back(), coarse_n)) {
    if (pd && fs.back().n % 2 != 0)
      throw Error(kErrUnsupported, "space-time multigrid with P^disc: nested coarsening (even cell counts) only");
    fs.push_back(forest_coarsen(fs.back()));
  }
  // temporal steps on the coarsest mesh, unless (vertex stars) a star there holds every cell
  const bool time_steps = pd || !vertex_star_covers_all(fs.back());
  const std::vector<StLevelSpec> seq = stmg_sequence(k0, st.r, (int)fs.size(), time_steps);
  auto mg = std::make_unique<Stmg>();
  mg->nu_s = nu_s;
  mg->inv_prec = inv_prec;
  mg->omega = omega;
  mg->tau = st.tau;
  for (const StLevelSpec& sp : seq) {
    auto L = std::make_unique<StmgLevel>();
    L->k = sp.k;
    L->r = sp.r;
    L->Q = sp.r + 1;
    std::string err;
    if (!temporal_matrices(sp.r, L->T, &err)) throw Error(kErrArg, err);
    if (pd) {
      build_pdisc_level(*L, fs[sp.forest], sp.k, st.nu, bud);
    } else {
      L->A = std::make_unique<OpLevel>();
      build_oplevel(*L->A, fs[sp.forest], OP_STOKES, sp.k, phys, bud);
      L->M = std::make_unique<OpLevel>();
      build_oplevel(*L->M, fs[sp.forest], OP_VMASS, sp.k, phys, bud);
      L->n = L->A->n_dofs;
    }
    const size_t qn = (size_t)L->Q * L->n * 8;
    for (DevBuf* v : {&L->vx, &L->vb, &L->vr, &L->vt, &L->vz, &L->vmx}) {
      v->alloc(bud, qn);
      MFNS_CUDA(cudaMemsetAsync(v->get(), 0, qn, s));
    }
    mg->lv.push_back(std::move(L));
  }
  for (size_t l = 0; l + 1 < mg->lv.size(); ++l) {
    StmgLevel& F = *mg->lv[l];
    StmgLevel& C = *mg->lv[l + 1];
    if (F.r != C.r) {
      F.tkind = 1;
      F.Qc = C.Q;
      const std::vector<double> Pt = time_prolongation(C.r, F.r);
      for (int q = 0; q < F.Q; ++q)
        for (int j = 0; j < C.Q; ++j) F.Pt.g[q][j] = Pt[(size_t)q * C.Q + j];
    } else {
      F.tkind = 2;
      F.tv = std::make_unique<Transfer>();
      build_transfer(*F.tv, *F.A, *C.A, bud);
      if (pd) {
        const int dim = F.pg.dim;
        if (F.pg.n == C.pg.n) {  // degree step on one mesh
          F.ep_hstep = false;
          F.Ep = upload(bud, pdisc_degree_embedding(dim, F.k - 1, C.k - 1));
        } else if (F.pg.n == 2 * C.pg.n && F.k == C.k) {  // nested h-step
          F.ep_hstep = true;
          std::vector<double> E;
          for (int child = 0; child < (1 << dim); ++child) {
            const std::vector<double> e = pdisc_child_embedding(dim, F.k - 1, child);
            E.insert(E.end(), e.begin(), e.end());
          }
          F.Ep = upload(bud, E);
        } else {
          throw Error(kErrUnsupported, "P^disc transfer: nested h-steps or degree steps only");
        }
      } else {
        for (StmgLevel* X : {&F, &C})
          if (!X->P) {
            X->P = std::make_unique<OpLevel>();
            build_oplevel(*X->P, X->A->forest, OP_PMASS, X->k - 1, phys, bud);
          }
        F.tp = std::make_unique<Transfer>();
        build_transfer(*F.tp, *F.P, *C.P, bud);
      }
    }
    build_schwarz(*mg, F, bud, s);
  }
  // free pressure entries of a level: their constant (one per stage) is the null space of K
  auto pressure_entries = [](const StmgLevel& L) {
    if (L.kind == 0) return L.A->pres_host;
    std::vector<int32_t> e;
    const int64_t cells = (L.n - L.pg.n_main) / L.pg.npc;
    for (int64_t c = 0; c < cells; ++c) e.push_back((int32_t)(L.pg.n_main + c * L.pg.npc));  // constant monomial
    return e;
  };
  // coarsest level: dense operator by unit vectors, plus the constant pressures of every stage
  StmgLevel& C = *mg->lv.back();
  const int64_t N = (int64_t)C.Q * C.n;
  if (N > 8192) throw Error(kErrUnsupported, "space-time multigrid: coarsest level too large for a dense solve");
  std::vector<double> K((size_t)N * N), col(N);
  for (int64_t j = 0; j < N; ++j) {
    MFNS_CUDA(cudaMemsetAsync(C.vz.get(), 0, (size_t)N * 8, s));
    const double one = 1.0;
    MFNS_CUDA(cudaMemcpyAsync(C.vz.as<double>() + j, &one, 8, cudaMemcpyHostToDevice, s));
    level_vmult(*mg, C, C.vz.as<double>(), C.vt.as<double>(), s);
    MFNS_CUDA(cudaMemcpyAsync(col.data(), C.vt.get(), (size_t)N * 8, cudaMemcpyDeviceToHost, s));
    MFNS_CUDA(cudaStreamSynchronize(s));
    for (int64_t i = 0; i < N; ++i) K[(size_t)i * N + j] = col[i];
  }
  const std::vector<int32_t> pres = pressure_entries(C);
  if (!pres.empty()) {
    const double v = 1.0 / double(pres.size());
    for (int q = 0; q < C.Q; ++q)
      for (int32_t a : pres)
        for (int32_t b : pres) K[(size_t)(q * C.n + a) * N + (q * C.n + b)] += v;
  }
  if (!invert_dense_rel(K, N, 1e-15)) throw Error(kErrArg, "space-time multigrid: singular coarse matrix");
  mg->cinv = upload(bud, K);
  mg->cn = N;
  mg->pres = upload(bud, pres);
  mg->n_pres = (int64_t)pres.size();
  mg->part.alloc(bud, (size_t)kRedBlocks * kMaxDots * 8);
  mg->scal.alloc(bud, 64);
  const std::vector<int32_t> pres0 = pressure_entries(*mg->lv[0]);
  mg->pres0 = upload(bud, pres0);
  mg->n_pres0 = (int64_t)pres0.size();
  MFNS_CUDA(cudaStreamSynchronize(s));
  st.mg = std::move(mg);
}

}  // namespace mfns

// a vector argument whose length differs from the one the call expects
static int st_len_fail(const char* what, int64_t got, int64_t want) {
  return mfns::capi_fail(mfns::kErrArg, (std::string(what) + " has " + std::to_string(got) + " entries, expected " +
                                         std::to_string(want)).c_str());
}

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
    st->ctx = p->ctx;
    st->bud = P.bud;
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

extern "C" int mfns_spacetime_vmult(mfns_spacetime* st, int prec, const void* x, void* y, int64_t n, void* stream) {
  using namespace mfns;
  try {
    (void)cudaGetLastError();
    if (!st || !x || !y || x == y || (prec != 0 && prec != 1)) return capi_fail(kErrArg, "bad arguments");
    if (n != (int64_t)st->Q * st->n) return st_len_fail("x/y", n, (int64_t)st->Q * st->n);
    MFNS_CUDA(cudaSetDevice(st->ctx->device));
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

#define ST_BEGIN \
  using namespace mfns; \
  try {                 \
    (void)cudaGetLastError();
#define ST_END                                                  \
  }                                                             \
  catch (const Error& e) { return capi_fail(e.code, e.what()); } \
  catch (const std::exception& e) { return capi_fail(kErrArg, e.what()); } \
  return MFNS_OK;

extern "C" int mfns_spacetime_mg_build(mfns_spacetime* st, int nu_s, double omega, int coarse_n, int inverse_precision,
                                       void* stream) {
  ST_BEGIN
  if (!st || (inverse_precision != 0 && inverse_precision != 1)) return capi_fail(kErrArg, "bad arguments");
  MFNS_CUDA(cudaSetDevice(st->ctx->device));
  st->mg.reset();
  build_stmg(*st, nu_s, omega, coarse_n, inverse_precision, reinterpret_cast<cudaStream_t>(stream));
  ST_END
}

extern "C" int mfns_spacetime_mg_level(const mfns_spacetime* st, int level, int* n_levels, int* k, int* r,
                                       int64_t* n_stage) {
  if (!st || !st->mg) return mfns::capi_fail(mfns::kErrArg, "no space-time multigrid (mfns_spacetime_mg_build)");
  const int nl = (int)st->mg->lv.size();
  if (n_levels) *n_levels = nl;
  if (level < 0 || level >= nl) return level == -1 ? MFNS_OK : mfns::capi_fail(mfns::kErrArg, "level out of range");
  const mfns::StmgLevel& L = *st->mg->lv[level];
  if (k) *k = L.k;
  if (r) *r = L.r;
  if (n_stage) *n_stage = L.n;
  return MFNS_OK;
}

extern "C" int mfns_spacetime_mg_support_points(const mfns_spacetime* st, int level, double* xyz_host, int* field_host) {
  ST_BEGIN
  if (!st || !st->mg || level < 0 || level >= (int)st->mg->lv.size() || !xyz_host || !field_host)
    return capi_fail(kErrArg, "bad arguments");
  level_support(*st->mg->lv[level], xyz_host, field_host);
  ST_END
}

extern "C" int mfns_spacetime_mg_apply(mfns_spacetime* st, int level, int what, const void* in, int64_t n_in,
                                       void* out, int64_t n_out, void* stream) {
  ST_BEGIN
  if (!st || !st->mg || !in || !out || in == out || level < 0 || level >= (int)st->mg->lv.size())
    return capi_fail(kErrArg, "bad arguments");
  Stmg& mg = *st->mg;
  StmgLevel& L = *mg.lv[level];
  const bool has_coarse = level + 1 < (int)mg.lv.size();
  {
    const int64_t nl = (int64_t)L.Q * L.n;
    const int64_t nc = has_coarse ? (int64_t)mg.lv[level + 1]->Q * mg.lv[level + 1]->n : 0;
    const int64_t want_in = what == 2 ? nc : nl, want_out = what == 3 ? nc : nl;
    if ((what == 2 || what == 3) && !has_coarse)
      return capi_fail(kErrArg, "the coarsest level has no coarser level");
    if (n_in != want_in) return st_len_fail("in", n_in, want_in);
    if (n_out != want_out) return st_len_fail("out", n_out, want_out);
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  MFNS_CUDA(cudaSetDevice(st->ctx->device));
  switch (what) {
    case 0: level_vmult(mg, L, (const double*)in, (double*)out, s); break;
    case 1:
      if (!has_coarse) return capi_fail(kErrArg, "the coarsest level has no smoother");
      schwarz(mg, L, (const double*)in, (double*)out, s);
      break;
    case 2:
      if (!has_coarse) return capi_fail(kErrArg, "the coarsest level has no coarser level");
      level_prolongate_add(L, *mg.lv[level + 1], (const double*)in, (double*)out, s);
      break;
    case 3:
      if (!has_coarse) return capi_fail(kErrArg, "the coarsest level has no coarser level");
      level_restrict(L, *mg.lv[level + 1], (const double*)in, (double*)out, s);
      break;
    default: return capi_fail(kErrArg, "what: 0 operator, 1 Schwarz, 2 prolongate-add, 3 restrict");
  }
  ST_END
}

extern "C" int mfns_spacetime_vcycle(mfns_spacetime* st, const void* b, void* x, int64_t n, void* stream) {
  ST_BEGIN
  if (!st || !st->mg || !b || !x || b == x) return capi_fail(kErrArg, "bad arguments");
  Stmg& mg = *st->mg;
  StmgLevel& L = *mg.lv[0];
  if (n != (int64_t)L.Q * L.n) return st_len_fail("b/x", n, (int64_t)L.Q * L.n);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  MFNS_CUDA(cudaSetDevice(st->ctx->device));
  const size_t bytes = (size_t)L.Q * L.n * 8;
  MFNS_CUDA(cudaMemcpyAsync(L.vb.get(), b, bytes, cudaMemcpyDeviceToDevice, s));
  stmg_vcycle(mg, s);
  MFNS_CUDA(cudaMemcpyAsync(x, L.vx.get(), bytes, cudaMemcpyDeviceToDevice, s));
  ST_END
}

extern "C" int mfns_spacetime_solve(mfns_spacetime* st, const void* b, void* x, int64_t n, double tol, int maxit,
                                    int* iterations, double* relres, int* converged, void* stream) {
  ST_BEGIN
  if (!st || !st->mg || !b || !x || b == x || !(tol > 0.0) || maxit < 1) return capi_fail(kErrArg, "bad arguments");
  if (n != (int64_t)st->Q * st->n) return st_len_fail("b/x", n, (int64_t)st->Q * st->n);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  MFNS_CUDA(cudaSetDevice(st->ctx->device));
  double rel = 0.0;
  bool conv = false;
  const int its = stmg_fgmres(*st, (const double*)b, (double*)x, tol, maxit, &rel, &conv, s);
  if (iterations) *iterations = its;
  if (relres) *relres = rel;
  if (converged) *converged = conv ? 1 : 0;
  if (!conv) return capi_fail(MFNS_ERR_NOT_CONVERGED, "space-time FGMRES did not reach the tolerance");
  ST_END
}

extern "C" int mfns_spacetime_create_pdisc(mfns_ctx* ctx, const mfns_mesh* mesh, int k, double nu, int r, double tau,
                                           mfns_spacetime** out) {
  ST_BEGIN
  if (!ctx || !mesh || !out || !(tau > 0.0) || !(nu > 0.0)) return capi_fail(kErrArg, "bad arguments");
  *out = nullptr;
  if (r < 0 || r + 1 > kMaxStages) return capi_fail(kErrArg, "temporal degree must lie in 0..7");
  MFNS_CUDA(cudaSetDevice(ctx->device));
  auto st = std::make_unique<mfns_spacetime>();
  st->ctx = ctx;
  st->bud = &ctx->budget;
  st->nu = nu;
  st->r = r;
  st->Q = r + 1;
  st->tau = tau;
  std::string err;
  if (!temporal_matrices(r, st->T, &err)) return capi_fail(kErrArg, err.c_str());
  auto L = std::make_unique<StmgLevel>();
  L->k = k;
  L->r = r;
  L->Q = r + 1;
  L->T = st->T;
  build_pdisc_level(*L, mesh->forest, k, nu, st->bud);
  L->vmx.alloc(st->bud, (size_t)L->Q * L->n * 8);
  st->n = L->n;
  st->top = std::move(L);
  *out = st.release();
  ST_END
}

extern "C" int mfns_spacetime_support_points(const mfns_spacetime* st, double* xyz_host, int* field_host) {
  ST_BEGIN
  if (!st || !xyz_host || !field_host) return capi_fail(kErrArg, "bad arguments");
  if (st->top)
    level_support(*st->top, xyz_host, field_host);
  else
    oplevel_support(*st->problem->p->system, xyz_host, field_host);
  ST_END
}

extern "C" int mfns_spacetime_mg_smoother_bytes(const mfns_spacetime* st, int level, int64_t* inverse_bytes,
                                                int64_t* n_patches) {
  if (!st || !st->mg || level < 0 || level >= (int)st->mg->lv.size())
    return mfns::capi_fail(mfns::kErrArg, "bad arguments");
  const mfns::StmgLevel& L = *st->mg->lv[level];
  if (inverse_bytes) *inverse_bytes = L.kinv_bytes;
  if (n_patches) *n_patches = L.n_patch;
  return MFNS_OK;
}
