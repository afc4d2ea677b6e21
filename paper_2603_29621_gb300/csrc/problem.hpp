// Problem = operator + global-coarsening hierarchy + smoothers + coarse solver
// + workspaces, all resident on one device.
#pragma once
#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "common.hpp"
#include "hp_space.hpp"
#include "mesh.hpp"
#include "opkind.hpp"
#include "op_launch.hpp"

namespace mfns {

struct HpData;
struct HpTransfer;

struct Physics {
  double nu = 1.0, dt = 0.0, div_sign = -1.0;
  int terms = 127;
  bool precompute_frozen = true;  // stabilised NS: store the frozen state's point values
};

// One operator on one mesh (one multigrid level, the system operator or the pressure mass).
struct OpLevel {
  int op = 0, dim = 3, k = 1, NU = 1;
  Forest forest;
  NodeSpace nu, np;                     // main nodes, Taylor--Hood pressure nodes
  int64_t n_dofs = 0, n_main_dofs = 0;  // vector length, main-node block length
  OpLaunch L;
  std::vector<int32_t> perm;            // colour-sorted position -> forest cell id
  DevBuf cell_u, cell_p, cell_f, mask, hcell[2], frozen[2], fq[2];
  DevBuf gexp[2];                       // stabilised NS: explicit BDF field g (allocated on first use)
  DevBuf lastc;                         // per main node: last colour touching it (fused epilogues)
  std::vector<int32_t> constrained_host;
  DevBuf constrained;                   // identity rows
  DevBuf keep_mask;                     // uniform meshes: bitmask of the identity rows (see oplevel_vmult)
  DevBuf defer[2];                      // small uniform 3D stabilised levels: per-cell contributions (FP64 / FP32)
  int64_t n_hang = 0;
  DevBuf hang_dof, hang_ptr, hang_src, hang_w[2];
  std::vector<int32_t> pres_host;
  DevBuf pres;                          // free pressure entries (constant-pressure null space)
  int64_t n_pres = 0;
  // transfer support: true fine node per slot with flags (bit 31 skip, bit 30 boundary)
  DevBuf tnodes, tpnodes;
  // smoother
  DevBuf dinv[2];
  double lmax = 0.0;
  std::unique_ptr<KernelTimer> timer = std::make_unique<KernelTimer>();
  // hp level (cells of several degrees): operator, diagonal and support points come from here
  std::unique_ptr<HpData> hp;
  size_t bytes() const;
};

// hp levels (Section 3).  The cells of one degree form a group applied by that degree's cell
// kernel with their own node ids (no constraint masks).  The constraints of h- and
// p-adaptivity are applied around the cell kernels: the input's constrained entries are first
// completed from their masters (distribute), the products on constrained entries are then folded
// into the masters with the same weights (the transpose), and constrained rows are identity rows.
struct HpGroup {
  int k = 1;
  OpLaunch L;
  std::vector<int32_t> cells;           // forest cell ids, colour order
  DevBuf cell_u, cell_p, mask, hcell[2];
  std::unique_ptr<KernelTimer> timer = std::make_unique<KernelTimer>();
};
struct HpData {
  HpSpace space;                        // the main field's nodes (velocity, or the scalar field)
  HpSpace pspace;                       // Taylor--Hood: the pressure nodes (degrees k - 1)
  std::vector<std::unique_ptr<HpGroup>> groups;
  DevBuf tmp[2];                        // distributed input
  DevBuf diag[2];                       // exact diagonal of C^T K C (identity rows 1), FP64 / FP32
  // transpose of the constraints: for master dof ct_master[i], slaves ct_slave[j] with weights
  // ct_w[j], j in [ct_ptr[i], ct_ptr[i+1])
  DevBuf ct_master, ct_ptr, ct_slave, ct_w[2];
  int64_t n_ct = 0;
  // Section 3's blended smoother (built on request): additive Schwarz blocks on the combined faces,
  // point Jacobi on the entries in no block
  struct Asm {
    int64_t n_block = 0, max_block = 0;
    DevBuf b_ptr, b_idx, k_ptr, kinv[2];  // blocks (entries), inverses of A_BB (row-major, FP64 / FP32)
    DevBuf e_ptr, e_base;                 // per entry: the block results to add (indices into zloc)
    DevBuf jdinv[2];                      // 1 / A_ii on entries in no block, 0 on block entries
    DevBuf zloc[2];                       // block results
  };
  std::unique_ptr<Asm> asm_;
};
// op: OP_STOKES_A (vector Laplacian, degree per cell), OP_STOKES (Taylor--Hood: velocity degree per
// cell, pressure one lower) or OP_PMASS (scalar mass, degree per cell)
void build_hp_oplevel(OpLevel& lv, const Forest& f, const std::vector<int32_t>& degree, const Physics& ph,
                      Budget* bud, int op = OP_STOKES_A);
void hp_vmult(const OpLevel& lv, int prec, const void* src, void* dst, cudaStream_t s);
void hp_diag(const OpLevel& lv, int prec, void* diag, cudaStream_t s);
// y[m] += sum of w * y[slave] over the slaves of every master m (hp levels)
void hp_condense(const OpLevel& lv, int prec, void* y, cudaStream_t s);
// x[slave] = sum of w * x[master] for every constrained (non-Dirichlet) entry
void hp_distribute(const OpLevel& lv, int prec, void* x, cudaStream_t s);
// the blended smoother's blocks of an hp level of the vector Laplacian (lv.dinv[0] must hold the
// diagonal inverse); no-op on a level without combined faces
void build_hp_asm(OpLevel& lv, Budget* bud, cudaStream_t s);
// z = P^{-1} r of the blended smoother (requires lv.hp->asm_)
void hp_asm_apply(const OpLevel& lv, int prec, const void* r, void* z, cudaStream_t s);

// edge_dirichlet (level forests of local smoothing): nodes on the refinement edge are constrained
// like Dirichlet nodes (identity rows, zero in the operator's input)
void build_oplevel(OpLevel& lv, const Forest& f, int op, int k, const Physics& ph, Budget* bud,
                   bool edge_dirichlet = false);
void oplevel_vmult(const OpLevel& lv, int prec, const void* src, void* dst, cudaStream_t s);
void oplevel_diag(const OpLevel& lv, int prec, void* diag, cudaStream_t s);
// One smoothing step with the update fused into the operator application (t: scratch):
// d = c1 d + c2 dinv (b - A x), xout = x + d  (xout must not alias x)
void oplevel_smooth_step(const OpLevel& lv, int prec, const void* x, void* xout, void* d, const void* b,
                         const void* dinv, void* t, double c1, double c2, cudaStream_t s);
// r = b - A x with the subtraction fused into the operator application (t: scratch)
void oplevel_residual_fused(const OpLevel& lv, int prec, const void* x, const void* b, void* r, void* t,
                            cudaStream_t s);
// Y[:, j] = A X[:, j] for ncols columns of length n_dofs (column-major blocks)
void oplevel_vmult_cols(const OpLevel& lv, int prec, const void* X, void* Y, int ncols, cudaStream_t s);
void oplevel_distribute(const OpLevel& lv, int prec, void* x, cudaStream_t s);
void oplevel_support(const OpLevel& lv, double* xyz, int* field);

// Separable transfer between uniform meshes: 1D stencils P1 (fine x coarse) and P1^T per axis.
struct SepTransfer {
  int dim = 3, ncomp = 1, nvel = 0;
  int64_t Mf = 0, Mc = 0;               // 1D node counts
  DevBuf p_ptr, p_idx, p_w[2];          // rows = fine nodes
  DevBuf r_ptr, r_idx, r_w[2];          // rows = coarse nodes
  DevBuf i_ptr, i_idx, i_w;             // fine-to-coarse interpolation, rows = coarse nodes (fp64)
  DevBuf tmp1[2], tmp2[2];              // intermediate grids per precision
};

// Transfer between fine level (index l) and coarse level (l+1), Eq. 4.
struct Transfer {
  bool separable = false;
  SepTransfer sep;
  bool hkind = true;                    // true: h (children), false: p (same cells)
  int dim = 3, kf = 1, kc = 1, ncomp = 1;
  int64_t n_coarse_cells = 0;
  std::vector<int32_t> color_ptr;       // colours of the coarse level
  DevBuf child_cell;                    // n_coarse * 2^dim fine cell ids (-1: none)
  DevBuf child_code;                    // per child: child bits, or 8 = same cell
  std::vector<double> E;                // h: P_half[2][NF][NC]; p: S[NF][NC]
  std::vector<double> Pc;               // coarse hanging interpolation P[2][NC][NC]
  DevBuf own_c;                         // state interpolation: owner flag per coarse (cell, slot)
  std::unique_ptr<HpTransfer> hp;       // p-step from an hp level (groups of degree pairs)
};
// p-transfer from an hp level to the level with every degree lowered by one (hp or uniform)
void build_hp_transfer(Transfer& t, const OpLevel& fine, const OpLevel& coarse, Budget* bud);
// one (fine degree, coarse degree) pair of an hp p-transfer: the same cells on both levels
struct HpTGroup {
  Transfer t;                           // degree change (or identity) per cell, coarse colours
  OpLevel fine_view, coarse_view;       // fine owner table (tnodes); coarse cell table and masks
};
struct HpTransfer {
  std::vector<std::unique_ptr<HpTGroup>> groups;
};
// allow_unrefined (local smoothing): coarse cells without children in the fine level are skipped
void build_transfer(Transfer& t, const OpLevel& fine, const OpLevel& coarse, Budget* bud,
                    bool allow_unrefined = false);
bool build_separable(SepTransfer& t, const OpLevel& fine, const OpLevel& coarse, Budget* bud);
void sep_restrict(const SepTransfer& t, int prec, const void* fine, void* coarse, cudaStream_t s);
// coarse = the fine FE function evaluated at the coarse nodes (all components, no masking; fp64)
void sep_interpolate(const SepTransfer& t, const double* fine, double* coarse, cudaStream_t s);
// the same for any transfer (separable passes, or per coarse cell through its children); the fine
// values must have consistent hanging-node entries; coarse hanging entries are left to the caller
void cell_interpolate(Transfer& t, const OpLevel& fine, const OpLevel& coarse, const double* uf, double* uc,
                      Budget* bud, cudaStream_t s);
void sep_prolongate_add(const SepTransfer& t, int prec, const void* coarse, void* fine, cudaStream_t s);
void transfer_prolongate_add(const Transfer& t, const OpLevel& fine, const OpLevel& coarse, int prec,
                             const void* xc, void* xf, cudaStream_t s);
void transfer_restrict(const Transfer& t, const OpLevel& fine, const OpLevel& coarse, int prec,
                       const void* rf, void* rc, cudaStream_t s);

struct Workspace {
  DevBuf r, d, t, b, x;                 // per level, per precision
};

// FGMRES state of one solve (resumable: one Arnoldi step per round)
struct Krylov {
  bool active = false, converged = false;
  int it = 0, j = 0;
  double bnorm = 0.0, relres = 0.0;
  std::vector<double> H, cs, sn, g;
  double* x = nullptr;
  cudaStream_t stream = nullptr;
};

// Multi-problem operator application (batch.cu): one launch per colour over several problems'
// structured levels sharing (dim, degree, operator, precision, frozen-data mode, block size).
struct MultiOp;
MultiOp* multi_op_create(const std::vector<const OpLevel*>& lv, const std::vector<const void*>& src,
                         const std::vector<void*>& dst, int prec, Budget* bud);
void multi_op_destroy(MultiOp* m);
// dst_i = A_i src_i for every member (constrained rows dst = src)
void multi_vmult(const MultiOp& m, cudaStream_t s);
struct MultiOpDel {
  void operator()(MultiOp* m) const { multi_op_destroy(m); }
};
using MultiOpPtr = std::unique_ptr<MultiOp, MultiOpDel>;

struct LocalSmoothing;

struct Problem {
  uint64_t uid = 0;                     // process-unique id (batch plans are keyed by it)
  uint64_t graph_epoch = 0;             // incremented whenever the captured graphs are dropped
  int kind = 0, dim = 3, k = 2;
  Physics phys;
  int smoother = 0, smoother_degree = 5, mg_precision = 0, restart = 30, maxit = 500, cg_iterations = 10;
  bool fused_smoother = false;          // fuse smoother update / V-cycle residual into the cell kernel
  double tol = 1e-8;
  Budget* bud = nullptr;
  std::unique_ptr<OpLevel> system;      // the problem's operator on the finest mesh
  std::unique_ptr<OpLevel> pmass;       // Stokes: pressure mass
  std::vector<std::unique_ptr<OpLevel>> levels;  // multigrid levels (0 = finest)
  std::vector<std::unique_ptr<Transfer>> transfers;  // transfers[l]: level l <-> l+1
  // coarse solver
  bool coarse_dense = true;
  int64_t coarse_n = 0;
  DevBuf coarse_inv[2];
  DevBuf coarse_cols;                   // set-up scratch: operator columns of the coarse level
  int coarse_cheby_degree = 30;
  // workspaces [precision][level]
  std::vector<Workspace> ws[2];
  // FGMRES / Krylov (fp64)
  DevBuf V, Z, w, tmp, hvec, yvec, part, ptrV, ptrZ, scal;
  DevBuf sys_r, sys_z;                  // fp64 system-size temporaries
  DevBuf mg_b32, mg_x32;                // fp32 copies for the mixed-precision preconditioner
  DevBuf cg_r, cg_z, cg_p, cg_q, cg_x;  // Stokes Schur CG (mg precision)
  DevBuf stokes_u_rhs, stokes_u_sol;    // Stokes A-block rhs/solution (mg precision)
  // CUDA graphs: the preconditioner (fp64 in/out) and the V-cycle per precision
  bool use_graphs = true;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t pc_graph = nullptr;
  cudaGraphExec_t vc_graph[2] = {nullptr, nullptr};
  DevBuf pc_in, pc_out, vc_in[2], vc_out[2];
  Krylov kry;
  double* hh_host = nullptr;            // pinned: Gram--Schmidt coefficients of the last step
  // Newton / BDF (stabilised NS; allocated on first use): explicit field, residual, increment
  DevBuf nt_g, nt_F, nt_d;
  cudaEvent_t ev_step = nullptr;        // batched rounds: the step's input is in pc_in
  double st_dt = -1.0, st_alpha = -1.0;  // dt, alpha and explicit-field use of the last set_state
  bool st_g = false;
  // local-smoothing hierarchy (null: global coarsening over `levels`)
  std::unique_ptr<LocalSmoothing> ls;
  size_t bytes = 0;
  ~Problem();
};

// Local smoothing (Section 2) for the vector Laplacian on a locally refined mesh.  Level l >= 1 is
// the set of cells of refinement level l (a partial forest), smoothed with homogeneous Dirichlet
// conditions on its refinement edge; level 0 is the unrefined base mesh, whose own
// global-coarsening hierarchy (p and h) completes the cycle.  Every free DoF of the fine mesh is
// owned by exactly one level: the coarsest level among the active cells holding it, where it is
// not on the refinement edge.
struct LsLevel {
  std::unique_ptr<OpLevel> op;          // refinement edge and boundary constrained: the smoother's operator
  std::unique_ptr<OpLevel> full;        // boundary constrained only: residual rows on the edge, transfers
  Transfer down;                        // this level (fine) <-> the next coarser level
  DevBuf copy_fine, copy_lvl;           // owned DoFs: fine node id, level node id
  int64_t n_copy = 0;
  Workspace ws[2];                      // b defect, x iterate, r residual, t product, d smoother direction
  DevBuf z[2], c[2];                    // smoother right-hand side; restricted contribution / correction
};
struct LocalSmoothing {
  std::unique_ptr<Problem> base;        // level 0 and below: the base mesh's global-coarsening hierarchy
  std::vector<std::unique_ptr<LsLevel>> lv;  // lv[l - 1]: refinement level l
  DevBuf copy_fine, copy_lvl;           // DoFs owned by level 0
  int64_t n_copy = 0;
  DevBuf b[2], x[2], c[2];              // level-0 defect, iterate, restricted contribution
};
// Multigrid levels as seen by the API (information, smoother bounds): global coarsening: `levels`;
// local smoothing: the refined levels finest first, then the base hierarchy.
int mg_level_count(const Problem& p);
OpLevel& mg_level(Problem& p, int i);

// Build everything for a mesh and a description; throws Error.
// hp-adaptive vector Laplacian (Section 3): degree[c] per forest cell; hierarchy: every degree
// lowered by one per level until all are linear, then global coarsening
// kind 1: the vector Laplacian; kind 0: Taylor--Hood Stokes (system and pressure mass on hp spaces,
// the A block on the hp hierarchy)
std::unique_ptr<Problem> build_problem_hp(const Forest& f, const std::vector<int32_t>& degree, const Physics& ph,
                                          int coarse_stop_n, Budget* bud, int kind = 1);
// hierarchy: 0 global coarsening, 1 local smoothing (vector Laplacian and the Stokes A block on a
// locally refined mesh; an unrefined mesh needs none and gets global coarsening)
std::unique_ptr<Problem> build_problem(const Forest& f, int kind, int k, const Physics& ph, int mg_order,
                                       int coarse_stop_n, Budget* bud, int hierarchy = 0);
// the level workspaces alone (r, d, t, b, x per level and precision)
void alloc_level_workspaces(Problem& p);

// Multigrid
void smooth(Problem& p, int level, int prec, const void* b, void* x, bool x_is_zero, cudaStream_t s);
void vcycle(Problem& p, int prec, const void* b, void* x, cudaStream_t s);
// V-cycle through its captured CUDA graph (captured on first use)
void vcycle_graph(Problem& p, int prec, const void* b, void* x, cudaStream_t s);
// Drop captured graphs (after a change of smoother bounds or settings)
void invalidate_graphs(Problem& p);
void estimate_lambda(Problem& p, cudaStream_t s);
// choose the cell kernel's block size for every operator of the problem (cached per process)
void autotune(Problem& p, cudaStream_t s);
void setup_coarse(Problem& p, cudaStream_t s);
// Stabilised NS (Section 5): set dt, the BDF coefficient alpha, the frozen state U and the explicit
// field g (null: none) on the finest level, carry them down the hierarchy by interpolation and
// refresh every level's point data, diagonal and the coarse inverse (uniform and refined meshes).
void set_state(Problem& p, double dt, double alpha, const double* U, const double* g, cudaStream_t s);
// the two halves of set_state: the finest level only (enough for the residual and the Jacobian),
// and the rest of the hierarchy with the diagonals and the coarse inverse
void set_state_fine(Problem& p, double dt, double alpha, const double* U, const double* g, cudaStream_t s);
void refresh_preconditioner(Problem& p, cudaStream_t s);
// dst = F(state): the nonlinear residual on the free rows, zero on constrained rows
void residual(Problem& p, int prec, void* dst, cudaStream_t s);
struct NewtonParams {
  double dt = 0.0, omega = 1.0, rtol = 1e-8, atol = 0.0, lin_tol = 1e-4;
  int max_newton = 10;
  bool extrapolate = false;
};
struct NewtonResult {
  int newton_iterations = 0, linear_iterations = 0;
  double residual0 = 0.0, residual = 0.0;
  bool converged = false;
};
// One variable-step BDF step (omega = dt_n / dt_{n-1}; 0: BDF1) solved by Newton-FGMRES.
// u: in = initial guess with the Dirichlet values at t_{n+1}, out = solution.
NewtonResult bdf_step(Problem& p, const NewtonParams& np, const double* u_n, const double* u_nm1,
                      const double* forcing, double* u, cudaStream_t s);
// max over velocity nodes of |u| (host value)
double max_velocity(Problem& p, const double* u, cudaStream_t s);
void alloc_workspaces(Problem& p);
// Solve (FP64 FGMRES); returns iterations, writes relres; throws on CUDA errors
int fgmres_solve(Problem& p, const double* b, double* x, double* relres, bool* converged, cudaStream_t s);
// Resumable FGMRES: begin (synchronises once), then per step enqueue (async) and complete (host,
// after the stream is synchronised); complete returns false once the solve has finished.
void krylov_begin(Problem& p, const double* b, double* x, cudaStream_t s);
void krylov_enqueue(Problem& p);
bool krylov_complete(Problem& p);
// The same step split around its preconditioner application, for rounds in which the
// preconditioners of several problems run as one batched, graph-captured V-cycle (D6):
// pre = the step's vector into p.pc_in (event p.ev_step recorded), post = the rest of the step,
// ordered after `ready` (recorded once the batched preconditioner has written p.pc_out).
void krylov_enqueue_pre(Problem& p);
void krylov_enqueue_post(Problem& p, cudaEvent_t ready);
// Problems whose preconditioner is one V-cycle on uniform levels (batched rounds)
bool batchable(const Problem& p);
// One V-cycle for each of several problems, in lock-step over the levels: at every level, the
// operator applications of all problems whose levels share (dim, degree, operator, precision,
// smoother) run as one launch per colour.  Results equal those of the problems' own V-cycles.
struct BatchVcycle;
struct BatchVcycleDel {
  void operator()(BatchVcycle* b) const;
};
using BatchVcyclePtr = std::unique_ptr<BatchVcycle, BatchVcycleDel>;
BatchVcyclePtr make_batch_vcycle(const std::vector<Problem*>& ps, int prec, const std::vector<const void*>& b,
                                 const std::vector<void*>& x, Budget* bud);
void batch_vcycle(BatchVcycle& B, cudaStream_t s);
// The preconditioners of the listed (batchable) problems in one captured CUDA graph: input
// p.pc_in, output p.pc_out of every problem.
struct BatchPrecond;
struct BatchPrecondDel {
  void operator()(BatchPrecond* b) const;
};
using BatchPrecondPtr = std::unique_ptr<BatchPrecond, BatchPrecondDel>;
BatchPrecondPtr make_batch_precond(const std::vector<Problem*>& ps);
void batch_precond_launch(BatchPrecond& B, cudaStream_t s);

}  // namespace mfns
