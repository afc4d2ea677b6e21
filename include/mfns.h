/*
 * mfns.h -- C ABI of the GB300 matrix-free Stokes / stabilised Navier--Stokes
 * multigrid library (libmfns.so).
 *
 * The operations follow the problem statement of the paper "Solving the
 * (Navier--)Stokes equations with space and time adaptivity using deal.II":
 *   - Eq. 1 (stationary Stokes) with Taylor--Hood Q_k / Q_{k-1} elements and the
 *     block system of Eq. 5 ([[A, B], [B^T, 0]]: continuity row -(div u, q));
 *   - the A block alone (vector Laplacian nu (grad u, grad v), Eq. 5);
 *   - Eq. 3 with the SUPG/PSPG terms of Section 5, BDF2 in time, linearised by
 *     Newton's method at a frozen state (equal-order Q_k Q_k);
 *   - matrix-free evaluation (Section 1), global-coarsening h- and
 *     p-multigrid with hanging-node constraints resolved in smoother and
 *     transfer (Section 2, Eq. 4), Chebyshev/Jacobi smoothing around point
 *     Jacobi (Sections 3 and 5), one V-cycle as preconditioner inside FGMRES
 *     (Section 3) and the block-triangular preconditioner of Eq. 5.
 *
 * Conventions (all entry points):
 *   - Every call returns an int status: MFNS_OK (0) or a negative error code.
 *     mfns_last_error() returns a thread-local message for the last failure.
 *     No C++ exception crosses this boundary.
 *   - Vectors passed as `const void*` / `void*` are DEVICE pointers owned by
 *     the caller (for example the data pointers of torch tensors), laid out as
 *     described in mfns_problem_info and aligned to 16 bytes.  They are read
 *     and written asynchronously on `stream` (a cudaStream_t, NULL = the
 *     legacy default stream); the caller synchronises.  src and dst must not
 *     alias.  Host pointers are only used where the name says so (`_host`).
 *   - Every call that takes device vectors also takes their lengths in
 *     elements (`n`, `n_fine`, ...).  The library checks each against the
 *     length the call expects (mfns_problem_info: n_dofs, level_dofs,
 *     cycle_dofs) and returns MFNS_ERR_ARG, touching nothing, when they
 *     differ: a wrong-sized buffer is reported instead of read or written
 *     out of bounds.  The library cannot see the allocation itself: the
 *     caller guarantees that each pointer holds n elements.
 *   - Precision: MFNS_FP64 vectors hold double, MFNS_FP32 vectors hold float.
 *   - The library owns meshes, hierarchies, diagonals, frozen states and
 *     workspaces; they are allocated against the context's HBM budget at
 *     create time (MFNS_ERR_BUDGET when it would be exceeded), so vmult,
 *     smooth, vcycle and solve allocate nothing.
 *   - One problem is used by one stream at a time (not thread-safe per
 *     problem); distinct problems may run concurrently on distinct streams.
 *
 * Vector layout of a problem's system operator (MFNS_OP_SYSTEM):
 *   STAB_NS:  node-interleaved [u_x, u_y, (u_z), p] per Q_k node.
 *   STOKES:   node-interleaved velocity [u_x, u_y, (u_z)] per Q_k node, then
 *             one pressure entry per Q_{k-1} node (offset = n_velocity_dofs).
 *   STOKES_A: node-interleaved velocity only.   PMASS: one entry per node.
 *   Node numbering is the library's own; mfns_dof_support_points exports the
 *   coordinates and field of every entry.  Constrained entries (Dirichlet
 *   velocity on the boundary, hanging nodes) are identity rows of every
 *   operator: vmult returns dst_i = src_i there and ignores them elsewhere.
 */
#ifndef MFNS_H
#define MFNS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define MFNS_OK 0
#define MFNS_ERR_ARG (-1)            /* invalid argument (null pointer, bad level, misaligned vector,
                                        vector length other than the one the call expects) */
#define MFNS_ERR_OOM (-2)            /* cudaMalloc failed */
#define MFNS_ERR_BUDGET (-3)         /* the context's HBM budget would be exceeded */
#define MFNS_ERR_UNSUPPORTED (-4)    /* (dim, degree, kind) not built */
#define MFNS_ERR_CUDA (-5)           /* a CUDA runtime call failed */
#define MFNS_ERR_TIMEOUT (-6)        /* a bounded device-side wait gave up */
#define MFNS_ERR_NOT_CONVERGED (-7)  /* solve hit maxit; the iterate is still written */

/* problem kinds */
#define MFNS_STOKES 0   /* Taylor--Hood Q_k/Q_{k-1}, Eq. 1 / Eq. 5 */
#define MFNS_STOKES_A 1 /* vector Laplacian (A block of Eq. 5) */
#define MFNS_STAB_NS 2  /* linearised SUPG/PSPG BDF2 Navier--Stokes, Q_k Q_k (Section 5) */
#define MFNS_PMASS 3    /* pressure mass matrix on Q_k */

/* precisions */
#define MFNS_FP64 0
#define MFNS_FP32 1

/* operator selectors for mfns_vmult / mfns_diagonal (levels are >= 0) */
#define MFNS_OP_SYSTEM (-1) /* the problem's own operator on the finest mesh */
#define MFNS_OP_PMASS (-2)  /* STOKES only: pressure mass matrix (Schur approximation) */

/* stabilised-NS term flags (Section 5); default MFNS_TERMS_ALL */
#define MFNS_TERM_MASS 1         /* BDF2 mass 3/(2 dt) (du, v) and its part of the residual */
#define MFNS_TERM_CONV 2         /* ub . grad du */
#define MFNS_TERM_NEWTON 4       /* du . grad ub */
#define MFNS_TERM_SUPG 8         /* tau (Rlin, ub . grad v) */
#define MFNS_TERM_SUPG_NEWTON 16 /* tau (Rbar, du . grad v) */
#define MFNS_TERM_PSPG 32        /* tau (Rlin, grad q) */
#define MFNS_TERM_STRONG_VISC 64 /* -nu lap du inside Rlin */
#define MFNS_TERMS_ALL 127

typedef struct mfns_ctx mfns_ctx;
typedef struct mfns_mesh mfns_mesh;
typedef struct mfns_problem mfns_problem;
typedef struct mfns_spacetime mfns_spacetime;

typedef struct {
  int kind;             /* MFNS_STOKES, MFNS_STOKES_A, MFNS_STAB_NS, MFNS_PMASS */
  int degree;           /* velocity degree k (STOKES: k >= 2, pressure k-1; PMASS: its own degree) */
  double nu;            /* viscosity */
  double dt;            /* time step of BDF2 (STAB_NS); <= 0 means stationary (no mass term) */
  int terms;            /* STAB_NS term flags; 0 is taken as MFNS_TERMS_ALL */
  double div_sign;      /* sign of the continuity row; 0 = default (STOKES -1, STAB_NS +1) */
  int smoother;         /* 0 = default for the kind: STAB_NS relaxation around point Jacobi (Section 5,
                           Exp. 3), otherwise Chebyshev around point Jacobi (Section 3);
                           1 = Chebyshev, 2 = Jacobi relaxation; 3 = Chebyshev around the blend of
                           Section 3 on the hp levels that have faces h-refined on one side and
                           p-refined on the other: additive Schwarz blocks there (the free unknowns
                           on the closed face of the coarse cell, block inverses summed where blocks
                           overlap), point Jacobi on the unknowns in no block; Chebyshev around point
                           Jacobi on every other level */
  int smoother_degree;  /* Chebyshev degree / relaxation sweeps; 0 = default (5) */
  int mg_order;         /* 0 default (STOKES_A: p then h; STAB_NS: h then p), 1 p_then_h, 2 h_then_p */
  int mg_precision;     /* MFNS_FP64 or MFNS_FP32: precision of the multigrid preconditioner */
  int coarse_stop_n;    /* uniform h-coarsening stops when n is odd or n <= this; 0 = 2 */
  int fgmres_restart;   /* 0 = 30 */
  double tol;           /* relative residual tolerance of mfns_solve; 0 = 1e-8 */
  int maxit;            /* 0 = 500 */
  int cg_iterations;    /* STOKES: Jacobi-CG steps for the Schur complement; 0 = 10 */
  double lambda_max;    /* > 0: use this lambda_max of D^-1 A on every level instead of the estimate */
  int recompute_frozen; /* STAB_NS: 1 = interpolate the frozen state inside every apply; 0 (default) =
                           store its point values (u, grad u, Rbar, tau) once per level (more HBM,
                           fewer shared-memory contractions per apply) */
  int fused_smoother;   /* 1: on uniform levels the Chebyshev / Jacobi update and the V-cycle residual
                           are applied by the cell kernel to each node in the colour that completes
                           its product (no separate vector pass); 0 (default): the product is
                           written out and a streaming kernel applies the update (faster on GB300:
                           the cell kernel is latency-bound) */
  int hierarchy;        /* multigrid levels on a locally refined mesh (Section 2): 0 (default) global
                           coarsening -- every level covers the whole domain, hanging nodes resolved
                           on each; 1 local smoothing (MFNS_STOKES, MFNS_STOKES_A and
                           MFNS_STAB_NS; for MFNS_STAB_NS with the frozen Taylor--Green state:
                           mfns_set_state / mfns_bdf_step return MFNS_ERR_UNSUPPORTED) -- level
                           l is the set of cells of refinement level l with homogeneous Dirichlet
                           conditions on its refinement edge (velocity, and pressure for
                           MFNS_STAB_NS), level 0 the unrefined base mesh with
                           its own global-coarsening hierarchy.  The levels reported by
                           mfns_problem_info and addressed by mfns_set_lambda_max are then the
                           refined levels (finest first) followed by the base hierarchy;
                           mfns_smooth, mfns_prolongate_add and mfns_restrict address global-
                           coarsening levels only and return MFNS_ERR_UNSUPPORTED or
                           MFNS_ERR_ARG.  On an unrefined mesh 1 is the same as 0. */
} mfns_problem_desc;

typedef struct {
  int dim, degree, kind;
  int n_levels;                 /* multigrid levels, 0 = finest */
  int64_t n_dofs;               /* system vector length */
  int64_t n_velocity_dofs;      /* STOKES: start of the pressure block */
  int64_t n_cells;
  int n_colors;                 /* colours of the finest level */
  int64_t level_dofs[32];       /* vector length of each multigrid level (mfns_smooth, transfers,
                                   mfns_set_lambda_max); under local smoothing level 0 is the finest
                                   refinement level, not the fine operator (see cycle_dofs) */
  int level_degree[32];
  int64_t level_cells[32];
  double lambda_max[32];        /* smoother bound per level (estimate x 1.2, or the override) */
  size_t device_bytes;          /* HBM held by this problem */
  int64_t cycle_dofs;           /* vector length of mfns_vcycle: the fine operator of the multigrid
                                   (the velocity A block for STOKES, n_dofs otherwise), for both
                                   hierarchies */
} mfns_info;

typedef struct {
  int iterations;
  double rel_residual;          /* ||b - A x|| / ||b||, true residual in FP64 */
  double seconds;
  int converged;
} mfns_solve_info;

/* Newton step of a BDF time step (Section 5), see mfns_bdf_step. */
typedef struct {
  double dt;           /* time step dt_n = t_{n+1} - t_n (> 0) */
  double omega;        /* step ratio dt_n / dt_{n-1}; 0 = BDF1 (implicit Euler), e.g. for the first step */
  double rtol;         /* stop when ||F(u_k)|| <= max(atol, rtol ||F(u_0)||); 0 = 1e-8 */
  double atol;
  double lin_tol;      /* relative tolerance of each FGMRES solve (inexact Newton); 0 = 1e-4 */
  int max_newton;      /* 0 = 10 */
  int extrapolate;     /* 1: start from (1 + omega) u^n - omega u^{n-1} on the free entries */
} mfns_newton_desc;

typedef struct {
  int newton_iterations;        /* Newton updates performed */
  int linear_iterations;        /* FGMRES iterations over all Newton updates */
  double residual0, residual;   /* ||F|| (l2, FP64) at the initial guess and at the result */
  double seconds;
  int converged;
} mfns_newton_info;

/* ---- context --------------------------------------------------------------------------- */
/* device: CUDA ordinal; hbm_budget_bytes: 0 = unlimited.  Errors: ARG, CUDA. */
int mfns_ctx_create(int device, size_t hbm_budget_bytes, mfns_ctx** out);
/* 1 (default): mfns_batch_step runs the preconditioners of eligible problems as one batched
 * V-cycle; 0: every problem's preconditioner on its own stream (for comparison). */
int mfns_ctx_set_batching(mfns_ctx* ctx, int enable);
int mfns_ctx_destroy(mfns_ctx* ctx);
/* bytes currently charged to the context */
int mfns_ctx_memory(const mfns_ctx* ctx, size_t* used, size_t* peak);
const char* mfns_last_error(void);

/* ---- meshes (host objects) -------------------------------------------------------------- */
/* Unit square (dim 2) or cube (dim 3) with n cells per direction. */
int mfns_mesh_uniform(mfns_ctx* ctx, int dim, int n, mfns_mesh** out);
/* Refine cells with centre strictly inside the ball, `levels` times (level by level),
 * then 2:1 closure over faces, edges and vertices.  centre[2] is ignored in 2D. */
int mfns_mesh_refine_ball(mfns_mesh* mesh, const double centre[3], double radius, int levels);
int mfns_mesh_info(const mfns_mesh* mesh, int64_t* n_cells, int* max_level);
/* The active cells in the mesh's canonical order (the order of mfns_problem_create_hp's degree
 * array): 4 int32 per cell -- level and the integer coordinates x, y, z at that level (z = 0 in
 * 2D); writes up to cap cells to cells_host (may be NULL), the count to *n. */
int mfns_mesh_cells(const mfns_mesh* mesh, int32_t* cells_host, int64_t cap, int64_t* n);
int mfns_mesh_destroy(mfns_mesh* mesh);

/* ---- problems ------------------------------------------------------------------------------ */
/* Builds the operator, its global-coarsening hierarchy, diagonals, smoother bounds,
 * the dense coarse inverse and all workspaces.  The mesh may be destroyed afterwards. */
int mfns_problem_create(mfns_ctx* ctx, const mfns_mesh* mesh, const mfns_problem_desc* desc,
                        mfns_problem** out);
/* hp-adaptive problems (Section 3): cell_degree[c] (1..4; host array of n_cells entries in
 * the order of mfns_mesh_cells) is the degree of cell c.  A node is constrained when a cell whose
 * closed box holds it does not have it as a node and dominates every cell that does (coarser, or
 * same level and lower degree); it takes that cell's finite-element function at its position.
 * Where a hanging face has a coarse cell of higher degree than a fine cell (the combined h+p
 * face), that rule does not give a conforming space; the constraints of the whole space then
 * come from eliminating the continuity conditions of every face piece, the least preferred nodes
 * (finer, then higher degree, then face before edge before vertex, then higher node id) becoming
 * the constrained ones; every constrained node is expressed in nodes of its own face or edge.
 * The multigrid hierarchy lowers every degree by one per level until all cells are linear, then
 * coarsens globally.  desc->kind must be MFNS_STOKES_A or MFNS_STOKES (Taylor--Hood: velocity
 * degree per cell >= 2, pressure one lower, the A block on the hp hierarchy) and desc->hierarchy 0
 * (MFNS_ERR_UNSUPPORTED otherwise); one degree everywhere is the same as mfns_problem_create. */
int mfns_problem_create_hp(mfns_ctx* ctx, const mfns_mesh* mesh, const mfns_problem_desc* desc,
                           const int32_t* cell_degree, int64_t n_cells, mfns_problem** out);
int mfns_problem_info(const mfns_problem* p, mfns_info* out);
/* Support point (xyz_host[3*i..], z = 0 in 2D) and field (0..dim-1 velocity component,
 * dim pressure) of every entry of the vector of `which` (MFNS_OP_SYSTEM, MFNS_OP_PMASS
 * or a level).  Host arrays of length n (n = that vector's length). */
int mfns_dof_support_points(const mfns_problem* p, int which, double* xyz_host, int* field_host);
/* Constrained entries (identity rows) of `which`: writes up to cap indices, returns count in *n. */
int mfns_constrained_dofs(const mfns_problem* p, int which, int64_t* idx_host, int64_t cap, int64_t* n);
/* Replace the smoother bound of one level (parity tests pass the bound explicitly). */
int mfns_set_lambda_max(mfns_problem* p, int level, double lambda_max);
int mfns_problem_destroy(mfns_problem* p);

/* ---- operators ----------------------------------------------------------------------------- */
/* dst = A src (matrix-free, Section 1 / Eq. 4 per cell); constrained rows dst_i = src_i.
 * n: entries of src and of dst (n_dofs for MFNS_OP_SYSTEM, n_dofs - n_velocity_dofs for
 * MFNS_OP_PMASS, level_dofs[which] for a level).  On a uniform mesh the colour launches after
 * the first start while their predecessor drains (programmatic dependent launches). */
int mfns_vmult(mfns_problem* p, int which, int precision, const void* src, void* dst, int64_t n,
               void* stream);
/* dst_host[i] = A src_host[i], i < count, for vectors in HOST memory (a list of requests to the same
 * operator, the call a host-side client makes): the library copies each input to the device,
 * applies the operator exactly as mfns_vmult does (bitwise the same result) and copies the result
 * back, pipelined over two device staging sets -- the input copy of vector i+1 and the read-back of
 * vector i-1 overlap the product of vector i -- on two internal copy streams ordered after the work
 * already in `stream`; when `stream` reaches the end of the call, every dst_host[i] is written.
 * The staging (4 n entries of the precision) is allocated against the context's budget on the first
 * call for a (which, precision) and kept until the problem is destroyed or another pair is used.
 * Host vectors should be page-locked (cudaHostAlloc / cudaHostRegister) for the copies to run
 * asynchronously; pageable memory works, with the copies staged by the driver.  n as for
 * mfns_vmult; a dst_host[i] must not overlap any src_host[j] of the call (the same source may be
 * listed several times).  Calls on one problem must be ordered (the same stream, or the caller
 * orders them).  Error: ARG (null pointers, count < 1, precision, n), OOM (staging beyond the
 * budget). */
int mfns_vmult_host(mfns_problem* p, int which, int precision, const void* const* src_host,
                    void* const* dst_host, int count, int64_t n, void* stream);
/* diag = diag(A) (exact, per-cell unit-vector evaluation; 1 on constrained rows); n as in
 * mfns_vmult. */
int mfns_diagonal(mfns_problem* p, int which, int precision, void* diag, int64_t n, void* stream);
/* Hanging entries of x from their masters (x_h = sum_j w_hj x_j), Dirichlet entries kept; n as in
 * mfns_vmult. */
int mfns_apply_constraints(mfns_problem* p, int which, int precision, void* x, int64_t n, void* stream);

/* Per-kernel timing of the operator-kernel launches of `which` with CUDA events recorded on
 * the launching stream: mode 1 = reset and enable, 0 = disable, 2 = read (synchronises on the
 * recorded events; writes the summed kernel time in ms and the number of timed launches,
 * then resets).  The timed launches are the colour launches of the cell kernel only. */
int mfns_kernel_timing(mfns_problem* p, int which, int mode, double* total_ms, int64_t* launches);

/* ---- multigrid ----------------------------------------------------------------------------- */
/* One smoothing step on level `level`: Chebyshev of the problem's degree (or the Jacobi
 * relaxation) around point Jacobi, starting from x (x_is_zero = 1 skips the first product);
 * b and x have n = level_dofs[level] entries. */
int mfns_smooth(mfns_problem* p, int level, int precision, const void* b, void* x, int64_t n, int x_is_zero,
                void* stream);
/* Same smoothing step as mfns_smooth, for callers that must not allocate device memory
 * when they call in -- for example code running while a stream is being captured into a
 * CUDA graph, or a service that forbids cudaMalloc/cudaFree after start-up -- and that
 * should not depend on per-call workspace.  The paper has no counterpart; this is an
 * operational variant.  Its two scratch vectors (the Chebyshev direction and the operator
 * product) live in one fixed device array of 16 MiB that every GPU loading the library
 * holds until exit, so the level may have at most 1,048,576 entries (larger levels are
 * rejected with MFNS_ERR_ARG and a message).  The call performs no cudaMalloc/cudaFree.
 * The first call on a device looks up that array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  All calls share the array and it keeps
 * the last call's contents: calls whose GPU work overlaps in time (different streams,
 * different problems) race on it and must be serialised by the caller. */
int mfns_smooth_noalloc(mfns_problem* p, int level, int precision, const void* b, void* x, int64_t n,
                        int x_is_zero, void* stream);
/* Transfers between level `level` (fine) and level+1 (coarse), Eq. 4:
 * fine += P coarse;  coarse = P^T fine.  n_fine = level_dofs[level], n_coarse =
 * level_dofs[level + 1]. */
int mfns_prolongate_add(mfns_problem* p, int level, int precision, const void* coarse, int64_t n_coarse,
                        void* fine, int64_t n_fine, void* stream);
int mfns_restrict(mfns_problem* p, int level, int precision, const void* fine, int64_t n_fine, void* coarse,
                  int64_t n_coarse, void* stream);
/* x = V-cycle(b) on the multigrid hierarchy (zero initial guess); b and x have
 * mfns_info.cycle_dofs entries. */
int mfns_vcycle(mfns_problem* p, int precision, const void* b, void* x, int64_t n, void* stream);

/* ---- solve ---------------------------------------------------------------------------------- */
/* FGMRES(m) in FP64 on the system operator, preconditioned by one V-cycle (STAB_NS, STOKES_A)
 * or the block-triangular preconditioner of Eq. 5 (STOKES), with the multigrid in
 * desc.mg_precision.  b and x are FP64 device vectors; x is overwritten (zero start).
 * The pressure l2 mean of b and of every preconditioned vector is removed when the
 * pressure is only fixed up to a constant.  Returns MFNS_ERR_NOT_CONVERGED when maxit is hit.
 * n = n_dofs (both vectors). */
int mfns_solve(mfns_problem* p, const void* b, void* x, int64_t n, mfns_solve_info* info, void* stream);

/* ---- nonlinear and time-dependent stabilised Navier--Stokes (Section 5) ---------------------- */
/* STAB_NS on uniform meshes: set the time step dt, the BDF coefficient alpha of u^{n+1} (3/2 for
 * BDF2 with equal steps, 1 for BDF1) and the state at which the operator is linearised.
 * `state` is an FP64 device vector in the system layout (velocity with its Dirichlet values, and
 * pressure).  `explicit_field` (FP64 device, system layout, velocity entries used; may be NULL)
 * holds g = (beta_n u^n + beta_{n-1} u^{n-1}) / dt - f_h, the explicit part of the BDF time
 * derivative and the nodal forcing: the strong momentum residual becomes
 * R = (alpha/dt) u + g + u.grad u + grad p - nu lap u.  Without it the time derivative in R is
 * zero (as for the default Taylor--Green state).  The state and g are interpolated to every
 * multigrid level (coarse-node evaluation of the fine FE function); each level's stored point
 * values, smoother diagonal (evaluated in FP32 whatever the multigrid precision: it only scales
 * the smoother's correction) and the coarse inverse are recomputed.  The call synchronises
 * `stream`.  On refined meshes the hanging-node entries of the state and of g are set from their
 * masters first; a coarse level receives the fine function evaluated at its nodes cell by cell
 * (through the children of each coarse cell).  Returns MFNS_ERR_UNSUPPORTED for other kinds.
 * n = n_dofs (state and explicit_field). */
int mfns_set_state(mfns_problem* p, double dt, double alpha, const void* state, const void* explicit_field,
                   int64_t n, void* stream);
/* dst = F(state), the nonlinear residual of the SUPG/PSPG BDF discretisation at the state of the
 * last mfns_set_state, on the free rows; constrained rows are set to 0.  With tau frozen at the
 * state, mfns_vmult applies its Jacobian.  dst: device vector in `precision`, system layout, of
 * n = n_dofs entries. */
int mfns_residual(mfns_problem* p, int precision, void* dst, int64_t n, void* stream);
/* One variable-step BDF step for u^{n+1} (Section 5): Newton's method on F(u) = 0 with
 * g = (beta_n u^n + beta_{n-1} u^{n-1}) / dt - forcing, each update solving J(u_k) d = -F(u_k) by
 * FGMRES with the multigrid preconditioner at the current state (mg_precision of the problem).
 * alpha = (1 + 2 w)/(1 + w), beta_n = -(1 + w), beta_{n-1} = w^2/(1 + w) for w = desc.omega > 0;
 * w = 0: alpha = 1, beta_n = -1 (BDF1, u_nm1 unused).  u_n, u_nm1, forcing (may be NULL) and u
 * are FP64 device vectors in the system layout; u holds the initial guess with the Dirichlet
 * values at t_{n+1} on entry (the increments vanish on constrained entries) and the result on
 * return.  The pressure is fixed up to a constant when the velocity is Dirichlet everywhere.
 * Synchronises `stream`; returns MFNS_ERR_NOT_CONVERGED (result written) after max_newton
 * updates.  Buffers for g, F and the increment are allocated on the first call.  n = n_dofs (every
 * vector argument). */
int mfns_bdf_step(mfns_problem* p, const mfns_newton_desc* desc, const void* u_n, const void* u_nm1,
                  const void* forcing, void* u, int64_t n, mfns_newton_info* info, void* stream);
/* *umax (host) = max over velocity nodes of |u| for an FP64 device vector u in the system layout
 * (time-step control by a CFL number: dt = CFL h / umax), n = n_dofs.  Synchronises `stream`. */
int mfns_max_velocity(mfns_problem* p, const void* u, int64_t n, double* umax, void* stream);

/* ---- batched solves (continuous batching of many problems) ---------------------------------- */
/* Start a solve as in mfns_solve (same FGMRES, same preconditioner), without iterating: the
 * right-hand side is projected, x set to zero and the initial residual norm read back (one
 * synchronisation).  All later device work of this solve runs on `stream`; give every problem
 * of a batch its own stream so their work overlaps on the device.  n = n_dofs. */
int mfns_solve_begin(mfns_problem* p, const void* b, void* x, int64_t n, void* stream);
/* One round: every listed problem whose solve is still running performs one FGMRES iteration
 * (Section 3).  The device work of all of them is enqueued first, each on its own stream, then
 * each is completed on the host (Givens rotation, and at the end of a restart cycle the update
 * of x and the true residual).  The preconditioners of the running STAB_NS / STOKES_A problems
 * on uniform meshes (two or more) run as one batched V-cycle (see mfns_batch_vcycle) replayed
 * from a CUDA graph that is captured when the set of such problems changes.  running[i]
 * (optional) is set to 1 while problem i iterates.  Problems are independent: the result of
 * each is the same alone and in any batch. */
int mfns_batch_step(mfns_problem** problems, int n, int* running);
/* One V-cycle (zero initial guess) for each of n problems of one context, batched: the
 * operator applications of all problems whose current multigrid levels share dimension, degree,
 * operator, precision and smoother run as one launch per level and colour over the cells of all
 * of them, each block reading its problem from a descriptor table (uneven sizes share launches).
 * Results equal n separate mfns_vcycle calls (bitwise: the per-cell arithmetic and its order are
 * those of a single-problem launch).  b[i], x[i]: device vectors of problem i in `precision`, of
 * lengths[i] (host array) entries each, which must equal problem i's cycle_dofs.
 * Problems: STAB_NS or STOKES_A on uniform meshes, fused_smoother = 0 (else
 * MFNS_ERR_UNSUPPORTED).  mfns_batch_step uses the same batching, captured into a CUDA graph, for
 * the preconditioners of such problems.  Synchronises `stream`. */
int mfns_batch_vcycle(mfns_problem** problems, int n, int precision, void* const* b, void* const* x,
                      const int64_t* lengths, void* stream);
/* Iterations, relative residual and convergence of the last (or current) solve of p. */
int mfns_solve_status(const mfns_problem* p, mfns_solve_info* info);

/* ---- space-time slabs (Section 4) ----------------------------------------------------------- */
/* One time slab of the transient Stokes equations on the Taylor--Hood space of `stokes` (an
 * MFNS_STOKES problem built by mfns_problem_create; hp problems: MFNS_ERR_UNSUPPORTED), with
 * DG(r) in time, 0 <= r <= 7: Q = r + 1 stages, the Lagrange basis at the Q right Gauss--Radau
 * points of the slab (the last stage is the slab's end value; this is the Q-stage Radau IIA
 * method), slab length tau > 0.  Vectors are stage-major: Q blocks of the problem's system vector
 * (length Q * n, n = mfns_dof_support_points' length for MFNS_OP_SYSTEM).  The slab operator of
 * Eq. 6 after mass scaling with M_Q^{-1}:
 *     K = G_Q (x) M + tau I_Q (x) A,   G_Q = M_Q^{-1} A_Q,
 * with reference-slab matrices M_Q[j][i] = int phi_i phi_j and A_Q[j][i] = int phi_i' phi_j +
 * phi_i(0) phi_j(0), M the velocity mass (zero pressure rows, zero constrained rows) and A the
 * problem's Stokes operator (identity rows on constrained entries), so constrained rows of K are
 * tau times identity rows.  The problem must outlive the slab.  Errors: ARG, UNSUPPORTED, OOM,
 * BUDGET, CUDA. */
int mfns_spacetime_create(mfns_problem* stokes, int r, double tau, mfns_spacetime** out);
/* The same slab on the paper's spatial pair Q_k^dim / P^disc_{k-1} (Section 4): velocity of degree
 * k (2..4) with homogeneous Dirichlet conditions, pressure of total degree k - 1 per cell in the
 * monomials of the cell's centred, scaled coordinates (graded order), no continuity; the symmetric
 * form nu (grad u, grad v) - (p, div v) - (div u, q).  Uniform meshes only (MFNS_ERR_UNSUPPORTED
 * otherwise), FP64 only.  Spatial vector: the velocity block (nodes of the (k n + 1)^dim grid,
 * lexicographic, dim interleaved components) then npc coefficients per cell (lexicographic cells).
 * The slab owns its spatial operators; the mesh may be destroyed afterwards. */
int mfns_spacetime_create_pdisc(mfns_ctx* ctx, const mfns_mesh* mesh, int k, double nu, int r, double tau,
                                mfns_spacetime** out);
/* Support point and field of every spatial entry of the slab (host arrays of n_stage entries, xyz 3
 * per entry, z = 0 in 2D): field < dim velocity, dim pressure (Taylor--Hood), dim + a the
 * coefficient a of the cell's pressure polynomial at the cell centre (P^disc). */
int mfns_spacetime_support_points(const mfns_spacetime* st, double* xyz_host, int* field_host);
/* Stage count, spatial vector length and (host arrays, may be NULL) the Q temporal nodes on
 * [0, 1] and G_Q (Q x Q, row-major). */
int mfns_spacetime_info(const mfns_spacetime* st, int* stages, int64_t* n_stage, double* nodes_host,
                        double* g_host);
/* y = K x (device vectors of length n = Q * n_stage in `precision`; x and y must not overlap).  P^disc slabs:
 * FP64 only (MFNS_ERR_UNSUPPORTED otherwise). */
int mfns_spacetime_vmult(mfns_spacetime* st, int precision, const void* x, void* y, int64_t n, void* stream);
int mfns_spacetime_destroy(mfns_spacetime* st);
/* Space-time multigrid for the slab (Section 4), FP64, uniform meshes (MFNS_ERR_UNSUPPORTED
 * otherwise).  Levels, finest first (space before time, polynomial before geometric): the spatial
 * degree halved while above 2, then global coarsening in space while the mesh has more than
 * coarse_n (>= 2) cells per direction, then the temporal degree halved down to DG(0) on that
 * coarsest mesh -- left out when one vertex star there holds every cell (its patch would be
 * singular; the coarsest level is then solved at the fine temporal degree); no coarsening of tau.  Transfers: P_tau (x) I for a temporal step (the coarse temporal polynomial
 * at the fine nodes), I_Q (x) P_h for a spatial one (Eq. 4 for velocity and pressure); restriction
 * is the transpose.  Smoother: nu_s steps x += omega S (b - K x) before and after the coarse
 * correction, S the additive Schwarz method over vertex stars (for every mesh vertex, the free
 * entries all of whose cells contain it, all stages together, each block solved exactly), each
 * entry weighted by the inverse number of patches holding it, constrained rows solved exactly;
 * the coarsest level is solved directly (pseudo-inverse: the constant pressure of every stage is
 * a null direction).  The set-up probes the spatial operators on the device, inverts the patch
 * blocks on the host (in FP64) and synchronises `stream`.  inverse_precision: the patch inverses
 * are stored and applied in FP64 (0) or rounded to FP32 and applied in FP32 (1: half the bytes
 * of every patch solve; the vectors, the transfers, the coarse solve and the outer FGMRES stay
 * FP64).  Error: ARG for another inverse_precision. */
int mfns_spacetime_mg_build(mfns_spacetime* st, int nu_s, double omega, int coarse_n, int inverse_precision,
                            void* stream);
/* Number of levels; for 0 <= level < *n_levels also its spatial degree, temporal degree and
 * spatial vector length (level -1: the count only).  ARG if the multigrid is not built. */
int mfns_spacetime_mg_level(const mfns_spacetime* st, int level, int* n_levels, int* k, int* r, int64_t* n_stage);
/* Support point and field of every spatial entry of a level (host arrays of n_stage entries;
 * xyz 3 per entry, z = 0 in 2D; field < dim velocity, dim pressure). */
int mfns_spacetime_mg_support_points(const mfns_spacetime* st, int level, double* xyz_host, int* field_host);
/* One piece of the cycle on device FP64 vectors (stage-major): what = 0: out = K_l in; 1: out =
 * S_l in (Schwarz; not on the coarsest level); 2: out += P_l in (in on level l+1, out on level l);
 * 3: out = P_l^T in (in on level l, out on level l+1).  in and out must not overlap; n_in and n_out
 * are their lengths (Q_l * n_stage of the level each lives on). */
int mfns_spacetime_mg_apply(mfns_spacetime* st, int level, int what, const void* in, int64_t n_in, void* out,
                            int64_t n_out, void* stream);
/* Bytes of the Schwarz patch inverses of a level (each smoother application reads them once:
 * the algorithmic traffic of the HBM-bound patch solve) and the number of patches (0 on the
 * coarsest level). */
int mfns_spacetime_mg_smoother_bytes(const mfns_spacetime* st, int level, int64_t* inverse_bytes, int64_t* n_patches);
/* x = one V-cycle of the space-time multigrid applied to b (zero initial guess; FP64, length
 * Q * n of the finest level). */
int mfns_spacetime_vcycle(mfns_spacetime* st, const void* b, void* x, int64_t n, void* stream);
/* K x = b on the slab by FGMRES(30) in FP64 (classical Gram--Schmidt twice), right-preconditioned
 * by one space-time V-cycle; the constant pressure of every stage (the null space of K) is removed
 * from b and from every preconditioned vector, so x has none.  Stops when ||b - K x|| <= tol ||b||
 * or after maxit iterations (then MFNS_ERR_NOT_CONVERGED, x the last iterate).  iterations,
 * relres, converged: host outputs (may be NULL).  Synchronises `stream` once per iteration. */
int mfns_spacetime_solve(mfns_spacetime* st, const void* b, void* x, int64_t n, double tol, int maxit,
                         int* iterations, double* relres, int* converged, void* stream);
/* The DG(r) reference-slab matrices on the host, no device needed (any pointer may be NULL):
 * nodes (Q), m_Q (Q, m_Q[j] = phi_j(0)), M_Q, A_Q and G_Q (Q x Q, row-major [j][i]).  Error: ARG
 * for r outside 0..7. */
int mfns_spacetime_temporal(int r, double* nodes_host, double* m_host, double* mq_host, double* aq_host,
                            double* g_host);

#ifdef __cplusplus
}
#endif
#endif /* MFNS_H */
