// Host description of one operator on one mesh level, as needed to launch the
// operator kernels (filled by level.cpp, consumed by the templated launchers).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace mfns {

// CUDA-event timer of the operator-kernel launches of one level (per-kernel tracing).
struct KernelTimer {
  bool enabled = false;
  std::vector<cudaEvent_t> ev;   // pairs (start, stop)
  size_t used = 0;               // events recorded since the last read
  void record_pair_begin(cudaStream_t s);
  void record_pair_end(cudaStream_t s);
  double read_ms(int64_t* launches);  // synchronises, sums and resets
  ~KernelTimer();
};

// Fused epilogue of an operator application (see OpArgs): mode 1 = Chebyshev / Jacobi step,
// mode 2 = residual; pointers in the launch precision.
struct OpEpilogue {
  int mode = 0;
  // the product is preceded in the stream by the library's own clearing kernel of dst (which
  // lets dependents start early): the first colour is a programmatic dependent launch as well
  bool after_clear = false;
  const void* b = nullptr;
  const void* dinv = nullptr;
  void* d = nullptr;
  void* xout = nullptr;
  double c1 = 0.0, c2 = 0.0;
};

struct OpLaunch {
  int dim = 3, k = 2, op = 0;        // main-field degree k, op = OpKind
  bool structured = false;          // uniform mesh with lexicographic numbering
  int n = 0;                        // structured: cells per direction
  double h = 0.0;                   // structured: edge length
  int64_t n_cells = 0;
  int n_colors = 0;
  std::vector<int32_t> color_ptr;   // indexed: colour c = cells [color_ptr[c], color_ptr[c+1])
  const int32_t* cell_u = nullptr;  // device, colour-sorted
  const int32_t* cell_p = nullptr;
  const int32_t* cell_f = nullptr;
  const uint32_t* mask = nullptr;
  const void* hcell[2] = {nullptr, nullptr};     // fp64 / fp32 edge lengths
  const void* frozen[2] = {nullptr, nullptr};    // fp64 / fp32 frozen state
  int64_t p_offset = 0;
  double nu = 1.0, dt = 0.0, div_sign = -1.0;    // dt <= 0: stationary
  double alpha = 1.5;                            // BDF coefficient of u^{n+1}: c_m = alpha / dt
  const void* gexp[2] = {nullptr, nullptr};      // stabilised NS: explicit field g (fp64 / fp32) or none
  int terms = 127;
  // 1D tables in double (converted to the kernel precision at launch)
  int Q = 3, N = 3, NP = 3;
  std::vector<double> S, Sp, D, D2, W, P, Pp;
  KernelTimer* timer = nullptr;     // optional per-launch timing
  void* fq[2] = {nullptr, nullptr}; // stabilised NS: precomputed frozen point data (fp64 / fp32)
  int warps[2] = {0, 0};            // warps per block per precision (0 = not tuned yet: use 4)
  const uint8_t* lastc = nullptr;   // per main node: index of the last colour whose cells touch it
};

// The current device's word in which the cell kernels report a bounded wait that ran out (bit 0);
// allocated on first use (4 bytes per device, held until exit).
int* op_wait_flag();
// Reads and clears the current device's word (synchronous); throws Error(kErrTimeout) if set.
void op_check_wait_flag();

// Autotuner: pick the warps per block (1, 2 or 4) of the cell kernel for this operator and
// precision by timing a few applications on scratch vectors; results are cached per
// (dim, degree, operator, precision, structured) for the process.
int autotune_warps(OpLaunch& L, int prec, void* src, void* dst, int64_t n, cudaStream_t s);

// Stabilised NS: number of precomputed values per cell (lanes x points x values per point).
int64_t frozen_point_values_per_cell(int dim, int k);
// Fill L.fq[prec] (device buffer of n_cells * frozen_point_values_per_cell) from the frozen state.
void op_precompute_frozen(const OpLaunch& L, int prec, cudaStream_t s);

// Stabilised NS: dst = F(frozen state), the nonlinear residual on the free rows (dst zeroed by the
// caller; constrained rows untouched).
void op_residual(const OpLaunch& L, int prec, void* dst, cudaStream_t s);

// Fill the 1D tables of `L` for its degree (needs L.dim, L.k, L.op).
void fill_tables(OpLaunch& L);

// dst = A src on the free rows (dst must be zeroed by the caller); diag = true
// accumulates the diagonal instead (src ignored).  Constrained rows untouched.
// ncols > 1: ncols products at once, column j reading src + j col_stride and writing dst + j col_stride.
template <int DIM, int K, int OP, typename T>
void op_launch(const OpLaunch& L, const T* src, T* dst, bool diag, cudaStream_t s, int fq_mode = -1, int ncols = 1,
               int64_t col_stride = 0, const OpEpilogue* epi = nullptr);

// One colour of a multi-problem launch (structured cells, plain products): `probs` is the device
// descriptor table (one ProbArgs of the launch precision per problem), `block_pid` the problem of
// every block, `nblocks` the blocks of all problems.  `L` (any member) provides the 1D tables and
// the block size; all members share (dim, k, op, precision) and the frozen-data mode.
struct MultiColour {
  const void* probs = nullptr;
  const int32_t* block_pid = nullptr;
  unsigned nblocks = 0;
};
template <int DIM, int K, int OP, typename T>
void op_launch_multi(const OpLaunch& L, int color, const MultiColour& mc, cudaStream_t s);

// Deferred product of a uniform 3D stabilised, vector-Laplacian or pressure-mass level (small
// levels, where the eight colour launches are latency, not work): one launch over every colour writes each cell's
// contributions to `defer` (n_cells * (k+1)^3 * NU entries of the precision), then one gather pass
// forms dst = A src, every node summing its cells' contributions in colour order -- the additions
// and the order of the colour-ordered scatter onto a cleared vector, so the result is the same bit
// for bit -- with the identity rows (velocity of boundary nodes) src.
template <int DIM, int K, int OP, typename T>
void op_launch_deferred(const OpLaunch& L, const T* src, T* defer, cudaStream_t s);
void op_apply_deferred(const OpLaunch& L, int prec, const void* src, void* dst, void* defer, cudaStream_t s);
void op_apply_multi(const OpLaunch& L, int prec, int color, const MultiColour& mc, cudaStream_t s);

// Runtime dispatch over (dim, k, op, precision); prec 0 = fp64, 1 = fp32.
void op_apply(const OpLaunch& L, int prec, const void* src, void* dst, bool diag, cudaStream_t s);
// dst = 0, then dst += A src on the free rows: a clearing kernel followed by the colour launches,
// all of them programmatic dependent launches after the clear (constrained rows untouched).  With
// keep (a bitmask of n rows that the colour launches do not write: a uniform level's constrained
// rows), the clearing kernel sets those rows to src instead of 0.
void op_apply_cleared(const OpLaunch& L, int prec, const void* src, void* dst, int64_t n, cudaStream_t s,
                      const uint32_t* keep = nullptr);
// dst (zeroed by the caller) receives partial sums; the epilogue writes the fused result
void op_apply_epi(const OpLaunch& L, int prec, const void* src, void* dst, const OpEpilogue& epi, cudaStream_t s);
// ncols applications at once (column j: src + j col_stride -> dst + j col_stride), dst zeroed by the caller
void op_apply_cols(const OpLaunch& L, int prec, const void* src, void* dst, int ncols, int64_t col_stride,
                   cudaStream_t s);

}  // namespace mfns
