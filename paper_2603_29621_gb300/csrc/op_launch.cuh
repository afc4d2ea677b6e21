// Templated launcher of the operator kernel; included by the per-operator
// instantiation units (op_<kind>_<dim>d.cu).
#pragma once
#include <atomic>

#include "common.hpp"
#include "op_apply.cuh"
#include "op_launch.hpp"

namespace mfns {

template <typename T, int Q, int N, int NP>
static void build_tables(const OpLaunch& L, Tables<T, Q, N, NP>& t) {
  for (int q = 0; q < Q; ++q) {
    for (int a = 0; a < N; ++a) t.S[q][a] = (T)L.S[q * N + a];
    for (int a = 0; a < NP; ++a) t.Sp[q][a] = L.Sp.empty() ? T(0) : (T)L.Sp[q * NP + a];
    for (int r = 0; r < Q; ++r) {
      t.D[q][r] = (T)L.D[q * Q + r];
      t.D2[q][r] = (T)L.D2[q * Q + r];
    }
    t.W[q] = (T)L.W[q];
  }
  for (int h = 0; h < 2; ++h) {
    for (int s = 0; s < N; ++s)
      for (int m = 0; m < N; ++m) t.P[h][s][m] = (T)L.P[(h * N + s) * N + m];
    for (int s = 0; s < NP; ++s)
      for (int m = 0; m < NP; ++m) t.Pp[h][s][m] = L.Pp.empty() ? T(0) : (T)L.Pp[(h * NP + s) * NP + m];
  }
}

// Launch of one colour; pdl: as a programmatic dependent launch of the previous kernel in `s`.
template <typename Kern, typename Args>
static void launch_op(Kern kern, dim3 grid, unsigned block, size_t smem, cudaStream_t s, const Args& a, bool pdl) {
  if (!pdl) {
    kern<<<grid, block, smem, s>>>(a);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  MFNS_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
}

// The kernel arguments every launch of L shares: tables, mesh tables, physics.
template <typename T, int Q, int N, int NP>
static void fill_common(const OpLaunch& L, OpArgs<T, Q, N, NP>& a) {
  if (L.Q != Q || L.N != N || L.NP != NP) throw Error(kErrArg, "operator tables do not match the degree");
  build_tables(L, a.tab);
  const int prec = sizeof(T) == 8 ? 0 : 1;
  a.frozen = reinterpret_cast<const T*>(L.frozen[prec]);
  a.cell_u = L.cell_u;
  a.cell_p = L.cell_p;
  a.cell_f = L.cell_f;
  a.mask = L.mask;
  a.hcell = reinterpret_cast<const T*>(L.hcell[prec]);
  a.n = L.n;
  a.p_offset = L.p_offset;
  a.h = (T)L.h;
  a.nu = (T)L.nu;
  const double dt_inv = L.dt > 0 ? 1.0 / L.dt : 0.0;
  a.dt_inv = (T)dt_inv;
  a.cm = (T)(L.alpha * dt_inv);
  a.div_sign = (T)L.div_sign;
  for (int b = 0; b < 7; ++b) a.cf[b] = (L.terms >> b) & 1 ? T(1) : T(0);
  a.err = op_wait_flag();
  a.fq = reinterpret_cast<T*>(L.fq[prec]);
  a.gexp = reinterpret_cast<const T*>(L.gexp[prec]);
}

template <int DIM, int K, int OP, typename T>
void op_launch(const OpLaunch& L, const T* src, T* dst, bool diag, cudaStream_t s, int fq_mode, int ncols,
               int64_t col_stride, const OpEpilogue* epi) {
  constexpr int Q = K + 1, N = K + 1, NP = OP == OP_STOKES ? K : K + 1;
  OpArgs<T, Q, N, NP> a{};
  fill_common(L, a);
  const int prec = sizeof(T) == 8 ? 0 : 1;
  a.src = src;
  a.dst = dst;
  a.diag = diag;
  if (ncols < 1 || (ncols > 1 && (diag || fq_mode == 2 || fq_mode == 3)))
    throw Error(kErrArg, "several columns only for operator applications");
  a.col_stride = ncols > 1 ? col_stride : 0;
  const bool fused = epi && epi->mode;
  if (epi && epi->after_clear && (fused || diag || ncols != 1 || fq_mode == 2 || fq_mode == 3))
    throw Error(kErrArg, "products after the clearing kernel: single operator applications");
  if (fused) {
    if (diag || ncols > 1 || fq_mode == 2 || fq_mode == 3 || OpTraits<OP, DIM>::SPLIT_P || !L.lastc ||
        !L.structured)
      throw Error(kErrArg, "fused epilogue: single-column application on a uniform mesh, main-node operator");
    a.epi = epi->mode;
    a.lastc = L.lastc;
    a.eb = static_cast<const T*>(epi->b);
    a.edinv = static_cast<const T*>(epi->dinv);
    a.ed = static_cast<T*>(epi->d);
    a.exout = static_cast<T*>(epi->xout);
    a.ec1 = (T)epi->c1;
    a.ec2 = (T)epi->c2;
  }
  // frozen state: -1 = use the precomputed point data when present; 2 = write it (set-up pass)
  // 3 = residual pass: the state is read from the frozen buffer (src unused, pointed there)
  const int fq = OP != OP_STAB_NS ? 0 : (fq_mode == 2 || fq_mode == 3) ? fq_mode : (a.fq ? 1 : 0);
  if (fq == 3 && diag) throw Error(kErrArg, "residual pass in diagonal mode");
  if (fq == 2 || fq == 3) a.src = a.frozen;
  using TM = Team<DIM, Q>;
  const int warps = L.warps[prec] > 0 ? L.warps[prec] : kOpWarps;
  const int cells_per_block = warps * TM::CPW;
  const size_t smem = op_smem_bytes<DIM, K, OP, T>(warps, false);
  const size_t smem_fq = op_smem_bytes<DIM, K, OP, T>(warps, true);
  if constexpr (OP == OP_STAB_NS) {
    // the staged-frozen kernels may need more than the default 48 KB of dynamic shared memory;
    // the attribute is per device and set once for the largest block size
    static std::atomic<uint64_t> attr_done{0};
    int dev = 0;
    MFNS_CUDA(cudaGetDevice(&dev));
    const uint64_t bit = 1ull << (dev & 63);
    if (fq == 1 && !(attr_done.load() & bit)) {
      const int mx = (int)op_smem_bytes<DIM, K, OP, T>(kOpWarps, true);
      MFNS_CUDA(cudaFuncSetAttribute(op_kernel<DIM, K, OP, T, true, false, 1>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
      MFNS_CUDA(cudaFuncSetAttribute(op_kernel<DIM, K, OP, T, false, true, 1>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
      MFNS_CUDA(cudaFuncSetAttribute(op_kernel<DIM, K, OP, T, false, false, 1>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
      MFNS_CUDA(cudaFuncSetAttribute(op_kernel<DIM, K, OP, T, true, false, 1, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
      // the structured product's blocks are one warp with its staged blocks: ask for the largest
      // shared-memory carveout so that shared memory never caps the resident blocks below the
      // register limit
      MFNS_CUDA(cudaFuncSetAttribute(op_kernel<DIM, K, OP, T, true, false, 1>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout, 100));
      attr_done.fetch_or(bit);
    }
  }
  const bool structured = L.structured && !diag;
  int64_t color_offset = 0;
  bool launched = epi && epi->after_clear;  // the clearing kernel before colour 0 lets it start early
  for (int c = 0; c < L.n_colors; ++c) {
    int64_t ncell;
    if (structured) {
      a.color = c;
      a.color_offset = color_offset;
      ncell = 1;
      for (int d = 0; d < DIM; ++d) ncell *= (L.n - ((c >> d) & 1) + 1) / 2;
      color_offset += ncell;
    } else {
      a.color = c;
      a.cell_begin = L.color_ptr[c];
      a.cell_end = L.color_ptr[c + 1];
      ncell = a.cell_end - a.cell_begin;
    }
    if (ncell <= 0) continue;
    const unsigned gx = (unsigned)((ncell + cells_per_block - 1) / cells_per_block);
    // diagonal of a level with few cells: split the unit-vector passes over blockIdx.y (only on
    // uniform meshes, where no two slots of a cell share a DoF, so the blocks write disjoint entries)
    unsigned gy = (unsigned)ncols;
    if (diag && L.structured) {
      using Tr = OpTraits<OP, DIM>;
      constexpr int NLOC = Tr::NU * ipow(N, DIM) + (Tr::SPLIT_P ? ipow(NP, DIM) : 0);
      const unsigned want = 152u * 8u;
      gy = gx >= want ? 1u : std::min<unsigned>((unsigned)NLOC, (want + gx - 1) / gx);
    }
    const dim3 grid(gx, gy);
    const bool timed = L.timer && L.timer->enabled;
    if (timed) L.timer->record_pair_begin(s);
    // colours after the first are programmatic dependent launches: their blocks may start while
    // the previous colour drains and wait (griddepcontrol.wait) only before touching dst; src and
    // the frozen data are not written by the colour launches.  Timed launches stay serialised.
    const bool pdl = launched && !timed;
    launched = true;
    auto go = [&](auto kern, size_t sm) { launch_op(kern, grid, warps * 32, sm, s, a, pdl); };
    if constexpr (OP == OP_STAB_NS) {
      if (fq == 2) {
        if (L.structured)
          go(op_kernel<DIM, K, OP, T, true, false, 2>, smem);
        else
          go(op_kernel<DIM, K, OP, T, false, false, 2>, smem);
      } else if (fq == 3) {
        if (L.structured)
          go(op_kernel<DIM, K, OP, T, true, false, 3>, smem);
        else
          go(op_kernel<DIM, K, OP, T, false, false, 3>, smem);
      } else if (fq == 1) {
        if (structured && fused)
          go(op_kernel<DIM, K, OP, T, true, false, 1, true>, smem_fq);
        else if (structured)
          go(op_kernel<DIM, K, OP, T, true, false, 1>, smem_fq);
        else if (diag)
          go(op_kernel<DIM, K, OP, T, false, true, 1>, smem_fq);
        else
          go(op_kernel<DIM, K, OP, T, false, false, 1>, smem_fq);
      } else {
        if (structured && fused)
          go(op_kernel<DIM, K, OP, T, true, false, 0, true>, smem);
        else if (structured)
          go(op_kernel<DIM, K, OP, T, true, false, 0>, smem);
        else if (diag)
          go(op_kernel<DIM, K, OP, T, false, true, 0>, smem);
        else
          go(op_kernel<DIM, K, OP, T, false, false, 0>, smem);
      }
    } else {
      if (structured && fused)
        go(op_kernel<DIM, K, OP, T, true, false, 0, true>, smem);
      else if (structured)
        go(op_kernel<DIM, K, OP, T, true, false>, smem);
      else if (diag)
        go(op_kernel<DIM, K, OP, T, false, true>, smem);
      else
        go(op_kernel<DIM, K, OP, T, false, false>, smem);
    }
    MFNS_CUDA(cudaGetLastError());
    if (L.timer && L.timer->enabled) L.timer->record_pair_end(s);
  }
}

// Deferred product of a uniform 3D stabilised level: one launch over every colour (blockIdx.y =
// colour) writing each cell's contributions to `defer`; k_gather_cells forms dst from them.
template <int DIM, int K, int OP, typename T>
void op_launch_deferred(const OpLaunch& L, const T* src, T* defer, cudaStream_t s) {
  if constexpr (!(DIM == 3 && (OP == OP_STAB_NS || OP == OP_STOKES_A || OP == OP_PMASS))) {
    throw Error(kErrUnsupported, "deferred products: 3D stabilised, vector-Laplacian or pressure-mass levels only");
  } else {
    constexpr int Q = K + 1, N = K + 1, NP = K + 1;
    if (!L.structured || L.n_colors != 8) throw Error(kErrArg, "deferred products: uniform levels only");
    OpArgs<T, Q, N, NP> a{};
    fill_common(L, a);
    a.src = src;
    a.defer = defer;
    using TM = Team<DIM, Q>;
    const int prec = sizeof(T) == 8 ? 0 : 1;
    const int warps = L.warps[prec] > 0 ? L.warps[prec] : kOpWarps;
    const int cells_per_block = warps * TM::CPW;
    int64_t off = 0, maxc = 0;
    for (int c = 0; c < 8; ++c) {
      int64_t nc = 1;
      for (int d = 0; d < DIM; ++d) nc *= (L.n - ((c >> d) & 1) + 1) / 2;
      a.defer_off[c] = off;
      off += nc;
      maxc = std::max(maxc, nc);
    }
    const dim3 grid((unsigned)((maxc + cells_per_block - 1) / cells_per_block), 8u);
    if constexpr (OP == OP_STAB_NS) {
      if (a.fq) {  // the precomputed frozen point data, staged per cell
        const size_t sm = op_smem_bytes<DIM, K, OP, T>(warps, true);
        auto kern = op_kernel<DIM, K, OP, T, true, false, 1, false, false, true>;
        static std::atomic<uint64_t> attr_done{0};  // per device, for the largest block size
        int dev = 0;
        MFNS_CUDA(cudaGetDevice(&dev));
        const uint64_t bit = 1ull << (dev & 63);
        if (!(attr_done.load() & bit)) {
          MFNS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)op_smem_bytes<DIM, K, OP, T>(kOpWarps, true)));
          attr_done.fetch_or(bit);
        }
        kern<<<grid, warps * 32, sm, s>>>(a);
        MFNS_CUDA(cudaGetLastError());
        return;
      }
    }
    op_kernel<DIM, K, OP, T, true, false, 0, false, false, true>
        <<<grid, warps * 32, op_smem_bytes<DIM, K, OP, T>(warps, false), s>>>(a);
    MFNS_CUDA(cudaGetLastError());
  }
}

template <int DIM, int K, int OP, typename T>
void op_launch_multi(const OpLaunch& L, int color, const MultiColour& mc, cudaStream_t s) {
  constexpr int Q = K + 1, N = K + 1, NP = OP == OP_STOKES ? K : K + 1;
  if constexpr (OpTraits<OP, DIM>::SPLIT_P) {
    throw Error(kErrArg, "multi-problem launch: Taylor--Hood system operator");
  } else {
    if (!L.structured) throw Error(kErrArg, "multi-problem launch: non-uniform level");
    if (mc.nblocks == 0) return;
    OpArgs<T, Q, N, NP> a{};
    if (L.Q != Q || L.N != N || L.NP != NP) throw Error(kErrArg, "operator tables do not match the degree");
    build_tables(L, a.tab);
    const int prec = sizeof(T) == 8 ? 0 : 1;
    a.color = color;
    a.probs = static_cast<const ProbArgs<T>*>(mc.probs);
    a.block_pid = mc.block_pid;
    a.err = op_wait_flag();
    const int warps = L.warps[prec] > 0 ? L.warps[prec] : kOpWarps;
    bool staged = false;
    if constexpr (OP == OP_STAB_NS) staged = L.fq[prec] != nullptr;
    if (staged) {
      static std::atomic<uint64_t> attr_done{0};
      int dev = 0;
      MFNS_CUDA(cudaGetDevice(&dev));
      const uint64_t bit = 1ull << (dev & 63);
      if constexpr (OP == OP_STAB_NS) {
        if (!(attr_done.load() & bit)) {
          MFNS_CUDA(cudaFuncSetAttribute(op_kernel<DIM, K, OP, T, true, false, 1, false, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)op_smem_bytes<DIM, K, OP, T>(kOpWarps, true)));
          attr_done.fetch_or(bit);
        }
      }
      if constexpr (OP == OP_STAB_NS)
        op_kernel<DIM, K, OP, T, true, false, 1, false, true>
            <<<mc.nblocks, warps * 32, op_smem_bytes<DIM, K, OP, T>(warps, true), s>>>(a);
    } else {
      op_kernel<DIM, K, OP, T, true, false, 0, false, true>
          <<<mc.nblocks, warps * 32, op_smem_bytes<DIM, K, OP, T>(warps, false), s>>>(a);
    }
    MFNS_CUDA(cudaGetLastError());
  }
}

#define MFNS_INSTANTIATE_DEFERRED(DIM, K, OP)                                                                  \
  template void op_launch_deferred<DIM, K, OP, double>(const OpLaunch&, const double*, double*, cudaStream_t);    \
  template void op_launch_deferred<DIM, K, OP, float>(const OpLaunch&, const float*, float*, cudaStream_t);

#define MFNS_INSTANTIATE_OP(DIM, K, OP)                                                                        \
  template void op_launch<DIM, K, OP, double>(const OpLaunch&, const double*, double*, bool, cudaStream_t, int, int, \
                                               int64_t, const OpEpilogue*);                                        \
  template void op_launch<DIM, K, OP, float>(const OpLaunch&, const float*, float*, bool, cudaStream_t, int, int,    \
                                              int64_t, const OpEpilogue*);                                         \
  template void op_launch_multi<DIM, K, OP, double>(const OpLaunch&, int, const MultiColour&, cudaStream_t);       \
  template void op_launch_multi<DIM, K, OP, float>(const OpLaunch&, int, const MultiColour&, cudaStream_t);

}  // namespace mfns

