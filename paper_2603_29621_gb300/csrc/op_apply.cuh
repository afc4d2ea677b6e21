// The operator kernel (see op_kernel.cuh for the building blocks).
#pragma once
#include "op_kernel.cuh"

namespace mfns {

constexpr int kOpWarps = 4;  // largest number of warps per block (the block size is tuned at run time)
// The stabilised kernel's x-direction exchanges go through warp shuffles (the x-row of a team is
// adjacent lanes), the y-direction ones through shared memory: measured on the 64^3 FP32 apply,
// 0.199 ms against 0.204 ms with both through shared memory.
constexpr bool kXShfl = true;
// Products scatter with reductions done by the L2 (red.global.add.v4.f32 for four FP32 components
// per node, scalar red.global.add.f32 / .f64 otherwise, see scatter_add) instead of reading dst
// after the grid-dependency wait: the same single rounding per contribution, and the colours stay
// ordered by that wait, so results are unchanged bit for bit; the late, exposed dst loads go away
// (64^3 stabilised FP32 apply: 0.186 against 0.196 ms).  The fused epilogue needs the completed sum
// and keeps the read-modify-write, and so do FP64 nodes of four components (two 16-byte accesses;
// that apply is bound by the FP64 rate).
constexpr bool kScatterRed = kScatterRedF32;

template <int DIM, int Q>
struct Team {
  static constexpr int TPC = ipow(Q, DIM - 1);   // lanes per cell
  static constexpr int CPW = 32 / TPC;           // cells per warp
  static constexpr int BUF = ipow(Q, DIM);       // elements per team buffer
  static constexpr int NBUF = 4;                 // buffers per team (4 fields per exchange stage)
  // Team stride padded so that the teams of a warp start TPC banks apart: lanes of different
  // teams touching the same relative element then hit disjoint banks.
  template <typename T>
  __host__ __device__ static constexpr int stride() {
    constexpr int w = sizeof(T) / 4, m = 32 / w;
    return NBUF * BUF + (((TPC - NBUF * BUF) % m) + m) % m;
  }
  // Staged frozen blocks live in a later shared-memory region, one per team.  A block is read in
  // 16-byte quads, the TPC lanes of a team reading consecutive quads; the per-team stride is the
  // block (a multiple of 16 bytes) rounded up to 16 modulo 128 bytes, so that the next team's
  // first quad continues the bank sequence where this team's lanes end and the quarter-warp
  // phases of a 128-bit load hit 8 distinct bank groups.
  template <typename T>
  __host__ __device__ static constexpr size_t stage_stride_bytes(size_t block_bytes) {
    return block_bytes + (16 + 128 - block_bytes % 128) % 128;
  }
};

// Minimum resident blocks per SM for the register allocator (occupancy vs spills), per
// instantiation; 1 lets the compiler use up to 255 registers.  The 3D Q2 stabilised kernel in
// FP32 (the headline product) runs best at 6 x 128 threads' worth (80 registers, 8 bytes of
// spill): measured on the 64^3 apply, 4 / 5 / 6 / 7 / 8 gave 0.222 / 0.208 / 0.199 / 0.214 /
// 0.232 ms (the latency of the late dst loads and the shared-memory exchanges wants warps).
// The fused-epilogue instantiation gets one block less (its update operands need registers).
template <int DIM, int K, int OP, typename T>
struct OpMinBlocks {
  static constexpr int value = 1;
};
#ifndef MFNS_STABNS_Q2_F32_MINBLOCKS
#define MFNS_STABNS_Q2_F32_MINBLOCKS 6
#endif
template <>
struct OpMinBlocks<3, 2, OP_STAB_NS, float> {
  static constexpr int value = MFNS_STABNS_Q2_F32_MINBLOCKS;
};

template <int OP, int DIM, int N, int NP>
struct Layout {
  using Tr = OpTraits<OP, DIM>;
  static constexpr int NB = ipow(N, DIM);
  static constexpr int NBP = ipow(NP, DIM);
  // team buffers: scratch (3) + frozen needs none extra (kept in registers)
  static constexpr int NBUF = 3;
};

// Node id of slot (a,b,c) of a structured cell, and whether it is on the boundary.
template <int DIM, int K>
__device__ __forceinline__ int64_t structured_node(int n, const int cc[3], int a, int b, int c, bool& bnd) {
  const int64_t M = (int64_t)K * n + 1;
  const int64_t ix = (int64_t)K * cc[0] + a, iy = (int64_t)K * cc[1] + b, iz = DIM == 3 ? (int64_t)K * cc[2] + c : 0;
  bnd = ix == 0 || ix == M - 1 || iy == 0 || iy == M - 1 || (DIM == 3 && (iz == 0 || iz == M - 1));
  return ix + M * (iy + M * iz);
}

// FQ: 0 = frozen state interpolated in the kernel, 1 = read the precomputed point values,
// 2 = compute the point values, write them to args.fq and stop (set-up pass),
// 3 = nonlinear residual at the frozen state (Section 5; src unused).
template <int DIM>
struct FrozenPoint {
  static constexpr int NFQ = DIM + DIM * DIM + DIM + 1;  // u, grad u, Rbar, tau
  static constexpr int NQ = (NFQ + 3) / 4;                // quads of 4 values per point and lane
  // one cell's block: [point l][quad][lane][4 values] (values NFQ..4 NQ-1 unused): a lane reads
  // its point's values as NQ aligned 4-vectors, the lanes of a team consecutive ones
  template <typename T>
  __host__ __device__ static constexpr int block(int q) {
    return ipow(q, DIM - 1) * q * NQ * 4;
  }
  // offset of value k of point l of lane `lane` (tpc lanes per cell)
  __host__ __device__ static constexpr int at(int l, int k, int lane, int tpc) {
    return ((l * NQ + (k >> 2)) * tpc + lane) * 4 + (k & 3);
  }
};

// Completion of a team's staged block: bounded wait on its mbarrier (phase 0).  A wait that runs
// out sets bit 0 of *err (when given) and waits once more, so that the copy is not left writing
// into the block of a finished CTA; the computation then goes on (no early exit: every lane of
// the warp must reach the same __syncwarp calls).
__device__ __forceinline__ bool mbar_try_wait0(unsigned addr) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(addr)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void mbar_wait0_bounded(unsigned addr, int* err) {
  constexpr uint32_t kLimit = 1u << 22;
  for (uint32_t it = 0; it < kLimit; ++it)
    if (mbar_try_wait0(addr)) return;
  if (err) atomicOr(err, 1);
  for (uint32_t it = 0; it < kLimit; ++it)
    if (mbar_try_wait0(addr)) return;
}

// EPI: the fused smoother / residual epilogue is compiled in (structured launches only).
// MULTI: one launch over the cells of several problems (structured, plain products); each block
// reads its problem's fields from args.probs.
// DEFER: one launch over every colour of a uniform level (blockIdx.y = colour) that writes each
// cell's contributions to args.defer instead of adding them into dst (k_gather_cells sums them).
template <int DIM, int K, int OP, typename T, bool STRUCT, bool DIAG, int FQ = 0, bool EPI = false,
          bool MULTI = false, bool DEFER = false>
__global__ void __launch_bounds__(kOpWarps * 32, (EPI && OpMinBlocks<DIM, K, OP, T>::value > 1)
                                                     ? OpMinBlocks<DIM, K, OP, T>::value - 1
                                                     : OpMinBlocks<DIM, K, OP, T>::value)
op_kernel(const OpArgs<T, K + 1, K + 1, (OP == OP_STOKES ? K : K + 1)> args) {
  constexpr int Q = K + 1, N = K + 1, NP = OP == OP_STOKES ? K : K + 1;
  using Tr = OpTraits<OP, DIM>;
  using TM = Team<DIM, Q>;
  constexpr int NU = Tr::NU;
  constexpr int NB = ipow(N, DIM);
  constexpr int NBP = ipow(NP, DIM);
  constexpr int BUF = TM::BUF;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  // per-problem fields: kernel parameters, or the descriptor of the problem owning this block
  const T* srcp;
  T* dstp;
  const T *frozen, *gexp;
  T* fqd;
  int nmesh;
  int64_t color_offset, p_offset, bx;
  T hs, nu_, cm_, dt_inv_, div_sign_, cf_[7];
  if constexpr (MULTI) {
    static_assert(STRUCT && !DIAG && !EPI, "multi-problem launches: structured products only");
    const ProbArgs<T>* pa = args.probs + args.block_pid[blockIdx.x];
    srcp = pa->src;
    dstp = pa->dst;
    frozen = pa->frozen;
    gexp = pa->gexp;
    fqd = pa->fq;
    nmesh = pa->n;
    color_offset = pa->color_offset;
    p_offset = pa->p_offset;
    bx = (int64_t)blockIdx.x - pa->first_block;
    hs = pa->h;
    nu_ = pa->nu;
    cm_ = pa->cm;
    dt_inv_ = pa->dt_inv;
    div_sign_ = pa->div_sign;
#pragma unroll
    for (int i = 0; i < 7; ++i) cf_[i] = pa->cf[i];
  } else {
    srcp = args.src + (DEFER ? 0 : (int64_t)blockIdx.y * args.col_stride);
    dstp = args.dst + (DEFER ? 0 : (int64_t)blockIdx.y * args.col_stride);
    frozen = args.frozen;
    gexp = args.gexp;
    fqd = args.fq;
    nmesh = args.n;
    color_offset = DEFER ? args.defer_off[blockIdx.y] : args.color_offset;
    p_offset = args.p_offset;
    bx = (int64_t)blockIdx.x;
    hs = args.h;
    nu_ = args.nu;
    cm_ = args.cm;
    dt_inv_ = args.dt_inv;
    div_sign_ = args.div_sign;
#pragma unroll
    for (int i = 0; i < 7; ++i) cf_[i] = args.cf[i];
  }

  const int lane = lane_id();
  const int warp = threadIdx.x >> 5;
  int team = lane / TM::TPC;
  const int tid = lane % TM::TPC;
  const bool lane_active = team < TM::CPW;
  if (!lane_active) team = TM::CPW;  // dummy team for the spare lanes
  const int ti = tid % Q;
  const int tj = DIM == 3 ? tid / Q : 0;
  constexpr int FQB = (Tr::FROZEN && FQ == 1) ? FrozenPoint<DIM>::template block<T>(Q) : 0;
  T* buf0 = smem + (size_t)(warp * (TM::CPW + 1) + team) * TM::template stride<T>();
  T* buf1 = buf0 + BUF;
  T* buf2 = buf1 + BUF;
  // staged frozen blocks (FQ == 1): after the team buffers, one mbarrier per team, then one block
  // per team (16-byte aligned, see Team::stage_stride_bytes); the spare lanes use team 0's
  const size_t region1 = ((sizeof(T) * (size_t)(blockDim.x >> 5) * (TM::CPW + 1) * TM::template stride<T>() + 15) / 16) * 16;
  const int team_slot = warp * TM::CPW + (lane_active ? team : 0);
  const size_t mbar_bytes = ((size_t)(blockDim.x >> 5) * TM::CPW * 8 + 15) / 16 * 16;
  const unsigned mbar_addr = (unsigned)__cvta_generic_to_shared(smem_raw + region1) + 8u * (unsigned)team_slot;
  T* fqs = reinterpret_cast<T*>(smem_raw + region1 + mbar_bytes +
                                (size_t)team_slot * TM::template stage_stride_bytes<T>(sizeof(T) * FQB));

  // ---- which cell
  int64_t cell;
  bool valid;
  int cc[3] = {0, 0, 0};
  int64_t cellpos;  // position in the colour-major enumeration (precomputed frozen data)
  {
    const int64_t t = bx * ((blockDim.x >> 5) * TM::CPW) + warp * TM::CPW + (lane_active ? team : 0);
    if (STRUCT) {
      const int n = nmesh;
      int m[3], bits[3];
      int64_t total = 1;
      for (int d = 0; d < 3; ++d) {
        bits[d] = d < DIM ? ((DEFER ? (int)blockIdx.y : args.color) >> d) & 1 : 0;
        m[d] = d < DIM ? (n - bits[d] + 1) / 2 : 1;
        total *= m[d];
      }
      // a deferred launch spans all colours, some of which may hold no cell (n = 1): such a
      // colour's blocks leave before touching memory (total is uniform over the block)
      if (DEFER && total == 0) return;
      valid = lane_active && t < total;
      const int64_t tt = t < total ? t : total - 1;
      cc[0] = 2 * (int)(tt % m[0]) + bits[0];
      cc[1] = 2 * (int)((tt / m[0]) % m[1]) + bits[1];
      cc[2] = DIM == 3 ? 2 * (int)(tt / ((int64_t)m[0] * m[1])) + bits[2] : 0;
      cell = cc[0] + (int64_t)n * (cc[1] + (int64_t)n * cc[2]);
      cellpos = color_offset + tt;
    } else {
      const int64_t c = args.cell_begin + t;
      valid = lane_active && c < args.cell_end;
      cell = c < args.cell_end ? c : args.cell_end - 1;
      cellpos = cell;
    }
  }
  // the next colour's grid may be scheduled once every block of this one has started (it waits
  // for this grid's completion before it touches dst)
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  const T h = STRUCT ? hs : args.hcell[cell];
  const uint32_t mask = STRUCT ? 0u : args.mask[cell];
  // warp-uniform: every team of the warp takes the constraint path if one needs it
  // (a team with mask 0 leaves its values unchanged), so all __syncwarp calls match
  const bool constrained = __any_sync(0xffffffffu, (mask & 0x3FFFFu) != 0);
  const T inv_h = T(1) / h;
  T hd = h;
#pragma unroll
  for (int d = 1; d < DIM; ++d) hd *= h;

  const bool own = ti < N && tj < N;      // lane owns a nodal line of the main field
  const bool ownp = ti < NP && tj < NP;   // ... of the pressure field (Taylor--Hood)
  const int ti_n = ti < N ? ti : 0, tj_n = tj < N ? tj : 0;
  const int ti_p = ti < NP ? ti : 0, tj_p = tj < NP ? tj : 0;

  // ---- node ids of the owned slots
  int64_t node[N];
  bool bnd[N];
  int64_t fnode[N];
#pragma unroll
  for (int c = 0; c < N; ++c) {
    const int slot = DIM == 3 ? (c * N + tj_n) * N + ti_n : c * N + ti_n;
    if (STRUCT) {
      node[c] = DIM == 3 ? structured_node<DIM, K>(nmesh, cc, ti_n, tj_n, c, bnd[c])
                         : structured_node<DIM, K>(nmesh, cc, ti_n, c, 0, bnd[c]);
      fnode[c] = node[c];
    } else {
      const int32_t v = args.cell_u[cell * NB + slot];
      node[c] = v & 0x7fffffff;
      bnd[c] = v < 0;
      fnode[c] = (Tr::FROZEN && args.cell_f) ? (int64_t)args.cell_f[cell * NB + slot] : node[c];
    }
  }
  int64_t pnode[NP];
  if (Tr::SPLIT_P) {
#pragma unroll
    for (int c = 0; c < NP; ++c) {
      const int slot = DIM == 3 ? (c * NP + tj_p) * NP + ti_p : c * NP + ti_p;
      if (STRUCT) {
        bool dummy;
        pnode[c] = DIM == 3 ? structured_node<DIM, K - 1>(nmesh, cc, ti_p, tj_p, c, dummy)
                            : structured_node<DIM, K - 1>(nmesh, cc, ti_p, c, 0, dummy);
      } else {
        pnode[c] = args.cell_p[cell * NBP + slot];
      }
    }
  }

  const auto& tab = args.tab;
  const T nu = nu_;

  // weights of the lane's column
  T jxw[Q];
#pragma unroll
  for (int l = 0; l < Q; ++l) jxw[l] = (DIM == 3 ? tab.W[ti] * tab.W[tj] : tab.W[ti]) * tab.W[l] * hd;

  // ---- gather (or unit vectors in diagonal mode)
  constexpr int NLOC = NU * NB + (Tr::SPLIT_P ? NBP : 0);
  T dacc[NU][N];   // diagonal mode: accumulated diagonal entries of the owned slots
  T daccp[NP];
#pragma unroll
  for (int f = 0; f < NU; ++f)
#pragma unroll
    for (int c = 0; c < N; ++c) dacc[f][c] = 0;
#pragma unroll
  for (int c = 0; c < NP; ++c) daccp[c] = 0;

  // vmult: issue the loads of src and of the dst values to be updated together with the
  // frozen state, so that each cell waits for global memory once
  T u0[NU][N];
  T pv0[NP];
  T d0[NU][N];
  if (!DIAG && FQ != 2) {  // the set-up pass reads neither src nor dst
#pragma unroll
    for (int c = 0; c < N; ++c) {
      if constexpr (NU == 4) {
        if constexpr (sizeof(T) == 4) {
          const float4 v = own ? __ldg(reinterpret_cast<const float4*>(srcp + node[c] * 4)) : make_float4(0, 0, 0, 0);
          u0[0][c] = v.x; u0[1][c] = v.y; u0[2][c] = v.z; u0[3][c] = v.w;
        } else {
          const double2 v0 = own ? __ldg(reinterpret_cast<const double2*>(srcp + node[c] * 4)) : make_double2(0, 0);
          const double2 v1 = own ? __ldg(reinterpret_cast<const double2*>(srcp + node[c] * 4 + 2)) : make_double2(0, 0);
          u0[0][c] = v0.x; u0[1][c] = v0.y; u0[2][c] = v1.x; u0[3][c] = v1.y;
        }
      } else {
#pragma unroll
        for (int f = 0; f < NU; ++f) {
          u0[f][c] = own ? srcp[node[c] * NU + f] : T(0);
          d0[f][c] = 0;
        }
      }
      if (OP != OP_PMASS && bnd[c]) {
#pragma unroll
        for (int f = 0; f < DIM; ++f) u0[f][c] = 0;
      }
    }
    if (Tr::SPLIT_P) {
#pragma unroll
      for (int c = 0; c < NP; ++c) pv0[c] = ownp ? srcp[p_offset + pnode[c]] : T(0);
    }
  }

  // fused epilogue: which of the lane's nodes this colour completes (bit c), and an early L2
  // prefetch of their update operands (read-only here, and touched by no other colour)
  uint32_t epi_last = 0;
  if constexpr (EPI) {
    if (own && valid) {
#pragma unroll
      for (int c = 0; c < N; ++c)
        if (args.lastc[node[c]] == (uint8_t)args.color) {
          epi_last |= 1u << c;
          const int64_t o = node[c] * NU;
          asm volatile("prefetch.global.L2 [%0];" ::"l"(args.eb + o));
          if (args.epi == 1) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(args.edinv + o));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(args.ed + o));
          }
        }
    }
  }

  // frozen state (stabilised NS) at the lane's Gauss points; pressure value, pressure gradient and
  // velocity Laplacian are kept for the residual pass
  T Ub[DIM][Q], Gb[DIM][DIM][Q], Rb[DIM][Q], tau[Q];
  T gp[DIM][Q], lb[DIM][Q], pb[Q];
  constexpr int NFQ = FrozenPoint<DIM>::NFQ;
  if constexpr (Tr::FROZEN && FQ == 1) {
    // the team's cell block (contiguous in global memory, a multiple of 16 bytes, 16-byte aligned)
    // comes in with one TMA bulk copy issued by the team's first lane and tracked by the team's
    // mbarrier; it overlaps the interpolation of the trial fields and is awaited before first use
    constexpr unsigned BB = (unsigned)(FQB * sizeof(T));
    static_assert(BB % 16 == 0, "bulk copies move multiples of 16 bytes");
    if (lane_active && tid == 0) {
      const unsigned sdst = (unsigned)__cvta_generic_to_shared(fqs);
      const T* gsrc = fqd + (size_t)cellpos * FQB;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar_addr) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar_addr), "r"(BB) : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(sdst),
          "l"(gsrc), "r"(BB), "r"(mbar_addr)
          : "memory");
    }
  }
  if constexpr (Tr::FROZEN && FQ != 1) {
    T fz[DIM + 1][N];
#pragma unroll
    for (int c = 0; c < N; ++c) {
      if constexpr (NU == 4) {
        if constexpr (sizeof(T) == 4) {
          const float4 v = own ? *reinterpret_cast<const float4*>(frozen + fnode[c] * 4) : make_float4(0, 0, 0, 0);
          fz[0][c] = v.x; fz[1][c] = v.y; fz[2][c] = v.z; fz[3][c] = v.w;
        } else {
          const double2 v0 = own ? *reinterpret_cast<const double2*>(frozen + fnode[c] * 4) : make_double2(0, 0);
          const double2 v1 = own ? *reinterpret_cast<const double2*>(frozen + fnode[c] * 4 + 2) : make_double2(0, 0);
          fz[0][c] = v0.x; fz[1][c] = v0.y; fz[2][c] = v1.x; fz[3][c] = v1.y;
        }
      } else {
#pragma unroll
        for (int f = 0; f <= DIM; ++f) fz[f][c] = own ? frozen[fnode[c] * NU + f] : T(0);
      }
    }
#pragma unroll
    for (int f = 0; f <= DIM; ++f) {
      T val[Q], g[DIM][Q], h2[DIM][Q];
      values<DIM, Q, N, T>(fz[f], val, buf0, ti, tj, tab.S);
      if (f < DIM) {
        derivatives<DIM, Q, true, T>(val, g, h2, buf1, ti, tj, tab.D, tab.D2);
#pragma unroll
        for (int l = 0; l < Q; ++l) {
          Ub[f][l] = val[l];
          T lap = 0;
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            Gb[f][d][l] = g[d][l] * inv_h;
            lap += h2[d][l];
          }
          lb[f][l] = lap * inv_h * inv_h;
        }
      } else {
        derivatives<DIM, Q, false, T>(val, g, h2, buf1, ti, tj, tab.D, tab.D2);
#pragma unroll
        for (int l = 0; l < Q; ++l) {
          pb[l] = val[l];
#pragma unroll
          for (int d = 0; d < DIM; ++d) gp[d][l] = g[d][l] * inv_h;
        }
      }
    }
    // time derivative in the strong residual: c_m u + g with the explicit field g (BDF history
    // and forcing); without g the state's history equals the state and the term vanishes
    T tq[DIM][Q];
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
      for (int l = 0; l < Q; ++l) tq[i][l] = 0;
    if (gexp) {  // kernel parameter: uniform over the warp
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        T gz[N], gv[Q];
#pragma unroll
        for (int c = 0; c < N; ++c) gz[c] = own ? gexp[fnode[c] * NU + i] : T(0);
        values<DIM, Q, N, T>(gz, gv, buf0, ti, tj, tab.S);
#pragma unroll
        for (int l = 0; l < Q; ++l) tq[i][l] = cm_ * Ub[i][l] + gv[l];
      }
    }
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      T un2 = 0;
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        T s = tq[i][l] + gp[i][l] - nu * lb[i][l];
#pragma unroll
        for (int j = 0; j < DIM; ++j) s += Ub[j][l] * Gb[i][j][l];
        Rb[i][l] = s;
        un2 += Ub[i][l] * Ub[i][l];
      }
      const T a = T(2) * dt_inv_, b2 = T(4) * un2 * inv_h * inv_h, c = T(12) * nu * inv_h * inv_h;
      tau[l] = T(1) / sqrt(a * a + b2 + c * c);
    }
    if constexpr (FQ == 2) {
      if (valid) {
        constexpr int B = FrozenPoint<DIM>::template block<T>(Q);
        T* fp = fqd + (size_t)cellpos * B;
        auto at = [&](int l, int k) -> T& { return fp[FrozenPoint<DIM>::at(l, k, tid, TM::TPC)]; };
#pragma unroll
        for (int l = 0; l < Q; ++l) {
#pragma unroll
          for (int i = 0; i < DIM; ++i) {
            at(l, i) = Ub[i][l];
#pragma unroll
            for (int j = 0; j < DIM; ++j) at(l, DIM + i * DIM + j) = Gb[i][j][l];
            at(l, DIM + DIM * DIM + i) = Rb[i][l];
          }
          at(l, NFQ - 1) = tau[l];
        }
      }
      return;  // set-up pass: nothing else to do (no __syncwarp follows)
    }
  }

  // the local loop: one pass for vmult, NLOC passes (unit vectors) for the diagonal; in diagonal
  // mode blockIdx.y takes the passes [pass_begin, pass_end) (levels with few cells split them)
  int pass_begin = 0, pass_end = 1;
  if (DIAG) {
    const int per = (NLOC + (int)gridDim.y - 1) / (int)gridDim.y;
    pass_begin = (int)blockIdx.y * per;
    pass_end = min(NLOC, pass_begin + per);
  }
  for (int pass = pass_begin; pass < pass_end; ++pass) {
    T u[NU][N];
    T pv[NP];
    if (!DIAG) {
#pragma unroll
      for (int f = 0; f < NU; ++f)
#pragma unroll
        for (int c = 0; c < N; ++c) u[f][c] = u0[f][c];
#pragma unroll
      for (int c = 0; c < NP; ++c) pv[c] = pv0[c];
    } else {
      // unit vector of local DoF `pass` (component-major over the main nodes, then pressure)
#pragma unroll
      for (int f = 0; f < NU; ++f)
#pragma unroll
        for (int c = 0; c < N; ++c) {
          const int slot = DIM == 3 ? (c * N + tj_n) * N + ti_n : c * N + ti_n;
          u[f][c] = (own && pass == f * NB + slot) ? T(1) : T(0);
          if (OP != OP_PMASS && f < DIM && bnd[c]) u[f][c] = 0;
        }
      if (Tr::SPLIT_P) {
#pragma unroll
        for (int c = 0; c < NP; ++c) {
          const int slot = DIM == 3 ? (c * NP + tj_p) * NP + ti_p : c * NP + ti_p;
          pv[c] = (ownp && pass == NU * NB + slot) ? T(1) : T(0);
        }
      }
    }
    if (!STRUCT && constrained) {
#pragma unroll
      for (int f = 0; f < NU; ++f) apply_constraints<DIM, N, false, T>(u[f], buf0, mask, ti_n, tj_n, tab.P, own);
      if (Tr::SPLIT_P) apply_constraints<DIM, NP, false, T>(pv, buf0, mask, ti_p, tj_p, tab.Pp, ownp);
    }

    // ---- physics; result r[f][c] per component (and rp for the pressure block)
    T r[NU][N];
    T rp[NP];
    if constexpr (OP == OP_STOKES_A) {
#pragma unroll
      for (int f = 0; f < NU; ++f) {
        T val[Q], g[DIM][Q], h2[DIM][Q], c0[Q];
        values<DIM, Q, N, T>(u[f], val, buf0, ti, tj, tab.S);
        derivatives<DIM, Q, false, T>(val, g, h2, buf1, ti, tj, tab.D, tab.D2);
#pragma unroll
        for (int l = 0; l < Q; ++l) {
          const T s = nu * jxw[l] * inv_h * inv_h;
#pragma unroll
          for (int d = 0; d < DIM; ++d) g[d][l] *= s;
        }
        integrate<DIM, Q, N, false, true, T>(c0, g, r[f], buf1, buf2, ti, tj, tab.S, tab.D);
      }
    } else if constexpr (OP == OP_PMASS) {
      T val[Q], c0[Q], g[DIM][Q];
      values<DIM, Q, N, T>(u[0], val, buf0, ti, tj, tab.S);
#pragma unroll
      for (int l = 0; l < Q; ++l) c0[l] = val[l] * jxw[l];
      integrate<DIM, Q, N, true, false, T>(c0, g, r[0], buf1, buf2, ti, tj, tab.S, tab.D);
    } else if constexpr (OP == OP_VMASS) {
#pragma unroll
      for (int f = 0; f < NU; ++f) {
        T val[Q], c0[Q], g[DIM][Q];
        values<DIM, Q, N, T>(u[f], val, buf0, ti, tj, tab.S);
#pragma unroll
        for (int l = 0; l < Q; ++l) c0[l] = val[l] * jxw[l];
        integrate<DIM, Q, N, true, false, T>(c0, g, r[f], buf1, buf2, ti, tj, tab.S, tab.D);
      }
    } else if constexpr (OP == OP_STOKES) {
      T gu[DIM][DIM][Q];
      T div[Q];
#pragma unroll
      for (int l = 0; l < Q; ++l) div[l] = 0;
#pragma unroll
      for (int f = 0; f < DIM; ++f) {
        T val[Q], g[DIM][Q], h2[DIM][Q];
        values<DIM, Q, N, T>(u[f], val, buf0, ti, tj, tab.S);
        derivatives<DIM, Q, false, T>(val, g, h2, buf1, ti, tj, tab.D, tab.D2);
#pragma unroll
        for (int l = 0; l < Q; ++l) {
#pragma unroll
          for (int d = 0; d < DIM; ++d) gu[f][d][l] = g[d][l] * inv_h;
          div[l] += g[f][l] * inv_h;
        }
      }
      T p[Q];
      values<DIM, Q, NP, T>(pv, p, buf0, ti, tj, tab.Sp);
#pragma unroll
      for (int f = 0; f < DIM; ++f) {
        T cg[DIM][Q], c0[Q];
#pragma unroll
        for (int l = 0; l < Q; ++l) {
          const T s = jxw[l] * inv_h;
#pragma unroll
          for (int d = 0; d < DIM; ++d) cg[d][l] = (nu * gu[f][d][l] - (d == f ? p[l] : T(0))) * s;
        }
        integrate<DIM, Q, N, false, true, T>(c0, cg, r[f], buf1, buf2, ti, tj, tab.S, tab.D);
      }
      {
        T c0[Q], cg[DIM][Q];
#pragma unroll
        for (int l = 0; l < Q; ++l) c0[l] = div_sign_ * div[l] * jxw[l];
        integrate<DIM, Q, NP, true, false, T>(c0, cg, rp, buf1, buf2, ti, tj, tab.Sp, tab.D);
      }
    } else if constexpr (FQ == 3) {  // OP_STAB_NS, nonlinear residual at the frozen state
      // (c_m u + g + u.grad u, v) + nu (grad u, grad v) - (p, div v) + (tau R, u.grad v)
      // + s (div u, q) + (tau R, grad q), with R the strong residual computed above
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        T c0[Q], cg[DIM][Q];
#pragma unroll
        for (int l = 0; l < Q; ++l) {
          c0[l] = (Rb[i][l] - gp[i][l] + nu * lb[i][l]) * jxw[l];  // c_m u + g + u.grad u
          const T st = tau[l] * Rb[i][l];
#pragma unroll
          for (int d = 0; d < DIM; ++d)
            cg[d][l] = (nu * Gb[i][d][l] - (d == i ? pb[l] : T(0)) + st * Ub[d][l]) * jxw[l] * inv_h;
        }
        integrate<DIM, Q, N, true, true, T>(c0, cg, r[i], buf1, buf2, ti, tj, tab.S, tab.D);
      }
      {
        T c0[Q], cg[DIM][Q];
#pragma unroll
        for (int l = 0; l < Q; ++l) {
          T dv = 0;
#pragma unroll
          for (int j = 0; j < DIM; ++j) dv += Gb[j][j][l];
          c0[l] = div_sign_ * dv * jxw[l];
#pragma unroll
          for (int d = 0; d < DIM; ++d) cg[d][l] = tau[l] * Rb[d][l] * jxw[l] * inv_h;
        }
        integrate<DIM, Q, N, true, true, T>(c0, cg, r[DIM], buf1, buf2, ti, tj, tab.S, tab.D);
      }
    } else {  // OP_STAB_NS, the Jacobian at the frozen state (Section 5)
      // Phase 1: every trial field at the lane's points -- velocity values, physical gradients and
      // the part of the strong residual that needs no frozen data (grad p - nu lap u); pressure.
      const T cmm = cf_[0] * cm_, cfc = cf_[1], cfn = cf_[2], cfs = cf_[3], cfsn = cf_[4], cfp = cf_[5];
      const T lapc = cf_[6] * nu * inv_h * inv_h;
      // All DIM + 1 fields go through each exchange stage together (one warp barrier per stage).
      T tv[DIM][Q], tg[DIM][DIM][Q], tr[DIM][Q];
      T pval[Q];
      {
        T val[DIM + 1][Q], g[DIM + 1][DIM][Q], h2[DIM + 1][DIM][Q];
        values_multi<DIM, Q, DIM + 1, T, kXShfl>(u, val, buf0, BUF, ti, tj, tab.S);
        derivatives_multi<DIM, Q, DIM + 1, DIM, T, kXShfl>(val, g, h2, buf0, BUF, ti, tj, tab.D, tab.D2);
#pragma unroll
        for (int j = 0; j < DIM; ++j)
#pragma unroll
          for (int l = 0; l < Q; ++l) {
            T lap = 0;
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
              tg[j][d][l] = g[j][d][l] * inv_h;
              lap += h2[j][d][l];
            }
            tv[j][l] = val[j][l];
            tr[j][l] = -lapc * lap;
          }
        // the arithmetic below is written with explicit fused multiply-adds: every instantiation
        // of this kernel (single problem, multi-problem, fused epilogue) then rounds identically
#pragma unroll
        for (int l = 0; l < Q; ++l) {
          pval[l] = val[DIM][l];
#pragma unroll
          for (int i = 0; i < DIM; ++i) tr[i][l] = fma(g[DIM][i][l], inv_h, tr[i][l]);
        }
      }
      if constexpr (FQ == 1) mbar_wait0_bounded(mbar_addr, args.err);
      // Phase 2: point by point, the frozen values of the point (read once: NQ aligned 4-vectors
      // from the staged block, or the registers of the recomputing variant) and the 4 (DIM + 1)
      // integrand coefficients of the test functions: value c0 and reference gradient cg
      T c0[DIM + 1][Q], cg[DIM + 1][DIM][Q];
#pragma unroll
      for (int l = 0; l < Q; ++l) {
        T F[FrozenPoint<DIM>::NQ * 4];
        if constexpr (FQ == 1) {
          // the spare lanes of the warp read nothing (their results are discarded): the 128-bit
          // loads of the teams then stay free of bank conflicts
          const T* fb = fqs + FrozenPoint<DIM>::at(l, 0, tid, TM::TPC);
#pragma unroll
          for (int q4 = 0; q4 < FrozenPoint<DIM>::NQ; ++q4) {
            const T* src4 = fb + q4 * TM::TPC * 4;
            if constexpr (sizeof(T) == 4) {
              const float4 v = lane_active ? *reinterpret_cast<const float4*>(src4) : make_float4(0, 0, 0, 0);
              F[4 * q4] = v.x; F[4 * q4 + 1] = v.y; F[4 * q4 + 2] = v.z; F[4 * q4 + 3] = v.w;
            } else {
              const double2 v0 = lane_active ? *reinterpret_cast<const double2*>(src4) : make_double2(0, 0);
              const double2 v1 = lane_active ? *reinterpret_cast<const double2*>(src4 + 2) : make_double2(0, 0);
              F[4 * q4] = v0.x; F[4 * q4 + 1] = v0.y; F[4 * q4 + 2] = v1.x; F[4 * q4 + 3] = v1.y;
            }
          }
        } else {
#pragma unroll
          for (int i = 0; i < DIM; ++i) {
            F[i] = Ub[i][l];
#pragma unroll
            for (int j = 0; j < DIM; ++j) F[DIM + i * DIM + j] = Gb[i][j][l];
            F[DIM + DIM * DIM + i] = Rb[i][l];
          }
          F[NFQ - 1] = tau[l];
        }
        const T* U = F;                      // frozen velocity
        const T* G = F + DIM;                // its gradient, G[i * DIM + j] = d u_i / d x_j
        const T* RB = F + DIM + DIM * DIM;   // frozen strong residual
        const T ta = F[NFQ - 1];             // tau
        T Rl[DIM];
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          T ugu = U[0] * tg[i][0][l], nt = tv[0][l] * G[i * DIM];
#pragma unroll
          for (int d = 1; d < DIM; ++d) {
            ugu = fma(U[d], tg[i][d][l], ugu);       // (ub . grad) du_i
            nt = fma(tv[d][l], G[i * DIM + d], nt);  // (du . grad) ub_i
          }
          const T vci = fma(cmm, tv[i][l], fma(cfc, ugu, cfn * nt));   // Galerkin value coefficient
          c0[i][l] = vci * jxw[l];
          Rl[i] = vci + tr[i][l];                                      // linearised strong residual
        }
        const T sg = jxw[l] * inv_h;
        T dv = tg[0][0][l];
#pragma unroll
        for (int i = 1; i < DIM; ++i) dv += tg[i][i][l];
        const T cst = cfs * ta, csn = cfsn * ta;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          const T st = cst * Rl[i];       // SUPG: tau Rlin_i (ub . grad v_i)
          const T sn = csn * RB[i];       // SUPG, Newton part: tau Rbar_i (du . grad v_i)
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            T a = fma(nu, tg[i][d][l], d == i ? -pval[l] : T(0));
            a = fma(sn, tv[d][l], a);
            a = fma(st, U[d], a);
            cg[i][d][l] = a * sg;
          }
        }
        c0[DIM][l] = div_sign_ * dv * jxw[l];
        const T sp = cfp * ta * sg;            // PSPG: tau Rlin . grad q
#pragma unroll
        for (int d = 0; d < DIM; ++d) cg[DIM][d][l] = sp * Rl[d];
      }
      // Phase 3: integrate the test fields, two per exchange stage
#pragma unroll
      for (int i0 = 0; i0 <= DIM; i0 += 2) {
        constexpr int F2 = 2;
        T c0p[F2][Q], cgp[F2][DIM][Q], rp2[F2][Q];
#pragma unroll
        for (int f = 0; f < F2; ++f)
#pragma unroll
          for (int l = 0; l < Q; ++l) {
            const int i = i0 + f <= DIM ? i0 + f : DIM;
            c0p[f][l] = c0[i][l];
#pragma unroll
            for (int d = 0; d < DIM; ++d) cgp[f][d][l] = cg[i][d][l];
          }
        integrate_multi<DIM, Q, F2, T, kXShfl>(c0p, cgp, rp2, buf0, BUF, ti, tj, tab.S, tab.D);
#pragma unroll
        for (int f = 0; f < F2; ++f)
          if (i0 + f <= DIM)
#pragma unroll
            for (int c = 0; c < N; ++c) r[i0 + f][c] = rp2[f][c];
      }
    }

    if (!STRUCT && constrained) {
#pragma unroll
      for (int f = 0; f < NU; ++f) apply_constraints<DIM, N, true, T>(r[f], buf0, mask, ti_n, tj_n, tab.P, own);
      if (Tr::SPLIT_P) apply_constraints<DIM, NP, true, T>(rp, buf0, mask, ti_p, tj_p, tab.Pp, ownp);
    }

    // dst: the previous colour's grid (a programmatic dependency when this is a later colour of
    // the same product) must be complete and visible before dst is read or written
    if (pass == pass_begin) asm volatile("griddepcontrol.wait;\n" ::: "memory");
    if constexpr (NU == 4 && !DEFER && !(kScatterRed && !EPI && sizeof(T) == 4)) {
      if (!DIAG && FQ != 2) {
#pragma unroll
        for (int c = 0; c < N; ++c) {
          // dst holds the partial sums of earlier colours; with the L2 reduction scatter only the
          // nodes this colour completes need them (the fused epilogue adds them in registers)
          const bool rd = own && valid && (!(kScatterRed && sizeof(T) == 4) || ((epi_last >> c) & 1u));
          if constexpr (sizeof(T) == 4) {
            const float4 w = rd ? *reinterpret_cast<const float4*>(dstp + node[c] * 4) : make_float4(0, 0, 0, 0);
            d0[0][c] = w.x; d0[1][c] = w.y; d0[2][c] = w.z; d0[3][c] = w.w;
          } else {
            const double2 w0 = rd ? *reinterpret_cast<const double2*>(dstp + node[c] * 4) : make_double2(0, 0);
            const double2 w1 = rd ? *reinterpret_cast<const double2*>(dstp + node[c] * 4 + 2) : make_double2(0, 0);
            d0[0][c] = w0.x; d0[1][c] = w0.y; d0[2][c] = w1.x; d0[3][c] = w1.y;
          }
        }
      }
    }
    if (DIAG) {
#pragma unroll
      for (int f = 0; f < NU; ++f)
#pragma unroll
        for (int c = 0; c < N; ++c) {
          const int slot = DIM == 3 ? (c * N + tj_n) * N + ti_n : c * N + ti_n;
          if (own && pass == f * NB + slot) dacc[f][c] = r[f][c];
        }
      if (Tr::SPLIT_P) {
#pragma unroll
        for (int c = 0; c < NP; ++c) {
          const int slot = DIM == 3 ? (c * NP + tj_p) * NP + ti_p : c * NP + ti_p;
          if (ownp && pass == NU * NB + slot) daccp[c] = rp[c];
        }
      }
    } else if (valid) {
      // ---- scatter (no other cell of this colour touches these DoFs: reductions or read-modify-write)
      if (own) {
#pragma unroll
        for (int c = 0; c < N; ++c) {
          T* d = dstp + node[c] * NU;
          if (EPI && ((epi_last >> c) & 1u)) {
            // fused epilogue: this colour completes (A src) at the node
            const int64_t o = node[c] * NU;
            const bool cbnd = OP != OP_PMASS && bnd[c];  // velocity entries are identity rows
            if constexpr (NU == 4 && sizeof(T) == 4) {
              const float4 b4 = *reinterpret_cast<const float4*>(args.eb + o);
              const float ax[4] = {d0[0][c] + r[0][c], d0[1][c] + r[1][c], d0[2][c] + r[2][c], d0[3][c] + r[3][c]};
              const float bb[4] = {b4.x, b4.y, b4.z, b4.w};
              float xo[4];
              if (args.epi == 1) {
                const float4 q4 = *reinterpret_cast<const float4*>(args.edinv + o);
                const float4 e4 = *reinterpret_cast<const float4*>(args.ed + o);
                const float qq[4] = {q4.x, q4.y, q4.z, q4.w}, ee[4] = {e4.x, e4.y, e4.z, e4.w};
                float dn[4];
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                  const bool keep = cbnd && f < DIM;
                  dn[f] = keep ? ee[f] : args.ec1 * ee[f] + args.ec2 * qq[f] * (bb[f] - ax[f]);
                }
                // x' = x + d with x read again (a cache hit: the gather read it) rather than held
                // in registers through the cell; identity rows are rewritten by a separate pass
                const float4 x4 = __ldg(reinterpret_cast<const float4*>(srcp + o));
                const float xx[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
                for (int f = 0; f < 4; ++f) xo[f] = xx[f] + dn[f];
                *reinterpret_cast<float4*>(args.ed + o) = make_float4(dn[0], dn[1], dn[2], dn[3]);
              } else {
#pragma unroll
                for (int f = 0; f < 4; ++f) xo[f] = bb[f] - ax[f];
              }
              *reinterpret_cast<float4*>(args.exout + o) = make_float4(xo[0], xo[1], xo[2], xo[3]);
            } else {
#pragma unroll
              for (int f = 0; f < NU; ++f) {
                if (cbnd && f < DIM) continue;
                const T ax = (NU == 4 ? d0[f][c] : d[f]) + r[f][c];
                if (args.epi == 1) {
                  const T dn = args.ec1 * args.ed[o + f] + args.ec2 * args.edinv[o + f] * (args.eb[o + f] - ax);
                  args.ed[o + f] = dn;
                  args.exout[o + f] = srcp[o + f] + dn;
                } else {
                  args.exout[o + f] = args.eb[o + f] - ax;
                }
              }
            }
            continue;
          }
          // uniform meshes: the velocity rows of boundary nodes are the level's constrained (identity)
          // rows, set by the clearing kernel or by a copy after the colours; the colours add zero there
          // (selects, not a branch: every lane of the warp issues the same scatter)
          if constexpr (STRUCT && OP != OP_PMASS) {
#pragma unroll
            for (int f = 0; f < DIM && f < NU; ++f) r[f][c] = bnd[c] ? T(0) : r[f][c];
          }
          if constexpr (DEFER) {
            const int slot = DIM == 3 ? (c * N + tj_n) * N + ti_n : c * N + ti_n;
            T* pc = args.defer + ((size_t)cellpos * NB + slot) * NU;
            if constexpr (NU == 4 && sizeof(T) == 4) {
              *reinterpret_cast<float4*>(pc) = make_float4(r[0][c], r[1][c], r[2][c], r[3][c]);
            } else {
#pragma unroll
              for (int f = 0; f < NU; ++f) pc[f] = r[f][c];
            }
          } else if constexpr (NU == 4 && kScatterRed && sizeof(T) == 4) {
            // the addition done by the L2 (one rounding, as the read-modify-write below)
            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(d), "f"(r[0][c]), "f"(r[1][c]),
                         "f"(r[2][c]), "f"(r[3][c])
                         : "memory");
          } else if constexpr (NU == 4) {
            // dst values loaded after the grid-dependency wait (no other cell of this colour touches them)
            T o[4];
#pragma unroll
            for (int f = 0; f < 4; ++f) o[f] = d0[f][c] + r[f][c];
            if constexpr (sizeof(T) == 4) {
              *reinterpret_cast<float4*>(d) = make_float4(o[0], o[1], o[2], o[3]);
            } else {
              *reinterpret_cast<double2*>(d) = make_double2(o[0], o[1]);
              *reinterpret_cast<double2*>(d + 2) = make_double2(o[2], o[3]);
            }
          } else {
#pragma unroll
            for (int f = 0; f < NU; ++f) scatter_add(d + f, r[f][c]);
          }
        }
      }
      if (Tr::SPLIT_P && ownp) {
#pragma unroll
        for (int c = 0; c < NP; ++c) scatter_add(dstp + p_offset + pnode[c], rp[c]);
      }
    }
  }
  if (DIAG && valid) {
    // only the entries of this block's passes (another block of the same cell owns the others)
    if (own) {
#pragma unroll
      for (int c = 0; c < N; ++c) {
        const int slot = DIM == 3 ? (c * N + tj_n) * N + ti_n : c * N + ti_n;
#pragma unroll
        for (int f = 0; f < NU; ++f) {
          const int ps = f * NB + slot;
          if (ps >= pass_begin && ps < pass_end) dstp[node[c] * NU + f] += dacc[f][c];
        }
      }
    }
    if (Tr::SPLIT_P && ownp) {
#pragma unroll
      for (int c = 0; c < NP; ++c) {
        const int slot = DIM == 3 ? (c * NP + tj_p) * NP + ti_p : c * NP + ti_p;
        const int ps = NU * NB + slot;
        if (ps >= pass_begin && ps < pass_end) dstp[p_offset + pnode[c]] += daccp[c];
      }
    }
  }
}

template <int DIM, int K, int OP, typename T>
constexpr size_t op_smem_bytes(int warps = kOpWarps, bool staged_frozen = false) {
  using TM = Team<DIM, K + 1>;
  const size_t region1 = ((sizeof(T) * (size_t)warps * (TM::CPW + 1) * TM::template stride<T>() + 15) / 16) * 16;
  if (!staged_frozen) return region1;
  const size_t block = sizeof(T) * FrozenPoint<DIM>::template block<T>(K + 1);
  const size_t mbar_bytes = ((size_t)warps * TM::CPW * 8 + 15) / 16 * 16;
  return region1 + mbar_bytes + (size_t)warps * TM::CPW * TM::template stage_stride_bytes<T>(block);
}

}  // namespace mfns
