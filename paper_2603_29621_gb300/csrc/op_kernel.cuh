// Cell-batched, sum-factorised operator evaluation for Q_k quadrilaterals and
// hexahedra (the "matrix-free approach" of Section 1/2).
//
// Per cell:  gather G -> constraints C -> interpolation to the Gauss points ->
// pointwise physics -> integration -> C^T -> scatter S  (the cell-wise
// structure of Eq. 4, applied to the operator itself).
//
// Thread mapping: a "team" of Q^(dim-1) lanes works on one cell, Q = k_u + 1
// Gauss points per direction.  Lane (i, j) owns the column of points
// (i, j, 0..Q-1) (3D) or (i, 0..Q-1) (2D) in registers; contractions along
// x and y go through the team's shared-memory buffers (x by warp shuffles in
// the stabilised kernel), along the last direction they stay in registers.  A
// warp holds floor(32 / team) teams and synchronises with __syncwarp only.
// Gradients use the collocation derivative at the Gauss points (exact, Q = k+1).
//
// Scatter: cells of one colour share no DoF, so each lane's addition into dst
// (an L2 reduction, or a read-modify-write) meets no other; colours run one
// launch after the other, which fixes the summation order (deterministic).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "opkind.hpp"

namespace mfns {

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

template <int OP, int DIM>
struct OpTraits {
  static constexpr int NC = (OP == OP_STOKES_A || OP == OP_VMASS) ? DIM : OP == OP_PMASS ? 1 : DIM + 1;  // components
  static constexpr bool SPLIT_P = OP == OP_STOKES;   // pressure of lower degree in its own block
  static constexpr bool FROZEN = OP == OP_STAB_NS;
  static constexpr int NU = OP == OP_STOKES ? DIM : NC;  // components carried by the main nodes
};

// 1D tables, passed by value (kernel-parameter constant bank, uniform reads).
template <typename T, int Q, int N, int NP>
struct Tables {
  T S[Q][N];        // main-field basis at the Gauss points
  T Sp[Q][NP];      // pressure basis (Taylor--Hood)
  T D[Q][Q];        // collocation derivative at the Gauss points (reference)
  T D2[Q][Q];       // D * D
  T W[Q];           // Gauss weights on [0,1]
  T P[2][N][N];     // hanging-node interpolation to child half h, main field
  T Pp[2][NP][NP];  // same for the pressure degree
};

// Per-problem fields of one colour launch over several problems (structured cells): the
// descriptor table of a multi-problem launch (blocks [first_block, next problem's first_block)).
template <typename T>
struct ProbArgs {
  const T* src;
  T* dst;
  const T* frozen;
  const T* gexp;
  T* fq;
  int64_t color_offset;  // cells of this problem's earlier colours
  int64_t p_offset;
  int64_t first_block;
  int32_t n;
  T h, nu, cm, dt_inv, div_sign;
  T cf[7];
};

template <typename T, int Q, int N, int NP>
struct OpArgs {
  Tables<T, Q, N, NP> tab;
  const T* src;
  T* dst;
  const T* frozen;             // stabilised NS: frozen state, same layout as src
  const T* gexp;               // stabilised NS: explicit BDF history + forcing g (velocity slots), or null
  const int32_t* cell_u;       // indexed: master node per slot, bit 31 = boundary node
  const int32_t* cell_p;       // indexed Taylor--Hood: pressure master per slot
  const int32_t* cell_f;       // indexed stabilised NS: true node per slot (frozen gather)
  const uint32_t* mask;        // indexed: constraint mask per cell
  const T* hcell;              // indexed: edge length per cell
  int32_t cell_begin, cell_end;  // indexed: range of this colour
  int32_t n;                   // structured: cells per direction
  int32_t color;               // structured: parity bits of this colour
  int64_t p_offset;            // Taylor--Hood: first pressure entry
  T h;                         // structured: edge length
  T nu, cm, dt_inv, div_sign;  // physics (cm = alpha / dt, alpha = 3/2 for BDF2 with equal steps)
  T cf[7];                     // term factors: mass conv newton supg supgN pspg strongvisc
  // diagonal mode: compute (C e_m)^T A_cell (C e_m) for every local slot m
  int diag;
  // stabilised NS: frozen quantities at the Gauss points, precomputed (u, grad u, Rbar, tau per
  // point), laid out [cell position][lane][point][NFQ] with cell position = colour offset + index
  T* fq;
  int64_t color_offset;  // structured: cells of the colours before this one
  // several right-hand sides in one launch: blockIdx.y selects src/dst + blockIdx.y * col_stride
  // (0 in diagonal mode, where blockIdx.y splits the unit-vector passes instead)
  int64_t col_stride;
  // fused epilogue, applied to a node by the colour that completes its product (lastc[node] ==
  // colour); dst then only carries partial sums.  epi 1: Chebyshev / Jacobi step
  // ed = ec1 ed + ec2 edinv (eb - A src), exout = src + ed;  epi 2: residual exout = eb - A src.
  // Constrained rows are left to a separate pass (identity rows).
  int epi;
  const uint8_t* lastc;
  const T* eb;
  const T* edinv;
  T* ed;
  T* exout;
  T ec1, ec2;
  // multi-problem launch: descriptor of the problem owning each block
  const ProbArgs<T>* probs;
  const int32_t* block_pid;
  // device word in which a bounded wait that ran out sets bit 0 (or null)
  int* err;
  // deferred product of a uniform level (one launch over every colour, blockIdx.y = colour): each
  // cell's contributions go to defer[(cell position * nodes per cell + slot) * NU + f]; the cells of
  // colour c start at cell position defer_off[c]
  T* defer;
  int64_t defer_off[8];
};

// ------------------------------------------------------------ small helpers
template <typename T> struct V4;
template <> struct V4<float> { using type = float4; };
template <> struct V4<double> { using type = double2; };  // two loads per node

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Scatters whose every destination entry receives one contribution per launch (a colour of a cell
// kernel, the owners of a transfer): the addition is done by the L2 (red.global.add.f32 / .f64:
// one rounding, as a read-modify-write, without the load whose latency the end of a block would
// otherwise wait for).  Measured on the ball-refined 32^3 Stokes mesh: the FP32 apply 1.79e10 ->
// 2.49e10 DoF/s, the FP64 apply 2.49e9 -> 2.57e9 DoF/s.
constexpr bool kScatterRedF32 = true;
template <typename T>
__device__ __forceinline__ void scatter_add(T* p, T v) {
  if constexpr (sizeof(T) == 4)
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
  else
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

// Flags of the hanging-node constraint lines through a slot (see mesh.hpp for the mask layout).
template <int DIM, int N>
struct LineFlags {
  // x-line at (b, c): faces y-,y+,z-,z+ and edges parallel to x
  __device__ static bool x(uint32_t m, int b, int c) {
    bool f = false;
    f |= (b == 0) && (m & (1u << 2));
    f |= (b == N - 1) && (m & (1u << 3));
    if (DIM == 3) {
      f |= (c == 0) && (m & (1u << 4));
      f |= (c == N - 1) && (m & (1u << 5));
      if ((b == 0 || b == N - 1) && (c == 0 || c == N - 1))
        f |= (m >> (6 + 0 + 2 * (c == N - 1) + (b == N - 1))) & 1u;
    }
    return f;
  }
  // y-line at (a, c): faces x-,x+,z-,z+ and edges parallel to y
  __device__ static bool y(uint32_t m, int a, int c) {
    bool f = false;
    f |= (a == 0) && (m & 1u);
    f |= (a == N - 1) && (m & 2u);
    if (DIM == 3) {
      f |= (c == 0) && (m & (1u << 4));
      f |= (c == N - 1) && (m & (1u << 5));
      if ((a == 0 || a == N - 1) && (c == 0 || c == N - 1))
        f |= (m >> (6 + 4 + 2 * (c == N - 1) + (a == N - 1))) & 1u;
    }
    return f;
  }
  // z-line at (a, b): faces x-,x+,y-,y+ and edges parallel to z
  __device__ static bool z(uint32_t m, int a, int b) {
    bool f = false;
    f |= (a == 0) && (m & 1u);
    f |= (a == N - 1) && (m & 2u);
    f |= (b == 0) && (m & 4u);
    f |= (b == N - 1) && (m & 8u);
    if ((a == 0 || a == N - 1) && (b == 0 || b == N - 1))
      f |= (m >> (6 + 8 + 2 * (b == N - 1) + (a == N - 1))) & 1u;
    return f;
  }
};

// Apply C (forward) or C^T (transpose) to one component held as nodal values:
// lane (ti, tj) holds the last-direction line vals[0..N-1] at (a = ti, b = tj)
// (2D: lane ti holds the y-line at a = ti).  `buf` is a team buffer of >= N^DIM.
template <int DIM, int N, bool TRANSPOSE, typename T>
__device__ __forceinline__ void apply_constraints(T (&v)[N], T* buf, uint32_t m, int ti, int tj,
                                                  const T (&P)[2][N][N], bool own) {
  const int hx = (m >> 24) & 1u, hy = (m >> 25) & 1u, hz = (m >> 26) & 1u;
  if constexpr (DIM == 3) {
    if (TRANSPOSE) {  // reverse order: z, y, x with P^T
      if (own && LineFlags<3, N>::z(m, ti, tj)) {
        T o[N];
#pragma unroll
        for (int c = 0; c < N; ++c) {
          T s = 0;
#pragma unroll
          for (int l = 0; l < N; ++l) s += P[hz][l][c] * v[l];
          o[c] = s;
        }
#pragma unroll
        for (int c = 0; c < N; ++c) v[c] = o[c];
      }
    }
    // x and y passes through shared memory
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
      const int dir = TRANSPOSE ? 1 - pass : pass;  // forward: x then y; transpose: y then x
      if (own)
#pragma unroll
        for (int c = 0; c < N; ++c) buf[(c * N + tj) * N + ti] = v[c];
      __syncwarp();
      if (own) {
#pragma unroll
        for (int c = 0; c < N; ++c) {
          if (dir == 0 && LineFlags<3, N>::x(m, tj, c)) {
            T s = 0;
#pragma unroll
            for (int a = 0; a < N; ++a)
              s += (TRANSPOSE ? P[hx][a][ti] : P[hx][ti][a]) * buf[(c * N + tj) * N + a];
            v[c] = s;
          }
          if (dir == 1 && LineFlags<3, N>::y(m, ti, c)) {
            T s = 0;
#pragma unroll
            for (int b = 0; b < N; ++b)
              s += (TRANSPOSE ? P[hy][b][tj] : P[hy][tj][b]) * buf[(c * N + b) * N + ti];
            v[c] = s;
          }
        }
      }
      __syncwarp();
    }
    if (!TRANSPOSE) {
      if (own && LineFlags<3, N>::z(m, ti, tj)) {
        T o[N];
#pragma unroll
        for (int c = 0; c < N; ++c) {
          T s = 0;
#pragma unroll
          for (int l = 0; l < N; ++l) s += P[hz][c][l] * v[l];
          o[c] = s;
        }
#pragma unroll
        for (int c = 0; c < N; ++c) v[c] = o[c];
      }
    }
  } else {
    // 2D: lane ti holds the y-line (a = ti); x-lines at b, y-lines at a
    if (TRANSPOSE) {
      if (own && LineFlags<2, N>::y(m, ti, 0)) {
        T o[N];
#pragma unroll
        for (int c = 0; c < N; ++c) {
          T s = 0;
#pragma unroll
          for (int l = 0; l < N; ++l) s += P[hy][l][c] * v[l];
          o[c] = s;
        }
#pragma unroll
        for (int c = 0; c < N; ++c) v[c] = o[c];
      }
    }
    if (own)
#pragma unroll
      for (int b = 0; b < N; ++b) buf[b * N + ti] = v[b];
    __syncwarp();
    if (own) {
#pragma unroll
      for (int b = 0; b < N; ++b)
        if (LineFlags<2, N>::x(m, b, 0)) {
          T s = 0;
#pragma unroll
          for (int a = 0; a < N; ++a) s += (TRANSPOSE ? P[hx][a][ti] : P[hx][ti][a]) * buf[b * N + a];
          v[b] = s;
        }
    }
    __syncwarp();
    if (!TRANSPOSE) {
      if (own && LineFlags<2, N>::y(m, ti, 0)) {
        T o[N];
#pragma unroll
        for (int c = 0; c < N; ++c) {
          T s = 0;
#pragma unroll
          for (int l = 0; l < N; ++l) s += P[hy][c][l] * v[l];
          o[c] = s;
        }
#pragma unroll
        for (int c = 0; c < N; ++c) v[c] = o[c];
      }
    }
  }
}

// Values at the lane's Gauss-point column from nodal values (lane (ti,tj) holds
// the nodal line (ti, tj, 0..N-1) when ti, tj < N).
template <int DIM, int Q, int N, typename T>
__device__ __forceinline__ void values(const T (&nod)[N], T (&val)[Q], T* buf, int ti, int tj,
                                       const T (&S)[Q][N]) {
  if constexpr (DIM == 3) {
    // x-stage: t1(i, b, c) = sum_a S(i,a) u(a,b,c); lane (i, b) for b < N
    const bool own = ti < N && tj < N;
    if (own)
#pragma unroll
      for (int c = 0; c < N; ++c) buf[(c * N + tj) * N + ti] = nod[c];
    __syncwarp();
    T t1[N];
#pragma unroll
    for (int c = 0; c < N; ++c) {
      T s = 0;
#pragma unroll
      for (int a = 0; a < N; ++a) s += S[ti][a] * buf[(c * N + (tj < N ? tj : 0)) * N + a];
      t1[c] = s;
    }
    __syncwarp();
    if (tj < N)
#pragma unroll
      for (int c = 0; c < N; ++c) buf[(c * N + tj) * Q + ti] = t1[c];
    __syncwarp();
    // y-stage: t2(i, j, c) = sum_b S(j,b) t1(i,b,c)
    T t2[N];
#pragma unroll
    for (int c = 0; c < N; ++c) {
      T s = 0;
#pragma unroll
      for (int b = 0; b < N; ++b) s += S[tj][b] * buf[(c * N + b) * Q + ti];
      t2[c] = s;
    }
    __syncwarp();
    // z-stage in registers
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      T s = 0;
#pragma unroll
      for (int c = 0; c < N; ++c) s += S[l][c] * t2[c];
      val[l] = s;
    }
  } else {
    const bool own = ti < N;
    if (own)
#pragma unroll
      for (int b = 0; b < N; ++b) buf[b * N + ti] = nod[b];
    __syncwarp();
    T t1[N];
#pragma unroll
    for (int b = 0; b < N; ++b) {
      T s = 0;
#pragma unroll
      for (int a = 0; a < N; ++a) s += S[ti][a] * buf[b * N + a];
      t1[b] = s;
    }
    __syncwarp();
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      T s = 0;
#pragma unroll
      for (int b = 0; b < N; ++b) s += S[l][b] * t1[b];
      val[l] = s;
    }
  }
}

// Reference first (and optionally second) derivatives at the lane's column from values.
template <int DIM, int Q, bool SECOND, typename T>
__device__ __forceinline__ void derivatives(const T (&val)[Q], T (&g)[DIM][Q], T (&h2)[DIM][Q], T* buf, int ti,
                                            int tj, const T (&D)[Q][Q], const T (&D2)[Q][Q]) {
  if constexpr (DIM == 3) {
#pragma unroll
    for (int l = 0; l < Q; ++l) buf[(l * Q + tj) * Q + ti] = val[l];
    __syncwarp();
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      T sx = 0, sy = 0, sxx = 0, syy = 0;
#pragma unroll
      for (int r = 0; r < Q; ++r) {
        const T vx = buf[(l * Q + tj) * Q + r];
        const T vy = buf[(l * Q + r) * Q + ti];
        sx += D[ti][r] * vx;
        sy += D[tj][r] * vy;
        if (SECOND) {
          sxx += D2[ti][r] * vx;
          syy += D2[tj][r] * vy;
        }
      }
      g[0][l] = sx;
      g[1][l] = sy;
      if (SECOND) {
        h2[0][l] = sxx;
        h2[1][l] = syy;
      }
      T sz = 0, szz = 0;
#pragma unroll
      for (int r = 0; r < Q; ++r) {
        sz += D[l][r] * val[r];
        if (SECOND) szz += D2[l][r] * val[r];
      }
      g[2][l] = sz;
      if (SECOND) h2[2][l] = szz;
    }
    __syncwarp();
  } else {
#pragma unroll
    for (int l = 0; l < Q; ++l) buf[l * Q + ti] = val[l];
    __syncwarp();
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      T sx = 0, sxx = 0;
#pragma unroll
      for (int r = 0; r < Q; ++r) {
        const T vx = buf[l * Q + r];
        sx += D[ti][r] * vx;
        if (SECOND) sxx += D2[ti][r] * vx;
      }
      g[0][l] = sx;
      if (SECOND) h2[0][l] = sxx;
      T sy = 0, syy = 0;
#pragma unroll
      for (int r = 0; r < Q; ++r) {
        sy += D[l][r] * val[r];
        if (SECOND) syy += D2[l][r] * val[r];
      }
      g[1][l] = sy;
      if (SECOND) h2[1][l] = syy;
    }
    __syncwarp();
  }
}

// Integration of one test component: c0 (value) and cg (reference-gradient)
// coefficients at the lane's column -> nodal contributions r (lane (ti,tj), ti,tj<N).
template <int DIM, int Q, int N, bool HAS_VAL, bool HAS_GRAD, typename T>
__device__ __forceinline__ void integrate(const T (&c0)[Q], const T (&cg)[DIM][Q], T (&r)[N], T* bufA, T* bufB,
                                          int ti, int tj, const T (&S)[Q][N], const T (&D)[Q][Q]) {
  T w[Q];
  if constexpr (DIM == 3) {
    if (HAS_GRAD) {
#pragma unroll
      for (int l = 0; l < Q; ++l) {
        bufA[(l * Q + tj) * Q + ti] = cg[0][l];
        bufB[(l * Q + tj) * Q + ti] = cg[1][l];
      }
      __syncwarp();
    }
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      T s = HAS_VAL ? c0[l] : T(0);
      if (HAS_GRAD) {
#pragma unroll
        for (int rr = 0; rr < Q; ++rr) {
          s += D[rr][ti] * bufA[(l * Q + tj) * Q + rr];
          s += D[rr][tj] * bufB[(l * Q + rr) * Q + ti];
          s += D[rr][l] * cg[2][rr];
        }
      }
      w[l] = s;
    }
    // z^T in registers
    T t2[N];
#pragma unroll
    for (int c = 0; c < N; ++c) {
      T s = 0;
#pragma unroll
      for (int l = 0; l < Q; ++l) s += S[l][c] * w[l];
      t2[c] = s;
    }
    __syncwarp();
#pragma unroll
    for (int c = 0; c < N; ++c) bufA[(c * Q + tj) * Q + ti] = t2[c];
    __syncwarp();
    // y^T: t1(i, b, c) = sum_j S(j, b) t2(i, j, c), lane (i, b) with b < N
    T t1[N];
    const int bb = tj < N ? tj : 0;
#pragma unroll
    for (int c = 0; c < N; ++c) {
      T s = 0;
#pragma unroll
      for (int j = 0; j < Q; ++j) s += S[j][bb] * bufA[(c * Q + j) * Q + ti];
      t1[c] = s;
    }
    if (tj < N)
#pragma unroll
      for (int c = 0; c < N; ++c) bufB[(c * N + tj) * Q + ti] = t1[c];
    __syncwarp();
    // x^T: r(a, b, c) = sum_i S(i, a) t1(i, b, c), lane (a, b) with a, b < N
    const int aa = ti < N ? ti : 0;
#pragma unroll
    for (int c = 0; c < N; ++c) {
      T s = 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) s += S[i][aa] * bufB[(c * N + bb) * Q + i];
      r[c] = s;
    }
    __syncwarp();
  } else {
    if (HAS_GRAD) {
#pragma unroll
      for (int l = 0; l < Q; ++l) bufA[l * Q + ti] = cg[0][l];
      __syncwarp();
    }
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      T s = HAS_VAL ? c0[l] : T(0);
      if (HAS_GRAD) {
#pragma unroll
        for (int rr = 0; rr < Q; ++rr) {
          s += D[rr][ti] * bufA[l * Q + rr];
          s += D[rr][l] * cg[1][rr];
        }
      }
      w[l] = s;
    }
    T t1[N];
#pragma unroll
    for (int b = 0; b < N; ++b) {
      T s = 0;
#pragma unroll
      for (int l = 0; l < Q; ++l) s += S[l][b] * w[l];
      t1[b] = s;
    }
    __syncwarp();
#pragma unroll
    for (int b = 0; b < N; ++b) bufA[b * Q + ti] = t1[b];
    __syncwarp();
    const int aa = ti < N ? ti : 0;
#pragma unroll
    for (int b = 0; b < N; ++b) {
      T s = 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) s += S[i][aa] * bufA[b * Q + i];
      r[b] = s;
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------ several fields per exchange
// The same contractions for F fields at once: every shared-memory stage writes the F fields into
// F team buffers (stride BUF elements from buf), synchronises the warp once and reads them back,
// so the F fields' loads are independent and in flight together (the single-field versions
// synchronise per field).  Arithmetic per field is that of values / derivatives / integrate.

// Values at the lane's Gauss-point column of F fields (3D or 2D; N = Q: the nodal and the point
// grid have the same size).
// XS (3D): the x-direction exchanges go through warp shuffles instead of shared memory (the Q
// lanes of an x-row of a team are adjacent lanes: lane - ti + a holds column a of the row).
template <int DIM, int Q, int F, typename T, bool XS = false>
__device__ __forceinline__ void values_multi(const T (&nod)[F][Q], T (&val)[F][Q], T* buf, int BUF, int ti,
                                             int tj, const T (&S)[Q][Q]) {
  if constexpr (DIM == 3) {
    T t1[F][Q];
    if constexpr (XS) {
      const int row = lane_id() - ti;
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int c = 0; c < Q; ++c) {
          T s = 0;
#pragma unroll
          for (int a = 0; a < Q; ++a) s += S[ti][a] * __shfl_sync(0xffffffffu, nod[f][c], row + a);
          t1[f][c] = s;
        }
    } else {
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int c = 0; c < Q; ++c) buf[f * BUF + (c * Q + tj) * Q + ti] = nod[f][c];
      __syncwarp();
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int c = 0; c < Q; ++c) {
          T s = 0;
#pragma unroll
          for (int a = 0; a < Q; ++a) s += S[ti][a] * buf[f * BUF + (c * Q + tj) * Q + a];
          t1[f][c] = s;
        }
      __syncwarp();
    }
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int c = 0; c < Q; ++c) buf[f * BUF + (c * Q + tj) * Q + ti] = t1[f][c];
    __syncwarp();
    T t2[F][Q];
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int c = 0; c < Q; ++c) {
        T s = 0;
#pragma unroll
        for (int b = 0; b < Q; ++b) s += S[tj][b] * buf[f * BUF + (c * Q + b) * Q + ti];
        t2[f][c] = s;
      }
    __syncwarp();
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int l = 0; l < Q; ++l) {
        T s = 0;
#pragma unroll
        for (int c = 0; c < Q; ++c) s += S[l][c] * t2[f][c];
        val[f][l] = s;
      }
  } else {
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int b = 0; b < Q; ++b) buf[f * BUF + b * Q + ti] = nod[f][b];
    __syncwarp();
    T t1[F][Q];
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int b = 0; b < Q; ++b) {
        T s = 0;
#pragma unroll
        for (int a = 0; a < Q; ++a) s += S[ti][a] * buf[f * BUF + b * Q + a];
        t1[f][b] = s;
      }
    __syncwarp();
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int l = 0; l < Q; ++l) {
        T s = 0;
#pragma unroll
        for (int b = 0; b < Q; ++b) s += S[l][b] * t1[f][b];
        val[f][l] = s;
      }
  }
}

// Reference first derivatives of F fields and, for the first F2 of them, the diagonal of the
// reference Hessian, at the lane's column.
template <int DIM, int Q, int F, int F2, typename T, bool XS = false>
__device__ __forceinline__ void derivatives_multi(const T (&val)[F][Q], T (&g)[F][DIM][Q], T (&h2)[F][DIM][Q],
                                                  T* buf, int BUF, int ti, int tj, const T (&D)[Q][Q],
                                                  const T (&D2)[Q][Q]) {
  if constexpr (DIM == 3) {
    const int row = lane_id() - ti;
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int l = 0; l < Q; ++l) buf[f * BUF + (l * Q + tj) * Q + ti] = val[f][l];
    __syncwarp();
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int l = 0; l < Q; ++l) {
        T sx = 0, sy = 0, sxx = 0, syy = 0;
#pragma unroll
        for (int r = 0; r < Q; ++r) {
          const T vx = XS ? __shfl_sync(0xffffffffu, val[f][l], row + r) : buf[f * BUF + (l * Q + tj) * Q + r];
          const T vy = buf[f * BUF + (l * Q + r) * Q + ti];
          sx += D[ti][r] * vx;
          sy += D[tj][r] * vy;
          if (f < F2) {
            sxx += D2[ti][r] * vx;
            syy += D2[tj][r] * vy;
          }
        }
        g[f][0][l] = sx;
        g[f][1][l] = sy;
        h2[f][0][l] = sxx;
        h2[f][1][l] = syy;
        T sz = 0, szz = 0;
#pragma unroll
        for (int r = 0; r < Q; ++r) {
          sz += D[l][r] * val[f][r];
          if (f < F2) szz += D2[l][r] * val[f][r];
        }
        g[f][2][l] = sz;
        h2[f][2][l] = szz;
      }
    __syncwarp();
  } else {
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int l = 0; l < Q; ++l) buf[f * BUF + l * Q + ti] = val[f][l];
    __syncwarp();
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int l = 0; l < Q; ++l) {
        T sx = 0, sxx = 0;
#pragma unroll
        for (int r = 0; r < Q; ++r) {
          const T vx = buf[f * BUF + l * Q + r];
          sx += D[ti][r] * vx;
          if (f < F2) sxx += D2[ti][r] * vx;
        }
        g[f][0][l] = sx;
        h2[f][0][l] = sxx;
        T sy = 0, syy = 0;
#pragma unroll
        for (int r = 0; r < Q; ++r) {
          sy += D[l][r] * val[f][r];
          if (f < F2) syy += D2[l][r] * val[f][r];
        }
        g[f][1][l] = sy;
        h2[f][1][l] = syy;
      }
    __syncwarp();
  }
}

// Integration of F test fields, each with a value (c0) and a reference-gradient (cg) coefficient:
// nodal contributions r (lane (ti, tj)); buf holds 2 F team buffers.
template <int DIM, int Q, int F, typename T, bool XS = false>
__device__ __forceinline__ void integrate_multi(const T (&c0)[F][Q], const T (&cg)[F][DIM][Q], T (&r)[F][Q], T* buf,
                                                int BUF, int ti, int tj, const T (&S)[Q][Q], const T (&D)[Q][Q]) {
  T w[F][Q];
  if constexpr (DIM == 3) {
    const int row = lane_id() - ti;
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int l = 0; l < Q; ++l) {
        if (!XS) buf[(2 * f) * BUF + (l * Q + tj) * Q + ti] = cg[f][0][l];
        buf[(2 * f + 1) * BUF + (l * Q + tj) * Q + ti] = cg[f][1][l];
      }
    __syncwarp();
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int l = 0; l < Q; ++l) {
        T s = c0[f][l];
#pragma unroll
        for (int rr = 0; rr < Q; ++rr) {
          s += D[rr][ti] * (XS ? __shfl_sync(0xffffffffu, cg[f][0][l], row + rr)
                               : buf[(2 * f) * BUF + (l * Q + tj) * Q + rr]);
          s += D[rr][tj] * buf[(2 * f + 1) * BUF + (l * Q + rr) * Q + ti];
          s += D[rr][l] * cg[f][2][rr];
        }
        w[f][l] = s;
      }
    T t2[F][Q];
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int c = 0; c < Q; ++c) {
        T s = 0;
#pragma unroll
        for (int l = 0; l < Q; ++l) s += S[l][c] * w[f][l];
        t2[f][c] = s;
      }
    if (!XS) __syncwarp();  // with XS nothing read buffer 2f in the gradient stage
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int c = 0; c < Q; ++c) buf[(2 * f) * BUF + (c * Q + tj) * Q + ti] = t2[f][c];
    __syncwarp();
    T t1[F][Q];
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int c = 0; c < Q; ++c) {
        T s = 0;
#pragma unroll
        for (int j = 0; j < Q; ++j) s += S[j][tj] * buf[(2 * f) * BUF + (c * Q + j) * Q + ti];
        t1[f][c] = s;
      }
    if constexpr (XS) {
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int c = 0; c < Q; ++c) {
          T s = 0;
#pragma unroll
          for (int i = 0; i < Q; ++i) s += S[i][ti] * __shfl_sync(0xffffffffu, t1[f][c], row + i);
          r[f][c] = s;
        }
    } else {
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int c = 0; c < Q; ++c) buf[(2 * f + 1) * BUF + (c * Q + tj) * Q + ti] = t1[f][c];
      __syncwarp();
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int c = 0; c < Q; ++c) {
          T s = 0;
#pragma unroll
          for (int i = 0; i < Q; ++i) s += S[i][ti] * buf[(2 * f + 1) * BUF + (c * Q + tj) * Q + i];
          r[f][c] = s;
        }
    }
    __syncwarp();
  } else {
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int l = 0; l < Q; ++l) buf[(2 * f) * BUF + l * Q + ti] = cg[f][0][l];
    __syncwarp();
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int l = 0; l < Q; ++l) {
        T s = c0[f][l];
#pragma unroll
        for (int rr = 0; rr < Q; ++rr) {
          s += D[rr][ti] * buf[(2 * f) * BUF + l * Q + rr];
          s += D[rr][l] * cg[f][1][rr];
        }
        w[f][l] = s;
      }
    T t1[F][Q];
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int b = 0; b < Q; ++b) {
        T s = 0;
#pragma unroll
        for (int l = 0; l < Q; ++l) s += S[l][b] * w[f][l];
        t1[f][b] = s;
      }
    __syncwarp();
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int b = 0; b < Q; ++b) buf[(2 * f + 1) * BUF + b * Q + ti] = t1[f][b];
    __syncwarp();
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int b = 0; b < Q; ++b) {
        T s = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) s += S[i][ti] * buf[(2 * f + 1) * BUF + b * Q + i];
        r[f][b] = s;
      }
    __syncwarp();
  }
}

}  // namespace mfns
