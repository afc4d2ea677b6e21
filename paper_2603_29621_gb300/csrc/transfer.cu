// Intergrid transfers, Eq. 4:  x_f = sum_e S_e W_e P_e C_e G_e x_c.
//
// One team per coarse cell (coarse colour order).  Prolongation gathers the
// coarse nodal values (G), resolves the coarse hanging-node constraints and
// Dirichlet zeros (C), interpolates to every child (P: h-refinement uses the
// 1D child-half matrices, p-refinement the degree-change matrix) and adds the
// values to the fine vector.  The weighting W is 0/1: every fine node is
// written by exactly one (coarse cell, child, slot) -- its owner -- and never
// when it is constrained in the fine space, so the fine vector receives the
// coarse finite-element function at its free nodes.  Restriction is the exact
// transpose; its scatter into the coarse vector follows the coarse colours.
#include <algorithm>
#include <cstdlib>
#include <map>
#include <numeric>
#include <cstring>
#include <unordered_map>

#include "op_kernel.cuh"
#include "problem.hpp"
#include "vec.hpp"

namespace mfns {

template <typename T, int NF, int NC>
struct TransferTabs {
  T E[2][NF][NC];   // h: child half 0/1; p: E[0] = degree change
  T Pc[2][NC][NC];  // coarse hanging-node interpolation
};

template <typename T, int NF, int NC>
struct TransferArgs {
  TransferTabs<T, NF, NC> tab;
  const T* src;
  T* dst;
  const int32_t* cu;          // coarse: master | boundary bit (colour order)
  const uint32_t* cmask;      // coarse masks
  const int32_t* child_cell;  // per coarse cell (colour order) 2^dim fine cell positions (colour order of fine)
  const uint8_t* child_code;  // child bits, 8 = same cell (identity / p-transfer)
  const int32_t* fnodes;      // fine true node per slot: bit 31 skip, bit 30 boundary
  int32_t cell_begin, cell_end;
  int hkind;
};

// out = (Mz x My x Mx) in, matrices per direction selected by `sel` (0/1 half, 2 identity).
// in: lane (ti, tj) < NI holds the last-direction line; out: lane < NO.
template <int DIM, int NI, int NO, bool TR, typename T, typename Mat>
__device__ __forceinline__ void tensor_apply(const T (&in)[NI], T (&out)[NO], T* buf, int ti, int tj,
                                             const Mat& M, const int (&sel)[3]) {
  // M(d, sel, row, col) with row in [0, NF), col in [0, NC); forward maps NC->NF, TR maps NF->NC
  auto m = [&](int d, int r, int c) -> T {
    if (sel[d] == 2) return r == c ? T(1) : T(0);
    return TR ? M(sel[d], c, r) : M(sel[d], r, c);
  };
  constexpr int L = NI > NO ? NI : NO;
  if constexpr (DIM == 3) {
    // x-stage: s1(i, b, c) = sum_a m_x(i, a) in(a, b, c), lane (i, b) with b < NI
    if (ti < NI && tj < NI)
#pragma unroll
      for (int c = 0; c < NI; ++c) buf[(c * NI + tj) * NI + ti] = in[c];
    __syncwarp();
    T s1[NI];
    const int bb = tj < NI ? tj : 0;
#pragma unroll
    for (int c = 0; c < NI; ++c) {
      T s = 0;
#pragma unroll
      for (int a = 0; a < NI; ++a) s += m(0, ti < NO ? ti : 0, a) * buf[(c * NI + bb) * NI + a];
      s1[c] = s;
    }
    __syncwarp();
    if (ti < NO && tj < NI)
#pragma unroll
      for (int c = 0; c < NI; ++c) buf[(c * NI + tj) * L + ti] = s1[c];
    __syncwarp();
    // y-stage: s2(i, j, c) = sum_b m_y(j, b) s1(i, b, c), lane (i, j) < NO
    T s2[NI];
#pragma unroll
    for (int c = 0; c < NI; ++c) {
      T s = 0;
#pragma unroll
      for (int b = 0; b < NI; ++b) s += m(1, tj < NO ? tj : 0, b) * buf[(c * NI + b) * L + (ti < NO ? ti : 0)];
      s2[c] = s;
    }
    __syncwarp();
#pragma unroll
    for (int l = 0; l < NO; ++l) {
      T s = 0;
#pragma unroll
      for (int c = 0; c < NI; ++c) s += m(2, l, c) * s2[c];
      out[l] = s;
    }
  } else {
    if (ti < NI)
#pragma unroll
      for (int b = 0; b < NI; ++b) buf[b * NI + ti] = in[b];
    __syncwarp();
    T s1[NI];
#pragma unroll
    for (int b = 0; b < NI; ++b) {
      T s = 0;
#pragma unroll
      for (int a = 0; a < NI; ++a) s += m(0, ti < NO ? ti : 0, a) * buf[b * NI + a];
      s1[b] = s;
    }
    __syncwarp();
#pragma unroll
    for (int l = 0; l < NO; ++l) {
      T s = 0;
#pragma unroll
      for (int b = 0; b < NI; ++b) s += m(1, l, b) * s1[b];
      out[l] = s;
    }
  }
}

template <int DIM, int NF, int NC, int NCOMP, int NVEL, typename T, bool RESTRICT>
__global__ void __launch_bounds__(128) transfer_kernel(const TransferArgs<T, NF, NC> a) {
  constexpr int TPC = ipow(NF, DIM - 1);
  constexpr int CPW = 32 / TPC;
  constexpr int BUF = ipow(NF, DIM);
  constexpr int NBC = ipow(NC, DIM), NBF = ipow(NF, DIM);
  constexpr int NCH = 1 << DIM;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  int team = lane / TPC;
  const int tid = lane % TPC;
  const bool lane_active = team < CPW;
  if (!lane_active) team = CPW;
  const int ti = tid % NF, tj = DIM == 3 ? tid / NF : 0;
  T* buf = smem + (size_t)(warp * (CPW + 1) + team) * BUF;
  const int64_t t = (int64_t)blockIdx.x * (4 * CPW) + warp * CPW + (lane_active ? team : 0);
  const int64_t c0 = a.cell_begin + t;
  const bool valid = lane_active && c0 < a.cell_end;
  const int64_t cell = c0 < a.cell_end ? c0 : a.cell_end - 1;
  const uint32_t mask = a.cmask[cell];
  // warp-uniform control flow around every __syncwarp: constraint path if any team needs it,
  // and the child loop runs to the largest child count of the warp (absent children write nothing)
  const bool constrained = __any_sync(0xffffffffu, (mask & 0x3FFFFu) != 0);
  int my_nch = 0;
  for (int ch = 0; ch < NCH; ++ch) my_nch += a.child_cell[cell * NCH + ch] >= 0 ? 1 : 0;
  const int nch_warp = __reduce_max_sync(0xffffffffu, my_nch);
  const bool ownc = ti < NC && tj < NC;
  const bool ownf = ti < NF && tj < NF;
  const int tic = ti < NC ? ti : 0, tjc = tj < NC ? tj : 0;
  auto E = [&](int s, int r, int c) -> T { return a.tab.E[s][r][c]; };

  // coarse slot ids (colour-ordered coarse cell)
  int32_t cid[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int slot = DIM == 3 ? (c * NC + tjc) * NC + tic : c * NC + tic;
    cid[c] = a.cu[cell * NBC + slot];
  }
  if (!RESTRICT) {
    T u[NCOMP][NC];
#pragma unroll
    for (int f = 0; f < NCOMP; ++f)
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int32_t v = cid[c];
        const bool bnd = v < 0;
        T x = ownc ? a.src[(int64_t)(v & 0x7fffffff) * NCOMP + f] : T(0);
        if (bnd && f < NVEL) x = 0;
        u[f][c] = x;
      }
    if (constrained)
#pragma unroll
      for (int f = 0; f < NCOMP; ++f) apply_constraints<DIM, NC, false, T>(u[f], buf, mask, tic, tjc, a.tab.Pc, ownc);
    for (int ch = 0; ch < nch_warp; ++ch) {
      const int32_t fc = a.child_cell[cell * NCH + ch];
      const bool has = fc >= 0;
      const int code = has ? a.child_code[cell * NCH + ch] : 8;
      int sel[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) sel[d] = code == 8 ? (a.hkind ? 2 : 0) : (code >> d) & 1;
#pragma unroll
      for (int f = 0; f < NCOMP; ++f) {
        T o[NF];
        tensor_apply<DIM, NC, NF, false, T>(u[f], o, buf, ti, tj, E, sel);
        if (valid && ownf && has) {
#pragma unroll
          for (int c = 0; c < NF; ++c) {
            const int slot = DIM == 3 ? (c * NF + tj) * NF + ti : c * NF + ti;
            const int32_t v = a.fnodes[(int64_t)fc * NBF + slot];
            if (v < 0) continue;                 // not the owner, or a hanging fine node
            if ((v & 0x40000000) && f < NVEL) continue;  // Dirichlet fine entry
            scatter_add(a.dst + (int64_t)(v & 0x3fffffff) * NCOMP + f, o[c]);
          }
        }
      }
    }
  } else {
    T acc[NCOMP][NC];
#pragma unroll
    for (int f = 0; f < NCOMP; ++f)
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[f][c] = 0;
    for (int ch = 0; ch < nch_warp; ++ch) {
      const int32_t fc = a.child_cell[cell * NCH + ch];
      const bool has = fc >= 0;
      const int code = has ? a.child_code[cell * NCH + ch] : 8;
      int sel[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) sel[d] = code == 8 ? (a.hkind ? 2 : 0) : (code >> d) & 1;
#pragma unroll
      for (int f = 0; f < NCOMP; ++f) {
        T in[NF];
#pragma unroll
        for (int c = 0; c < NF; ++c) {
          const int slot = DIM == 3 ? (c * NF + (tj < NF ? tj : 0)) * NF + (ti < NF ? ti : 0) : c * NF + (ti < NF ? ti : 0);
          const int32_t v = has ? a.fnodes[(int64_t)fc * NBF + slot] : int32_t(0x80000000u);
          const bool skip = !ownf || v < 0 || ((v & 0x40000000) && f < NVEL);
          in[c] = skip ? T(0) : a.src[(int64_t)(v & 0x3fffffff) * NCOMP + f];
        }
        T o[NC];
        tensor_apply<DIM, NF, NC, true, T>(in, o, buf, ti, tj, E, sel);
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[f][c] += o[c];
      }
    }
    if (constrained)
#pragma unroll
      for (int f = 0; f < NCOMP; ++f) apply_constraints<DIM, NC, true, T>(acc[f], buf, mask, tic, tjc, a.tab.Pc, ownc);
    if (valid && ownc) {
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int f = 0; f < NCOMP; ++f) scatter_add(a.dst + (int64_t)(cid[c] & 0x7fffffff) * NCOMP + f, acc[f][c]);
    }
  }
}

// ------------------------------------------------------------------------ host side
void build_transfer(Transfer& t, const OpLevel& fine, const OpLevel& coarse, Budget* bud, bool allow_unrefined) {
  const int dim = fine.dim;
  if (!allow_unrefined && build_separable(t.sep, fine, coarse, bud)) {  // uniform -> uniform: tensor-product stencils
    t.separable = true;
    t.dim = dim;
    t.kf = fine.k;
    t.kc = coarse.k;
    t.ncomp = fine.NU;
    t.hkind = fine.k == coarse.k;
    return;
  }
  t.dim = dim;
  t.kf = fine.k;
  t.kc = coarse.k;
  t.ncomp = fine.NU;
  t.hkind = fine.k == coarse.k;
  if (!t.hkind && (fine.forest.n_cells() != coarse.forest.n_cells() || fine.k <= coarse.k))
    throw Error(kErrArg, "p-transfer needs the same mesh and a lower coarse degree");
  const int NF = fine.k + 1, NC = coarse.k + 1;
  const int NBF = fine.nu.nb;
  const int nch = 1 << dim;
  const Forest& ff = fine.forest;
  const Forest& fc = coarse.forest;
  const size_t ncc = fc.n_cells(), ncf = ff.n_cells();
  t.n_coarse_cells = ncc;
  t.color_ptr = coarse.L.color_ptr;
  // fine cell id -> colour-order position
  std::vector<int32_t> fpos(ncf);
  for (size_t i = 0; i < ncf; ++i) fpos[fine.perm[i]] = (int32_t)i;
  // locate fine cells of every coarse cell
  std::vector<int32_t> child(ncc * nch, -1);
  std::vector<uint8_t> code(ncc * nch, 0);
  if (!t.hkind) {
    for (size_t i = 0; i < ncc; ++i) {
      child[i * nch] = fpos[coarse.perm[i]];  // same forest, same cell ids
      code[i * nch] = 8;
    }
  } else {
    // map (level, coords) of fine cells; coarse cell = same cell or parent of 2^dim children
    const bool uniform_step = ff.uniform() && fc.uniform() && ff.n == 2 * fc.n;
    std::unordered_map<int64_t, int32_t> fmap;
    auto key = [](int l, int64_t x, int64_t y, int64_t z) { return (((int64_t)l * 4096 + z) * 4096 + y) * 4096 + x; };
    for (size_t c = 0; c < ncf; ++c)
      fmap[key(uniform_step ? 0 : ff.lev[c], ff.crd[3 * c], ff.crd[3 * c + 1], ff.crd[3 * c + 2])] = (int32_t)c;
    for (size_t i = 0; i < ncc; ++i) {
      const int32_t c = coarse.perm[i];
      const int l = fc.lev[c];
      const int64_t x = fc.crd[3 * c], y = fc.crd[3 * c + 1], z = fc.crd[3 * c + 2];
      auto same = uniform_step ? fmap.end() : fmap.find(key(l, x, y, z));
      if (same != fmap.end()) {
        child[i * nch] = fpos[same->second];
        code[i * nch] = 8;
        continue;
      }
      for (int ch = 0; ch < nch; ++ch) {
        const int64_t cx = 2 * x + (ch & 1), cy = 2 * y + ((ch >> 1) & 1), cz = dim == 3 ? 2 * z + ((ch >> 2) & 1) : 0;
        auto it = fmap.find(key(uniform_step ? 0 : l + 1, cx, cy, cz));
        if (it == fmap.end() && allow_unrefined && ch == 0) break;  // not refined: no children (-1)
        if (it == fmap.end()) throw Error(kErrArg, "h-transfer: coarse cell neither kept nor refined once");
        child[i * nch + ch] = fpos[it->second];
        code[i * nch + ch] = (uint8_t)ch;
      }
    }
  }
  t.child_cell = upload(bud, child);
  t.child_code = upload(bud, code);
  // owner flags on the fine level (true ids), in fine colour order
  std::vector<char> hangf(fine.nu.n_nodes, 0);
  for (int32_t g : fine.nu.hang_node) hangf[g] = 1;
  std::vector<char> seen(fine.nu.n_nodes, 0);
  std::vector<int32_t> fn(ncf * NBF, int32_t(0x80000000u));
  for (size_t i = 0; i < ncc; ++i)
    for (int ch = 0; ch < nch; ++ch) {
      const int32_t p = child[i * nch + ch];
      if (p < 0) break;
      const int32_t c = fine.perm[p];
      for (int b = 0; b < NBF; ++b) {
        const int32_t g = fine.nu.cell_nodes[(size_t)c * NBF + b];
        int32_t v = g;
        if (fine.op != OP_PMASS && fine.nu.boundary[g]) v |= 0x40000000;
        if (seen[g] || hangf[g]) v |= int32_t(0x80000000u);
        seen[g] = 1;
        fn[(size_t)p * NBF + b] = v;
      }
    }
  const_cast<OpLevel&>(fine).tnodes = upload(bud, fn);
  // 1D matrices
  std::vector<double> xf = gll_nodes(fine.k), xc = gll_nodes(coarse.k);
  t.E.assign(2 * NF * NC, 0.0);
  for (int h = 0; h < 2; ++h)
    for (int s = 0; s < NF; ++s)
      for (int m = 0; m < NC; ++m)
        t.E[(h * NF + s) * NC + m] = t.hkind ? lagrange(xc, m, 0.5 * (h + xf[s])) : lagrange(xc, m, xf[s]);
  t.Pc.assign(2 * NC * NC, 0.0);
  for (int h = 0; h < 2; ++h)
    for (int s = 0; s < NC; ++s)
      for (int m = 0; m < NC; ++m) t.Pc[(h * NC + s) * NC + m] = lagrange(xc, m, 0.5 * (h + xc[s]));
}

template <int DIM, int NF, int NC, int NCOMP, int NVEL, typename T>
static void launch_transfer(const Transfer& t, const OpLevel& fine, const OpLevel& coarse, const T* src, T* dst,
                            bool restrict_, cudaStream_t s) {
  TransferArgs<T, NF, NC> a{};
  for (int h = 0; h < 2; ++h) {
    for (int r = 0; r < NF; ++r)
      for (int c = 0; c < NC; ++c) a.tab.E[h][r][c] = (T)t.E[(h * NF + r) * NC + c];
    for (int r = 0; r < NC; ++r)
      for (int c = 0; c < NC; ++c) a.tab.Pc[h][r][c] = (T)t.Pc[(h * NC + r) * NC + c];
  }
  a.src = src;
  a.dst = dst;
  a.cu = coarse.cell_u.as<int32_t>();
  a.cmask = coarse.mask.as<uint32_t>();
  a.child_cell = t.child_cell.as<int32_t>();
  a.child_code = t.child_code.as<uint8_t>();
  a.fnodes = fine.tnodes.as<int32_t>();
  a.hkind = t.hkind;
  constexpr int TPC = ipow(NF, DIM - 1), CPW = 32 / TPC;
  const size_t smem = sizeof(T) * 4 * (CPW + 1) * ipow(NF, DIM);
  if (!restrict_) {
    // prolongation: no conflicts (owner writes), one launch over all coarse cells
    a.cell_begin = 0;
    a.cell_end = (int32_t)t.n_coarse_cells;
    const unsigned grid = (unsigned)((t.n_coarse_cells + 4 * CPW - 1) / (4 * CPW));
    if (grid) transfer_kernel<DIM, NF, NC, NCOMP, NVEL, T, false><<<grid, 128, smem, s>>>(a);
    MFNS_CUDA(cudaGetLastError());
    return;
  }
  for (size_t c = 0; c + 1 < t.color_ptr.size(); ++c) {
    a.cell_begin = t.color_ptr[c];
    a.cell_end = t.color_ptr[c + 1];
    const int64_t n = a.cell_end - a.cell_begin;
    if (n <= 0) continue;
    const unsigned grid = (unsigned)((n + 4 * CPW - 1) / (4 * CPW));
    transfer_kernel<DIM, NF, NC, NCOMP, NVEL, T, true><<<grid, 128, smem, s>>>(a);
    MFNS_CUDA(cudaGetLastError());
  }
}

template <typename T>
static void dispatch_transfer(const Transfer& t, const OpLevel& fine, const OpLevel& coarse, const T* src, T* dst,
                              bool restrict_, cudaStream_t s) {
  const int d = t.dim, nf = t.kf + 1, nc = t.kc + 1, ncomp = t.ncomp;
  const int nvel = fine.op == OP_PMASS ? 0 : d;
#define TCASE(DIM, NF, NC, NCOMP)                                                                  \
  if (d == DIM && nf == NF && nc == NC && ncomp == NCOMP)                                          \
    return launch_transfer<DIM, NF, NC, NCOMP, (NCOMP == 1 ? 0 : DIM), T>(t, fine, coarse, src, dst, restrict_, s);
  (void)nvel;
  // h-transfers (same degree) for the vector Laplacian (dim comps) and stabilised NS (dim+1)
  TCASE(3, 2, 2, 3) TCASE(3, 3, 3, 3) TCASE(3, 4, 4, 3) TCASE(3, 5, 5, 3)
  TCASE(3, 2, 2, 4) TCASE(3, 3, 3, 4) TCASE(3, 4, 4, 4)
  TCASE(2, 2, 2, 2) TCASE(2, 3, 3, 2) TCASE(2, 4, 4, 2) TCASE(2, 5, 5, 2)
  TCASE(2, 2, 2, 3) TCASE(2, 3, 3, 3) TCASE(2, 4, 4, 3) TCASE(2, 5, 5, 3)
  // p-transfers (degree k -> k-1 on the same mesh)
  TCASE(3, 3, 2, 3) TCASE(3, 4, 3, 3) TCASE(3, 5, 4, 3)
  TCASE(3, 3, 2, 4) TCASE(3, 4, 3, 4)
  TCASE(2, 3, 2, 2) TCASE(2, 4, 3, 2) TCASE(2, 5, 4, 2)
  TCASE(2, 3, 2, 3) TCASE(2, 4, 3, 3) TCASE(2, 5, 4, 3)
#undef TCASE
  throw Error(kErrUnsupported, "transfer not instantiated for this (dim, degrees, components)");
}

// ---- coarse nodal values of a fine finite-element function (Newton states on refined meshes)
struct GllPair {
  double xf[8], xc[8];
};

__device__ __forceinline__ double lagrange_at(const double* x, int n, int m, double e) {
  double v = 1.0;
  for (int j = 0; j < n; ++j)
    if (j != m) v *= (e - x[j]) / (x[m] - x[j]);
  return v;
}

// One thread per (coarse cell, coarse slot), coarse colour order.  The slot's reference point is
// located in a child of the coarse cell (or the same cell: p-steps, cells kept), the fine function
// is evaluated there from the child's nodal values, and the owner slot of the coarse node writes.
__global__ void k_cell_interpolate(const double* __restrict__ uf, double* __restrict__ uc, int64_t ncc, int dim,
                                   int nf, int ncn, int ncomp, const int32_t* __restrict__ child,
                                   const uint8_t* __restrict__ code, const int32_t* __restrict__ fnodes,
                                   const int32_t* __restrict__ cnodes, int32_t cmask,
                                   const uint8_t* __restrict__ own, GllPair tab) {
  const int nbc = dim == 3 ? ncn * ncn * ncn : ncn * ncn;
  const int nbf = dim == 3 ? nf * nf * nf : nf * nf;
  const int nch = 1 << dim;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ncc * nbc; t += (int64_t)gridDim.x * blockDim.x) {
    if (!own[t]) continue;
    const int64_t i = t / nbc;
    const int slot = (int)(t - i * nbc);
    const int idx[3] = {slot % ncn, (slot / ncn) % ncn, dim == 3 ? slot / (ncn * ncn) : 0};
    double eta[3] = {0.0, 0.0, 0.0};
    int32_t fcell;
    if (code[i * nch] == 8) {
      fcell = child[i * nch];
      for (int d = 0; d < dim; ++d) eta[d] = tab.xc[idx[d]];
    } else {
      int ch = 0;
      for (int d = 0; d < dim; ++d) {
        const double xi = tab.xc[idx[d]];
        const int h = xi > 0.5 ? 1 : 0;  // a node on the mid-plane lies in both halves: take the first
        ch |= h << d;
        eta[d] = 2.0 * xi - h;
      }
      fcell = child[i * nch + ch];
    }
    double phi[3][8];
    for (int d = 0; d < 3; ++d)
      for (int m = 0; m < nf; ++m) phi[d][m] = d < dim ? lagrange_at(tab.xf, nf, m, eta[d]) : (m == 0 ? 1.0 : 0.0);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int fs = 0; fs < nbf; ++fs) {
      const int a = fs % nf, b = (fs / nf) % nf, c = dim == 3 ? fs / (nf * nf) : 0;
      const double w = phi[0][a] * phi[1][b] * phi[2][c];
      const int64_t g = fnodes[(int64_t)fcell * nbf + fs] & 0x3fffffff;
      for (int q = 0; q < ncomp; ++q) acc[q] += w * uf[g * ncomp + q];
    }
    const int64_t gc = cnodes[t] & cmask;
    for (int q = 0; q < ncomp; ++q) uc[gc * ncomp + q] = acc[q];
  }
}

void cell_interpolate(Transfer& t, const OpLevel& fine, const OpLevel& coarse, const double* uf, double* uc,
                      Budget* bud, cudaStream_t s) {
  if (t.separable) return sep_interpolate(t.sep, uf, uc, s);
  const int dim = t.dim, nf = t.kf + 1, ncn = t.kc + 1;
  if (nf > 8 || ncn > 8 || t.ncomp > 4) throw Error(kErrUnsupported, "state interpolation: degree or components");
  const int nbc = coarse.nu.nb;
  const int64_t ncc = (int64_t)coarse.forest.n_cells();
  const bool coarse_f = coarse.cell_f.get() != nullptr;
  if (!t.own_c.get()) {  // owner slot of every coarse node (first occurrence in colour order)
    std::vector<uint8_t> own((size_t)ncc * nbc, 0);
    std::vector<char> seen(coarse.nu.n_nodes, 0);
    for (int64_t i = 0; i < ncc; ++i)
      for (int b = 0; b < nbc; ++b) {
        const int32_t g = coarse.nu.cell_nodes[(size_t)coarse.perm[i] * nbc + b];
        if (!seen[g]) own[(size_t)i * nbc + b] = 1;
        seen[g] = 1;
      }
    t.own_c = upload(bud, own);
  }
  GllPair tab{};
  const std::vector<double> xf = gll_nodes(t.kf), xc = gll_nodes(t.kc);
  for (int m = 0; m < nf; ++m) tab.xf[m] = xf[m];
  for (int m = 0; m < ncn; ++m) tab.xc[m] = xc[m];
  const int64_t work = ncc * nbc;
  const unsigned grid = (unsigned)std::min<int64_t>((work + 255) / 256, 152 * 32);
  if (work > 0)
    k_cell_interpolate<<<grid, 256, 0, s>>>(uf, uc, ncc, dim, nf, ncn, t.ncomp, t.child_cell.as<int32_t>(),
                                            t.child_code.as<uint8_t>(), fine.tnodes.as<int32_t>(),
                                            coarse_f ? coarse.cell_f.as<int32_t>() : coarse.cell_u.as<int32_t>(),
                                            coarse_f ? int32_t(-1) : int32_t(0x7fffffff), t.own_c.as<uint8_t>(), tab);
  MFNS_CUDA(cudaGetLastError());
}

// ---- hp p-transfers: groups of cells with one (fine degree, coarse degree) pair
void build_hp_transfer(Transfer& t, const OpLevel& fine, const OpLevel& coarse, Budget* bud) {
  if (!fine.hp) throw Error(kErrArg, "hp transfer needs an hp fine level");
  const HpSpace& fs = fine.hp->space;
  const Forest& ff = fine.forest;
  const Forest& fc = coarse.forest;
  if (ff.n_cells() != fc.n_cells() || ff.lev != fc.lev || ff.crd != fc.crd)
    throw Error(kErrArg, "hp p-transfer needs the same cells on both levels");
  const int dim = fine.dim, NU = fine.NU, nch = 1 << dim;
  const size_t nc = ff.n_cells();
  // coarse: degree, slot values (node | Dirichlet bit) and constraint masks per cell
  std::vector<int> kc(nc);
  std::vector<uint32_t> cmask(nc, 0u);
  if (coarse.hp) {
    for (size_t c = 0; c < nc; ++c) kc[c] = coarse.hp->space.degree[c];
  } else {
    for (size_t c = 0; c < nc; ++c) kc[c] = coarse.k;
    const Lattice lat = make_lattice(fc);
    cmask = constraint_masks(fc, lat);
  }
  auto coarse_slot = [&](size_t c, int b) -> int32_t {
    int32_t node;
    bool bnd;
    if (coarse.hp) {
      const HpSpace& cs = coarse.hp->space;
      node = cs.cell_nodes[cs.cell_ptr[c] + b];
      bnd = cs.boundary[node];
    } else {
      node = coarse.nu.cell_master[c * coarse.nu.nb + b];
      bnd = coarse.nu.boundary[node];
    }
    return node | (bnd ? int32_t(0x80000000u) : 0);
  };
  // fine owner flags over all cells: bit 31 not the owner or hanging, bit 30 Dirichlet
  std::vector<char> hangf(fs.n_nodes, 0), seen(fs.n_nodes, 0);
  for (int32_t g : fs.hang_node) hangf[g] = 1;
  std::vector<int32_t> fval(fs.cell_nodes.size());
  for (size_t c = 0; c < nc; ++c)
    for (int64_t j = fs.cell_ptr[c]; j < fs.cell_ptr[c + 1]; ++j) {
      const int32_t g = fs.cell_nodes[j];
      int32_t v = g;
      if (fs.boundary[g]) v |= 0x40000000;
      if (seen[g] || hangf[g]) v |= int32_t(0x80000000u);
      seen[g] = 1;
      fval[j] = v;
    }
  std::map<std::pair<int, int>, std::vector<int32_t>> pairs;
  for (size_t c = 0; c < nc; ++c) pairs[{fs.degree[c], kc[c]}].push_back((int32_t)c);
  auto H = std::make_unique<HpTransfer>();
  for (auto& kv : pairs) {
    const int kf = kv.first.first, kcg = kv.first.second;
    const std::vector<int32_t>& cells = kv.second;
    const int NF = kf + 1, NC = kcg + 1;
    const int NBF = dim == 3 ? NF * NF * NF : NF * NF, NBC = dim == 3 ? NC * NC * NC : NC * NC;
    // colours of the coarse scatter: no two cells of a colour write the same coarse entry
    std::map<int32_t, std::vector<int32_t>> node_cells;
    for (int32_t i = 0; i < (int32_t)cells.size(); ++i)
      for (int b = 0; b < NBC; ++b) node_cells[coarse_slot(cells[i], b) & 0x7fffffff].push_back(i);
    std::vector<int32_t> color(cells.size(), -1);
    int ncol = 0;
    for (int32_t i = 0; i < (int32_t)cells.size(); ++i) {
      std::vector<char> used(ncol + 1, 0);
      for (int b = 0; b < NBC; ++b)
        for (int32_t o : node_cells[coarse_slot(cells[i], b) & 0x7fffffff])
          if (color[o] >= 0) used[color[o]] = 1;
      int col = 0;
      while (used[col]) ++col;
      color[i] = col;
      ncol = std::max(ncol, col + 1);
    }
    std::vector<int32_t> order(cells.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return color[a] < color[b]; });
    auto G = std::make_unique<HpTGroup>();
    Transfer& tt = G->t;
    tt.dim = dim;
    tt.kf = kf;
    tt.kc = kcg;
    tt.ncomp = NU;
    tt.hkind = kf == kcg;  // same degree: identity (code 8 with the h tables)
    tt.n_coarse_cells = (int64_t)cells.size();
    tt.color_ptr.assign(ncol + 1, 0);
    std::vector<int32_t> cu(cells.size() * NBC), fn(cells.size() * NBF), child(cells.size() * nch, -1);
    std::vector<uint32_t> mk(cells.size());
    std::vector<uint8_t> code(cells.size() * nch, 0);
    for (size_t i = 0; i < cells.size(); ++i) {
      const int32_t c = cells[order[i]];
      tt.color_ptr[color[order[i]] + 1]++;
      for (int b = 0; b < NBC; ++b) cu[i * NBC + b] = coarse_slot(c, b);
      for (int b = 0; b < NBF; ++b) fn[i * NBF + b] = fval[fs.cell_ptr[c] + b];
      mk[i] = cmask[c];
      child[i * nch] = (int32_t)i;
      code[i * nch] = 8;
    }
    for (int c = 0; c < ncol; ++c) tt.color_ptr[c + 1] += tt.color_ptr[c];
    tt.child_cell = upload(bud, child);
    tt.child_code = upload(bud, code);
    const std::vector<double> xf = gll_nodes(kf), xc = gll_nodes(kcg);
    tt.E.assign(2 * NF * NC, 0.0);
    for (int h = 0; h < 2; ++h)
      for (int r = 0; r < NF; ++r)
        for (int m = 0; m < NC; ++m)
          tt.E[(h * NF + r) * NC + m] = tt.hkind ? lagrange(xc, m, 0.5 * (h + xf[r])) : lagrange(xc, m, xf[r]);
    tt.Pc.assign(2 * NC * NC, 0.0);
    for (int h = 0; h < 2; ++h)
      for (int r = 0; r < NC; ++r)
        for (int m = 0; m < NC; ++m) tt.Pc[(h * NC + r) * NC + m] = lagrange(xc, m, 0.5 * (h + xc[r]));
    for (OpLevel* v : {&G->fine_view, &G->coarse_view}) {
      v->op = OP_STOKES_A;
      v->dim = dim;
      v->NU = NU;
    }
    G->fine_view.k = kf;
    G->coarse_view.k = kcg;
    G->fine_view.tnodes = upload(bud, fn);
    G->coarse_view.cell_u = upload(bud, cu);
    G->coarse_view.mask = upload(bud, mk);
    H->groups.push_back(std::move(G));
  }
  t.dim = dim;
  t.kf = fine.k;
  t.kc = coarse.k;
  t.ncomp = NU;
  t.hkind = false;
  t.hp = std::move(H);
}

void transfer_prolongate_add(const Transfer& t, const OpLevel& fine, const OpLevel& coarse, int prec, const void* xc,
                             void* xf, cudaStream_t s) {
  if (t.hp) {
    const void* src = xc;
    if (coarse.hp) {  // the coarse function at every slot: complete its constrained entries first
      void* tmp = coarse.hp->tmp[prec].get();
      MFNS_CUDA(cudaMemcpyAsync(tmp, xc, coarse.n_dofs * esize(prec), cudaMemcpyDeviceToDevice, s));
      hp_distribute(coarse, prec, tmp, s);
      src = tmp;
    }
    for (auto& g : t.hp->groups)
      if (prec == 0)
        dispatch_transfer<double>(g->t, g->fine_view, g->coarse_view, (const double*)src, (double*)xf, false, s);
      else
        dispatch_transfer<float>(g->t, g->fine_view, g->coarse_view, (const float*)src, (float*)xf, false, s);
    return;
  }
  if (t.separable) return sep_prolongate_add(t.sep, prec, xc, xf, s);
  if (prec == 0)
    dispatch_transfer<double>(t, fine, coarse, (const double*)xc, (double*)xf, false, s);
  else
    dispatch_transfer<float>(t, fine, coarse, (const float*)xc, (float*)xf, false, s);
}

void transfer_restrict(const Transfer& t, const OpLevel& fine, const OpLevel& coarse, int prec, const void* rf,
                       void* rc, cudaStream_t s) {
  if (t.hp) {
    MFNS_CUDA(cudaMemsetAsync(rc, 0, coarse.n_dofs * esize(prec), s));
    for (auto& g : t.hp->groups)
      if (prec == 0)
        dispatch_transfer<double>(g->t, g->fine_view, g->coarse_view, (const double*)rf, (double*)rc, true, s);
      else
        dispatch_transfer<float>(g->t, g->fine_view, g->coarse_view, (const float*)rf, (float*)rc, true, s);
    if (coarse.hp) hp_condense(coarse, prec, rc, s);  // contributions of constrained entries to masters
  } else if (t.separable) {
    sep_restrict(t.sep, prec, rf, rc, s);
  } else {
    MFNS_CUDA(cudaMemsetAsync(rc, 0, coarse.n_dofs * esize(prec), s));
    if (prec == 0)
      dispatch_transfer<double>(t, fine, coarse, (const double*)rf, (double*)rc, true, s);
    else
      dispatch_transfer<float>(t, fine, coarse, (const float*)rf, (float*)rc, true, s);
  }
  const int64_t nc = (int64_t)coarse.constrained_host.size();
  if (prec == 0)
    vset_idx<double>((double*)rc, 0.0, coarse.constrained.as<int32_t>(), nc, s);
  else
    vset_idx<float>((float*)rc, 0.0f, coarse.constrained.as<int32_t>(), nc, s);
}

}  // namespace mfns
