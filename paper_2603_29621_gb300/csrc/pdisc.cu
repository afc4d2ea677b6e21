// Kernels of the Q_k / P^disc_{k-1} pair on uniform meshes (see pdisc_dev.hpp): the pressure-velocity
// coupling of one cell block B, one warp per cell, and the pressure transfers.
#include <algorithm>

#include "common.hpp"
#include "pdisc_dev.hpp"

namespace mfns {

namespace {

constexpr int kWarpsPerBlock = 4;

// node id and Dirichlet flag of local velocity slot b of cell (cx, cy, cz)
__device__ __forceinline__ int64_t slot_node(const PdiscGeom g, int cx, int cy, int cz, int b, bool& bnd) {
  const int np1 = g.k + 1;
  const int64_t M = (int64_t)g.k * g.n + 1;
  const int bx = b % np1, by = (b / np1) % np1, bz = g.dim == 3 ? b / (np1 * np1) : 0;
  const int64_t ix = (int64_t)g.k * cx + bx, iy = (int64_t)g.k * cy + by, iz = g.dim == 3 ? (int64_t)g.k * cz + bz : 0;
  bnd = ix == 0 || ix == M - 1 || iy == 0 || iy == M - 1 || (g.dim == 3 && (iz == 0 || iz == M - 1));
  return ix + M * (iy + M * iz);
}

__device__ __forceinline__ void cell_coords(const PdiscGeom g, int64_t cell, int& cx, int& cy, int& cz) {
  cx = (int)(cell % g.n);
  cy = (int)((cell / g.n) % g.n);
  cz = g.dim == 3 ? (int)(cell / ((int64_t)g.n * g.n)) : 0;
}

// y_p(cell) = B x_u(cell): every lane sums a strided share of the cell's velocity entries for
// every coefficient (NPC of them, in registers), then the warp adds the shares in a fixed order
template <int NPC>
__global__ void k_div(const PdiscGeom g, const double* __restrict__ B, const double* __restrict__ x,
                      double* __restrict__ y, int64_t n_cells) {
  const int lane = threadIdx.x & 31;
  const int64_t cell = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (cell >= n_cells) return;
  int cx, cy, cz;
  cell_coords(g, cell, cx, cy, cz);
  int nb = g.k + 1;
  nb = g.dim == 3 ? nb * nb * nb : nb * nb;
  const int nj = nb * g.dim;
  double acc[NPC];
#pragma unroll
  for (int a = 0; a < NPC; ++a) acc[a] = 0.0;
  for (int j = lane; j < nj; j += 32) {
    const int b = j / g.dim, d = j - b * g.dim;
    bool bnd;
    const int64_t node = slot_node(g, cx, cy, cz, b, bnd);
    const double u = bnd ? 0.0 : x[node * g.dim + d];
#pragma unroll
    for (int a = 0; a < NPC; ++a) acc[a] += B[(int64_t)a * nj + j] * u;
  }
#pragma unroll
  for (int a = 0; a < NPC; ++a) {
    double v = acc[a];
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) y[g.n_main + cell * NPC + a] = v;
  }
}

// y_u += B^T x_p(cell) on the cells of one parity class
__global__ void k_grad_add(const PdiscGeom g, const double* __restrict__ B, const double* __restrict__ x,
                           double* __restrict__ y, int parity, int64_t n_class) {
  const int lane = threadIdx.x & 31;
  const int64_t t = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (t >= n_class) return;
  // t-th cell of the class: coordinates 2 i + parity bit per direction
  const int hx = (g.n - (parity & 1) + 1) / 2, hy = (g.n - ((parity >> 1) & 1) + 1) / 2;
  const int cx = 2 * (int)(t % hx) + (parity & 1);
  const int cy = 2 * (int)((t / hx) % hy) + ((parity >> 1) & 1);
  const int cz = g.dim == 3 ? 2 * (int)(t / ((int64_t)hx * hy)) + ((parity >> 2) & 1) : 0;
  const int64_t cell = cx + (int64_t)g.n * (cy + (int64_t)g.n * cz);
  int nb = g.k + 1;
  nb = g.dim == 3 ? nb * nb * nb : nb * nb;
  const int nj = nb * g.dim;
  const double* p = x + g.n_main + cell * g.npc;
  for (int j = lane; j < nj; j += 32) {
    const int b = j / g.dim, d = j - b * g.dim;
    bool bnd;
    const int64_t node = slot_node(g, cx, cy, cz, b, bnd);
    if (bnd) continue;
    double v = 0.0;
    for (int a = 0; a < g.npc; ++a) v += B[(int64_t)a * nj + j] * p[a];
    y[node * g.dim + d] += v;
  }
}

__global__ void k_prolong_add(int dim, int nf, int npf, int npc, bool hstep, const double* __restrict__ E,
                              const double* __restrict__ pc, double* __restrict__ pf, int64_t n_fine_cells) {
  for (int64_t cf = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cf < n_fine_cells;
       cf += (int64_t)gridDim.x * blockDim.x) {
    int64_t cc = cf;
    int child = 0;
    if (hstep) {
      const int i = (int)(cf % nf), j = (int)((cf / nf) % nf), l = dim == 3 ? (int)(cf / ((int64_t)nf * nf)) : 0;
      const int nc = nf / 2;
      cc = (i / 2) + (int64_t)nc * ((j / 2) + (int64_t)nc * (l / 2));
      child = (i & 1) | ((j & 1) << 1) | ((l & 1) << 2);
    }
    const double* Ec = E + (int64_t)child * npf * npc;
    for (int b = 0; b < npf; ++b) {
      double v = 0.0;
      for (int a = 0; a < npc; ++a) v += Ec[b * npc + a] * pc[cc * npc + a];
      pf[cf * npf + b] += v;
    }
  }
}

__global__ void k_restrict(int dim, int nf, int npf, int npc, bool hstep, const double* __restrict__ E,
                           const double* __restrict__ pf, double* __restrict__ pc, int64_t n_coarse_cells) {
  for (int64_t cc = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cc < n_coarse_cells;
       cc += (int64_t)gridDim.x * blockDim.x) {
    const int nchild = hstep ? (1 << dim) : 1;
    for (int a = 0; a < npc; ++a) {
      double v = 0.0;
      for (int child = 0; child < nchild; ++child) {
        int64_t cf = cc;
        if (hstep) {
          const int nc = nf / 2;
          const int i = (int)(cc % nc), j = (int)((cc / nc) % nc), l = dim == 3 ? (int)(cc / ((int64_t)nc * nc)) : 0;
          cf = (2 * i + (child & 1)) + (int64_t)nf * ((2 * j + ((child >> 1) & 1)) + (int64_t)nf * (2 * l + ((child >> 2) & 1)));
        }
        const double* Ec = E + (int64_t)child * npf * npc;
        for (int b = 0; b < npf; ++b) v += Ec[b * npc + a] * pf[cf * npf + b];
      }
      pc[cc * npc + a] = v;
    }
  }
}

unsigned grid_for_items(int64_t items, int per_block) {
  return (unsigned)std::max<int64_t>(1, (items + per_block - 1) / per_block);
}

}  // namespace

void pdisc_div(const PdiscGeom& g, const double* B, const double* x, double* y, cudaStream_t s) {
  const int64_t n_cells = g.dim == 3 ? (int64_t)g.n * g.n * g.n : (int64_t)g.n * g.n;
  const unsigned grid = grid_for_items(n_cells, kWarpsPerBlock), block = 32 * kWarpsPerBlock;
  // coefficients per cell: total degree <= k - 1 in dim variables, k = 2..4
  switch (g.npc) {
    case 3: k_div<3><<<grid, block, 0, s>>>(g, B, x, y, n_cells); break;
    case 4: k_div<4><<<grid, block, 0, s>>>(g, B, x, y, n_cells); break;
    case 6: k_div<6><<<grid, block, 0, s>>>(g, B, x, y, n_cells); break;
    case 10: k_div<10><<<grid, block, 0, s>>>(g, B, x, y, n_cells); break;
    case 20: k_div<20><<<grid, block, 0, s>>>(g, B, x, y, n_cells); break;
    default: throw Error(kErrUnsupported, "P^disc: unsupported number of pressure coefficients per cell");
  }
  MFNS_CUDA(cudaGetLastError());
}

void pdisc_grad_add(const PdiscGeom& g, const double* B, const double* x, double* y, cudaStream_t s) {
  for (int parity = 0; parity < (1 << g.dim); ++parity) {
    const int64_t hx = (g.n - (parity & 1) + 1) / 2, hy = (g.n - ((parity >> 1) & 1) + 1) / 2;
    const int64_t hz = g.dim == 3 ? (g.n - ((parity >> 2) & 1) + 1) / 2 : 1;
    const int64_t n_class = hx * hy * hz;
    if (n_class <= 0) continue;
    k_grad_add<<<grid_for_items(n_class, kWarpsPerBlock), 32 * kWarpsPerBlock, 0, s>>>(g, B, x, y, parity, n_class);
    MFNS_CUDA(cudaGetLastError());
  }
}

void pdisc_prolongate_add(int dim, int nf, int npf, int npc, bool hstep, const double* E, const double* pc,
                          double* pf, cudaStream_t s) {
  const int64_t n_fine = dim == 3 ? (int64_t)nf * nf * nf : (int64_t)nf * nf;
  k_prolong_add<<<grid_for_items(n_fine, 256), 256, 0, s>>>(dim, nf, npf, npc, hstep, E, pc, pf, n_fine);
  MFNS_CUDA(cudaGetLastError());
}

void pdisc_restrict(int dim, int nf, int npf, int npc, bool hstep, const double* E, const double* pf, double* pc,
                    cudaStream_t s) {
  const int nc = hstep ? nf / 2 : nf;
  const int64_t n_coarse = dim == 3 ? (int64_t)nc * nc * nc : (int64_t)nc * nc;
  k_restrict<<<grid_for_items(n_coarse, 256), 256, 0, s>>>(dim, nf, npf, npc, hstep, E, pf, pc, n_coarse);
  MFNS_CUDA(cudaGetLastError());
}

}  // namespace mfns
