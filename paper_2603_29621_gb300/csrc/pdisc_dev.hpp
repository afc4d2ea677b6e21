// Device side of the Q_k / P^disc_{k-1} pair on uniform meshes (host tables in pdisc.hpp).
//
// Vector layout of one stage: the velocity block (lexicographic nodes of the (k n + 1)^dim grid,
// dim interleaved components, boundary nodes Dirichlet) of length n_main, then npc pressure
// coefficients per cell (lexicographic cells).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace mfns {

struct PdiscGeom {
  int dim = 3, k = 2, n = 1, npc = 1;
  int64_t n_main = 0;
};

// y_p = B x_u on every cell (overwrites the pressure block of y); B: device table of the cell block
// (pdisc_cell_B); Dirichlet velocity entries are read as zero.  FP64.
void pdisc_div(const PdiscGeom& g, const double* B, const double* x, double* y, cudaStream_t s);
// y_u += B^T x_p on every cell, Dirichlet velocity rows left alone (one launch per cell parity class:
// no two cells of a class share a node).  FP64.
void pdisc_grad_add(const PdiscGeom& g, const double* B, const double* x, double* y, cudaStream_t s);
// Pressure blocks between two levels: hstep (nested refinement, fine mesh 2 nc, E: 2^dim child
// embeddings npf x npc) or a degree step on one mesh (E: npf x npc).  prolongation: pf += E pc;
// restriction: pc = sum over children of E^T pf.  pf/pc point at the pressure blocks.
void pdisc_prolongate_add(int dim, int nf, int npf, int npc, bool hstep, const double* E, const double* pc,
                          double* pf, cudaStream_t s);
void pdisc_restrict(int dim, int nf, int npf, int npc, bool hstep, const double* E, const double* pf, double* pc,
                    cudaStream_t s);

}  // namespace mfns
