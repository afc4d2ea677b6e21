// Space-time finite elements for one time slab of the transient Stokes equations (Section 4).
//
// The slab I_n = (t_{n-1}, t_n], tau = t_n - t_{n-1}, carries a DG(r) discretisation in time with
// Q = r + 1 stages: the Lagrange basis phi_i at the Q right Gauss--Radau points of the slab (the
// last point is the slab's end, so the value passed on to the next slab is the last stage).  On
// the reference slab [0, 1]
//   M_Q[j][i] = int phi_i phi_j,   A_Q[j][i] = int phi_i' phi_j + phi_i(0) phi_j(0),   m_Q[j] = phi_j(0)
// (time derivative, upwind jump at the slab's start, previous end value); this is the Q-stage
// Radau IIA method.  Stage values of the spatial vector are stored stage-major, and after mass
// scaling with M_Q^{-1} the slab operator of Eq. 6 is
//   K = G_Q (x) M + tau I_Q (x) A,   G_Q = M_Q^{-1} A_Q,
// with M the velocity mass of the spatial Stokes space (zero pressure rows, zero constrained
// rows) and A the spatial Stokes operator (identity rows on constrained entries), so the
// constrained rows of K are tau times identity rows.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "mesh.hpp"

namespace mfns {

// The Q right Gauss--Radau points on [0, 1], ascending; the last one is 1.
std::vector<double> radau_right(int Q);

struct TemporalMatrices {
  int Q = 0;
  std::vector<double> t;        // Q nodes
  std::vector<double> M, A, G;  // Q x Q, row-major: M[j * Q + i]
  std::vector<double> m;        // Q
};

// DG(r) matrices on the reference slab, r in 0..7; false with a message otherwise.
bool temporal_matrices(int r, TemporalMatrices& out, std::string* err);

// P_tau (Q_f x Q_c, row-major): the coarse DG(rc) temporal polynomial at the fine DG(rf) nodes.
std::vector<double> time_prolongation(int rc, int rf);

// Levels of the space-time multigrid, finest first, by Section 4's rules -- space before time, and
// in each polynomially before geometrically: the spatial degree halved while above 2 (k >= 2 is
// kept: Q2 is the lowest Taylor--Hood velocity), then the coarser forests of global coarsening
// (index 1, 2, ... of the forest sequence, forest 0 being the fine mesh), then, when time_steps,
// the temporal degree halved (DG(r) -> DG(r / 2)) down to 0 on the coarsest forest; no coarsening
// of the slab length (time-marching).
struct StLevelSpec {
  int k = 2, r = 0, forest = 0;
};
std::vector<StLevelSpec> stmg_sequence(int k, int r, int n_forests, bool time_steps);

// Whether some vertex star (the cells having one vertex as a corner) holds every cell of f: its
// vertex-star patch would then hold every unknown and be singular.
bool vertex_star_covers_all(const Forest& f);

// Patches of the space-time Schwarz smoother on a Taylor--Hood space (velocity entries g * dim + c
// over the nodes of nu, then pressure entries n_main + g over the nodes of np): for every vertex
// of the mesh, the cells having it as a corner form a star, and the patch is the set of free
// entries (not Dirichlet, not hanging) every holding cell of which lies in the star.  Entries
// ascending; stars in lattice order; empty patches dropped.
std::vector<std::vector<int32_t>> vertex_star_patches(const Forest& f, const NodeSpace& nu, const NodeSpace& np);

// Colours of the patches for probing the patch blocks of a spatial operator on that space: two
// patches of one colour have no entry pair (row of one, column of the other) that any cell couples,
// a cell coupling the entries of every node it holds and the masters of the hanging nodes it
// holds.  colour[p] for every patch; returns the number of colours.
// In-place inverse of a dense n x n matrix (row-major) by Gauss--Jordan elimination with partial
// pivoting; false when a pivot falls below rel_tol times the largest entry (singular to that
// tolerance).
bool invert_dense_rel(std::vector<double>& A, int64_t n, double rel_tol);

int colour_patches_for_probing(const Forest& f, const NodeSpace& nu, const NodeSpace& np,
                               const std::vector<std::vector<int32_t>>& patches, std::vector<int32_t>& colour);

}  // namespace mfns
