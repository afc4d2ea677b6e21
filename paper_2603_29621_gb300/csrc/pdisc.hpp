// The spatial pair of Section 4, Q_k^dim velocity / P^disc_{k-1} pressure, on uniform meshes: host
// tables.
//
// Pressure on every cell: the polynomials of total degree <= k - 1 in the cell's centred, scaled
// coordinates s = (x - x_cell) / h, monomial basis s^a, exponents in graded order (total degree
// ascending, then the x exponent descending, then the y exponent descending).  Pressure entries
// follow the velocity block cell by cell (lexicographic cells, x fastest), npc coefficients per
// cell.  The symmetric form of Eq. 5 couples them through B = -(q, div u): on a uniform mesh every
// cell has the same block.
#pragma once
#include <array>
#include <cstdint>
#include <vector>

namespace mfns {

// Exponents of the monomials of total degree <= kp in dim variables, graded order.
std::vector<std::array<int, 3>> pdisc_exponents(int dim, int kp);

// B of one cell of size h for velocity degree k: B[(a * nb + b) * dim + d] = -int_cell s^{e_a}
// d(phi_b)/dx_d dx, nb = (k+1)^dim velocity nodes (GLL points, lexicographic, x fastest).
std::vector<double> pdisc_cell_B(int dim, int k, double h);

// Coefficients of a coarse cell's pressure polynomial on child `child` of the nested refinement
// (bit d of child: upper half in direction d): fine = E coarse, E npc x npc row-major (same
// degree kp on both cells; exact, by the binomial expansion of s_coarse = delta + s_fine / 2).
std::vector<double> pdisc_child_embedding(int dim, int kp, int child);

// Degree change on one cell, kpc <= kpf: fine = E coarse, E npc_f x npc_c row-major (the graded
// order makes the coarse exponents a prefix of the fine ones).
std::vector<double> pdisc_degree_embedding(int dim, int kpf, int kpc);

// Patches of the Schwarz smoother (one per cell, Section 4): the free velocity entries g * dim + c
// of the cell's nodes (uniform mesh, lexicographic nodes of the (k n + 1)^dim grid, boundary nodes
// Dirichlet) and the cell's npc pressure entries n_main + cell * npc + a; ascending.
std::vector<std::vector<int32_t>> pdisc_cell_patches(int dim, int n, int k);

}  // namespace mfns
