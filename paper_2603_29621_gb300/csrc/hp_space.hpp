// Host construction of hp-adaptive node spaces (Section 3): every cell of a forest carries its own
// degree; nodes are identified exactly; the constraints of h- and p-adaptivity are resolved to
// free masters.
//
// Constraint rules.  Local (dominance): a node is constrained when a cell whose closed box holds it
// does not have it as a node and dominates every cell that does (it is coarser, or of the same
// level and of lower degree); the node then takes that cell's finite-element function at its
// position.  Chains (a master that is itself constrained) are resolved transitively, so every
// listed master is free of hanging constraints.  This is a conforming space unless a hanging face
// has a coarse cell of higher degree than a fine cell on it (the combined h+p face).
// Elimination: the continuity conditions on every shared face piece, in reduced row echelon form
// with the columns ordered from the least to the most preferred node (coarser, then lower degree,
// then vertices before edge, face and cell interiors, then node id); the pivots are the
// constrained nodes, each expressed in nodes of its own face or edge.  It covers every configuration, including
// the combined face, and gives the local rule's constraints where that applies (boundary handling
// aside: with Dirichlet conditions boundary nodes are not unknowns and are neither constrained
// nor masters).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "mesh.hpp"

namespace mfns {

struct HpSpace {
  int dim = 3;
  int64_t n_nodes = 0;
  std::vector<int32_t> degree;       // per cell
  std::vector<int64_t> cell_ptr;     // per cell: offset of its (k_c+1)^dim slots in cell_nodes
  std::vector<int32_t> cell_nodes;   // node id of every slot (lexicographic, x fastest)
  std::vector<double> x;             // n_nodes * dim support points
  std::vector<uint8_t> boundary;     // node on the domain boundary
  // constrained nodes: value = sum over j in [hang_ptr[i], hang_ptr[i+1]) of hang_w[j] * value of
  // hang_master[j]; hang_node ascending
  std::vector<int32_t> hang_node, hang_ptr, hang_master;
  std::vector<double> hang_w;
};

enum class HpRule {
  kAuto = 0,         // the local rule, elimination where a combined h+p face makes it inapplicable
  kDominance = 1,    // the local rule only (fails on a combined face)
  kElimination = 2,  // elimination everywhere
};

// Builds the space; false with a message in err for an unsupported configuration or bad input.
// dirichlet: the field has homogeneous Dirichlet conditions on the domain boundary (used by the
// elimination rule, which then takes boundary nodes as zero rather than as unknowns).
bool make_hp_space(const Forest& f, const std::vector<int32_t>& degree, HpSpace& out, std::string* err,
                   HpRule rule = HpRule::kAuto, bool dirichlet = true);

// Greedy colouring of a subset of cells: no two cells of one colour share a node.  color[i] is the
// colour of cells[i]; returns the number of colours.
int hp_color_cells(const HpSpace& sp, const std::vector<int32_t>& cells, std::vector<int32_t>& color);

// Blocks of the additive Schwarz part of Section 3's blended smoother: for every combined h+p face
// (a cell face whose neighbours across it are finer and of lower degree), the free nodes (not
// constrained, not on the Dirichlet boundary) lying on the closed face of the coarse cell, each with
// its ncomp components (entries g * ncomp + c).  Entries ascending; faces in (cell, direction,
// side) order; faces without free nodes give no block.
std::vector<std::vector<int32_t>> hp_asm_blocks(const Forest& f, const HpSpace& sp, int ncomp);

}  // namespace mfns
