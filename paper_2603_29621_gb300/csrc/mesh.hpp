// Host-side geometry: forests of axis-aligned cells, Q_k node spaces with
// hanging-node constraint masks, cell colouring and transfer maps.
//
// Section 2 (global coarsening): smoothing runs on the whole mesh and the
// hanging-node constraints are resolved inside every operator evaluation
// and transfer.  A cell whose face (or edge) touches a coarser cell reads
// the coarse face's (edge's) nodal values in its own lexicographic slots and
// interpolates them with 1D matrices; the mask bits below say which faces
// and edges this applies to.
#pragma once
#include <array>
#include <cstdint>
#include <string>
#include <vector>

namespace mfns {

// Constraint-mask layout (per cell).
//   bits  0.. 5 : face (direction d, side s) constrained, bit = 2*d + s
//   bits  6..17 : edge parallel to direction d with sides (s1, s2) of the two
//                 other directions (ascending), bit = 6 + 4*d + 2*s2 + s1
//   bits 24..26 : position of the cell inside its parent (c_d & 1)
constexpr uint32_t kChildShift = 24;

struct Forest {
  int dim = 3;
  int n = 1;                      // root cells per direction
  bool partial = false;           // the cells need not cover the domain (a local-smoothing level)
  std::vector<int32_t> lev;       // level of every active cell
  std::vector<int32_t> crd;       // 3 integer coordinates per cell (at its level)
  size_t n_cells() const { return lev.size(); }
  int max_level() const;
  bool uniform() const { return max_level() == 0; }
  double h(size_t c) const;
  void sort();                    // canonical order: level, z, y, x
};

Forest forest_uniform(int dim, int n);
Forest forest_refine(const Forest& f, const std::vector<char>& mask);
Forest forest_balance(Forest f);  // 2:1 over faces, edges and vertices
Forest forest_refine_ball(Forest f, const double centre[3], double radius, int levels);
// Local smoothing (Section 2): the cells of refinement level l -- the active cells of level l
// and the level-l ancestors of finer ones -- as a partial forest
Forest forest_level(const Forest& f, int l);
// one global-coarsening step (finest level -> parents; uniform n -> ceil(n/2), non-nested for odd n)
bool forest_can_coarsen(const Forest& f, int stop_n);
Forest forest_coarsen(const Forest& f);

// Lattice of the finest level: cell id of every finest-level lattice cell.
struct Lattice {
  int dim, N;
  std::vector<int32_t> cell;      // N^dim, x fastest
  int32_t at(int i, int j, int k) const {
    return cell[(size_t)i + (size_t)N * ((size_t)j + (size_t)N * (size_t)k)];
  }
};
Lattice make_lattice(const Forest& f);

// Per-cell constraint masks of a forest (independent of the degree).
std::vector<uint32_t> constraint_masks(const Forest& f, const Lattice& lat);

// Q_k node space of a forest.
struct NodeSpace {
  int dim = 3, k = 1, nb = 0;     // nb = (k+1)^dim
  int64_t n_nodes = 0;
  bool lexicographic = false;     // uniform mesh: node id = lexicographic grid index
  std::vector<double> x;          // n_nodes * dim support points
  std::vector<uint8_t> boundary;  // node on the domain boundary
  std::vector<int32_t> cell_nodes;   // n_cells * nb: true node ids
  std::vector<int32_t> cell_master;  // n_cells * nb: master ids (hanging slots substituted)
  // hanging nodes: value = sum of weight * master value
  std::vector<int32_t> hang_node, hang_ptr, hang_master;
  std::vector<double> hang_w;
};
NodeSpace make_nodes(const Forest& f, const Lattice& lat, const std::vector<uint32_t>& masks, int k,
                     std::string* err);

// Nodes of a single-level partial forest on its refinement edge: some cell of that level inside
// the domain whose closure holds the node is not one of the forest's cells.
std::vector<uint8_t> refinement_edge(const Forest& f, const NodeSpace& ns);

// Local smoothing: the DoFs a level owns.  For the active cells of the fine forest at refinement
// level l, every slot whose fine node is free (not hanging; not on the boundary unless
// own_boundary) and whose level node (same cell of the level forest `lf`, same slot) is not on the
// refinement edge appends the pair (fine node, level node) to (cf, cl) and records owner[fine
// node] = l.  own_boundary: the field has components without a boundary condition (the pressure of
// the stabilised equal-order system), so boundary nodes carry free DoFs and need an owner too; their
// Dirichlet components are restored from the right-hand side after the cycle.  A node listed by two
// levels, or an active cell missing from `lf`, is an error (false, message in err).
bool ls_owned_nodes(const Forest& fine, const NodeSpace& fns, const Forest& lf, const NodeSpace& lns,
                    const std::vector<uint8_t>& edge, int l, std::vector<int32_t>& owner,
                    std::vector<int32_t>& cf, std::vector<int32_t>& cl, std::string* err,
                    bool own_boundary = false);
// every free node of the fine space has an owner (boundary nodes included when own_boundary)
bool ls_all_owned(const NodeSpace& fns, const std::vector<int32_t>& owner, bool own_boundary = false);

// 1D helpers shared by the host code (GLL nodes, Gauss rule, Lagrange values).
std::vector<double> gll_nodes(int k);
void gauss_rule(int q, std::vector<double>& x, std::vector<double>& w);
double lagrange(const std::vector<double>& nodes, int a, double x);
double lagrange_deriv(const std::vector<double>& nodes, int a, double x);

// Greedy colouring of cells so that no two cells of a colour share a node of
// any of the given spaces.  Returns colour per cell and the number of colours.
int color_cells(const Forest& f, const std::vector<const NodeSpace*>& spaces, std::vector<int32_t>& color);

}  // namespace mfns
