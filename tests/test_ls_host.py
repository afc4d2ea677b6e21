"""Host-side set-up of local smoothing (csrc/mesh.cpp, compiled with g++), checked against the oracle.

For ball-refined forests in 2D and 3D and degrees 1-3:
* the cells of every refinement level, their Q_k nodes and the refinement-edge and boundary flags
  equal the oracle's level spaces (``oracle.ls.LevelSpace``), node by node;
* level forests have no hanging nodes (all constraint masks zero) and every cell-node index is in
  range;
* every free fine DoF is owned by exactly one level, the coarsest level of the active cells that
  hold it (the oracle's ``owner_level``), and constrained fine DoFs by none -- with boundary nodes
  owned as well when the field has a component without a boundary condition (the stabilised
  system's pressure).
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import ls, mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2603_29621_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <string>
#include "mesh.hpp"
using namespace mfns;
static void fail(const char* m) { std::printf("FAIL %s\n", m); std::exit(0); }
static NodeSpace nodes_of(const Forest& f, int k, bool zero_masks) {
  Lattice lat = make_lattice(f);
  std::vector<uint32_t> masks = constraint_masks(f, lat);
  if (zero_masks)
    for (uint32_t m : masks) if (m & 0x3FFFFu) fail("level forest with a constrained face");
  std::string err;
  NodeSpace ns = make_nodes(f, lat, masks, k, &err);
  if (!err.empty()) fail(err.c_str());
  for (int32_t g : ns.cell_nodes) if (g < 0 || g >= ns.n_nodes) fail("node index out of range");
  return ns;
}
int main() {
  int dim, n, k, nc, ob;
  if (std::scanf("%d %d %d %d %d", &dim, &n, &k, &nc, &ob) != 5) return 1;
  Forest f;
  f.dim = dim;
  f.n = n;
  for (int c = 0; c < nc; ++c) {
    int l, x, y, z;
    if (std::scanf("%d %d %d %d", &l, &x, &y, &z) != 4) return 1;
    f.lev.push_back(l);
    f.crd.push_back(x); f.crd.push_back(y); f.crd.push_back(z);
  }
  f.sort();
  const int L = f.max_level();
  NodeSpace fns = nodes_of(f, k, false);
  std::vector<int32_t> owner(fns.n_nodes, -1);
  std::string err;
  for (int l = 0; l <= L; ++l) {
    Forest lf = l == 0 ? forest_uniform(dim, n) : forest_level(f, l);
    NodeSpace lns = nodes_of(lf, k, true);
    std::vector<uint8_t> edge = l == 0 ? std::vector<uint8_t>(lns.n_nodes, 0) : refinement_edge(lf, lns);
    std::vector<int32_t> cf, cl;
    if (!ls_owned_nodes(f, fns, lf, lns, edge, l, owner, cf, cl, &err, ob != 0)) fail(err.c_str());
    for (size_t i = 0; i < cf.size(); ++i)
      if (cf[i] < 0 || cf[i] >= fns.n_nodes || cl[i] < 0 || cl[i] >= lns.n_nodes || edge[cl[i]]) fail("copy pair");
    std::printf("LEVEL %d %zu %lld %zu\n", l, lf.n_cells(), (long long)lns.n_nodes, cf.size());
    for (int64_t g = 0; g < lns.n_nodes; ++g) {
      for (int d = 0; d < dim; ++d) std::printf("%.17g ", lns.x[g * dim + d]);
      std::printf("%d %d\n", (int)edge[g], (int)lns.boundary[g]);
    }
  }
  if (!ls_all_owned(fns, owner, ob != 0)) fail("a free fine node without owner");
  std::printf("FINE %lld\n", (long long)fns.n_nodes);
  for (int64_t g = 0; g < fns.n_nodes; ++g) {
    for (int d = 0; d < dim; ++d) std::printf("%.17g ", fns.x[g * dim + d]);
    std::printf("%d\n", owner[g]);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("lshost")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, str(src), os.path.join(CSRC, "mesh.cpp"), "-o", str(exe)],
                   check=True)

    def run(forest, k, own_boundary=False):
        cells = forest.cells
        rows = [f"{c[0]} {c[1]} {c[2]} {c[3] if forest.dim == 3 else 0}" for c in cells]
        inp = f"{forest.dim} {forest.n} {k} {len(cells)} {int(own_boundary)}\n" + "\n".join(rows) + "\n"
        out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
        assert not out[0].startswith("FAIL"), out[0]
        levels, i = {}, 0
        while out[i].startswith("LEVEL"):
            _, l, ncell, nn, ncopy = out[i].split()
            l, nn = int(l), int(nn)
            rows = np.array([[float(v) for v in out[i + 1 + j].split()] for j in range(nn)])
            levels[l] = dict(cells=int(ncell), x=rows[:, :forest.dim], edge=rows[:, forest.dim].astype(bool),
                             boundary=rows[:, forest.dim + 1].astype(bool), n_copy=int(ncopy))
            i += 1 + nn
        assert out[i].startswith("FINE"), out[i]
        nn = int(out[i].split()[1])
        rows = np.array([[float(v) for v in out[i + 1 + j].split()] for j in range(nn)])
        return levels, rows[:, :forest.dim], rows[:, forest.dim].astype(int)
    return run


def _key(x):
    return [tuple(v) for v in np.rint(np.asarray(x) * 2 ** 30).astype(np.int64)]


CASES = [(2, 3, 2, 2), (2, 4, 2, 1), (2, 2, 3, 3), (3, 2, 2, 2), (3, 3, 1, 1), (3, 2, 1, 3)]


@pytest.mark.parametrize("dim,n,levels,k", CASES)
def test_level_nodes_and_edges_match_the_oracle(harness, dim, n, levels, k):
    f = mesh.refine_ball(mesh.uniform(dim, n), (0.3, 0.35, 0.4), 0.3, levels)
    got, _, _ = harness(f, k)
    assert sorted(got) == list(range(f.max_level + 1))
    for l in range(1, f.max_level + 1):
        sp_ = ls.LevelSpace(f, l, k)
        g = got[l]
        assert g["cells"] == len(sp_.cells) and len(g["x"]) == sp_.n_nodes
        ref = dict(zip(_key(sp_.x), zip(sp_.edge, sp_.boundary)))
        for key, e, b in zip(_key(g["x"]), g["edge"], g["boundary"]):
            assert ref[key] == (e, b)


@pytest.mark.parametrize("own_boundary", [False, True])
@pytest.mark.parametrize("dim,n,levels,k", CASES)
def test_every_free_fine_dof_has_one_owner(harness, dim, n, levels, k, own_boundary):
    f = mesh.refine_ball(mesh.uniform(dim, n), (0.3, 0.35, 0.4), 0.3, levels)
    got, xf, owner = harness(f, k, own_boundary)
    ns = mesh.NodeSet(f, k)
    free = np.ones(ns.n_nodes, dtype=bool) if own_boundary else ~ns.boundary
    free[list(ns.hanging)] = False
    ref = dict(zip(_key(ns.x), zip(free, ns.owner_level)))
    assert len(xf) == ns.n_nodes
    counts = np.zeros(f.max_level + 1, dtype=int)
    for key, o in zip(_key(xf), owner):
        is_free, lev = ref[key]
        assert o == (lev if is_free else -1)
        if o >= 0:
            counts[o] += 1
    assert [got[l]["n_copy"] for l in range(f.max_level + 1)] == counts.tolist()
