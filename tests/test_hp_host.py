"""Host construction of hp spaces (csrc/hp_space.cpp, compiled with g++) against the oracle.

For ball-refined forests in 2D and 3D with degree fields that vary across same-level and hanging
faces: the library's nodes, boundary flags and constraints (every constrained node, its free
masters and weights, chains resolved) equal the oracle's ``hp.HpNodeSet`` node by node; every
cell-slot index is in range; the configuration the construction does not cover is rejected.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import hp, mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2603_29621_gb300", "csrc")

HARNESS = r"""
#include <algorithm>
#include <cstdio>
#include <string>
#include "hp_space.hpp"
using namespace mfns;
int main() {
  int dim, n, nc, rule, dbc;
  if (std::scanf("%d %d %d %d %d", &dim, &n, &nc, &rule, &dbc) != 5) return 1;
  Forest f;
  f.dim = dim;
  f.n = n;
  std::vector<int32_t> deg(nc);
  for (int c = 0; c < nc; ++c) {
    int l, x, y, z, k;
    if (std::scanf("%d %d %d %d %d", &l, &x, &y, &z, &k) != 5) return 1;
    f.lev.push_back(l);
    f.crd.push_back(x); f.crd.push_back(y); f.crd.push_back(z);
    deg[c] = k;
  }
  HpSpace sp;
  std::string err;
  if (!make_hp_space(f, deg, sp, &err, (HpRule)rule, dbc != 0)) { std::printf("FAIL %s\n", err.c_str()); return 0; }
  for (int32_t g : sp.cell_nodes) if (g < 0 || g >= sp.n_nodes) { std::printf("FAIL index\n"); return 0; }
  std::printf("NODES %lld\n", (long long)sp.n_nodes);
  for (int64_t g = 0; g < sp.n_nodes; ++g) {
    for (int d = 0; d < dim; ++d) std::printf("%.17g ", sp.x[g * dim + d]);
    std::printf("%d\n", (int)sp.boundary[g]);
  }
  // colourings: cells of each degree (no shared node within a colour), checked by brute force
  {
    int kmax = 0;
    for (int32_t k : deg) kmax = std::max(kmax, k);
    for (int k = 1; k <= kmax; ++k) {
      std::vector<int32_t> cells, color;
      for (int c = 0; c < nc; ++c) if (deg[c] == k) cells.push_back(c);
      if (cells.empty()) continue;
      hp_color_cells(sp, cells, color);
      std::vector<std::pair<int32_t, int32_t>> owner;  // (node, colour) pairs must be unique
      for (size_t i = 0; i < cells.size(); ++i)
        for (int64_t j = sp.cell_ptr[cells[i]]; j < sp.cell_ptr[cells[i] + 1]; ++j)
          owner.push_back({sp.cell_nodes[j] * 1024 + color[i], (int32_t)i});
      std::sort(owner.begin(), owner.end());
      for (size_t q = 1; q < owner.size(); ++q)
        if (owner[q].first == owner[q - 1].first && owner[q].second != owner[q - 1].second) {
          std::printf("FAIL colouring\n");
          return 0;
        }
    }
  }
  std::printf("HANG %zu\n", sp.hang_node.size());
  for (size_t i = 0; i < sp.hang_node.size(); ++i) {
    std::printf("%d %d", sp.hang_node[i], sp.hang_ptr[i + 1] - sp.hang_ptr[i]);
    for (int j = sp.hang_ptr[i]; j < sp.hang_ptr[i + 1]; ++j) std::printf(" %d %.17g", sp.hang_master[j], sp.hang_w[j]);
    std::printf("\n");
  }
  auto blocks = hp_asm_blocks(f, sp, dim);
  std::printf("ASM %zu\n", blocks.size());
  for (auto& b : blocks) {
    for (int32_t i : b) std::printf("%d ", i);
    std::printf("\n");
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("hphost")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, str(src), os.path.join(CSRC, "mesh.cpp"),
                    os.path.join(CSRC, "hp_space.cpp"), "-o", str(exe)], check=True)

    def run(forest, deg, rule=0, dirichlet=True):
        """rule: 0 auto, 1 the local rule only, 2 elimination everywhere."""
        rows = [f"{c[0]} {c[1]} {c[2]} {c[3] if forest.dim == 3 else 0} {k}" for c, k in zip(forest.cells, deg)]
        inp = f"{forest.dim} {forest.n} {len(rows)} {rule} {int(dirichlet)}\n" + "\n".join(rows) + "\n"
        out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
        if out[0].startswith("FAIL"):
            return out[0]
        nn = int(out[0].split()[1])
        rows = np.array([[float(v) for v in out[1 + i].split()] for i in range(nn)])
        x, bnd = rows[:, :forest.dim], rows[:, forest.dim].astype(bool)
        i = 1 + nn
        nh = int(out[i].split()[1])
        hang = {}
        for j in range(nh):
            t = out[i + 1 + j].split()
            g, m = int(t[0]), int(t[1])
            hang[g] = [(int(t[2 + 2 * q]), float(t[3 + 2 * q])) for q in range(m)]
        i += 1 + nh
        nblk = int(out[i].split()[1])
        run.asm = [[int(v) for v in out[i + 1 + j].split()] for j in range(nblk)]
        run.x = x
        return x, bnd, hang
    return run


def _key(x):
    return [tuple(v) for v in np.rint(np.asarray(x) * 2 ** 30).astype(np.int64)]


def _degrees(f, base):
    lev = f.cells[:, 0]
    return base + lev + ((f.cells[:, 1] >> lev) % 2)


@pytest.mark.parametrize("dim,n,levels,base", [(2, 3, 2, 1), (2, 4, 1, 2), (2, 2, 2, 2), (3, 2, 1, 1),
                                               (3, 3, 1, 2), (3, 2, 2, 1)])
def test_hp_space_matches_the_oracle(harness, dim, n, levels, base):
    f = mesh.refine_ball(mesh.uniform(dim, n), (0.3, 0.35, 0.4), 0.3, levels)
    deg = _degrees(f, base)
    got = harness(f, deg)
    assert not isinstance(got, str), got
    x, bnd, hang = got
    ns = hp.HpNodeSet(f, deg)
    assert len(x) == ns.n_nodes
    idx = dict(zip(_key(ns.x), range(ns.n_nodes)))
    m = np.array([idx[k] for k in _key(x)])              # library node -> oracle node
    assert len(set(m.tolist())) == len(m)
    assert np.array_equal(bnd, ns.boundary[m])
    assert set(m[list(hang)].tolist()) == set(ns.hanging)
    assert len(hang) > 0
    for g, masters in hang.items():
        ref = dict(ns.hanging[m[g]])
        mine = {int(m[q]): w for q, w in masters}
        assert set(mine) == set(ref)
        assert max(abs(mine[q] - ref[q]) for q in ref) <= 1e-12


def _compare(got, ns):
    """Library space against an oracle node set: same nodes, boundary flags, constrained nodes and
    weights (a master of weight zero may be listed on one side only)."""
    assert not isinstance(got, str), got
    x, bnd, hang = got
    assert len(x) == ns.n_nodes
    idx = dict(zip(_key(ns.x), range(ns.n_nodes)))
    m = np.array([idx[k] for k in _key(x)])
    assert len(set(m.tolist())) == len(m)
    assert np.array_equal(bnd, ns.boundary[m])
    assert set(m[list(hang)].tolist()) == set(ns.hanging)
    for g, masters in hang.items():
        ref = dict(ns.hanging[m[g]])
        mine = {int(m[q]): w for q, w in masters}
        assert max(abs(mine.get(q, 0.0) - ref.get(q, 0.0)) for q in set(ref) | set(mine)) <= 1e-12
    return len(hang)


def _combined(f, kind):
    lev = f.cells[:, 0]
    return {"3-2": 3 - lev, "4-2": 4 - 2 * lev, "4-3": 4 - lev, "2-1": 2 - lev}[kind]


def test_coarse_higher_degree_across_a_hanging_face_is_rejected_by_the_local_rule(harness):
    f = mesh.refine_ball(mesh.uniform(2, 3), (0.3, 0.35, 0.4), 0.3, 1)
    out = harness(f, 3 - f.cells[:, 0], rule=1)
    assert isinstance(out, str) and "unsupported" in out


@pytest.mark.parametrize("dirichlet", [True, False])
@pytest.mark.parametrize("dim,n,levels,base", [(2, 3, 2, 1), (2, 2, 2, 2), (3, 2, 1, 1), (3, 3, 1, 2)])
def test_elimination_matches_the_oracle_where_the_local_rule_applies(harness, dim, n, levels, base, dirichlet):
    """Forced elimination against the oracle's elimination (dense reduced row echelon form over
    other sample points): the reduced form is unique, so slaves and weights agree."""
    f = mesh.refine_ball(mesh.uniform(dim, n), (0.3, 0.35, 0.4), 0.3, levels)
    deg = _degrees(f, base)
    ns = hp.HpNodeSet(f, deg, "elimination", dirichlet=dirichlet)
    assert _compare(harness(f, deg, rule=2, dirichlet=dirichlet), ns) > 0


@pytest.mark.parametrize("dirichlet", [True, False])
@pytest.mark.parametrize("dim,n,kind", [(2, 3, "3-2"), (2, 4, "4-2"), (2, 3, "4-3"), (3, 2, "3-2"),
                                        (3, 3, "3-2"), (2, 4, "2-1"), (3, 3, "2-1")])
def test_combined_faces_by_elimination_match_the_oracle(harness, dim, n, kind, dirichlet):
    """Coarse cells of higher degree than the refined ones: the automatic rule switches to
    elimination and gives the oracle's constraints -- also for coarse degree 2 against fine degree
    1, where every node of the fine cells is a node of the coarse cell and no node hangs, yet the
    coarse trace must be reduced to a piecewise linear one."""
    f = mesh.refine_ball(mesh.uniform(dim, n), (0.3, 0.35, 0.4), 0.3, 1)
    deg = _combined(f, kind)
    ns = hp.HpNodeSet(f, deg, "elimination", dirichlet=dirichlet)
    assert _compare(harness(f, deg, rule=0, dirichlet=dirichlet), ns) > 0


def test_the_local_rule_stays_in_use_where_it_applies(harness):
    """With no combined face the automatic rule is the local one: boundary constrained nodes are
    listed (the local rule does not know the field's boundary condition)."""
    f = mesh.refine_ball(mesh.uniform(3, 2), (0.3, 0.35, 0.4), 0.3, 1)
    deg = _degrees(f, 1)
    x, bnd, hang = harness(f, deg, rule=0)
    assert any(bnd[g] for g in hang)


@pytest.mark.parametrize("dim,n,kind", [(2, 4, "3-2"), (2, 3, "4-2"), (3, 2, "3-2"), (3, 3, "3-2")])
def test_asm_blocks_match_the_oracle(harness, dim, n, kind):
    """The blocks of Section 3's blended smoother: for every combined face, the free unknowns on the
    closed face of its coarse cell (all components) -- the oracle's blocks, entry by entry."""
    f = mesh.refine_ball(mesh.uniform(dim, n), (0.3, 0.35, 0.4), 0.3, 1)
    deg = _combined(f, kind)
    got = harness(f, deg, rule=0)
    assert not isinstance(got, str), got
    x = harness.x
    P = hp.HpProblem(f, deg, "stokes_a", rule="elimination")
    ns = P.dofs.nodesets[0]
    key = lambda xx, c: (tuple(np.rint(np.asarray(xx) * 2 ** 30).astype(np.int64)), int(c))
    mine = {frozenset(key(x[i // dim], i % dim) for i in b) for b in harness.asm}
    ref = set()
    for B in hp.asm_blocks(P):
        g, c = (B - P.dofs.offsets[0]) % ns.n_nodes, (B - P.dofs.offsets[0]) // ns.n_nodes
        ref.add(frozenset(key(ns.x[gg], cc) for gg, cc in zip(g, c)))
    assert len(ref) > 0 and mine == ref
    assert len(harness.asm) == len(hp.asm_blocks(P))
