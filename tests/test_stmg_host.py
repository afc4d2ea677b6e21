"""Host set-up of the space-time multigrid (csrc/spacetime_host.cpp, compiled with g++) against the
oracle (Section 4): the level sequence (spatial degree, then temporal degree, then h) and the vertex
stars of the Schwarz smoother on Taylor--Hood spaces -- every patch, as a set of free entries
identified by support point and field, equals one of the oracle's, on uniform meshes and on
ball-refined meshes with hanging nodes, 2D and 3D."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import assemble, mesh, solvers, spacetime

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2603_29621_gb300", "csrc")
CENTRE = (0.3, 0.35, 0.4)

HARNESS = r"""
#include <cstdio>
#include <string>
#include "spacetime.hpp"
using namespace mfns;
int main() {
  int dim, n, nc, k, r, nf, ts;
  if (std::scanf("%d %d %d %d %d %d %d", &dim, &n, &nc, &k, &r, &nf, &ts) != 7) return 1;
  Forest f;
  f.dim = dim;
  f.n = n;
  for (int c = 0; c < nc; ++c) {
    int l, x, y, z;
    if (std::scanf("%d %d %d %d", &l, &x, &y, &z) != 4) return 1;
    f.lev.push_back(l);
    f.crd.push_back(x); f.crd.push_back(y); f.crd.push_back(z);
  }
  for (auto& s : stmg_sequence(k, r, nf, ts != 0)) std::printf("%d %d %d;", s.k, s.r, s.forest);
  std::printf("%d\n", (int)vertex_star_covers_all(f));
  Lattice lat = make_lattice(f);
  std::vector<uint32_t> masks = constraint_masks(f, lat);
  std::string err;
  NodeSpace nu = make_nodes(f, lat, masks, k, &err);
  NodeSpace np = make_nodes(f, lat, masks, k - 1, &err);
  if (!err.empty()) { std::printf("FAIL %s\n", err.c_str()); return 0; }
  std::printf("%lld %lld\n", (long long)nu.n_nodes, (long long)np.n_nodes);
  for (double v : nu.x) std::printf("%.17g ", v);
  std::printf("\n");
  for (double v : np.x) std::printf("%.17g ", v);
  std::printf("\n");
  auto patches = vertex_star_patches(f, nu, np);
  std::printf("%zu\n", patches.size());
  for (auto& p : patches) {
    for (int32_t i : p) std::printf("%d ", i);
    std::printf("\n");
  }
  std::vector<int32_t> colour;
  colour_patches_for_probing(f, nu, np, patches, colour);
  for (int32_t c : colour) std::printf("%d ", c);
  std::printf("\n");
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("stmghost")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, str(src), os.path.join(CSRC, "mesh.cpp"),
                    os.path.join(CSRC, "spacetime_host.cpp"), "-o", str(exe)], check=True)

    def run(forest, k, r, nf, ts=True):
        rows = [f"{c[0]} {c[1]} {c[2]} {c[3] if forest.dim == 3 else 0}" for c in forest.cells]
        inp = f"{forest.dim} {forest.n} {len(rows)} {k} {r} {nf} {int(ts)}\n" + "\n".join(rows) + "\n"
        out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
        parts = out[0].split(";")
        run.covers_all = bool(int(parts[-1]))
        seq = [tuple(int(v) for v in t.split()) for t in parts[:-1] if t.strip()]
        assert not out[1].startswith("FAIL"), out[1]
        nnu, nnp = (int(v) for v in out[1].split())
        dim = forest.dim
        xu = np.array([float(v) for v in out[2].split()]).reshape(nnu, dim)
        xp = np.array([float(v) for v in out[3].split()]).reshape(nnp, dim)
        npatch = int(out[4])
        patches = [[int(v) for v in out[5 + i].split()] for i in range(npatch)]
        run.colours = np.array([int(v) for v in out[5 + npatch].split()])
        return seq, xu, xp, patches
    return run


def _forest(dim, n, ball):
    f = mesh.uniform(dim, n)
    return mesh.refine_ball(f, CENTRE, 0.3, 1) if ball else f


@pytest.mark.parametrize("n,stop_n", [(8, 2), (8, 4), (6, 3)])
@pytest.mark.parametrize("k,r", [(2, 0), (2, 3), (4, 1), (3, 2)])
def test_level_sequence_matches_the_oracle(harness, k, r, n, stop_n):
    """Spatial degree, then h down to stop_n, then the temporal degree on the coarsest mesh unless a
    vertex star there holds every cell -- the oracle's sequence for vertex-star patches."""
    f = mesh.uniform(2, n)
    fs = solvers.coarse_forests(f, stop_n)
    ts = not spacetime._star_covers_all(fs[-1])
    seq = harness(f, k, r, len(fs), ts)[0]
    lv = spacetime.stmg_levels(f, k, r, tau=0.1, stop_n=stop_n, pressure="continuous")
    assert [(a, b) for a, b, _ in seq] == [(l.k, l.r) for l in lv]
    assert [fs[i].n for _, _, i in seq] == [l.st.space.forest.n for l in lv]


@pytest.mark.parametrize("dim,n,ball", [(2, 2, False), (2, 3, False), (3, 2, False), (2, 4, True), (3, 2, True)])
def test_vertex_star_covering_matches_the_oracle(harness, dim, n, ball):
    f = _forest(dim, n, ball)
    harness(f, 2, 0, 1)
    assert harness.covers_all == spacetime._star_covers_all(f)


@pytest.mark.parametrize("dim,n,ball,k", [(2, 4, False, 2), (2, 3, True, 2), (2, 3, False, 3), (3, 2, False, 2),
                                          (3, 2, True, 2)])
def test_vertex_star_patches_match_the_oracle(harness, dim, n, ball, k):
    f = _forest(dim, n, ball)
    _, xu, xp, patches = harness(f, k, 0, 1)
    prob = assemble.Problem(f, "stokes", k)
    xo, fo = prob.dofs.support_points()
    key = {(tuple(np.rint(x * 2 ** 30).astype(np.int64)), int(c)): i for i, (x, c) in enumerate(zip(xo, fo))}
    n_main = len(xu) * dim

    def oracle_index(i):
        if i < n_main:
            g, c = divmod(i, dim)
            return key[(tuple(np.rint(xu[g] * 2 ** 30).astype(np.int64)), c)]
        return key[(tuple(np.rint(xp[i - n_main] * 2 ** 30).astype(np.int64)), dim)]

    mine = {frozenset(oracle_index(i) for i in p) for p in patches}
    # probing colours: within a colour class no operator entry couples two different patches
    A = abs(prob.assemble()).tocsr()
    Mv = abs(spacetime.SpaceTimeStokes(f, k, 0, pressure="continuous").M).tocsr()
    colours = harness.colours
    assert len(colours) == len(patches) and colours.max() < 64
    idx = [np.array([oracle_index(i) for i in p]) for p in patches]
    for col in range(colours.max() + 1):
        members = np.nonzero(colours == col)[0]
        owner = -np.ones(A.shape[0], dtype=np.int64)
        for pi in members:
            assert np.all(owner[idx[pi]] < 0)              # patches of one colour are disjoint
            owner[idx[pi]] = pi
        for pi in members:
            for Mat in (A, Mv):
                cols = Mat[idx[pi]].nonzero()[1]
                hit = owner[cols]
                assert np.all((hit < 0) | (hit == pi)), (col, pi)
    ref_list = spacetime._patch_dofs(prob, "vertex")
    ref = {frozenset(p.tolist()) for p in ref_list}
    assert mine == ref
    # the same multiplicities (they set the Schwarz weights): no patch repeated on either side
    assert len(patches) == len(mine) and len(ref_list) == len(ref)


@pytest.mark.parametrize("n,stop_n", [(8, 2), (8, 4)])
@pytest.mark.parametrize("k,r", [(2, 1), (4, 3), (3, 2)])
def test_level_sequence_with_cell_patches_matches_the_oracle(harness, k, r, n, stop_n):
    """Cell patches (the paper's pair Q_k / P^disc_{k-1}): the temporal steps always follow the
    spatial ones on the coarsest mesh."""
    f = mesh.uniform(2, n)
    fs = solvers.coarse_forests(f, stop_n)
    seq = harness(f, k, r, len(fs), True)[0]
    lv = spacetime.stmg_levels(f, k, r, tau=0.1, stop_n=stop_n, pressure="disc")
    assert [(a, b) for a, b, _ in seq] == [(l.k, l.r) for l in lv]
    assert [fs[i].n for _, _, i in seq] == [l.st.space.forest.n for l in lv]
