"""Host tables of the Q_k / P^disc_{k-1} pair (csrc/pdisc_host.cpp, compiled with g++) against the
oracle's assembled operator and transfers (Section 4's spatial pair), on uniform meshes: monomial
order; the cell block B of -(q, div u) equal to every pressure-velocity entry of the oracle's matrix;
the child and degree embeddings equal to the pressure block of the oracle's prolongation; the
cell patches of the Schwarz smoother equal to the oracle's."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import fe, mesh, pdisc, spacetime

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2603_29621_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include "pdisc.hpp"
using namespace mfns;
int main() {
  int dim, n, k;
  if (std::scanf("%d %d %d", &dim, &n, &k) != 3) return 1;
  auto ex = pdisc_exponents(dim, k - 1);
  for (auto& e : ex) std::printf("%d %d %d;", e[0], e[1], e[2]);
  std::printf("\n");
  for (double v : pdisc_cell_B(dim, k, 1.0 / n)) std::printf("%.17g ", v);
  std::printf("\n");
  for (int c = 0; c < (1 << dim); ++c) {
    for (double v : pdisc_child_embedding(dim, k - 1, c)) std::printf("%.17g ", v);
    std::printf("\n");
  }
  for (double v : pdisc_degree_embedding(dim, k - 1, 1)) std::printf("%.17g ", v);
  std::printf("\n");
  auto P = pdisc_cell_patches(dim, n, k);
  std::printf("%zu\n", P.size());
  for (auto& p : P) {
    for (int32_t i : p) std::printf("%d ", i);
    std::printf("\n");
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("pdischost")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, str(src), os.path.join(CSRC, "mesh.cpp"),
                    os.path.join(CSRC, "pdisc_host.cpp"), "-o", str(exe)], check=True)

    def run(dim, n, k):
        out = subprocess.run([str(exe)], input=f"{dim} {n} {k}\n", capture_output=True, text=True,
                             check=True).stdout.split("\n")
        ex = [tuple(int(v) for v in t.split()) for t in out[0].split(";") if t.strip()]
        B = np.array([float(v) for v in out[1].split()])
        E = [np.array([float(v) for v in out[2 + c].split()]) for c in range(1 << dim)]
        Ed = np.array([float(v) for v in out[2 + (1 << dim)].split()])
        i = 3 + (1 << dim)
        npatch = int(out[i])
        patches = [[int(v) for v in out[i + 1 + j].split()] for j in range(npatch)]
        return ex, B, E, Ed, patches
    return run


CASES = [(2, 3, 2), (2, 2, 3), (3, 2, 2), (2, 2, 4)]


def _vel_key(x, c):
    return (tuple(np.rint(np.asarray(x) * 2 ** 30).astype(np.int64)), int(c))


@pytest.mark.parametrize("dim,n,k", CASES)
def test_cell_block_equals_the_oracle_matrix(harness, dim, n, k):
    ex, B, E, Ed, _ = harness(dim, n, k)
    oex = pdisc.exponents(dim, k - 1)
    assert [e[:dim] for e in ex] == [tuple(int(v) for v in e) for e in oex]
    f = mesh.uniform(dim, n)
    S = pdisc.StokesPdisc(f, k)
    K = S.assemble_K().tocsr()
    xo, fo = S.vel.support_points()
    key = {_vel_key(x, c): i for i, (x, c) in enumerate(zip(xo, fo))}
    npc, nb = S.npc, (k + 1) ** dim
    B = B.reshape(npc, nb, dim)
    gll = np.asarray(fe.gll_points(k))                  # the k + 1 velocity nodes of a cell
    h, org = f.h(), f.origin()
    worst = 0.0
    for c in range(f.n_cells):
        for b in range(nb):
            bi = [(b // (k + 1) ** e) % (k + 1) for e in range(dim)]
            x = org[c] + h[c] * gll[bi]
            for d in range(dim):
                col = key[_vel_key(x, d)]
                for a in range(npc):
                    worst = max(worst, abs(K[S.p_offset + c * npc + a, col] - B[a, b, d]))
    assert worst <= 1e-14


@pytest.mark.parametrize("dim,n,k", CASES)
def test_embeddings_equal_the_oracle_prolongation(harness, dim, n, k):
    _, _, E, Ed, _ = harness(dim, n, k)
    npc = len(pdisc.exponents(dim, k - 1))
    coarse = pdisc.StokesPdisc(mesh.uniform(dim, n), k)
    fine = pdisc.StokesPdisc(mesh.uniform(dim, 2 * n), k)
    P = pdisc.prolongation(coarse, fine).tocsr()
    worst = 0.0
    for cf in range(fine.forest.n_cells):
        ijk = fine.forest.cells[cf, 1:]
        cc = int(np.ravel_multi_index(tuple((ijk // 2)[::-1]), (n,) * dim))
        child = sum(int(ijk[e] % 2) << e for e in range(dim))
        blk = P[fine.p_offset + cf * npc:fine.p_offset + (cf + 1) * npc,
                coarse.p_offset + cc * npc:coarse.p_offset + (cc + 1) * npc].toarray()
        worst = max(worst, np.abs(blk - E[child].reshape(npc, npc)).max())
    assert worst <= 1e-13
    if k >= 3:                                          # degree k -> 2 on one mesh: pressure k-1 -> 1
        f = mesh.uniform(dim, n)
        c2, fk = pdisc.StokesPdisc(f, 2), pdisc.StokesPdisc(f, k)
        P = pdisc.prolongation(c2, fk).tocsr()
        nc = c2.npc
        blk = P[fk.p_offset:fk.p_offset + npc, c2.p_offset:c2.p_offset + nc].toarray()
        assert np.abs(blk - Ed.reshape(npc, nc)).max() <= 1e-13


@pytest.mark.parametrize("dim,n,k", CASES)
def test_cell_patches_equal_the_oracle(harness, dim, n, k):
    _, _, _, _, patches = harness(dim, n, k)
    f = mesh.uniform(dim, n)
    S = pdisc.StokesPdisc(f, k)
    xo, fo = S.vel.support_points()
    key = {_vel_key(x, c): i for i, (x, c) in enumerate(zip(xo, fo))}
    M = k * n + 1
    n_main = M ** dim * dim
    npc = S.npc

    gll = np.asarray(fe.gll_points(k))

    def position(ix):                                  # grid index -> coordinate (GLL nodes per cell)
        cx, bx = (ix // k, ix % k) if ix < k * n else (n - 1, k)
        return (cx + gll[bx]) / n

    def oracle_index(i):
        if i < n_main:
            g, c = divmod(i, dim)
            ijk = [(g // M ** e) % M for e in range(dim)]
            return key[_vel_key(np.array([position(v) for v in ijk]), c)]
        cell, a = divmod(i - n_main, npc)
        return S.p_offset + cell * npc + a

    mine = [sorted(oracle_index(i) for i in p) for p in patches]
    ref = [sorted(p.tolist()) for p in spacetime._patch_dofs(S, "cell")]
    assert mine == ref
