"""Host temporal matrices of the space-time slab (csrc/spacetime_host.cpp, compiled with g++).

DG(r) on right Gauss--Radau points (Section 4): the points in closed form (Q = 1, 2, 3); the
one-slab amplification y_Q of y' = lambda y computed from the library's M_Q, A_Q, m_Q is the (r, r+1)
Pade approximant of exp (the Radau IIA stability function), r = 0..5; G_Q = M_Q^{-1} A_Q; the
matrices and the time prolongations equal the oracle's."""
import os
import shutil
import subprocess
from math import factorial

import numpy as np
import pytest

from oracle import spacetime

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2603_29621_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <string>
#include "spacetime.hpp"
using namespace mfns;
int main() {
  int r;
  while (std::scanf("%d", &r) == 1) {
    TemporalMatrices T;
    std::string err;
    if (!temporal_matrices(r, T, &err)) { std::printf("FAIL %s\n", err.c_str()); continue; }
    std::printf("%d\n", T.Q);
    for (double v : T.t) std::printf("%.17g ", v);
    std::printf("\n");
    for (auto* M : {&T.M, &T.A, &T.G}) {
      for (double v : *M) std::printf("%.17g ", v);
      std::printf("\n");
    }
    for (double v : T.m) std::printf("%.17g ", v);
    std::printf("\n");
    for (int rc = 0; rc < r; ++rc) {
      for (double v : time_prolongation(rc, r)) std::printf("%.17g ", v);
      std::printf("\n");
    }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def temporal(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("sthost")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, str(src), os.path.join(CSRC, "mesh.cpp"),
                    os.path.join(CSRC, "spacetime_host.cpp"), "-o", str(exe)], check=True)

    def run(r):
        out = subprocess.run([str(exe)], input=f"{r}\n", capture_output=True, text=True, check=True).stdout
        lines = out.strip().split("\n")
        Q = int(lines[0])
        vec = lambda s: np.array([float(v) for v in s.split()])
        t = vec(lines[1])
        M, A, G = (vec(lines[2 + i]).reshape(Q, Q) for i in range(3))
        m = vec(lines[5])
        P = [vec(lines[6 + rc]).reshape(Q, rc + 1) for rc in range(r)]
        return t, M, A, G, m, P
    return run


def _pade(k, m, w):
    num = sum(factorial(k + m - j) * factorial(k) / (factorial(k + m) * factorial(j) * factorial(k - j)) * w ** j
              for j in range(k + 1))
    den = sum(factorial(k + m - j) * factorial(m) / (factorial(k + m) * factorial(j) * factorial(m - j)) * (-w) ** j
              for j in range(m + 1))
    return num / den


def test_radau_points_closed_form(temporal):
    assert np.array_equal(temporal(0)[0], [1.0])
    assert np.allclose(temporal(1)[0], [1 / 3, 1.0], rtol=0, atol=1e-15)
    s6 = np.sqrt(6.0)
    assert np.allclose(temporal(2)[0], [(4 - s6) / 10, (4 + s6) / 10, 1.0], rtol=0, atol=1e-15)


@pytest.mark.parametrize("r", [0, 1, 2, 3, 4, 5])
def test_amplification_is_the_radau_pade_approximant(temporal, r):
    t, M, A, G, m, _ = temporal(r)
    for w in (-0.3, -1.0, -4.0, -25.0, 0.4):
        y = np.linalg.solve(A - w * M, m)
        assert abs(y[-1] - _pade(r, r + 1, w)) <= 1e-12 * max(1.0, abs(y[-1]))
    assert np.abs(M @ G - A).max() <= 1e-13


@pytest.mark.parametrize("r", [0, 1, 2, 3])
def test_matrices_and_transfers_equal_the_oracle(temporal, r):
    t, M, A, G, m, P = temporal(r)
    to, Mo, Ao, mo = spacetime.temporal_matrices(r)
    for a, b in ((t, to), (M, Mo), (A, Ao), (m, mo), (G, np.linalg.solve(Mo, Ao))):
        assert np.abs(a - b).max() <= 1e-13 * max(1.0, np.abs(b).max())
    for rc in range(r):
        assert np.abs(P[rc] - spacetime.time_prolongation(rc, r)).max() <= 1e-14


def test_c_abi_temporal_matrices_without_a_device():
    """mfns_spacetime_temporal through the built shared library (host code, no device needed)."""
    import __graft_entry__ as g
    from paper_2603_29621_gb300 import _lib as L, api

    g.build()
    for r in (0, 1, 3):
        t, m, M, A, G = api.temporal_matrices(r)
        to, Mo, Ao, mo = spacetime.temporal_matrices(r)
        assert np.abs(t - to).max() <= 1e-14 and np.abs(m - mo).max() <= 1e-13
        assert np.abs(M - Mo).max() <= 1e-14 and np.abs(A - Ao).max() <= 1e-13
        assert np.abs(G - np.linalg.solve(Mo, Ao)).max() <= 1e-12 * np.abs(G).max()
    with pytest.raises(L.MfnsError) as e:
        api.temporal_matrices(8)
    assert e.value.code == L.ERR_ARG
