"""Host helpers of the smoother bounds (csrc/ritz.hpp), compiled with g++ and checked against
numpy: eigenvalues of small Hessenberg matrices (the Ritz values of an Arnoldi run) and the
relaxation weight that minimises max |1 - omega theta| over the upper half of the spectrum."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2603_29621_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include "ritz.hpp"
int main() {
  int m;
  if (std::scanf("%d", &m) != 1) return 1;
  std::vector<double> H((size_t)m * m);
  for (auto& v : H) if (std::scanf("%lf", &v) != 1) return 1;
  auto e = mfns::hessenberg_eigenvalues(H, m);
  std::printf("%zu\n", e.size());
  for (auto& z : e) std::printf("%.17g %.17g\n", z.real(), z.imag());
  std::printf("%.17g\n", mfns::relaxation_weight(e));
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("ritz")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def run(H):
        m = H.shape[0]
        inp = f"{m}\n" + " ".join(f"{v:.17g}" for v in H.ravel()) + "\n"
        out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
        k = int(out[0])
        ev = np.array([complex(*map(float, out[1 + i].split())) for i in range(k)])
        return ev, float(out[1 + k])
    return run


def _hessenberg(m, seed):
    rng = np.random.default_rng(seed)
    return np.triu(rng.uniform(-1, 1, (m, m)), -1)


def _match(a, b):
    """max over a of the distance to the nearest element of b (and vice versa)."""
    d = np.abs(a[:, None] - b[None, :])
    return max(d.min(axis=1).max(), d.min(axis=0).max())


@pytest.mark.parametrize("m,seed", [(1, 0), (2, 1), (5, 2), (12, 3), (30, 4), (30, 5)])
def test_eigenvalues_match_numpy(harness, m, seed):
    H = _hessenberg(m, seed)
    ev, _ = harness(H)
    ref = np.linalg.eigvals(H)
    assert len(ev) == m
    assert _match(ev, ref) <= 1e-9 * max(1.0, np.abs(H).max())
    if m >= 5:
        assert np.abs(ref.imag).max() > 1e-3  # complex pairs occur


def test_arnoldi_of_a_nonsymmetric_operator(harness):
    """Ritz values of 20 Arnoldi steps of a non-normal matrix equal the eigenvalues of its H."""
    rng = np.random.default_rng(6)
    n, m = 200, 20
    A = np.diag(np.linspace(0.1, 2.0, n)) + 0.3 * np.diag(rng.uniform(-1, 1, n - 1), 1) \
        - 0.3 * np.diag(rng.uniform(0, 1, n - 1), -1)
    V = np.zeros((n, m + 1))
    Hh = np.zeros((m + 1, m))
    v = rng.uniform(-1, 1, n)
    V[:, 0] = v / np.linalg.norm(v)
    for j in range(m):
        w = A @ V[:, j]
        for _ in range(2):
            h = V[:, :j + 1].T @ w
            w -= V[:, :j + 1] @ h
            Hh[:j + 1, j] += h
        Hh[j + 1, j] = np.linalg.norm(w)
        V[:, j + 1] = w / Hh[j + 1, j]
    H = Hh[:m, :m]
    ev, _ = harness(H)
    assert _match(ev, np.linalg.eigvals(H)) <= 1e-9


def test_relaxation_weight_is_the_minimax(harness):
    H = _hessenberg(30, 7)
    ev, w = harness(H)
    rho = np.abs(ev).max()
    S = ev[np.abs(ev) >= 0.5 * rho]
    grid = np.linspace(1e-6, 2.0 / np.abs(S).min(), 200001)
    f = np.abs(1 - grid[:, None] * S[None, :]).max(axis=1)
    fw = np.abs(1 - w * S).max()
    assert fw <= f.min() + 1e-9


def test_relaxation_weight_closed_form(harness):
    """Real eigenvalues: the minimax weight over S = {theta >= rho/2} is 2 / (min S + max S)."""
    rho = 3.0
    vals = np.linspace(0.1, rho, 40)           # diagonal H: its eigenvalues are these values
    ev, w = harness(np.diag(vals))
    S = vals[vals >= 0.5 * rho]
    assert w == pytest.approx(2.0 / (S.min() + S.max()), rel=1e-9)
