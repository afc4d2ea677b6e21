"""Pins of the oracle's 1D/tensor finite-element ingredients against closed forms."""
import numpy as np
import pytest

from oracle import fe


def test_gll_closed_forms():
    # GLL points are the end points and the roots of P_k'; closed forms for k <= 4
    assert np.allclose(fe.gll_points(1), [0, 1])
    assert np.allclose(fe.gll_points(2), [0, 0.5, 1])
    s5 = 1 / np.sqrt(5)
    assert np.allclose(fe.gll_points(3), [0, (1 - s5) / 2, (1 + s5) / 2, 1], atol=1e-15)
    s37 = np.sqrt(3 / 7)
    assert np.allclose(fe.gll_points(4), [0, (1 - s37) / 2, 0.5, (1 + s37) / 2, 1], atol=1e-15)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 6])
def test_gauss_exact_monomials(q):
    x, w = fe.gauss(q)
    assert abs(w.sum() - 1) < 1e-15
    for p in range(2 * q):
        assert abs((w * x ** p).sum() - 1.0 / (p + 1)) < 1e-14
    # and not exact one degree higher (pins the number of points)
    assert abs((w * x ** (2 * q)).sum() - 1.0 / (2 * q + 1)) > 1e-8


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_lagrange_property_and_reproduction(k):
    nodes = fe.gll_points(k)
    val, d1, d2 = fe.basis_1d(nodes, nodes)
    assert np.allclose(val, np.eye(k + 1), atol=1e-14)
    xs = np.linspace(0, 1, 17)
    val, d1, d2 = fe.basis_1d(nodes, xs)
    assert np.allclose(val.sum(0), 1, atol=1e-13)         # partition of unity
    assert np.allclose(d1.sum(0), 0, atol=1e-11)
    for p in range(k + 1):                                 # exact for x^p, p <= k
        coef = nodes ** p
        assert np.allclose(coef @ val, xs ** p, atol=1e-12)
        assert np.allclose(coef @ d1, p * xs ** max(p - 1, 0) if p > 0 else 0, atol=1e-10)
        assert np.allclose(coef @ d2, p * (p - 1) * xs ** max(p - 2, 0) if p > 1 else 0, atol=1e-8)


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 3), (3, 2)])
def test_tensor_tables(dim, k):
    q = k + 1
    phi, dphi, d2phi, w, xq = fe.reference_tables(dim, k, q)
    nb = (k + 1) ** dim
    assert phi.shape == (q ** dim, nb)
    assert np.allclose(phi.sum(1), 1)
    assert abs(w.sum() - 1) < 1e-14
    # node ordering x fastest: basis function 1 is the node at xi_0 = GLL[1]
    nodes = fe.gll_points(k)
    vals = fe.eval_basis_at(dim, k, np.array([[nodes[1]] + [0.0] * (dim - 1)]))
    assert np.argmax(vals[0]) == 1
    # gradients of the interpolant of x*y (+z) reproduce the exact gradient
    ni = fe.tensor_index(dim, k + 1)
    X = nodes[ni]
    u = X[:, 0] * X[:, 1] + (X[:, 2] if dim == 3 else 0)
    g = np.einsum("qbd,b->qd", dphi, u)
    exact = np.stack([xq[:, 1], xq[:, 0]] + ([np.ones(len(xq))] if dim == 3 else []), axis=1)
    assert np.allclose(g, exact, atol=1e-12)
