"""1D finite-element ingredients on the unit interval [0, 1].

Oracle (test infrastructure only).  Q_k elements use Lagrange polynomials on
Gauss--Lobatto--Legendre (GLL) points; integrals use Gauss--Legendre
quadrature with q = k_u + 1 points per direction (the velocity degree plus
one), the standard choice for the matrix-free operators of Section 1/2.
"""
import numpy as np
from numpy.polynomial import legendre as L
from numpy.polynomial import Polynomial


def gll_points(k):
    """GLL points of degree k on [0, 1]: the end points and the roots of P_k'."""
    if k < 1:
        raise ValueError("degree must be >= 1")
    if k == 1:
        return np.array([0.0, 1.0])
    inner = np.sort(L.Legendre.basis(k).deriv().roots().real)
    pts = np.concatenate(([-1.0], inner, [1.0]))
    x = 0.5 * (pts + 1.0)
    # enforce exact symmetry and the exact midpoint for even k
    x = 0.5 * (x + (1.0 - x[::-1]))
    if k % 2 == 0:
        x[k // 2] = 0.5
    x[0], x[-1] = 0.0, 1.0
    return x


def gauss(q):
    """Gauss--Legendre points and weights on [0, 1] with q points."""
    t, w = L.leggauss(q)
    return 0.5 * (t + 1.0), 0.5 * w


def lagrange_value(nodes, a, x):
    """Value of the a-th Lagrange polynomial on ``nodes`` at x, product form.

    The product form returns an exact 0 at the other nodes and an exact 1 at
    node a, which keeps hanging-node weights free of round-off noise."""
    x = np.asarray(x, dtype=float)
    v = np.ones_like(x)
    for m, xm in enumerate(nodes):
        if m != a:
            v = v * (x - xm) / (nodes[a] - xm)
    return v


def lagrange_poly(nodes, a):
    """The a-th Lagrange polynomial as a numpy Polynomial (for derivatives)."""
    p = Polynomial([1.0])
    for m, xm in enumerate(nodes):
        if m != a:
            p = p * Polynomial([-xm, 1.0]) / (nodes[a] - xm)
    return p


def basis_1d(nodes, x):
    """Tables (n_nodes, len(x)) of values, first and second derivatives."""
    n = len(nodes)
    val = np.array([lagrange_value(nodes, a, x) for a in range(n)])
    d1 = np.array([lagrange_poly(nodes, a).deriv(1)(x) for a in range(n)])
    d2 = np.array([lagrange_poly(nodes, a).deriv(2)(x) if n > 2 else np.zeros_like(x)
                   for a in range(n)])
    return val, d1, d2


def tensor_index(dim, n):
    """Lexicographic multi-indices (x fastest) of an n^dim tensor grid, shape (n^dim, dim)."""
    grids = np.meshgrid(*([np.arange(n)] * dim), indexing="ij")
    # index = a0 + n*a1 + n^2*a2  ->  a0 varies fastest
    idx = np.stack([g.ravel() for g in grids[::-1]], axis=1)
    return idx


def reference_tables(dim, k, q):
    """Basis tables of the tensor-product Q_k element at the q^dim Gauss points.

    Returns (phi, dphi, d2phi, w, xq):
      phi   (nq, nb)        values
      dphi  (nq, nb, dim)   reference gradients
      d2phi (nq, nb, dim)   diagonal of the reference Hessian (d^2/dx_d^2)
      w     (nq,)           reference quadrature weights
      xq    (nq, dim)       reference quadrature points
    Node and point ordering is lexicographic with x fastest.
    """
    nodes = gll_points(k)
    xg, wg = gauss(q)
    v1, d1, h1 = basis_1d(nodes, xg)          # (k+1, q)
    bi = tensor_index(dim, k + 1)             # (nb, dim)
    qi = tensor_index(dim, q)                 # (nq, dim)
    nb, nq = bi.shape[0], qi.shape[0]
    phi = np.ones((nq, nb))
    for d in range(dim):
        phi *= v1[bi[:, d]][:, qi[:, d]].T
    dphi = np.ones((nq, nb, dim))
    d2phi = np.ones((nq, nb, dim))
    for g in range(dim):           # derivative direction
        for d in range(dim):       # factor direction
            fac_d = (d1 if d == g else v1)[bi[:, d]][:, qi[:, d]].T
            fac_h = (h1 if d == g else v1)[bi[:, d]][:, qi[:, d]].T
            dphi[:, :, g] *= fac_d
            d2phi[:, :, g] *= fac_h
    w = np.ones(nq)
    for d in range(dim):
        w *= wg[qi[:, d]]
    xq = xg[qi]
    return phi, dphi, d2phi, w, xq


def eval_basis_at(dim, k, xi):
    """Values of all Q_k basis functions at reference points xi (npts, dim), product form."""
    nodes = gll_points(k)
    bi = tensor_index(dim, k + 1)
    xi = np.atleast_2d(xi)
    out = np.ones((xi.shape[0], bi.shape[0]))
    for d in range(dim):
        tab = np.array([lagrange_value(nodes, a, xi[:, d]) for a in range(k + 1)])  # (k+1, npts)
        out *= tab[bi[:, d]].T
    return out
