"""Pins of the oracle's Stokes pair with a discontinuous pressure, Q_k / P^disc_{k-1} (Section 4).

* Inf-sup stability on small meshes: the operator's null space is exactly the constant pressure
  (rank deficiency one, by brute force), in 2D and 3D.
* Closed-form energy: u = (phi, 2 phi), phi = x(1-x)y(1-y), p = x - 1/2 gives
  x^T K x = nu int |grad u|^2 - 2 int p div u = nu / 9 + 1/18.
* Transfers (velocity by interpolation, pressure by L2 projection) reproduce coarse-space
  polynomials exactly, for h- and p-steps.
"""
import numpy as np
import pytest

from oracle import mesh, pdisc


@pytest.mark.parametrize("dim,n,k", [(2, 3, 2), (2, 2, 3), (3, 2, 2)])
def test_null_space_is_the_constant_pressure(dim, n, k):
    P = pdisc.StokesPdisc(mesh.uniform(dim, n), k, nu=0.9)
    A = P.assemble().toarray()
    assert A.shape[0] - np.linalg.matrix_rank(A) == 1
    e = P.pressure_null()
    assert np.abs(A @ e).max() <= 1e-12 and np.abs(A.T @ e).max() <= 1e-12


def test_energy_closed_form():
    nu = 0.6
    P = pdisc.StokesPdisc(mesh.refine_ball(mesh.uniform(2, 3), (0.3, 0.35, 0.4), 0.3, 1), 2, nu=nu)
    phi = lambda x: np.prod(x * (1 - x), axis=1)
    xv = np.zeros(P.dofs.n_dofs)
    xv[:P.p_offset] = P.vel.interpolate(lambda x: np.stack([phi(x), 2 * phi(x)], axis=1))
    xv[P.p_offset:] = P.project_pressure(lambda x: x[:, 0] - 0.5)
    assert np.abs(P.dofs.distribute(xv) - xv).max() <= 1e-14
    energy = xv @ (P.assemble_K() @ xv)
    exact = nu / 9.0 + 1.0 / 18.0
    assert abs(energy - exact) <= 1e-12 * exact


@pytest.mark.parametrize("coarse,fine", [((2, 2), (4, 2)), ((3, 2), (3, 3)), ((2, 3), (4, 3))])
def test_transfers_exact_for_coarse_polynomials(coarse, fine):
    C = pdisc.StokesPdisc(mesh.uniform(2, coarse[0]), coarse[1])
    F = pdisc.StokesPdisc(mesh.uniform(2, fine[0]), fine[1])
    Pm = pdisc.prolongation(C, F)
    phi = lambda x: np.prod(x * (1 - x), axis=1)
    u = lambda x: np.stack([phi(x), -phi(x) * (1 + x[:, 1])], axis=1) if C.k >= 3 else \
        np.stack([phi(x), -phi(x)], axis=1)
    p = lambda x: x[:, 0] - 2 * x[:, 1] + 0.3 * x[:, 0] * x[:, 1] * (C.k >= 3)
    xc = np.zeros(C.dofs.n_dofs)
    xc[:C.p_offset] = C.vel.interpolate(u)
    xc[C.p_offset:] = C.project_pressure(p)
    xf = np.zeros(F.dofs.n_dofs)
    xf[:F.p_offset] = F.vel.interpolate(u) * F.vel.free
    xf[F.p_offset:] = F.project_pressure(p)
    assert np.abs(Pm @ xc - xf).max() <= 1e-12
