"""Pins of the oracle's smoothers and Krylov solvers against closed forms."""
import numpy as np
import numpy.polynomial.chebyshev as C
import pytest
import scipy.sparse as sp

from oracle import assemble, mesh, solvers


@pytest.mark.parametrize("degree", [1, 3, 5])
def test_chebyshev_closed_form_on_diagonal(degree):
    lam = np.linspace(0.05, 1.9, 40)
    A = sp.diags(lam)
    lmax = 2.0
    lmin = lmax / 20
    e0 = np.random.default_rng(0).uniform(-1, 1, len(lam))
    x = solvers.chebyshev(A, np.ones_like(lam), np.zeros_like(lam), e0, degree, lmax)  # b = 0: x is the error
    theta, delta = (lmax + lmin) / 2, (lmax - lmin) / 2
    Td = lambda t: C.chebval(t, [0] * degree + [1])
    expect = Td((theta - lam) / delta) / Td(theta / delta) * e0
    assert np.allclose(x, expect, atol=1e-14)
    # from a zero start, degree d uses d - 1 products and equals the same polynomial on b
    b = e0 * lam
    calls = []

    class Counting:
        def __matmul__(self, v):
            calls.append(1)
            return A @ v

    x0 = solvers.chebyshev(Counting(), np.ones_like(lam), b, np.zeros_like(lam), degree, lmax, x_is_zero=True)
    assert len(calls) == degree - 1
    exact = b / lam
    assert np.allclose(x0 - exact, expect * (-1) * (exact / e0), atol=1e-13)


def test_jacobi_relaxation_closed_form():
    lam = np.linspace(0.1, 1.5, 20)
    e0 = np.ones(20)
    x = solvers.jacobi_relaxation(sp.diags(lam), np.ones(20), np.zeros(20), e0, 5, 2.0)
    w = 2 / (2.0 + 0.1)
    assert np.allclose(x, (1 - w * lam) ** 5 * e0, atol=1e-15)


def test_cg_fixed_finite_termination():
    rng = np.random.default_rng(3)
    B = rng.normal(size=(8, 8))
    M = B @ B.T + 8 * np.eye(8)
    b = rng.normal(size=8)
    x = solvers.cg_jacobi_fixed(M, 1 / np.diag(M), b, 8)
    assert np.allclose(x, np.linalg.solve(M, b), atol=1e-10)


def test_fgmres_exact_preconditioner_one_iteration():
    rng = np.random.default_rng(4)
    A = rng.normal(size=(30, 30)) + 10 * np.eye(30)
    b = rng.normal(size=30)
    Ainv = np.linalg.inv(A)
    x, it, rel = solvers.fgmres(A, b, lambda v: Ainv @ v, tol=1e-12)
    assert it == 1 and rel < 1e-12
    x2, it2, rel2 = solvers.fgmres(A, b, lambda v: v, tol=1e-12, restart=7)
    assert rel2 < 1e-12 and np.allclose(x2, np.linalg.solve(A, b), atol=1e-10)


def test_fgmres_stab_ns_matches_direct_with_vcycle():
    f = mesh.uniform(2, 4)
    levels = solvers.hierarchy(f, "stab_ns", 2, nu=0.05, dt=0.05)
    lmax = [1.2 * solvers.power_lmax(lv.A, lv.dinv) for lv in levels[:-1]]
    vc = solvers.VCycle(levels, lmax, ("chebyshev", 3))
    p = levels[0].problem
    A = levels[0].A
    b = np.random.default_rng(5).uniform(-1, 1, A.shape[0])
    b[p.dofs.constrained] = 0
    x, it, rel = solvers.fgmres(A, b, vc, tol=1e-11, project=p.project_pressure_mean)
    xd = assemble.solve_direct(p, b, A)
    d = p.project_pressure_mean(x) - p.project_pressure_mean(xd)
    assert rel < 1e-11 and it < 40 and np.abs(d).max() < 1e-8 * np.abs(xd).max()


def test_stokes_block_preconditioned_fgmres():
    f = mesh.refine_ball(mesh.uniform(2, 4), (0.3, 0.3, 0.3), 0.3, 1)
    nu = 1.0
    prob = assemble.Problem(f, "stokes", 2, nu=nu)
    A = prob.assemble()
    levels = solvers.hierarchy(f, "stokes_a", 2, nu=nu)
    lmax = [1.2 * solvers.power_lmax(lv.A, lv.dinv) for lv in levels[:-1]]
    vc = solvers.VCycle(levels, lmax, ("chebyshev", 5))
    Mp = assemble.Problem(f, "pmass", 1).assemble()
    M = solvers.StokesBlockPreconditioner(prob, A, vc, Mp)
    b = np.random.default_rng(6).uniform(-1, 1, A.shape[0])
    b[prob.dofs.constrained] = 0
    x, it, rel = solvers.fgmres(A, b, M, tol=1e-10, project=prob.project_pressure_mean)
    xd = assemble.solve_direct(prob, b, A)
    d = prob.project_pressure_mean(x) - prob.project_pressure_mean(xd)
    assert rel < 1e-10 and it < 60 and np.abs(d).max() < 1e-7 * np.abs(xd).max(), (it, rel)


def test_vcycle_convergence_factor():
    f = mesh.uniform(3, 4)
    levels = solvers.hierarchy(f, "stokes_a", 2, nu=1.0)
    assert [lv.problem.k for lv in levels] == [2, 1, 1]
    lmax = [1.2 * solvers.power_lmax(lv.A, lv.dinv) for lv in levels[:-1]]
    vc = solvers.VCycle(levels, lmax, ("chebyshev", 5))
    A = levels[0].A
    rng = np.random.default_rng(7)
    b = rng.uniform(-1, 1, A.shape[0])
    x = np.zeros_like(b)
    res = [np.linalg.norm(b)]
    for _ in range(6):
        x = x + vc(b - A @ x)
        res.append(np.linalg.norm(b - A @ x))
    rate = (res[-1] / res[1]) ** (1 / 5)
    assert rate < 0.15, res
