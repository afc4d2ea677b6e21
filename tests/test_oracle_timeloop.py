"""Pins of the oracle's nonlinear residual, Newton iteration and variable-step BDF2.

* The linearised operator (already pinned by the operator tests) is the derivative of the
  residual with tau frozen: central differences agree to round-off, on uniform and hanging
  meshes, in 2D and 3D.
* A flow linear in space and quadratic in time (divergence-free, pressure linear in space,
  forcing from the equations) is reproduced exactly by BDF2 with variable steps: the BDF2
  formula is exact for quadratics in time and the fields lie in Q_k, so the strong residual
  vanishes at every point.  BDF1 is exact for flows linear in time.
* Newton converges quadratically.
* The 2D Taylor--Green vortex (exact Navier--Stokes solution, time-dependent boundary
  values) is approximated with an error that falls as h and dt are refined.
"""
import numpy as np
import pytest

from oracle import assemble, mesh, timeloop


def _linear_flow(dim, seed, quadratic=True):
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1, 1, (3, dim))
    e = rng.uniform(-1, 1, (3, dim))
    B = rng.uniform(-1, 1, (3, dim, dim))
    for q in range(3):
        B[q] -= np.eye(dim) * np.trace(B[q]) / dim
    if not quadratic:
        a[2] = e[2] = 0.0
        B[2] = 0.0

    def ev(C, t):
        return C[0] + C[1] * t + C[2] * t * t

    def dv(C, t):
        return C[1] + 2 * C[2] * t

    def fields(p, t):
        x = p.dofs.nodesets[0].x
        u = ev(a, t)[None] + x @ ev(B, t).T
        pr = x @ ev(e, t)
        f = dv(a, t)[None] + x @ dv(B, t).T + u @ ev(B, t).T + ev(e, t)[None]
        return np.concatenate([u.T.ravel(), pr]), np.concatenate([f.T.ravel(), np.zeros(len(pr))])

    return fields


@pytest.mark.parametrize("dim,n,k,ball", [(2, 3, 2, False), (3, 2, 2, False), (2, 2, 3, True), (3, 2, 1, True)])
def test_jacobian_is_the_derivative_of_the_residual(dim, n, k, ball):
    f = mesh.uniform(dim, n)
    if ball:
        f = mesh.refine_ball(f, (0.3, 0.3, 0.3), 0.3, 1)
    p = assemble.Problem(f, "stab_ns", k, nu=2e-2, dt=0.05, alpha=1.5)
    d = p.dofs
    rng = np.random.default_rng(3)
    U0 = d.set_hanging(p.state_vector() + 0.2 * rng.uniform(-1, 1, d.n_dofs))
    g = rng.uniform(-1, 1, d.n_dofs)
    V = rng.uniform(-1, 1, d.n_dofs)
    V[d.dirichlet] = 0.0
    V = d.set_hanging(V)
    p.set_state(U0, g)
    JV = p.assemble() @ V
    eps = 1e-5
    p.set_state(U0 + eps * V, g)
    Fp = p.residual(tau_state=U0)
    p.set_state(U0 - eps * V, g)
    Fm = p.residual(tau_state=U0)
    fd = (Fp - Fm) / (2 * eps)
    fr = d.free
    assert np.linalg.norm(fd[fr] - JV[fr]) <= 1e-9 * np.linalg.norm(JV[fr])
    assert np.all(Fp[d.constrained] == 0.0)


@pytest.mark.parametrize("dim,n,k", [(2, 3, 2), (3, 2, 2), (2, 2, 3)])
def test_residual_vanishes_for_a_linear_flow(dim, n, k):
    p = assemble.Problem(mesh.uniform(dim, n), "stab_ns", k, nu=0.05, dt=0.1, alpha=1.5)
    fields = _linear_flow(dim, 5)
    U, _ = fields(p, 0.0)
    # g chosen so that the strong residual vanishes: g = -(c_m u + u.grad u + grad p)
    x = p.dofs.nodesets[0].x
    rng = np.random.default_rng(5)
    B = rng.uniform(-1, 1, (dim, dim))
    B -= np.eye(dim) * np.trace(B) / dim
    a, e = rng.uniform(-1, 1, dim), rng.uniform(-1, 1, dim)
    u = a[None] + x @ B.T
    U = np.concatenate([u.T.ravel(), x @ e])
    gv = -(1.5 / 0.1 * u + u @ B.T + e[None])
    g = np.concatenate([gv.T.ravel(), np.zeros(len(x))])
    p.set_state(U, g)
    F = p.residual()
    scale = np.linalg.norm(p.assemble() @ U)
    assert np.linalg.norm(F) <= 1e-12 * scale
    # a wrong explicit field leaves a residual
    p.set_state(U, g * 1.01)
    assert np.linalg.norm(p.residual()) > 1e-6 * scale


@pytest.mark.parametrize("dim,n,k", [(2, 3, 2), (3, 2, 2)])
def test_bdf2_variable_steps_exact_for_quadratic_in_time_flow(dim, n, k):
    p = assemble.Problem(mesh.uniform(dim, n), "stab_ns", k, nu=0.05, dt=0.1)
    fields = _linear_flow(dim, 1)
    ts = [0.0, 0.1, 0.23, 0.30, 0.36]
    u_nm1, u_n = fields(p, ts[0])[0], fields(p, ts[1])[0]
    for j in range(2, len(ts)):
        dt = ts[j] - ts[j - 1]
        om = dt / (ts[j - 1] - ts[j - 2])
        Uex, f = fields(p, ts[j])
        guess = u_n.copy()
        guess[p.dofs.dirichlet] = Uex[p.dofs.dirichlet]
        U, hist = timeloop.bdf_step(p, u_n, u_nm1, dt, om, guess, forcing=f)
        assert len(hist) <= 6
        d = p.project_pressure_mean(U - Uex)
        assert np.linalg.norm(d) <= 1e-9 * np.linalg.norm(Uex)
        u_nm1, u_n = u_n, U


def test_bdf1_exact_for_linear_in_time_flow():
    p = assemble.Problem(mesh.uniform(2, 3), "stab_ns", 2, nu=0.05, dt=0.1)
    fields = _linear_flow(2, 2, quadratic=False)
    u0 = fields(p, 0.0)[0]
    Uex, f = fields(p, 0.1)
    guess = u0.copy()
    guess[p.dofs.dirichlet] = Uex[p.dofs.dirichlet]
    U, _ = timeloop.bdf_step(p, u0, None, 0.1, 0.0, guess, forcing=f)
    assert np.linalg.norm(p.project_pressure_mean(U - Uex)) <= 1e-9 * np.linalg.norm(Uex)


def test_newton_converges_quadratically():
    p = assemble.Problem(mesh.uniform(2, 4), "stab_ns", 2, nu=1e-2, dt=0.05)
    un = p.state_vector()
    U, hist = timeloop.bdf_step(p, un, 1.05 * un, 0.05, 1.0, un.copy())
    assert hist[-1] <= 1e-10 * hist[0] and len(hist) <= 6
    for r0, r1 in zip(hist[:-1], hist[1:]):
        if r1 > 1e-9 * hist[0]:
            assert r1 <= r0 * r0 / hist[0]


def _tg_exact(p, t, nu):
    x = p.dofs.nodesets[0].x
    F = np.exp(-2 * np.pi ** 2 * nu * t)
    X, Y = x[:, 0], x[:, 1]
    u = np.sin(np.pi * X) * np.cos(np.pi * Y) * F
    v = -np.cos(np.pi * X) * np.sin(np.pi * Y) * F
    pr = 0.25 * (np.cos(2 * np.pi * X) + np.cos(2 * np.pi * Y)) * F * F
    return np.concatenate([u, v, pr])


def test_taylor_green_vortex_error_falls_with_h_and_dt():
    nu, T = 0.05, 0.2
    errs = []
    for n, dt in ((4, 0.05), (8, 0.025)):
        p = assemble.Problem(mesh.uniform(2, n), "stab_ns", 2, nu=nu, dt=dt)
        d = p.dofs
        nv = 2 * d.nodesets[0].n_nodes
        u_nm1, u_n = _tg_exact(p, 0.0, nu), _tg_exact(p, dt, nu)
        steps = int(round(T / dt))
        for s in range(2, steps + 1):
            Uex = _tg_exact(p, s * dt, nu)
            guess = 2 * u_n - u_nm1
            guess[d.dirichlet] = Uex[d.dirichlet]
            U, _ = timeloop.bdf_step(p, u_n, u_nm1, dt, 1.0, guess)
            u_nm1, u_n = u_n, U
        errs.append(np.linalg.norm((U - Uex)[:nv]) / np.linalg.norm(Uex[:nv]))
    assert errs[0] < 5e-3 and errs[1] < 6e-4 and errs[0] / errs[1] > 4


def test_cfl_dt():
    p = assemble.Problem(mesh.uniform(2, 4), "stab_ns", 2, nu=1e-2, dt=0.05)
    U = p.state_vector()
    n = p.dofs.nodesets[0].n_nodes
    umax = np.sqrt(U[:n] ** 2 + U[n:2 * n] ** 2).max()
    assert timeloop.cfl_dt(p, U, 0.5) == pytest.approx(0.5 * 0.25 / umax)
