"""Pins of the oracle's space-time discretisation (Section 4).

* Right Gauss--Radau points in closed form (Q = 1, 2, 3).
* DG(r) in time on a scalar ODE y' = lambda y: the one-slab amplification is the (r, r+1) Pade
  approximant of exp (the Radau IIA stability function), for r = 0..3.
* DG(r) reproduces solutions that are polynomials of degree <= r in time.
* With r = 0 the Kronecker operator is backward Euler, M + tau A.
* One slab of the transient Stokes problem reproduces a manufactured discrete solution
  c(t) (U, P), c a polynomial of degree <= r (pressure up to one constant per stage), on a mesh with
  hanging nodes.
* Time transfers are exact for polynomials of the coarse temporal degree.
"""
from math import factorial

import numpy as np
import pytest

from oracle import mesh, spacetime


def test_radau_points_closed_form():
    assert np.allclose(spacetime.radau_right(1), [1.0], atol=0, rtol=0)
    assert np.allclose(spacetime.radau_right(2), [1 / 3, 1.0], atol=1e-15)
    s6 = np.sqrt(6.0)
    assert np.allclose(spacetime.radau_right(3), [(4 - s6) / 10, (4 + s6) / 10, 1.0], atol=1e-15)


def _pade(k, m, w):
    num = sum(factorial(k + m - j) * factorial(k) / (factorial(k + m) * factorial(j) * factorial(k - j)) * w ** j
              for j in range(k + 1))
    den = sum(factorial(k + m - j) * factorial(m) / (factorial(k + m) * factorial(j) * factorial(m - j)) * (-w) ** j
              for j in range(m + 1))
    return num / den


@pytest.mark.parametrize("r", [0, 1, 2, 3])
def test_amplification_is_the_radau_pade_approximant(r):
    t, M, A, m = spacetime.temporal_matrices(r)
    for w in (-0.3, -1.0, -4.0, -25.0, 0.4):
        y = np.linalg.solve(A - w * M, m)            # y' = lambda y, w = lambda tau, y(t_{n-1}) = 1
        assert abs(y[-1] - _pade(r, r + 1, w)) <= 1e-13 * max(1.0, abs(y[-1]))


@pytest.mark.parametrize("r", [0, 1, 2, 3])
def test_polynomials_of_degree_r_in_time_are_exact(r):
    t, M, A, m = spacetime.temporal_matrices(r)
    rng = np.random.default_rng(r)
    a = rng.uniform(-1, 1, r + 1)                    # y(s) = sum a_j s^j on the reference slab
    lam, tau = -2.5, 0.7
    y = lambda s: sum(a[j] * s ** j for j in range(r + 1))
    dy = lambda s: sum(j * a[j] * s ** (j - 1) for j in range(1, r + 1))
    # y' = lam y + f  on [0, tau], with s = t / tau:  f(t) = dy/tau - lam y
    from oracle import fe
    xg, wg = fe.gauss(r + 3)
    phi = np.array([[fe.lagrange_value(t, j, s) for s in xg] for j in range(r + 1)])
    F = tau * (phi * wg[None, :]) @ np.array([dy(s) / tau - lam * y(s) for s in xg])
    stages = np.linalg.solve(A - lam * tau * M, F + m * y(0.0))
    assert np.abs(stages - np.array([y(s) for s in t])).max() <= 1e-13


def test_dg0_kronecker_operator_is_backward_euler():
    st = spacetime.SpaceTimeStokes(mesh.uniform(2, 3), 2, 0, nu=0.7, tau=0.3, pressure="continuous")
    assert np.allclose(st.G_Q, [[1.0]])
    K = st.operator()
    assert abs(K - (st.M + 0.3 * st.A)).max() <= 1e-15


@pytest.mark.parametrize("pressure", ["continuous", "disc"])
@pytest.mark.parametrize("r", [0, 1, 2])
def test_slab_reproduces_a_manufactured_solution(r, pressure):
    f = mesh.refine_ball(mesh.uniform(2, 3), (0.3, 0.35, 0.4), 0.3, 1)
    tau, t0 = 0.25, 0.4
    st = spacetime.SpaceTimeStokes(f, 2, r, nu=0.8, tau=tau, pressure=pressure)
    d = st.space.dofs
    assert d.hanging.any()
    rng = np.random.default_rng(7 + r)
    X = d.distribute(rng.uniform(-1, 1, d.n_dofs))   # a discrete (U, P) with consistent hanging entries
    a = rng.uniform(-1, 1, r + 1)
    c = lambda t: sum(a[j] * (t - t0) ** j for j in range(r + 1))
    dc = lambda t: sum(j * a[j] * (t - t0) ** (j - 1) for j in range(1, r + 1))
    MX, AX = st.M @ X, st.A @ X
    load = lambda t: dc(t) * MX + c(t) * AX          # M u' + A x = f on the free rows
    b = st.rhs(load, c(t0) * X, t0)
    stage_t = t0 + st.nodes * tau
    b = st.set_constrained(b, [c(t) * X for t in stage_t])
    K = st.operator().toarray()
    x = np.linalg.lstsq(K, b, rcond=None)[0].reshape(st.Q, st.n)
    en = st.pressure_null()
    for q, t in enumerate(stage_t):
        e = x[q] - c(t) * X
        e -= (e @ en) / (en @ en) * en                 # the stage's pressure constant is free
        assert np.abs(e).max() <= 1e-10 * np.abs(X).max(), (q, np.abs(e).max())


@pytest.mark.parametrize("rc,rf", [(0, 1), (1, 2), (1, 3), (2, 3)])
def test_time_transfer_exact_for_coarse_polynomials(rc, rf):
    P = spacetime.time_prolongation(rc, rf)
    tc, tf = spacetime.radau_right(rc + 1), spacetime.radau_right(rf + 1)
    rng = np.random.default_rng(rc * 10 + rf)
    a = rng.uniform(-1, 1, rc + 1)
    poly = lambda s: sum(a[j] * s ** j for j in range(rc + 1))
    assert np.abs(P @ poly(tc) - poly(tf)).max() <= 1e-14


def test_stmg_level_sequence_follows_the_coarsening_rules():
    """Space before time (R1), polynomial before geometric in each (R2): the spatial degree halved
    (k >= 2 kept), then h in space, then the temporal degree on the coarsest mesh (time-marching: no
    coarsening of tau).  With vertex stars the temporal steps are left out when one star holds every
    cell of the coarsest mesh."""
    lv = spacetime.stmg_levels(mesh.uniform(2, 4), 4, 3, tau=0.1)
    seq = [(l.k, l.r, l.st.space.forest.n) for l in lv]
    assert seq == [(4, 3, 4), (2, 3, 4), (2, 3, 2), (2, 1, 2), (2, 0, 2)]
    assert all(l.st.tau == 0.1 for l in lv)
    lv = spacetime.stmg_levels(mesh.uniform(2, 4), 4, 3, tau=0.1, pressure="continuous")
    assert [(l.k, l.r, l.st.space.forest.n) for l in lv] == [(4, 3, 4), (2, 3, 4), (2, 3, 2)]
    lv = spacetime.stmg_levels(mesh.uniform(2, 8), 2, 1, tau=0.1, pressure="continuous", stop_n=4)
    assert [(l.k, l.r, l.st.space.forest.n) for l in lv] == [(2, 1, 8), (2, 1, 4), (2, 0, 4)]


def test_stmg_iterations_do_not_grow_under_refinement():
    """Section 4 reports iteration counts that do not grow under h-refinement (tau refined with h):
    with the paper's pair Q2/P1^disc, DG(1) and cell patches, FGMRES needs the same few iterations
    at n = 4, 8 and 16."""
    from oracle import solvers
    its = []
    for n in (4, 8, 16):
        lv = spacetime.stmg_levels(mesh.uniform(2, n), 2, 1, nu=1.0, tau=0.2 / n, pressure="disc")
        V = spacetime.STMG(lv)
        K = lv[0].K
        d = lv[0].st.space.dofs
        xs = V.project(np.tile(d.distribute(np.random.default_rng(1).uniform(-1, 1, d.n_dofs)), lv[0].st.Q))
        x, it, res = solvers.fgmres(K, K @ xs, V, tol=1e-10, maxit=100, project=V.project)
        assert res <= 1e-10
        its.append(it)
    assert max(its) <= 8 and max(its) - min(its) <= 2, its


@pytest.mark.parametrize("pressure,patch,omega", [("continuous", "vertex", 0.7), ("continuous", "cell", 0.5),
                                                   ("disc", "cell", 0.7)])
def test_damped_schwarz_contracts_except_the_pressure_constants(pressure, patch, omega):
    """I - omega S K on the free entries: one eigenvalue 1 per stage (the constant pressure, a null
    direction of K) and every other eigenvalue inside the unit disc.  (Cell patches on Taylor--Hood
    need the stronger damping: with omega = 0.7 their iteration is slightly expansive.)"""
    lv = spacetime.StLevel(mesh.uniform(2, 3), 2, 1, 1.0, 0.05, patch=patch, pressure=pressure)
    K = lv.K.toarray()
    N = K.shape[0]
    S = np.stack([lv.schwarz(e) for e in np.eye(N)], axis=1)
    free = ~lv.con
    E = (np.eye(N) - omega * S @ K)[np.ix_(free, free)]
    ev = np.sort(np.abs(np.linalg.eigvals(E)))[::-1]
    Q = lv.st.Q
    assert np.all(np.abs(ev[:Q] - 1.0) <= 1e-8)
    assert ev[Q] < 0.999


@pytest.mark.parametrize("dim", [2, 3])
def test_coarse_solve_is_the_pseudo_inverse(dim):
    """The coarsest solve returns the minimum-norm least-squares solution: K x is the part of b in
    the range of K (b minus its constant-pressure components, K being singular exactly along those)
    and x has no component along the constant pressures."""
    lv = spacetime.stmg_levels(mesh.uniform(dim, 4), 2, 1, nu=1.0, tau=0.05, pressure="continuous")
    V = spacetime.STMG(lv)
    C = lv[-1]
    K = C.K.toarray()
    b = np.random.default_rng(4).uniform(-1, 1, K.shape[0])
    x = V.coarse @ b
    e1 = C.st.pressure_null()
    Pb = b.copy()
    for q in range(C.st.Q):                          # one constant pressure per stage
        e = np.zeros(K.shape[0])
        e[q * C.st.n:(q + 1) * C.st.n] = e1 / np.linalg.norm(e1)
        Pb -= (b @ e) * e
        assert abs(x @ e) <= 1e-8 * np.abs(x).max()
    assert np.abs(K @ x - Pb).max() <= 1e-8 * np.abs(b).max()
    assert np.abs(x).max() <= 1e8 * np.abs(b).max()


@pytest.mark.parametrize("pressure", ["disc", "continuous"])
@pytest.mark.parametrize("n,k,r", [(8, 2, 1), (4, 3, 2), (8, 2, 0)])
def test_stmg_preconditioned_fgmres_converges(n, k, r, pressure):
    from oracle import solvers
    lv = spacetime.stmg_levels(mesh.uniform(2, n), k, r, nu=1.0, tau=0.05, pressure=pressure)
    V = spacetime.STMG(lv)
    K = lv[0].K
    d = lv[0].st.space.dofs
    rng = np.random.default_rng(1)
    xs = V.project(np.tile(d.distribute(rng.uniform(-1, 1, d.n_dofs)), lv[0].st.Q))
    # the error is bounded by the condition number (1e3..1e4 here) times the residual
    x, its, res = solvers.fgmres(K, K @ xs, V, tol=1e-12, maxit=200, project=V.project)
    assert res <= 1e-12 and its <= 50, its
    assert np.abs(V.project(x - xs)).max() <= 1e-8 * np.abs(xs).max()


def test_stmg_preconditioned_fgmres_converges_in_3d():
    from oracle import solvers
    lv = spacetime.stmg_levels(mesh.uniform(3, 4), 2, 1, nu=1.0, tau=0.05, pressure="continuous")
    V = spacetime.STMG(lv)
    K = lv[0].K
    d = lv[0].st.space.dofs
    rng = np.random.default_rng(1)
    xs = V.project(np.tile(d.distribute(rng.uniform(-1, 1, d.n_dofs)), lv[0].st.Q))
    x, its, res = solvers.fgmres(K, K @ xs, V, tol=1e-10, maxit=200, project=V.project)
    assert res <= 1e-10 and its <= 20, its
    assert np.abs(V.project(x - xs)).max() <= 1e-7 * np.abs(xs).max()
