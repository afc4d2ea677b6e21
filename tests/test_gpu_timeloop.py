"""GPU parity of the nonlinear residual, the state-dependent Jacobian and the Newton/BDF steps
(Section 5) against the oracle, through the C ABI.

* residual F(U) at a perturbed state with an explicit field g: FP64 <= 1e-12, FP32 <= 2e-5
  (relative l2), constrained rows zero;
* the Jacobian at that state (mfns_vmult after mfns_set_state): same bounds;
* every multigrid level after mfns_set_state with a state and g that all levels represent
  exactly (Q1 functions): the level operators equal the oracle's at that state (h- and
  p-levels, nested and non-nested coarsening);
* mfns_bdf_step reproduces a flow linear in space and quadratic in time exactly with variable
  steps (FP64 and FP32 multigrid), and follows the oracle's Newton/BDF2 on the Taylor--Green
  vortex to 1e-8."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import assemble, mesh, timeloop  # noqa: E402
from paper_2603_29621_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = {0: 1e-12, 1: 2e-5}


@pytest.fixture(scope="module")
def ctx():
    from paper_2603_29621_gb300 import api
    return api.Context(0)


def _pair(ctx, dim, n, k, nu, dt, alpha=1.5, mg_precision=1, **kw):
    from paper_2603_29621_gb300 import _lib as L, api
    m = api.Mesh(ctx, dim, n)
    prob = api.Problem(ctx, m, kind=L.STAB_NS, degree=k, nu=nu, dt=dt, mg_precision=mg_precision, **kw)
    op = assemble.Problem(mesh.uniform(dim, n), "stab_ns", k, nu=nu, dt=dt, alpha=alpha)
    xg, fg = prob.support_points()
    xo, fo = op.dofs.support_points()
    perm = inputs.match_dofs(xg, fg, xo, fo)   # library index of oracle DoF i
    return prob, op, perm, m


def _to_lib(x, perm, dtype=torch.float64):
    y = np.empty_like(x)
    y[perm] = x
    return torch.tensor(y, device="cuda", dtype=dtype)


def _from_lib(t, perm):
    return t.double().cpu().numpy()[perm]


CASES = [(2, 4, 2), (3, 2, 2), (3, 3, 1), (2, 3, 3), (2, 2, 4), (3, 2, 3)]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}d-n{c[1]}-k{c[2]}")
def test_residual_and_jacobian_at_a_state(ctx, case, prec):
    dim, n, k = case
    nu, dt, alpha = 2e-2, 0.05, 1.3
    prob, op, perm, _ = _pair(ctx, dim, n, k, nu, dt, alpha)
    rng = np.random.default_rng(11)
    U = op.state_vector() + 0.3 * rng.uniform(-1, 1, op.dofs.n_dofs)
    g = rng.uniform(-1, 1, op.dofs.n_dofs)
    op.set_state(U, g)
    Fo = op.residual()
    A = op.assemble()
    prob.set_state(dt, alpha, _to_lib(U, perm), _to_lib(g, perm))
    dt_ = torch.float64 if prec == 0 else torch.float32
    F = torch.full((len(perm),), 7.0, device="cuda", dtype=dt_)
    prob.residual(F)
    Fg = _from_lib(F, perm)
    assert np.linalg.norm(Fg - Fo) <= TOL[prec] * np.linalg.norm(Fo)
    assert np.all(Fg[op.dofs.constrained] == 0.0)
    x = inputs.uniform_vector(len(perm))
    y = torch.empty(len(perm), device="cuda", dtype=dt_)
    prob.vmult(_to_lib(x, perm, dt_), y)
    yo = A @ x
    assert np.linalg.norm(_from_lib(y, perm) - yo) <= TOL[prec] * np.linalg.norm(yo)


def _q1_field(x, coef):
    """Sum of coef[j] * monomial_j over the Q1 monomials (1, x, y, xy, [z, xz, yz, xyz])."""
    dim = x.shape[1]
    mons = [np.ones(len(x)), x[:, 0], x[:, 1], x[:, 0] * x[:, 1]]
    if dim == 3:
        z = x[:, 2]
        mons += [z, x[:, 0] * z, x[:, 1] * z, x[:, 0] * x[:, 1] * z]
    return sum(c * m for c, m in zip(coef, mons))


def _q1_state(op, rng_seed):
    rng = np.random.default_rng(rng_seed)
    dim = op.dim
    x = op.dofs.nodesets[0].x
    nm = 4 if dim == 2 else 8
    C = rng.uniform(-1, 1, (2, dim + 1, nm))
    U = np.concatenate([_q1_field(x, C[0, c]) for c in range(dim + 1)])
    g = np.concatenate([_q1_field(x, C[1, c]) for c in range(dim + 1)])
    return C, U, g


@pytest.mark.parametrize("case", [(3, 4, 2), (2, 3, 3), (3, 3, 2)], ids=lambda c: f"{c[0]}d-n{c[1]}-k{c[2]}")
def test_state_reaches_every_level(ctx, case):
    from paper_2603_29621_gb300 import _lib as L
    dim, n, k = case
    nu, dt, alpha = 5e-2, 0.1, 1.5
    prob, op, perm, _ = _pair(ctx, dim, n, k, nu, dt, alpha, mg_precision=0)
    C, U, g = _q1_state(op, 4)
    prob.set_state(dt, alpha, _to_lib(U, perm), _to_lib(g, perm))
    info = prob.get_info()
    seen = set()
    for lvl in range(info.n_levels):
        kl, cells = info.level_degree[lvl], info.level_cells[lvl]
        nl = int(round(cells ** (1.0 / dim)))
        seen.add((nl, kl))
        ol = assemble.Problem(mesh.uniform(dim, nl), "stab_ns", kl, nu=nu, dt=dt, alpha=alpha)
        xo = ol.dofs.nodesets[0].x
        ol.set_state(np.concatenate([_q1_field(xo, C[0, c]) for c in range(dim + 1)]),
                     np.concatenate([_q1_field(xo, C[1, c]) for c in range(dim + 1)]))
        xg, fg = prob.support_points(lvl)
        xs, fs = ol.dofs.support_points()
        pl = inputs.match_dofs(xg, fg, xs, fs)
        x = inputs.uniform_vector(len(pl), seed=lvl)
        y = torch.empty(len(pl), device="cuda", dtype=torch.float64)
        prob.vmult(_to_lib(x, pl), y, which=lvl)
        yo = ol.assemble() @ x
        assert np.linalg.norm(_from_lib(y, pl) - yo) <= 1e-12 * np.linalg.norm(yo), (lvl, nl, kl)
    assert len(seen) == info.n_levels >= 3


def _linear_flow(dim, seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1, 1, (3, dim))
    e = rng.uniform(-1, 1, (3, dim))
    B = rng.uniform(-1, 1, (3, dim, dim))
    for q in range(3):
        B[q] -= np.eye(dim) * np.trace(B[q]) / dim

    def ev(Cf, t):
        return Cf[0] + Cf[1] * t + Cf[2] * t * t

    def dv(Cf, t):
        return Cf[1] + 2 * Cf[2] * t

    def fields(op, t):
        x = op.dofs.nodesets[0].x
        u = ev(a, t)[None] + x @ ev(B, t).T
        pr = x @ ev(e, t)
        f = dv(a, t)[None] + x @ dv(B, t).T + u @ ev(B, t).T + ev(e, t)[None]
        return np.concatenate([u.T.ravel(), pr]), np.concatenate([f.T.ravel(), np.zeros(len(pr))])

    return fields


@pytest.mark.parametrize("mgp", [0, 1], ids=["fp64mg", "fp32mg"])
@pytest.mark.parametrize("case", [(2, 3, 2), (3, 4, 2)], ids=lambda c: f"{c[0]}d-n{c[1]}-k{c[2]}")
def test_bdf_step_exact_for_quadratic_in_time_flow(ctx, case, mgp):
    dim, n, k = case
    prob, op, perm, _ = _pair(ctx, dim, n, k, 0.05, 0.1, mg_precision=mgp)
    fields = _linear_flow(dim, 1)
    ts = [0.0, 0.1, 0.23, 0.30, 0.36]
    dirich = op.dofs.dirichlet
    u_nm1 = _to_lib(fields(op, ts[0])[0], perm)
    u_n = _to_lib(fields(op, ts[1])[0], perm)
    for j in range(2, len(ts)):
        dt = ts[j] - ts[j - 1]
        om = dt / (ts[j - 1] - ts[j - 2])
        Uex, f = fields(op, ts[j])
        guess = np.zeros_like(Uex)
        guess[dirich] = Uex[dirich]
        u = _to_lib(guess, perm)
        info = prob.bdf_step(u, u_n, u_nm1, forcing=_to_lib(f, perm), dt=dt, omega=om, rtol=1e-12,
                             lin_tol=1e-8, max_newton=12, extrapolate=True)
        assert info.converged and info.newton_iterations <= 8
        d = op.project_pressure_mean(_from_lib(u, perm) - Uex)
        assert np.linalg.norm(d) <= 1e-9 * np.linalg.norm(Uex)
        u_nm1, u_n = u_n, u


def _tg(op, t, nu):
    x = op.dofs.nodesets[0].x
    F = np.exp(-2 * np.pi ** 2 * nu * t)
    X, Y = x[:, 0], x[:, 1]
    u = np.sin(np.pi * X) * np.cos(np.pi * Y) * F
    v = -np.cos(np.pi * X) * np.sin(np.pi * Y) * F
    pr = 0.25 * (np.cos(2 * np.pi * X) + np.cos(2 * np.pi * Y)) * F * F
    return np.concatenate([u, v, pr])


def test_bdf_steps_follow_the_oracle_on_taylor_green(ctx):
    nu, dt = 0.05, 0.05
    prob, op, perm, _ = _pair(ctx, 2, 8, 2, nu, dt, mg_precision=1)
    d = op.dofs
    uo_nm1, uo_n = _tg(op, 0.0, nu), _tg(op, dt, nu)
    ug_nm1, ug_n = _to_lib(uo_nm1, perm), _to_lib(uo_n, perm)
    for s in range(2, 5):
        Uex = _tg(op, s * dt, nu)
        guess = 2 * uo_n - uo_nm1
        guess[d.dirichlet] = Uex[d.dirichlet]
        Uo, _ = timeloop.bdf_step(op, uo_n, uo_nm1, dt, 1.0, guess, rtol=1e-13, atol=1e-14)
        u = _to_lib(guess, perm)
        info = prob.bdf_step(u, ug_n, ug_nm1, dt=dt, omega=1.0, rtol=1e-11, lin_tol=1e-8, max_newton=12)
        assert info.converged
        diff = op.project_pressure_mean(_from_lib(u, perm) - Uo)
        assert np.linalg.norm(diff) <= 1e-8 * np.linalg.norm(Uo)
        uo_nm1, uo_n = uo_n, Uo
        ug_nm1, ug_n = ug_n, u
    nv = 2 * d.nodesets[0].n_nodes
    assert np.linalg.norm((uo_n - Uex)[:nv]) <= 2e-3 * np.linalg.norm(Uex[:nv])


def test_max_velocity(ctx):
    prob, op, perm, _ = _pair(ctx, 3, 3, 2, 0.05, 0.1)
    U = op.state_vector() * 1.7
    n = op.dofs.nodesets[0].n_nodes
    ref = np.sqrt(sum(U[c * n:(c + 1) * n] ** 2 for c in range(3))).max()
    assert prob.max_velocity(_to_lib(U, perm)) == pytest.approx(ref, rel=1e-15)


BALL2 = ((0.3, 0.3, 0.3), 0.3, 1)


def _pair_ball(ctx, dim, n, k, nu, dt, alpha=1.5, mg_precision=1):
    from paper_2603_29621_gb300 import _lib as L, api
    m = api.Mesh(ctx, dim, n)
    m.refine_ball(*BALL2)
    prob = api.Problem(ctx, m, kind=L.STAB_NS, degree=k, nu=nu, dt=dt, mg_precision=mg_precision)
    f = mesh.refine_ball(mesh.uniform(dim, n), *BALL2)
    op = assemble.Problem(f, "stab_ns", k, nu=nu, dt=dt, alpha=alpha)
    xg, fg = prob.support_points()
    xo, fo = op.dofs.support_points()
    return prob, op, inputs.match_dofs(xg, fg, xo, fo), m, f


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", [(2, 2, 3), (3, 2, 2)], ids=lambda c: f"{c[0]}d-n{c[1]}-k{c[2]}-ball")
def test_residual_and_jacobian_on_refined_meshes(ctx, case, prec):
    dim, n, k = case
    nu, dt, alpha = 2e-2, 0.05, 1.5
    prob, op, perm, _, _ = _pair_ball(ctx, dim, n, k, nu, dt, alpha)
    d = op.dofs
    assert len(d.nodesets[0].hanging) > 0
    rng = np.random.default_rng(12)
    U = d.set_hanging(op.state_vector() + 0.3 * rng.uniform(-1, 1, d.n_dofs))
    g = d.set_hanging(rng.uniform(-1, 1, d.n_dofs))
    op.set_state(U, g)
    Fo = op.residual()
    A = op.assemble()
    prob.set_state(dt, alpha, _to_lib(U, perm), _to_lib(g, perm))
    dt_ = torch.float64 if prec == 0 else torch.float32
    F = torch.full((len(perm),), 7.0, device="cuda", dtype=dt_)
    prob.residual(F)
    Fg = _from_lib(F, perm)
    assert np.linalg.norm(Fg - Fo) <= TOL[prec] * np.linalg.norm(Fo)
    x = inputs.uniform_vector(len(perm))
    y = torch.empty(len(perm), device="cuda", dtype=dt_)
    prob.vmult(_to_lib(x, perm, dt_), y)
    yo = A @ x
    assert np.linalg.norm(_from_lib(y, perm) - yo) <= TOL[prec] * np.linalg.norm(yo)


@pytest.mark.parametrize("case", [(3, 2, 2), (2, 3, 3)], ids=lambda c: f"{c[0]}d-n{c[1]}-k{c[2]}-ball")
def test_state_reaches_every_level_of_a_refined_hierarchy(ctx, case):
    """Q1 state and explicit field (exact on every level): after mfns_set_state every level's
    operator equals the oracle's at that state, through refined h-steps (children evaluated per
    coarse cell), uniform h-steps and p-steps."""
    from oracle import solvers
    dim, n, k = case
    nu, dt, alpha = 5e-2, 0.1, 1.5
    prob, op, perm, _, f = _pair_ball(ctx, dim, n, k, nu, dt, alpha, mg_precision=0)
    C, U, g = _q1_state(op, 6)
    prob.set_state(dt, alpha, _to_lib(U, perm), _to_lib(g, perm))
    levels = solvers.hierarchy(f, "stab_ns", k, nu=nu, dt=dt)
    info = prob.get_info()
    assert info.n_levels == len(levels) >= 3
    refined_steps = 0
    for lvl, lv in enumerate(levels):
        ol = lv.problem
        refined_steps += int(ol.forest.max_level > 0)
        xo = ol.dofs.nodesets[0].x
        ol.set_dt(dt, alpha)
        ol.set_state(np.concatenate([_q1_field(xo, C[0, c]) for c in range(dim + 1)]),
                     np.concatenate([_q1_field(xo, C[1, c]) for c in range(dim + 1)]))
        xg, fg = prob.support_points(lvl)
        xs, fs = ol.dofs.support_points()
        pl = inputs.match_dofs(xg, fg, xs, fs)
        x = inputs.uniform_vector(len(pl), seed=lvl)
        y = torch.empty(len(pl), device="cuda", dtype=torch.float64)
        prob.vmult(_to_lib(x, pl), y, which=lvl)
        yo = ol.assemble() @ x
        assert np.linalg.norm(_from_lib(y, pl) - yo) <= 1e-12 * np.linalg.norm(yo), lvl
    assert refined_steps >= 1


@pytest.mark.parametrize("case", [(2, 3, 2), (3, 2, 2)], ids=lambda c: f"{c[0]}d-n{c[1]}-k{c[2]}-ball")
def test_bdf_step_exact_on_refined_meshes(ctx, case):
    dim, n, k = case
    prob, op, perm, _, _ = _pair_ball(ctx, dim, n, k, 0.05, 0.1, mg_precision=1)
    fields = _linear_flow(dim, 3)
    ts = [0.0, 0.1, 0.22, 0.3]
    dirich = op.dofs.dirichlet
    u_nm1 = _to_lib(fields(op, ts[0])[0], perm)
    u_n = _to_lib(fields(op, ts[1])[0], perm)
    for j in range(2, len(ts)):
        dt = ts[j] - ts[j - 1]
        om = dt / (ts[j - 1] - ts[j - 2])
        Uex, fo = fields(op, ts[j])
        guess = np.zeros_like(Uex)
        guess[dirich] = Uex[dirich]
        u = _to_lib(guess, perm)
        info = prob.bdf_step(u, u_n, u_nm1, forcing=_to_lib(fo, perm), dt=dt, omega=om, rtol=1e-12,
                             lin_tol=1e-8, max_newton=12, extrapolate=True)
        assert info.converged
        # the pressure is fixed up to a constant: remove the offset of the free pressure entries
        # from every pressure entry (hanging ones included)
        d = _from_lib(u, perm) - Uex
        P = op.dofs.offsets[1]
        d[P:] -= d[op.pressure_dofs()].mean()
        assert np.linalg.norm(d) <= 1e-9 * np.linalg.norm(Uex)
        u_nm1, u_n = u_n, u
