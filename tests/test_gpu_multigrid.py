"""GPU multigrid parity against the oracle, through the C ABI: transfers (Eq. 4),
Chebyshev/Jacobi smoothing, V-cycle, FGMRES solves (FP64 and FP32 multigrid).

Smoother bounds lambda_max are passed explicitly to both sides (the estimate
itself is not part of the oracle).  Tolerances: transfers and one smoothing
step are linear maps evaluated in a different order -> 1e-12 relative; a
V-cycle composes O(10^2) operator applications -> 1e-10; solves compare
solutions, bounded by the solver tolerance."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import assemble, mesh, solvers  # noqa: E402
from paper_2603_29621_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu
KINDS = {"stokes": 0, "stokes_a": 1, "stab_ns": 2, "pmass": 3}


@pytest.fixture(scope="module")
def ctx():
    from paper_2603_29621_gb300 import api
    return api.Context(0)


def _forest(dim, n, refine):
    f = mesh.uniform(dim, n)
    if refine:
        f = mesh.refine_ball(f, *refine)
    return f


def _gpu_problem(ctx, kind, dim, n, refine, k, **kw):
    from paper_2603_29621_gb300 import api
    m = api.Mesh(ctx, dim, n)
    if refine:
        m.refine_ball(*refine)
    return api.Problem(ctx, m, kind=KINDS[kind], degree=k, **kw)


def _perm(prob, which, oprob, pressure_like=False):
    xg, fg = prob.support_points(which)
    xo, fo = oprob.dofs.support_points()
    return inputs.match_dofs(xg, fg, xo, fo)


def _to_gpu(x, perm, dtype=torch.float64):
    xd = np.empty_like(x)
    xd[perm] = x
    return torch.tensor(xd, device="cuda", dtype=dtype)


def _from_gpu(t, perm):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()[perm]


BALL = ((0.3, 0.3, 0.3), 0.3, 1)
HIER = [
    ("stab_ns", 3, 4, None, 2, dict(nu=1e-2, dt=1e-2)),
    ("stab_ns", 3, 5, None, 2, dict(nu=1e-2, dt=1e-2)),     # 5 -> 3 -> 2: non-nested h-steps
    ("stokes_a", 2, 7, None, 3, dict(nu=1.0)),
    ("stokes_a", 3, 2, BALL, 2, dict(nu=1.0)),
    ("stokes_a", 2, 4, BALL, 3, dict(nu=1.0)),
    ("stab_ns", 2, 4, BALL, 2, dict(nu=1e-2, dt=1e-1)),
    ("stab_ns", 3, 4, None, 1, dict(nu=0.4, dt=1e-2)),      # Q1Q1, viscosity-dominated tau
    ("stab_ns", 2, 5, None, 1, dict(nu=1e-2, dt=1e-2)),     # Q1Q1, 5 -> 3 -> 2 non-nested
]


@pytest.mark.parametrize("case", HIER, ids=lambda c: f"{c[0]}-{c[1]}d-n{c[2]}-k{c[4]}-{'ball' if c[3] else 'uni'}")
def test_transfers_match_oracle(ctx, case):
    kind, dim, n, refine, k, phys = case
    prob = _gpu_problem(ctx, kind, dim, n, refine, k, lambda_max=1.0, **phys)
    levels = solvers.hierarchy(_forest(dim, n, refine), kind, k, nu=phys["nu"], dt=phys.get("dt") or np.inf)
    assert prob.info.n_levels == len(levels)
    for l in range(len(levels) - 1):
        pf = _perm(prob, l, levels[l].problem)
        pc = _perm(prob, l + 1, levels[l + 1].problem)
        P = levels[l].P
        xc = inputs.uniform_vector(P.shape[1], seed=10 + l)
        xf0 = inputs.uniform_vector(P.shape[0], seed=20 + l)
        fine = _to_gpu(xf0, pf)
        prob.prolongate_add(l, _to_gpu(xc, pc), fine)
        got = _from_gpu(fine, pf)
        exp = xf0 + P @ xc
        assert np.abs(got - exp).max() <= 1e-12 * np.abs(exp).max(), (l, np.abs(got - exp).max())
        rf = inputs.uniform_vector(P.shape[0], seed=30 + l)
        coarse = torch.zeros(P.shape[1], dtype=torch.float64, device="cuda")
        prob.restrict(l, _to_gpu(rf, pf), coarse)
        got = _from_gpu(coarse, pc)
        exp = P.T @ rf
        assert np.abs(got - exp).max() <= 1e-12 * np.abs(exp).max(), (l, np.abs(got - exp).max())


@pytest.mark.parametrize("fused", [0, 1], ids=["separate", "fused"])
@pytest.mark.parametrize("smoother", [("chebyshev", 3), ("chebyshev", 5), ("jacobi", 4)])
@pytest.mark.parametrize("case", [HIER[0], HIER[3], HIER[2], HIER[6]],
                         ids=lambda c: f"{c[0]}-{c[1]}d-k{c[4]}-{'ball' if c[3] else 'uni'}")
def test_smoother_matches_oracle(ctx, case, smoother, fused):
    kind, dim, n, refine, k, phys = case
    prob = _gpu_problem(ctx, kind, dim, n, refine, k, lambda_max=1.0, smoother=1 if smoother[0] == "chebyshev" else 2,
                        smoother_degree=smoother[1], fused_smoother=fused, **phys)
    levels = solvers.hierarchy(_forest(dim, n, refine), kind, k, nu=phys["nu"], dt=phys.get("dt") or np.inf)
    lv = levels[0]
    lmax = 1.2 * solvers.power_lmax(lv.A, lv.dinv, iterations=50)
    prob.set_lambda_max(0, lmax)
    perm = _perm(prob, 0, lv.problem)
    b = inputs.uniform_vector(lv.A.shape[0], seed=3)
    x0 = inputs.uniform_vector(lv.A.shape[0], seed=4)
    for zero in (True, False):
        xg = _to_gpu(np.zeros_like(x0) if zero else x0, perm)
        prob.smooth(0, _to_gpu(b, perm), xg, x_is_zero=zero)
        got = _from_gpu(xg, perm)
        start = np.zeros_like(x0) if zero else x0
        if smoother[0] == "chebyshev":
            exp = solvers.chebyshev(lv.A, lv.dinv, b, start, smoother[1], lmax, x_is_zero=zero)
        else:
            exp = solvers.jacobi_relaxation(lv.A, lv.dinv, b, start, smoother[1], lmax)
        assert np.abs(got - exp).max() <= 1e-11 * np.abs(exp).max(), np.abs(got - exp).max()


@pytest.mark.parametrize("fused", [0, 1], ids=["separate", "fused"])
@pytest.mark.parametrize("case", HIER, ids=lambda c: f"{c[0]}-{c[1]}d-k{c[4]}-{'ball' if c[3] else 'uni'}")
def test_vcycle_matches_oracle(ctx, case, fused):
    kind, dim, n, refine, k, phys = case
    prob = _gpu_problem(ctx, kind, dim, n, refine, k, lambda_max=1.0, smoother=1, smoother_degree=3,
                        fused_smoother=fused, **phys)
    levels = solvers.hierarchy(_forest(dim, n, refine), kind, k, nu=phys["nu"], dt=phys.get("dt") or np.inf)
    lmax = [1.2 * solvers.power_lmax(lv.A, lv.dinv, iterations=50) for lv in levels[:-1]]
    for l, lm in enumerate(lmax):
        prob.set_lambda_max(l, lm)
    vc = solvers.VCycle(levels, lmax, ("chebyshev", 3))
    perm = _perm(prob, 0, levels[0].problem)
    b = inputs.uniform_vector(levels[0].A.shape[0], seed=5)
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    prob.vcycle(_to_gpu(b, perm), x)
    got = _from_gpu(x, perm)
    exp = vc(b)
    assert np.abs(got - exp).max() <= 1e-10 * np.abs(exp).max(), np.abs(got - exp).max()
    # FP32 V-cycle: same map within single-precision round-off
    x32 = torch.zeros(len(b), dtype=torch.float32, device="cuda")
    prob.vcycle(_to_gpu(b, perm, torch.float32), x32)
    got32 = _from_gpu(x32, perm)
    assert np.linalg.norm(got32 - exp) <= 1e-4 * np.linalg.norm(exp)


def _manufactured_2d(nu):
    u = lambda x: np.stack([x[:, 0] ** 2, -2 * x[:, 0] * x[:, 1]], axis=1)
    p = lambda x: x[:, 0] + x[:, 1] - 1
    f = lambda x: np.stack([np.full(len(x), 1 - 2 * nu), np.ones(len(x))], axis=1)
    return u, p, f


@pytest.mark.parametrize("tol,err_bound", [(1e-10, 1e-5), (1e-12, 1e-8)])
@pytest.mark.parametrize("mg_precision", [0, 1])
def test_config1_stokes_2d_manufactured_solve(ctx, mg_precision, tol, err_bound):
    """2D Stokes Q2/Q1 on 16x16, nu = 1: FGMRES with the block preconditioner of Eq. 5 reproduces
    the manufactured polynomial solution (in the FE space) and the oracle's direct solve.  The
    saddle-point system amplifies the residual: 1e-10 relative residual (the stated target) gives
    ~1e-6 error; 1e-12 gives <= 1e-8."""
    nu = 1.0
    f = mesh.uniform(2, 16)
    op = assemble.Problem(f, "stokes", 2, nu=nu)
    u, p, fr = _manufactured_2d(nu)
    F = assemble.load_vector(op, fr)
    b = assemble.dirichlet_system(op, F, u)
    x_direct = assemble.solve_direct(op, b)
    prob = _gpu_problem(ctx, "stokes", 2, 16, None, 2, nu=nu, tol=tol, mg_precision=mg_precision)
    perm = _perm(prob, -1, op)
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    info = prob.solve(_to_gpu(b, perm), x)
    assert info.converged and info.rel_residual <= tol
    assert info.iterations <= 80, info.iterations
    got = _from_gpu(x, perm)
    full = assemble.complete_solution(op, got, u)
    exact = op.dofs.interpolate(lambda X: np.concatenate([u(X), p(X)[:, None]], axis=1))
    pres = np.zeros(len(b), dtype=bool)
    pres[op.dofs.offsets[1]:] = True
    d = full - exact
    d[pres] -= d[pres].mean()
    assert np.abs(d).max() <= err_bound * np.abs(exact).max(), np.abs(d).max()
    dd = op.project_pressure_mean(got) - op.project_pressure_mean(x_direct)
    assert np.linalg.norm(dd) <= err_bound * np.linalg.norm(x_direct)


@pytest.mark.parametrize("mg_precision", [0, 1])
@pytest.mark.parametrize("case", [("stab_ns", 3, 4, None, 2, dict(nu=1e-2, dt=1e-2)),
                                  ("stokes", 3, 2, BALL, 2, dict(nu=1.0)),
                                  ("stab_ns", 3, 2, BALL, 2, dict(nu=1e-1, dt=1e-2))],
                         ids=lambda c: f"{c[0]}-{'ball' if c[3] else 'uni'}")
def test_solve_matches_direct(ctx, case, mg_precision):
    """FGMRES (FP64) with FP64 or FP32 multigrid: solution within 1e-8 of the oracle's direct solve."""
    kind, dim, n, refine, k, phys = case
    prob = _gpu_problem(ctx, kind, dim, n, refine, k, tol=1e-12, mg_precision=mg_precision, smoother_degree=3,
                        **phys)
    op = assemble.Problem(_forest(dim, n, refine), kind, k, nu=phys["nu"], dt=phys.get("dt") or np.inf)
    perm = _perm(prob, -1, op)
    A = op.assemble()
    xstar = op.project_pressure_mean(inputs.uniform_vector(A.shape[0], seed=7))
    xstar[op.dofs.hanging] = op.dofs.distribute(xstar)[op.dofs.hanging]
    b = A @ xstar
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    info = prob.solve(_to_gpu(b, perm), x)
    assert info.converged, (info.iterations, info.rel_residual)
    got = _from_gpu(x, perm)
    xd = assemble.solve_direct(op, b, A)
    err = np.linalg.norm(op.project_pressure_mean(got) - op.project_pressure_mean(xd)) / np.linalg.norm(xd)
    assert err <= 1e-8, (err, info.iterations)
