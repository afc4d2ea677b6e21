"""Local-smoothing multigrid (Section 2) on the GPU against the oracle, through the C ABI.

The cycle is a different composition of the same kernels (level operators on partial forests with
the refinement edge held at zero, transfers between levels, the base hierarchy's V-cycle), so a
cycle is compared with the oracle's multiplicative subspace correction to 1e-10, as the
global-coarsening V-cycle is.  Smoother bounds are passed explicitly to both sides."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import assemble, ls, mesh, solvers  # noqa: E402
from paper_2603_29621_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu
CENTRE = (0.3, 0.35, 0.4)


@pytest.fixture(scope="module")
def ctx():
    from paper_2603_29621_gb300 import api
    return api.Context(0)


def _gpu(ctx, kind, dim, n, levels, k, **kw):
    from paper_2603_29621_gb300 import _lib as L, api
    m = api.Mesh(ctx, dim, n)
    m.refine_ball(CENTRE, 0.3, levels)
    return api.Problem(ctx, m, kind=kind, degree=k, hierarchy=L.LOCAL_SMOOTHING, **kw)


def _perm(prob, which, oprob):
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


def _oracle(problem, smoother):
    tmp = ls.LocalSmoothing(problem, [1.0] * problem.forest.max_level, [1.0] * 8, smoother)
    lm_ls = [1.2 * solvers.power_lmax(lv.A, lv.dinv, iterations=50) for lv in tmp.levels]
    lm_base = [1.2 * solvers.power_lmax(lv.A, lv.dinv, iterations=50) for lv in tmp.base_levels[:-1]]
    return ls.LocalSmoothing(problem, lm_ls, lm_base, smoother), lm_ls, lm_base


def _set_bounds(prob, lm_ls, lm_base):
    """API level order: refined levels finest first, then the base hierarchy (its coarsest level is
    solved directly and takes no bound)."""
    L = len(lm_ls)
    assert prob.info.n_levels == L + len(lm_base) + 1
    for i in range(L):
        prob.set_lambda_max(i, lm_ls[L - 1 - i])
    for j, lm in enumerate(lm_base):
        prob.set_lambda_max(L + j, lm)


CASES = [(2, 4, 2, 2), (2, 2, 2, 3), (3, 2, 1, 2), (3, 2, 2, 2), (2, 5, 2, 1)]


@pytest.mark.parametrize("smoother", [("chebyshev", 3), ("jacobi", 2)])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}d-n{c[1]}-l{c[2]}-k{c[3]}")
def test_ls_cycle_matches_oracle(ctx, case, smoother):
    from paper_2603_29621_gb300 import _lib as L
    dim, n, levels, k = case
    f = mesh.refine_ball(mesh.uniform(dim, n), CENTRE, 0.3, levels)
    op = assemble.Problem(f, "stokes_a", k, nu=0.8)
    orc, lm_ls, lm_base = _oracle(op, smoother)
    prob = _gpu(ctx, L.STOKES_A, dim, n, levels, k, nu=0.8, lambda_max=1.0,
                smoother=1 if smoother[0] == "chebyshev" else 2, smoother_degree=smoother[1])
    _set_bounds(prob, lm_ls, lm_base)
    info = prob.info
    for i in range(len(lm_ls)):           # the refined levels are the oracle's level cell sets
        assert info.level_cells[i] == len(orc.levels[len(lm_ls) - 1 - i].space.cells)
    perm = _perm(prob, L.OP_SYSTEM, op)          # the fine operator (level indices name cycle levels)
    b = inputs.uniform_vector(op.dofs.n_dofs, seed=7)      # constrained entries nonzero too
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    prob.vcycle(_to_gpu(b, perm), x)
    got = _from_gpu(x, perm)
    exp = orc(b)
    assert np.abs(got - exp).max() <= 1e-10 * np.abs(exp).max(), np.abs(got - exp).max()
    # FP32 cycle: the same map within single-precision round-off
    x32 = torch.zeros(len(b), dtype=torch.float32, device="cuda")
    prob.vcycle(_to_gpu(b, perm, torch.float32), x32)
    got32 = _from_gpu(x32, perm)
    assert np.linalg.norm(got32 - exp) <= 1e-4 * np.linalg.norm(exp)


@pytest.mark.parametrize("mg_precision", [0, 1])
def test_ls_stokes_solve_matches_global_coarsening(ctx, mg_precision):
    """Stokes Q2/Q1 on a ball-refined 3D mesh: FGMRES with the block preconditioner of Eq. 5 and a
    local-smoothing cycle on the A block converges to the same solution as with global coarsening,
    in a similar number of iterations (Section 2, Tables 3 and 4)."""
    from paper_2603_29621_gb300 import _lib as L, api
    out = {}
    for h in (L.GLOBAL_COARSENING, L.LOCAL_SMOOTHING):
        m = api.Mesh(ctx, 3, 4)
        m.refine_ball(CENTRE, 0.3, 2)
        prob = api.Problem(ctx, m, kind=L.STOKES, degree=2, nu=1.0, tol=1e-10, mg_precision=mg_precision,
                           hierarchy=h)
        xyz, fld = prob.support_points()
        xs = torch.tensor(inputs.smooth_solution(xyz, fld, 3), device="cuda")
        b = torch.empty_like(xs)
        prob.vmult(xs, b)
        x = torch.zeros_like(xs)
        info = prob.solve(b, x, raise_on_nonconvergence=False)
        assert info.converged, (h, info.iterations, info.rel_residual)
        out[h] = (info.iterations, x.cpu().numpy(), xs.cpu().numpy(), fld)
    it_gc, x_gc, xs, fld = out[L.GLOBAL_COARSENING]
    it_ls, x_ls, _, _ = out[L.LOCAL_SMOOTHING]
    vel = fld < 3
    assert np.abs(x_ls[vel] - x_gc[vel]).max() <= 1e-6 * np.abs(xs[vel]).max()
    assert it_ls <= it_gc + 8, (it_ls, it_gc)


def test_ls_rejects_unsupported(ctx):
    from paper_2603_29621_gb300 import _lib as L
    with pytest.raises(L.MfnsError) as e:
        _gpu(ctx, L.PMASS, 3, 2, 1, 2, nu=1.0)
    assert e.value.code == L.ERR_UNSUPPORTED
    prob = _gpu(ctx, L.STOKES_A, 2, 4, 1, 2, nu=1.0)
    b = torch.zeros(prob.info.n_dofs, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(L.MfnsError) as e:
        prob.smooth(0, b, x)
    assert e.value.code == L.ERR_UNSUPPORTED
    # an unrefined mesh: local smoothing is the global-coarsening hierarchy itself
    from paper_2603_29621_gb300 import api
    m = api.Mesh(ctx, 2, 4)
    p0 = api.Problem(ctx, m, kind=L.STOKES_A, degree=2, hierarchy=L.LOCAL_SMOOTHING)
    p1 = api.Problem(ctx, api.Mesh(ctx, 2, 4), kind=L.STOKES_A, degree=2)
    assert p0.info.n_levels == p1.info.n_levels
