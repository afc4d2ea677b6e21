"""Local smoothing (Section 2) of the stabilised Navier--Stokes operator (Section 5) on the GPU against
the oracle's level recursion, through the C ABI.

Level operators are rediscretised on the cells of each refinement level (tau depends on the cell
size, so they are not Galerkin products); the refinement edge holds velocity and pressure at zero
in the smoothing operator, and a second operator with only the domain boundary constrained gives
the residual's edge rows and drives the transfers; level 0 is the base mesh's global-coarsening
hierarchy.  One cycle with Jacobi relaxation and the smoother bounds passed to both sides agrees
with the oracle to 1e-10, as the global-coarsening V-cycle does."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import assemble, ls, mesh  # noqa: E402
from paper_2603_29621_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu
CENTRE = (0.3, 0.35, 0.4)


@pytest.fixture(scope="module")
def ctx():
    from paper_2603_29621_gb300 import api
    return api.Context(0)


@pytest.mark.parametrize("dim,n,levels,k", [(2, 4, 2, 2), (3, 2, 1, 2), (2, 4, 2, 1)])
def test_ls_stabns_cycle_matches_oracle(ctx, dim, n, levels, k):
    from paper_2603_29621_gb300 import _lib as L, api
    params = dict(nu=1e-2, dt=1e-2)
    f = mesh.refine_ball(mesh.uniform(dim, n), CENTRE, 0.3, levels)
    op = assemble.Problem(f, "stab_ns", k, **params)
    sm = ("jacobi", 5)
    tmp = ls.LocalSmoothingLevels(op, [1.0] * f.max_level, [1.0] * 8, sm, **params)
    lm_ls = [3.0 + 0.1 * i for i in range(len(tmp.levels))]
    lm_b = [3.0 + 0.1 * i for i in range(len(tmp.base_levels) - 1)]
    orc = ls.LocalSmoothingLevels(op, lm_ls, lm_b, sm, **params)
    m = api.Mesh(ctx, dim, n)
    m.refine_ball(CENTRE, 0.3, levels)
    prob = api.Problem(ctx, m, kind=L.STAB_NS, degree=k, hierarchy=L.LOCAL_SMOOTHING, lambda_max=1.0,
                       smoother=2, smoother_degree=5, **params)
    Lv = len(lm_ls)
    assert prob.info.n_levels == Lv + len(lm_b) + 1
    for i in range(Lv):
        prob.set_lambda_max(i, lm_ls[Lv - 1 - i])
    for j, lm in enumerate(lm_b):
        prob.set_lambda_max(Lv + j, lm)
    xg, fg = prob.support_points(L.OP_SYSTEM)
    xo, fo = op.dofs.support_points()
    perm = inputs.match_dofs(xg, fg, xo, fo)
    b = inputs.uniform_vector(op.dofs.n_dofs, seed=7)
    bd = np.empty_like(b)
    bd[perm] = b
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    prob.vcycle(torch.tensor(bd, device="cuda"), x)
    torch.cuda.synchronize()
    got = x.cpu().numpy()[perm]
    exp = orc(b)
    assert np.abs(got - exp).max() <= 1e-10 * np.abs(exp).max()
