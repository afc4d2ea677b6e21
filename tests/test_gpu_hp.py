"""hp-adaptive vector Laplacian (Section 3) on the GPU against the oracle, through the C ABI.

Degree fields vary over same-level faces and across hanging faces (finer cells never of lower
degree).  Operator and exact diagonal: 1e-12 (FP64); transfers of the hp hierarchy (degrees
lowered one by one, then h): 1e-12; V-cycle: 1e-10 with the smoother bounds passed to both sides;
an FGMRES solve converges to the manufactured solution."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hp, mesh, solvers  # noqa: E402
from paper_2603_29621_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu
CENTRE = (0.3, 0.35, 0.4)


@pytest.fixture(scope="module")
def ctx():
    from paper_2603_29621_gb300 import api
    return api.Context(0)


def _degrees(cells, base):
    """base + level + parity of the root cell's x index (cells: level, x, y, ...)."""
    lev = cells[:, 0]
    return (base + lev + ((cells[:, 1] >> lev) % 2)).astype(np.int32)


def _pair(ctx, dim, n, levels, base, **desc):
    from paper_2603_29621_gb300 import _lib as L, api
    f = mesh.refine_ball(mesh.uniform(dim, n), CENTRE, 0.3, levels)
    m = api.Mesh(ctx, dim, n)
    m.refine_ball(CENTRE, 0.3, levels)
    cells = m.cells()
    assert np.array_equal(cells[:, :1 + dim], f.cells)     # one canonical cell order on both sides
    deg = _degrees(f.cells, base)
    prob = api.Problem(ctx, m, degrees=deg, kind=L.STOKES_A, degree=int(deg.max()), **desc)
    return f, deg, prob


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


CASES = [(2, 3, 2, 1), (2, 4, 1, 2), (3, 2, 1, 1), (3, 2, 1, 2)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}d-n{c[1]}-l{c[2]}-b{c[3]}")
def test_hp_operator_and_diagonal_match_oracle(ctx, case):
    dim, n, levels, base = case
    f, deg, prob = _pair(ctx, dim, n, levels, base, nu=0.7, lambda_max=1.0)
    op = hp.HpProblem(f, deg, "stokes_a", nu=0.7)
    A = op.assemble()
    perm = _perm(prob, -1, op)
    x = inputs.uniform_vector(A.shape[0], seed=3)
    y = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
    prob.vmult(_to_gpu(x, perm), y)
    exp = A @ x
    assert np.abs(_from_gpu(y, perm) - exp).max() <= 1e-12 * np.abs(exp).max()
    y32 = torch.empty(A.shape[0], dtype=torch.float32, device="cuda")
    prob.vmult(_to_gpu(x, perm, torch.float32), y32)
    assert np.linalg.norm(_from_gpu(y32, perm) - exp) <= 1e-5 * np.linalg.norm(exp)
    d = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
    prob.diagonal(d)
    assert np.abs(_from_gpu(d, perm) - A.diagonal()).max() <= 1e-12 * np.abs(A.diagonal()).max()


@pytest.mark.parametrize("case", CASES[:3], ids=lambda c: f"{c[0]}d-n{c[1]}-l{c[2]}-b{c[3]}")
def test_hp_transfers_and_vcycle_match_oracle(ctx, case):
    dim, n, levels, base = case
    f, deg, prob = _pair(ctx, dim, n, levels, base, nu=1.0, lambda_max=1.0, smoother=1, smoother_degree=3)
    lv = hp.hierarchy(f, deg)
    assert prob.info.n_levels == len(lv)
    for l in range(len(lv) - 1):
        pf = _perm(prob, l, lv[l].problem)
        pc = _perm(prob, l + 1, lv[l + 1].problem)
        P = lv[l].P
        xc = inputs.uniform_vector(P.shape[1], seed=10 + l)
        xf0 = inputs.uniform_vector(P.shape[0], seed=20 + l)
        fine = _to_gpu(xf0, pf)
        prob.prolongate_add(l, _to_gpu(xc, pc), fine)
        exp = xf0 + P @ xc
        assert np.abs(_from_gpu(fine, pf) - exp).max() <= 1e-12 * np.abs(exp).max(), l
        rf = inputs.uniform_vector(P.shape[0], seed=30 + l)
        coarse = torch.zeros(P.shape[1], dtype=torch.float64, device="cuda")
        prob.restrict(l, _to_gpu(rf, pf), coarse)
        exp = P.T @ rf
        assert np.abs(_from_gpu(coarse, pc) - exp).max() <= 1e-12 * np.abs(exp).max(), l
    lmax = [1.2 * solvers.power_lmax(l_.A, l_.dinv, iterations=50) for l_ in lv[:-1]]
    for l, lm in enumerate(lmax):
        prob.set_lambda_max(l, lm)
    V = solvers.VCycle(lv, lmax, ("chebyshev", 3))
    perm = _perm(prob, 0, lv[0].problem)
    b = inputs.uniform_vector(lv[0].A.shape[0], seed=5)
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    prob.vcycle(_to_gpu(b, perm), x)
    exp = V(b)
    assert np.abs(_from_gpu(x, perm) - exp).max() <= 1e-10 * np.abs(exp).max()


@pytest.mark.parametrize("mg_precision", [0, 1])
def test_hp_solve_converges(ctx, mg_precision):
    f, deg, prob = _pair(ctx, 3, 4, 1, 2, nu=1.0, tol=1e-10, mg_precision=mg_precision)
    xyz, fld = prob.support_points()
    xs = torch.tensor(inputs.smooth_solution(xyz, fld, 3), device="cuda")
    b = torch.empty_like(xs)
    prob.vmult(xs, b)
    x = torch.zeros_like(xs)
    info = prob.solve(b, x)
    assert info.converged and info.iterations <= 40, info.iterations
    assert float((x - xs).abs().max()) <= 1e-7 * float(xs.abs().max())


def test_hp_rejects_unsupported(ctx):
    """hp problems use global coarsening (local smoothing of hp levels is not built)."""
    from paper_2603_29621_gb300 import _lib as L, api
    m = api.Mesh(ctx, 2, 3)
    m.refine_ball(CENTRE, 0.3, 1)
    cells = m.cells()
    with pytest.raises(L.MfnsError) as e:
        api.Problem(ctx, m, degrees=(2 + cells[:, 0]).astype(np.int32), kind=L.STOKES_A, degree=3,
                    hierarchy=L.LOCAL_SMOOTHING)
    assert e.value.code == L.ERR_UNSUPPORTED
