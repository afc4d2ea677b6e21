"""hp spaces with combined h+p faces (Section 3) on the GPU against the oracle, through the C ABI.

Coarse cells of degree 3 (or 4) next to refined cells of degree 2: the library switches its
constraint construction to elimination for the whole space; the oracle eliminates with its dense
reduced row echelon form.  The kernels are those of every hp level (cell groups per degree,
constraint passes around them), so the bars are the hp bars: operator and exact diagonal 1e-11
(FP64), every transfer of the hierarchy 1e-11, one V-cycle 1e-10 with the smoother bounds passed
to both sides, and an FGMRES solve to the manufactured solution."""
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


def _combined(cells, kind):
    lev = cells[:, 0]
    return {"3-2": 3 - lev, "4-2": 4 - 2 * lev}[kind].astype(np.int32)


def _pair(ctx, dim, n, kind, **desc):
    from paper_2603_29621_gb300 import _lib as L, api
    f = mesh.refine_ball(mesh.uniform(dim, n), CENTRE, 0.3, 1)
    m = api.Mesh(ctx, dim, n)
    m.refine_ball(CENTRE, 0.3, 1)
    cells = m.cells()
    assert np.array_equal(cells[:, :1 + dim], f.cells)
    deg = _combined(f.cells, kind)
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


CASES = [(2, 4, "3-2"), (2, 4, "4-2"), (3, 3, "3-2")]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}d-n{c[1]}-{c[2]}")
def test_combined_operator_and_diagonal_match_oracle(ctx, case):
    dim, n, kind = case
    f, deg, prob = _pair(ctx, dim, n, kind, nu=0.7, lambda_max=1.0)
    op = hp.HpProblem(f, deg, "stokes_a", nu=0.7, rule="elimination")
    A = op.assemble()
    perm = _perm(prob, -1, op)
    # the same constrained entries (perm[i]: library entry of oracle entry i)
    assert set(prob.constrained().tolist()) == set(perm[np.nonzero(op.dofs.constrained)[0]].tolist())
    x = inputs.uniform_vector(A.shape[0], seed=3)
    y = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
    prob.vmult(_to_gpu(x, perm), y)
    exp = A @ x
    assert np.abs(_from_gpu(y, perm) - exp).max() <= 1e-11 * np.abs(exp).max()
    d = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
    prob.diagonal(d)
    assert np.abs(_from_gpu(d, perm) - A.diagonal()).max() <= 1e-11 * np.abs(A.diagonal()).max()


@pytest.mark.parametrize("case", CASES[:2] + [(3, 2, "3-2")], ids=lambda c: f"{c[0]}d-n{c[1]}-{c[2]}")
def test_combined_transfers_and_vcycle_match_oracle(ctx, case):
    dim, n, kind = case
    f, deg, prob = _pair(ctx, dim, n, kind, nu=1.0, lambda_max=1.0, smoother=1, smoother_degree=3)
    lv = hp.hierarchy(f, deg, rule="elimination")
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
        assert np.abs(_from_gpu(fine, pf) - exp).max() <= 1e-11 * np.abs(exp).max(), l
        rf = inputs.uniform_vector(P.shape[0], seed=30 + l)
        coarse = torch.zeros(P.shape[1], dtype=torch.float64, device="cuda")
        prob.restrict(l, _to_gpu(rf, pf), coarse)
        exp = P.T @ rf
        assert np.abs(_from_gpu(coarse, pc) - exp).max() <= 1e-11 * np.abs(exp).max(), l
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
def test_combined_solve_converges(ctx, mg_precision):
    f, deg, prob = _pair(ctx, 3, 4, "3-2", nu=1.0, tol=1e-10, mg_precision=mg_precision)
    xyz, fld = prob.support_points()
    xs = torch.tensor(inputs.smooth_solution(xyz, fld, 3), device="cuda")
    b = torch.empty_like(xs)
    prob.vmult(xs, b)
    x = torch.zeros_like(xs)
    info = prob.solve(b, x)
    assert info.converged and info.iterations <= 40, info.iterations
    assert float((x - xs).abs().max()) <= 1e-7 * float(xs.abs().max())


@pytest.mark.parametrize("case", [(2, 4, "3-2"), (2, 4, "4-2"), (3, 2, "3-2")], ids=lambda c: f"{c[0]}d-n{c[1]}-{c[2]}")
def test_blended_smoother_vcycle_matches_oracle(ctx, case):
    """Section 3's Chebyshev around point Jacobi blended with Schwarz blocks on the combined faces
    (smoother 3): one V-cycle against the oracle's with the same smoother bounds (1e-10; the blocks
    are principal submatrices of the SPD operator, well conditioned)."""
    dim, n, kind = case
    f, deg, prob = _pair(ctx, dim, n, kind, nu=1.0, lambda_max=1.0, smoother=3, smoother_degree=3)
    lv = hp.hierarchy(f, deg, rule="elimination", smoother="asm")
    assert prob.info.n_levels == len(lv)
    assert any(isinstance(l.dinv, hp.JacobiASM) for l in lv)
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
def test_blended_smoother_solve_converges(ctx, mg_precision):
    f, deg, prob = _pair(ctx, 3, 4, "3-2", nu=1.0, tol=1e-10, smoother=3, mg_precision=mg_precision)
    xyz, fld = prob.support_points()
    xs = torch.tensor(inputs.smooth_solution(xyz, fld, 3), device="cuda")
    b = torch.empty_like(xs)
    prob.vmult(xs, b)
    x = torch.zeros_like(xs)
    info = prob.solve(b, x)
    assert info.converged and info.iterations <= 40, info.iterations
    assert float((x - xs).abs().max()) <= 1e-7 * float(xs.abs().max())
