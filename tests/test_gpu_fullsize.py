"""Full-size parity through the C ABI, in the launch configuration the benchmark times.

The oracle cannot assemble these operators, so it computes sampled rows one by one
(element matrices of the cells around each row, constraints resolved):

* 64^3 Q2Q2 stabilised Navier-Stokes (nu = 1e-2, dt = 1e-2, Taylor-Green frozen state):
  FP64 and FP32 vmult of the seeded U(-1,1) vector, launched as the benchmark launches it
  (structured colour launches, autotuned block size, precomputed frozen point data).  Sampled
  rows: random ones, every row of the 2x2x2 cell block at the (1,1,1) corner (the last cell of
  each of the 8 colours, i.e. the ragged tail of the last block of every launch) and of the
  block at the origin (the first cells).
* Stokes Q2/Q1 on the 32^3 mesh refined twice inside the ball |x - (1/2,1/2,1/2)| < 1/4 with
  2:1 closure (indexed cells, hanging-node constraints): FP64 and FP32 vmult; random rows
  plus master rows of hanging nodes.
* 48^3 stabilised NS solves at nu = 1e-1, 1e-2, 1e-3 (FP32 multigrid inside FP64 FGMRES,
  relative residual 1e-13, as the benchmark runs them): the right-hand side b = A x* of the
  manufactured x* is checked against the oracle on sampled rows, and the solution against x*
  to 1e-8 relative (the FP32-multigrid target); the ball-refined Stokes Q2/Q1 solve (FP32
  multigrid, 1e-14) to 1e-8 as well.

Bounds: relative l2 error over the sample <= 1e-12 (FP64) and <= 2e-5 (FP32), as in the
small-size tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import assemble, mesh  # noqa: E402
from paper_2603_29621_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 2e-5}
BALL = ((0.5, 0.5, 0.5), 0.25, 2)


@pytest.fixture(scope="module")
def ctx():
    from paper_2603_29621_gb300 import api
    return api.Context(0)


def _rows_in_box(xyz, lo, hi, constrained):
    sel = np.all((xyz >= lo - 1e-12) & (xyz <= hi + 1e-12), axis=1) & ~constrained
    return np.nonzero(sel)[0]


def _compare(prob, perm, oprob, rows, x, prec):
    from paper_2603_29621_gb300 import _lib as L
    dt = torch.float64 if prec == 0 else torch.float32
    xd = np.empty_like(x)
    xd[perm] = x
    src = torch.tensor(xd, device="cuda", dtype=dt)
    dst = torch.full_like(src, 7.0)
    prob.vmult(src, dst, prec=L.FP64 if prec == 0 else L.FP32)
    torch.cuda.synchronize()
    y = dst.double().cpu().numpy()[perm[rows]]
    return y


@pytest.fixture(scope="module")
def stab_ns_64(ctx):
    from paper_2603_29621_gb300 import _lib as L, api
    m = api.Mesh(ctx, 3, 64)
    prob = api.Problem(ctx, m, kind=L.STAB_NS, degree=2, nu=1e-2, dt=1e-2, smoother=1, smoother_degree=3,
                       mg_precision=L.FP32)
    op = assemble.Problem(mesh.uniform(3, 64), "stab_ns", 2, nu=1e-2, dt=1e-2)
    xg, fg = prob.support_points()
    xo, fo = op.dofs.support_points()
    perm = inputs.match_dofs(xg, fg, xo, fo)
    # the benchmark's input: U(-1,1) in the library's order
    x_lib = inputs.uniform_vector(len(perm))
    x = x_lib[perm]
    c = op.dofs.constrained
    h = 1.0 / 64
    rng = np.random.default_rng(7)
    rows = np.concatenate([
        rng.choice(len(perm), 150, replace=False),
        _rows_in_box(xo, 1 - 2 * h, 1.0, c),          # last cell of every colour
        _rows_in_box(xo, 0.0, 2 * h, c),              # first cells
        np.nonzero(c)[0][:20],                        # identity rows
    ])
    rows = np.unique(rows)
    yo = op.sampled_rows(rows, x)
    return prob, perm, op, rows, x, yo, m


@pytest.mark.parametrize("prec", [0, 1])
def test_stab_ns_64_vmult_sampled_rows(stab_ns_64, prec):
    prob, perm, op, rows, x, yo, _ = stab_ns_64
    assert len(rows) > 500
    y = _compare(prob, perm, op, rows, x, prec)
    rel = np.linalg.norm(y - yo) / np.linalg.norm(yo)
    assert rel <= TOL[prec], rel
    assert np.abs(y - yo).max() <= 10 * TOL[prec] * np.abs(yo).max()


@pytest.fixture(scope="module")
def stokes_ball_32(ctx):
    from paper_2603_29621_gb300 import _lib as L, api
    m = api.Mesh(ctx, 3, 32)
    m.refine_ball(*BALL)
    prob = api.Problem(ctx, m, kind=L.STOKES, degree=2, nu=1.0, mg_precision=L.FP32)
    op = assemble.Problem(mesh.refine_ball(mesh.uniform(3, 32), *BALL), "stokes", 2, nu=1.0)
    xg, fg = prob.support_points()
    xo, fo = op.dofs.support_points()
    perm = inputs.match_dofs(xg, fg, xo, fo)
    x = inputs.uniform_vector(len(perm))
    d = op.dofs
    ccsc = d.C.tocsc()
    deps = np.diff(ccsc.indptr)                              # 1 + number of hanging dependents
    masters = d.free_ids[deps > 1]
    rng = np.random.default_rng(8)
    rows = np.unique(np.concatenate([rng.choice(len(perm), 150, replace=False),
                                     rng.choice(masters, 60, replace=False),
                                     np.nonzero(d.constrained)[0][:20]]))
    yo = op.sampled_rows(rows, x)
    return prob, perm, op, rows, x, yo, m, len(masters)


@pytest.mark.parametrize("prec", [0, 1])
def test_stokes_ball_32_vmult_sampled_rows(stokes_ball_32, prec):
    prob, perm, op, rows, x, yo, _, n_masters = stokes_ball_32
    assert n_masters > 1000 and prob.info.n_cells > 150000
    y = _compare(prob, perm, op, rows, x, prec)
    rel = np.linalg.norm(y - yo) / np.linalg.norm(yo)
    assert rel <= TOL[prec], rel


@pytest.mark.parametrize("nu", [1e-1, 1e-2, 1e-3])
def test_stab_ns_48_solve_fp32_multigrid(ctx, nu):
    from paper_2603_29621_gb300 import _lib as L, api
    m = api.Mesh(ctx, 3, 48)
    prob = api.Problem(ctx, m, kind=L.STAB_NS, degree=2, nu=nu, dt=1e-2, mg_precision=L.FP32, tol=1e-13,
                       maxit=300)
    xyz, fld = prob.support_points()
    xs_np = inputs.smooth_solution(xyz, fld, 3)
    xs = torch.tensor(xs_np, device="cuda")
    b = torch.empty_like(xs)
    prob.vmult(xs, b)
    x = torch.zeros_like(xs)
    info = prob.solve(b, x)
    assert info.converged and info.iterations <= 20
    # b = A x* on sampled rows against the oracle
    op = assemble.Problem(mesh.uniform(3, 48), "stab_ns", 2, nu=nu, dt=1e-2)
    xo, fo = op.dofs.support_points()
    perm = inputs.match_dofs(xyz, fld, xo, fo)
    rows = np.unique(np.random.default_rng(9).choice(len(perm), 120, replace=False))
    bo = op.sampled_rows(rows, xs_np[perm])
    bg = b.cpu().numpy()[perm[rows]]
    assert np.linalg.norm(bg - bo) <= 1e-12 * np.linalg.norm(bo)
    # solution against x* (pressure mean removed on both)
    d = (x - xs).cpu().numpy()
    xr = xs_np.copy()
    ps = slice(3, None, 4)
    d[ps] -= d[ps].mean()
    xr[ps] -= xr[ps].mean()
    assert np.linalg.norm(d) <= 1e-8 * np.linalg.norm(xr), np.linalg.norm(d) / np.linalg.norm(xr)


def test_stokes_ball_32_solve_fp32_multigrid(ctx):
    """Config 3's Stokes system with the FP32 multigrid: the solution of b = A x* to 1e-8 of x*
    (A itself is pinned against the oracle on sampled rows above)."""
    from paper_2603_29621_gb300 import _lib as L, api
    m = api.Mesh(ctx, 3, 32)
    m.refine_ball(*BALL)
    prob = api.Problem(ctx, m, kind=L.STOKES, degree=2, nu=1.0, mg_precision=L.FP32, tol=1e-14, maxit=300)
    xyz, fld = prob.support_points()
    xs_np = inputs.smooth_solution(xyz, fld, 3, 1.0)
    xs = torch.tensor(xs_np, device="cuda")
    b = torch.empty_like(xs)
    prob.vmult(xs, b)
    x = torch.zeros_like(xs)
    info = prob.solve(b, x, raise_on_nonconvergence=False)
    assert info.iterations <= 60, info.iterations
    d = (x - xs).cpu().numpy()
    xr = xs_np.copy()
    ps = slice(prob.info.n_velocity_dofs, None)
    d[ps] -= d[ps].mean()
    xr[ps] -= xr[ps].mean()
    assert np.linalg.norm(d) <= 1e-8 * np.linalg.norm(xr), np.linalg.norm(d) / np.linalg.norm(xr)
