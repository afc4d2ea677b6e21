"""The space-time slab operator (Section 4, Eq. 6) on the GPU against the oracle, through the C ABI.

K = G_Q (x) M + tau I_Q (x) A on stage-major vectors, Taylor--Hood in space (uniform meshes and a
ball-refined mesh with hanging nodes), DG(r) in time on right Radau points, r = 0..3: every entry
of K x agrees with the oracle's assembled Kronecker operator to 1e-12 relative (FP64) and 1e-5 in
the 2-norm (FP32)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mesh, spacetime  # noqa: E402
from paper_2603_29621_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu
CENTRE = (0.3, 0.35, 0.4)


@pytest.fixture(scope="module")
def ctx():
    from paper_2603_29621_gb300 import api
    return api.Context(0)


CASES = [(2, 4, False, 2, 1), (2, 3, True, 2, 2), (2, 4, False, 3, 0), (3, 2, False, 2, 1), (3, 2, True, 2, 3),
         (3, 2, False, 3, 1)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}d-n{c[1]}-{'ball' if c[2] else 'uni'}-k{c[3]}-r{c[4]}")
def test_slab_operator_matches_oracle(ctx, case):
    from paper_2603_29621_gb300 import _lib as L, api
    dim, n, ball, k, r = case
    nu, tau = 0.8, 0.3
    f = mesh.uniform(dim, n)
    m = api.Mesh(ctx, dim, n)
    if ball:
        f = mesh.refine_ball(f, CENTRE, 0.3, 1)
        m.refine_ball(CENTRE, 0.3, 1)
    prob = api.Problem(ctx, m, kind=L.STOKES, degree=k, nu=nu, lambda_max=1.0)
    st = api.SpaceTime(prob, r, tau)
    ost = spacetime.SpaceTimeStokes(f, k, r, nu=nu, tau=tau, pressure="continuous")
    assert st.Q == ost.Q and st.n == ost.n
    assert np.abs(st.nodes - ost.nodes).max() <= 1e-14
    assert np.abs(st.G - ost.G_Q).max() <= 1e-12 * np.abs(ost.G_Q).max()
    K = ost.operator()
    xg, fg = prob.support_points()
    xo, fo = ost.space.dofs.support_points()
    perm = inputs.match_dofs(xg, fg, xo, fo)                 # library entry of oracle entry i
    full = (np.arange(st.Q)[:, None] * st.n + perm[None, :]).ravel()
    x = inputs.uniform_vector(st.Q * st.n, seed=11)
    exp = K @ x
    for dtype, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        xd = np.empty_like(x)
        xd[full] = x
        src = torch.tensor(xd, device="cuda", dtype=dtype)
        dst = torch.full_like(src, 7.0)
        st.vmult(src, dst)
        torch.cuda.synchronize()
        got = dst.double().cpu().numpy()[full]
        if dtype == torch.float64:
            assert np.abs(got - exp).max() <= tol * np.abs(exp).max()
        else:
            assert np.linalg.norm(got - exp) <= tol * np.linalg.norm(exp)


def test_slab_rejects_other_problems(ctx):
    from paper_2603_29621_gb300 import _lib as L, api
    m = api.Mesh(ctx, 2, 3)
    prob = api.Problem(ctx, m, kind=L.STOKES_A, degree=2, lambda_max=1.0)
    with pytest.raises(L.MfnsError) as e:
        api.SpaceTime(prob, 1, 0.1)
    assert e.value.code == L.ERR_UNSUPPORTED


# (dim, n, k, r, coarse_n): with coarse_n = 4 the coarsest mesh has no star holding every cell, so
# the temporal levels (and their transfers) follow the spatial ones
STMG_CASES = [(2, 8, 2, 1, 2), (2, 4, 3, 2, 2), (3, 4, 2, 1, 2), (2, 8, 2, 1, 4), (2, 8, 3, 2, 4)]


@pytest.mark.parametrize("case", STMG_CASES, ids=lambda c: f"{c[0]}d-n{c[1]}-k{c[2]}-r{c[3]}-c{c[4]}")
def test_space_time_multigrid_matches_oracle(ctx, case):
    """Every level's slab operator (1e-12), Schwarz smoother and transfers (1e-12), and one V-cycle
    of the space-time multigrid against the oracle's (vertex stars, nu_s = 4, omega = 0.7, uniform
    meshes).  The patch blocks are saddle-point matrices of condition up to 6e4 here, inverted by
    different eliminations on the two sides (LAPACK LU, Gauss--Jordan): their products agree to
    about cond * eps * (block size), hence 1e-9 for the smoother and 1e-8 for the cycle (eight
    smoothing steps and a coarse solve of condition up to 2e4)."""
    from paper_2603_29621_gb300 import _lib as L, api
    dim, n, k, r, coarse_n = case
    nu, tau = 1.0, 0.05
    f = mesh.uniform(dim, n)
    m = api.Mesh(ctx, dim, n)
    prob = api.Problem(ctx, m, kind=L.STOKES, degree=k, nu=nu, lambda_max=1.0)
    st = api.SpaceTime(prob, r, tau)
    levels = st.mg_build(nu_s=4, omega=0.7, coarse_n=coarse_n)
    lv = spacetime.stmg_levels(f, k, r, nu=nu, tau=tau, pressure="continuous", stop_n=coarse_n)
    assert [(a, b) for a, b, _ in levels] == [(l.k, l.r) for l in lv]
    if coarse_n == 4:
        assert any(lv[l].r != lv[l + 1].r for l in range(len(lv) - 1))
    full = []
    for l, olv in enumerate(lv):
        xg, fg = st.mg_support_points(l)
        xo, fo = olv.st.space.dofs.support_points()
        perm = inputs.match_dofs(xg[:, :dim], fg, xo, fo)
        assert levels[l][2] == olv.st.n
        full.append((np.arange(olv.st.Q)[:, None] * olv.st.n + perm[None, :]).ravel())

    def to_gpu(x, l):
        xd = np.empty_like(x)
        xd[full[l]] = x
        return torch.tensor(xd, device="cuda")

    def from_gpu(t, l):
        torch.cuda.synchronize()
        return t.cpu().numpy()[full[l]]

    rng = np.random.default_rng(3)
    for l, olv in enumerate(lv):
        N = olv.K.shape[0]
        x = rng.uniform(-1, 1, N)
        y = torch.zeros(N, dtype=torch.float64, device="cuda")
        exp = olv.K @ x
        assert np.abs(from_gpu(st.mg_apply(l, 0, to_gpu(x, l), y), l) - exp).max() <= 1e-12 * np.abs(exp).max(), l
        if l == len(lv) - 1:
            break
        exp = olv.schwarz(x)
        got = from_gpu(st.mg_apply(l, 1, to_gpu(x, l), y), l)
        assert np.abs(got - exp).max() <= 1e-9 * np.abs(exp).max(), l
        Nc = lv[l + 1].K.shape[0]
        xc = rng.uniform(-1, 1, Nc)
        xf0 = rng.uniform(-1, 1, N)
        fine = to_gpu(xf0, l)
        st.mg_apply(l, 2, to_gpu(xc, l + 1), fine)
        exp = xf0 + olv.P @ xc
        assert np.abs(from_gpu(fine, l) - exp).max() <= 1e-12 * np.abs(exp).max(), l
        coarse = torch.zeros(Nc, dtype=torch.float64, device="cuda")
        st.mg_apply(l, 3, to_gpu(xf0, l), coarse)
        exp = olv.P.T @ xf0
        assert np.abs(from_gpu(coarse, l + 1) - exp).max() <= 1e-12 * np.abs(exp).max(), l
    V = spacetime.STMG(lv, nu_s=4, omega=0.7)
    # a right-hand side in the range of K (consistent hanging entries, no constant pressures)
    d = lv[0].st.space.dofs
    xs = V.project(np.tile(d.distribute(rng.uniform(-1, 1, d.n_dofs)), lv[0].st.Q))
    b = lv[0].K @ xs
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    st.vcycle(to_gpu(b, 0), x)
    exp = V(b)
    assert np.abs(from_gpu(x, 0) - exp).max() <= 1e-8 * np.abs(exp).max()


@pytest.mark.parametrize("case", [(2, 8, 2, 1), (3, 4, 2, 1)], ids=lambda c: f"{c[0]}d-n{c[1]}-k{c[2]}-r{c[3]}")
def test_space_time_solve_converges(ctx, case):
    """FGMRES with the space-time V-cycle: the manufactured slab solution (no constant pressures) is
    recovered, in about the oracle's number of iterations."""
    from oracle import solvers
    from paper_2603_29621_gb300 import _lib as L, api
    dim, n, k, r = case
    nu, tau = 1.0, 0.05
    f = mesh.uniform(dim, n)
    m = api.Mesh(ctx, dim, n)
    prob = api.Problem(ctx, m, kind=L.STOKES, degree=k, nu=nu, lambda_max=1.0)
    st = api.SpaceTime(prob, r, tau)
    st.mg_build(nu_s=4, omega=0.7)
    lv = spacetime.stmg_levels(f, k, r, nu=nu, tau=tau, pressure="continuous")
    V = spacetime.STMG(lv)
    K = lv[0].K
    d = lv[0].st.space.dofs
    xs = V.project(np.tile(d.distribute(np.random.default_rng(1).uniform(-1, 1, d.n_dofs)), lv[0].st.Q))
    b = K @ xs
    _, its_o, _ = solvers.fgmres(K, b, V, tol=1e-10, maxit=200, project=V.project)
    xg, fg = prob.support_points()
    xo, fo = d.support_points()
    perm = inputs.match_dofs(xg, fg, xo, fo)
    full = (np.arange(st.Q)[:, None] * st.n + perm[None, :]).ravel()
    bd = np.empty_like(b)
    bd[full] = b
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    its, rel = st.solve(torch.tensor(bd, device="cuda"), x, tol=1e-10, maxit=200)
    torch.cuda.synchronize()
    got = x.cpu().numpy()[full]
    assert rel <= 1e-10 and abs(its - its_o) <= 3, (its, its_o)
    assert np.abs(V.project(got) - xs).max() <= 1e-6 * np.abs(xs).max()


@pytest.mark.parametrize("case", [("th", 2, 8, 2, 1), ("th", 3, 4, 2, 1), ("pdisc", 3, 4, 2, 1)],
                         ids=lambda c: f"{c[0]}-{c[1]}d-n{c[2]}-k{c[3]}-r{c[4]}")
def test_fp32_patch_inverses(ctx, case):
    """FP32 Schwarz patch inverses: inverted in FP64, rounded to FP32, the patch products formed in
    FP32 (half the bytes of every patch solve; vectors, transfers, coarse solve and FGMRES stay
    FP64).  The smoother application agrees with the FP64 one to single-precision round-off
    amplified by the patch blocks (<= 2e-5 relative in the 2-norm on uniform random input), the
    reported inverse bytes halve, and the solve reaches the same tolerance in at most one more
    iteration, with the same solution (both have no constant pressure per stage) to 1e-6."""
    from paper_2603_29621_gb300 import _lib as L, api
    kind, dim, n, k, r = case
    m = api.Mesh(ctx, dim, n)
    prob = None
    if kind == "th":
        prob = api.Problem(ctx, m, kind=L.STOKES, degree=k, nu=1.0, lambda_max=1.0)
        st = api.SpaceTime(prob, r, 0.05)
    else:
        st = api.SpaceTime.pdisc(ctx, m, k, 1.0, r, 0.05)
    N = st.Q * st.n
    x = torch.tensor(inputs.uniform_vector(N, seed=5), device="cuda")
    xs = torch.tensor(inputs.uniform_vector(N, seed=6), device="cuda")
    b = torch.empty_like(xs)
    st.vmult(xs, b)
    res = {}
    for prec in (0, 1):
        st.mg_build(nu_s=4, omega=0.7, inverse_precision=prec)
        z = torch.zeros(N, dtype=torch.float64, device="cuda")
        st.mg_apply(0, 1, x, z)
        nbytes, npatch = st.mg_smoother_bytes(0)
        xsol = torch.zeros(N, dtype=torch.float64, device="cuda")
        its, rel = st.solve(b, xsol, tol=1e-10, maxit=200)
        torch.cuda.synchronize()
        res[prec] = (z, nbytes, npatch, its, rel, xsol)
    assert res[0][2] == res[1][2] > 0 and res[1][1] * 2 == res[0][1]
    z64, z32 = res[0][0], res[1][0]
    assert float(torch.linalg.norm(z32 - z64) / torch.linalg.norm(z64)) <= 2e-5
    assert res[1][4] <= 1e-10 and res[1][3] <= res[0][3] + 1, (res[0][3], res[1][3])
    assert float(torch.linalg.norm(res[1][5] - res[0][5]) / torch.linalg.norm(res[0][5])) <= 1e-6
    for prec in (0, 1):  # the reported residual is the true one
        kx = torch.empty_like(b)
        st.vmult(res[prec][5], kx)
        torch.cuda.synchronize()
        assert float(torch.linalg.norm(kx - b) / torch.linalg.norm(b)) <= 1e-9
    with pytest.raises(L.MfnsError) as e:
        st.mg_build(inverse_precision=2)
    assert e.value.code == L.ERR_ARG
    st.close()
    if prob is not None:
        prob.close()
    m.close()
