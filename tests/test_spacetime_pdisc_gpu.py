"""Space-time slabs on the paper's spatial pair Q_k / P^disc_{k-1} (Section 4) on the GPU against the
oracle, through the C ABI (uniform meshes, FP64): the slab operator (1e-12); the space-time
multigrid's levels, cell-patch Schwarz smoothers (1e-9: patch blocks of condition up to ~1e5,
inverted by different eliminations), transfers (1e-12) and one V-cycle (1e-8); an FGMRES solve whose
iteration count does not grow under refinement with tau refined with h (Section 4's report)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mesh, solvers, spacetime  # noqa: E402
from paper_2603_29621_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2603_29621_gb300 import api
    return api.Context(0)


def _oracle_points(space):
    """(support point, field) of every entry of an oracle StokesPdisc space: velocity entries at
    their nodes, pressure coefficient a of cell c at the cell centre with field dim + a."""
    dim = space.dim
    xv, fv = space.vel.support_points()
    f = space.forest
    centres = f.origin() + 0.5 * f.h()[:, None]
    xp = np.repeat(centres, space.npc, axis=0)
    fp = dim + np.tile(np.arange(space.npc), f.n_cells)
    return np.concatenate([xv, xp]), np.concatenate([fv, fp])


def _full_perm(xyz, fld, space, Q, dim):
    xo, fo = _oracle_points(space)
    perm = inputs.match_dofs(xyz[:, :dim], fld, xo, fo)
    n = len(perm)
    return (np.arange(Q)[:, None] * n + perm[None, :]).ravel()


@pytest.mark.parametrize("dim,n,k,r", [(2, 4, 2, 1), (2, 2, 3, 2), (3, 2, 2, 1), (2, 4, 4, 0)])
def test_pdisc_slab_operator_matches_oracle(ctx, dim, n, k, r):
    from paper_2603_29621_gb300 import api
    nu, tau = 0.8, 0.3
    m = api.Mesh(ctx, dim, n)
    st = api.SpaceTime.pdisc(ctx, m, k, nu, r, tau)
    ost = spacetime.SpaceTimeStokes(mesh.uniform(dim, n), k, r, nu=nu, tau=tau, pressure="disc")
    assert st.Q == ost.Q and st.n == ost.n
    xyz, fld = st.support_points()
    full = _full_perm(xyz, fld, ost.space, st.Q, dim)
    x = inputs.uniform_vector(st.Q * st.n, seed=12)
    xd = np.empty_like(x)
    xd[full] = x
    y = torch.full((len(x),), 7.0, dtype=torch.float64, device="cuda")
    st.vmult(torch.tensor(xd, device="cuda"), y)
    torch.cuda.synchronize()
    exp = ost.operator() @ x
    assert np.abs(y.cpu().numpy()[full] - exp).max() <= 1e-12 * np.abs(exp).max()


@pytest.mark.parametrize("dim,n,k,r", [(2, 8, 2, 1), (2, 4, 3, 2), (3, 4, 2, 1)])
def test_pdisc_space_time_multigrid_matches_oracle(ctx, dim, n, k, r):
    from paper_2603_29621_gb300 import api
    nu, tau = 1.0, 0.05
    m = api.Mesh(ctx, dim, n)
    st = api.SpaceTime.pdisc(ctx, m, k, nu, r, tau)
    levels = st.mg_build(nu_s=4, omega=0.7)
    lv = spacetime.stmg_levels(mesh.uniform(dim, n), k, r, nu=nu, tau=tau, pressure="disc")
    assert [(a, b) for a, b, _ in levels] == [(l.k, l.r) for l in lv]
    full = []
    for l, olv in enumerate(lv):
        xg, fg = st.mg_support_points(l)
        full.append(_full_perm(xg, fg, olv.st.space, olv.st.Q, dim))

    def to_gpu(x, l):
        xd = np.empty_like(x)
        xd[full[l]] = x
        return torch.tensor(xd, device="cuda")

    def from_gpu(t, l):
        torch.cuda.synchronize()
        return t.cpu().numpy()[full[l]]

    rng = np.random.default_rng(5)
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
    V = spacetime.STMG(lv)
    d = lv[0].st.space.dofs
    xs = V.project(np.tile(d.distribute(rng.uniform(-1, 1, d.n_dofs)), lv[0].st.Q))
    b = lv[0].K @ xs
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    st.vcycle(to_gpu(b, 0), x)
    exp = V(b)
    assert np.abs(from_gpu(x, 0) - exp).max() <= 1e-8 * np.abs(exp).max()


def test_pdisc_solve_iterations_do_not_grow(ctx):
    from paper_2603_29621_gb300 import api
    its = []
    for n in (4, 8):
        tau = 0.2 / n
        m = api.Mesh(ctx, 2, n)
        st = api.SpaceTime.pdisc(ctx, m, 2, 1.0, 1, tau)
        st.mg_build()
        lv = spacetime.stmg_levels(mesh.uniform(2, n), 2, 1, nu=1.0, tau=tau, pressure="disc")
        V = spacetime.STMG(lv)
        d = lv[0].st.space.dofs
        xs = V.project(np.tile(d.distribute(np.random.default_rng(1).uniform(-1, 1, d.n_dofs)), lv[0].st.Q))
        b = lv[0].K @ xs
        xyz, fld = st.support_points()
        full = _full_perm(xyz, fld, lv[0].st.space, st.Q, 2)
        bd = np.empty_like(b)
        bd[full] = b
        x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
        it, rel = st.solve(torch.tensor(bd, device="cuda"), x, tol=1e-10, maxit=100)
        torch.cuda.synchronize()
        assert rel <= 1e-10
        assert np.abs(V.project(x.cpu().numpy()[full]) - xs).max() <= 1e-6 * np.abs(xs).max()
        its.append(it)
    assert max(its) <= 8 and abs(its[1] - its[0]) <= 2, its
