"""Pins of the oracle's meshes, transfers and row sampling (brute force and polynomial exactness)."""
import numpy as np
import pytest

from oracle import assemble, fe, forms, mesh, solvers, transfer


def test_ball_refinement_brute_force():
    f0 = mesh.uniform(3, 4)
    f = mesh.refine_ball(f0, (0.5, 0.5, 0.5), 0.25, 2)
    assert mesh.is_balanced(f)
    assert abs((f.h() ** 3).sum() - 1.0) < 1e-14
    # brute force: every lattice point of level <= 1 whose cell centre lies in the ball is refined
    N, cell_at = f.lattice()
    lev = f.cells[:, 0][cell_at]
    for l in (0, 1):
        n = 4 * 2 ** l
        c = (np.arange(n) + 0.5) / n
        X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
        inside = np.sqrt((X - .5) ** 2 + (Y - .5) ** 2 + (Z - .5) ** 2) < 0.25
        s = N // n
        coarse_lev = lev[::s, ::s, ::s]  # level of the active cell at the lower corner of each level-l box
        if l == 0:
            assert (coarse_lev[inside] >= 1).all()
        else:
            # only level-1 boxes inside refined level-0 cells are candidates
            parent_refined = (lev[::2 * s, ::2 * s, ::2 * s] >= 1).repeat(2, 0).repeat(2, 1).repeat(2, 2)
            assert (coarse_lev[inside & parent_refined] >= 2).all()
    # 2:1 brute force over all touching pairs
    for cid in range(f.n_cells):
        l, *c = f.cells[cid]
        s = 2 ** (f.max_level - l)
        sl = tuple(slice(max(ci * s - 1, 0), min((ci + 1) * s + 1, N)) for ci in c)
        assert lev[sl].max() <= l + 1


def test_coarsening_sequence():
    f = mesh.refine_ball(mesh.uniform(3, 8), (0.5, 0.5, 0.5), 0.25, 2)
    seq = solvers.coarse_forests(f)
    assert [s.max_level for s in seq] == [2, 1, 0, 0, 0]
    assert [s.n for s in seq] == [8, 8, 8, 4, 2]
    assert [s.n for s in solvers.coarse_forests(mesh.uniform(3, 47))] == [47, 24, 12, 6, 3, 2]
    assert all(mesh.is_balanced(s) for s in seq)
    assert seq[2].n_cells == 512


def _poly(dim, deg, seed=0, bubble=False):
    rng = np.random.default_rng(seed)
    coef = rng.uniform(-1, 1, (deg + 1,) * dim)

    def f(x):
        out = np.zeros(len(x))
        for idx in np.ndindex(*coef.shape):
            out += coef[idx] * np.prod([x[:, d] ** idx[d] for d in range(dim)], axis=0)
        if bubble:
            out = out * np.prod(x * (1 - x), axis=1)
        return out
    return f


@pytest.mark.parametrize("kind,dim,n", [("stokes_a", 2, 5), ("stab_ns", 3, 3)])
def test_non_nested_prolongation_reproduces_polynomials(kind, dim, n):
    """Uniform n -> ceil(n/2) for odd n (non-nested meshes): P I_c(poly) = I_f(poly) still holds."""
    fine_forest = mesh.uniform(dim, n)
    coarse_forest = fine_forest.coarsen_finest()
    assert coarse_forest.n == (n + 1) // 2
    ncomp = dim if kind == "stokes_a" else dim + 1
    for k in (1, 2):
        pc = assemble.Problem(coarse_forest, kind, k)
        pf = assemble.Problem(fine_forest, kind, k)
        P = transfer.prolongation(pc, pf)
        base = _poly(dim, max(k - 2, 0), bubble=True) if k >= 2 else (lambda x: 0 * x[:, 0])
        pfun = _poly(dim, k, seed=4)
        fun = lambda x: np.concatenate([np.stack([base(x)] * dim, 1), pfun(x)[:, None]], 1)[:, :ncomp]
        y = P @ pc.dofs.interpolate(fun)
        xf = pf.dofs.interpolate(fun)
        free = pf.dofs.free
        assert np.abs(y[free] - xf[free]).max() < 1e-12
        # a non-nested P is not a plain injection: some fine nodes see several coarse nodes
        assert (np.diff(P.tocsr().indptr) > 1).any()


@pytest.mark.parametrize("kind,dim", [("stokes_a", 2), ("stab_ns", 3), ("stokes_a", 3)])
def test_h_and_p_prolongation_reproduce_polynomials(kind, dim):
    fine_forest = mesh.refine_ball(mesh.uniform(dim, 2), (0.3, 0.3, 0.3), 0.3, 1)
    coarse_forest = fine_forest.coarsen_finest()
    ncomp = dim if kind == "stokes_a" else dim + 1
    for (fc, kc), (ff, kf) in [((coarse_forest, 2), (fine_forest, 2)), ((fine_forest, 1), (fine_forest, 2)),
                               ((fine_forest, 2), (fine_forest, 3))]:
        pc = assemble.Problem(fc, kind, kc)
        pf = assemble.Problem(ff, kind, kf)
        P = transfer.prolongation(pc, pf)
        # bubble-weighted polynomial of total per-direction degree kc vanishes on the boundary
        base = _poly(dim, max(kc - 2, 0), bubble=True) if kc >= 2 else (lambda x: np.prod(x * (1 - x), axis=1) * 0)
        pfun = _poly(dim, kc, seed=3)
        fun = lambda x: np.concatenate([np.stack([base(x)] * dim, 1), pfun(x)[:, None]], 1)[:, :ncomp]
        xc = pc.dofs.interpolate(fun)
        xf = pf.dofs.interpolate(fun)
        y = P @ xc
        free = pf.dofs.free
        assert np.abs(y[free] - xf[free]).max() < 1e-12
        assert np.abs(y[~free]).max() == 0.0


@pytest.mark.parametrize("kind,dim,k", [("stab_ns", 3, 2), ("stokes", 3, 2), ("stokes", 2, 3)])
def test_row_sampling_matches_assembly(kind, dim, k):
    f = mesh.refine_ball(mesh.uniform(dim, 2), (0.3, 0.3, 0.3), 0.3, 1)
    p = assemble.Problem(f, kind, k, nu=0.05, dt=0.01)
    A = p.assemble()
    x = np.random.default_rng(1).uniform(-1, 1, p.dofs.n_dofs)
    rows = np.random.default_rng(2).choice(p.dofs.n_dofs, 40, replace=False)
    rows = np.concatenate([rows, np.nonzero(p.dofs.hanging)[0][:3], np.nonzero(p.dofs.dirichlet)[0][:3]])
    assert np.allclose(p.sampled_rows(rows, x), (A @ x)[rows], rtol=1e-13, atol=1e-12)
