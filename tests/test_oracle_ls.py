"""Pins of the oracle's local-smoothing multigrid (Section 2).

* The level operators: for the vector Laplacian, P_l^T A P_l on the interior level DoFs equals the
  operator assembled on the uniform level-l mesh (n 2^l cells per direction) restricted to the
  same nodes.  A wrong interpolation weight, a missed fine DoF or a refinement-edge node taken
  as interior changes the product.
* The level spaces together span the fine space: every free fine DoF is reached.
* On an unrefined mesh the cycle is the base mesh's global-coarsening V-cycle.
* The cycle is a symmetric operator (symmetric smoothers visited in mirrored order).
* As an FGMRES preconditioner it converges in about as many iterations as global coarsening
  (Section 2 and Tables 3/4: the two need similar iteration counts).
"""
import numpy as np
import pytest

from oracle import assemble, ls, mesh, solvers


def _ball(dim, n, levels, r=0.3):
    return mesh.refine_ball(mesh.uniform(dim, n), (0.3, 0.35, 0.4), r, levels)


def _bounds(levels_A_dinv):
    return [1.2 * solvers.power_lmax(A, dinv, iterations=60) for A, dinv in levels_A_dinv]


def _ls(problem, smoother=("chebyshev", 3)):
    """LocalSmoothing with bounds from power iterations on both hierarchies."""
    tmp = ls.LocalSmoothing(problem, [1.0] * problem.forest.max_level, [1.0] * 8, smoother)
    lm_ls = _bounds([(lv.A, lv.dinv) for lv in tmp.levels])
    lm_base = _bounds([(lv.A, lv.dinv) for lv in tmp.base_levels[:-1]])
    return ls.LocalSmoothing(problem, lm_ls, lm_base, smoother)


@pytest.mark.parametrize("dim,n,levels,k", [(2, 3, 2, 2), (2, 2, 2, 3), (3, 2, 1, 2), (2, 4, 1, 1)])
def test_level_operator_is_the_level_mesh_operator(dim, n, levels, k):
    f = _ball(dim, n, levels)
    p = assemble.Problem(f, "stokes_a", k, nu=0.7)
    A = p.assemble()
    for l in range(1, f.max_level + 1):
        lv = ls.LsLevel(p, A, l)
        sp_ = lv.space
        covers = len(sp_.cells) == sp_.N ** dim      # the level can cover the whole domain
        assert sp_.edge.any() != covers and sp_.interior.any()
        U = assemble.Problem(mesh.uniform(dim, n * 2 ** l), "stokes_a", k, nu=0.7)
        AU = U.assemble()
        nsU = U.dofs.nodesets[0]
        key = {tuple(np.rint(x * 1e9).astype(np.int64)): g for g, x in enumerate(nsU.x)}
        gU = np.array([key[tuple(np.rint(x * 1e9).astype(np.int64))] for x in sp_.x])
        inner = np.nonzero(sp_.interior)[0]
        I = np.concatenate([c * sp_.n_nodes + inner for c in range(dim)])
        J = np.concatenate([U.dofs.dof(0, c, gU[inner]) for c in range(dim)])
        Al = lv.A[I][:, I].toarray()
        Au = AU[J][:, J].toarray()
        assert np.abs(Al - Au).max() <= 1e-12 * np.abs(Au).max()


@pytest.mark.parametrize("dim,n,levels,k", [(2, 3, 2, 2), (3, 2, 1, 1)])
def test_level_spaces_span_the_fine_space(dim, n, levels, k):
    f = _ball(dim, n, levels)
    p = assemble.Problem(f, "stokes_a", k)
    A = p.assemble()
    L = ls.LocalSmoothing(p, [1.0] * f.max_level, [1.0] * 8)
    free = p.dofs.free_ids
    blocks = [L.P0] + [lv.P for lv in L.levels]
    M = np.concatenate([B[free].toarray() for B in blocks], axis=1)
    assert np.linalg.matrix_rank(M) == len(free)
    # the finest level alone does not (the refined part is a proper subdomain)
    assert np.linalg.matrix_rank(L.levels[-1].P[free].toarray()) < len(free)
    del A


def test_constrained_rows_are_inverted_exactly():
    """Dirichlet and hanging rows of A are identity rows outside every level space: the cycle
    returns b there, and its free part does not depend on b's constrained entries."""
    f = _ball(2, 3, 2)
    p = assemble.Problem(f, "stokes_a", 2)
    L = _ls(p)
    d = p.dofs
    assert d.hanging.any() and d.dirichlet.any()
    rng = np.random.default_rng(4)
    b = rng.uniform(-1, 1, d.n_dofs)
    x = L(b)
    assert np.all(x[d.constrained] == b[d.constrained])
    x_free = L(b * d.free)
    assert np.abs(x[d.free] - x_free[d.free]).max() <= 1e-14 * np.abs(x_free).max()


def test_uniform_mesh_cycle_is_the_base_vcycle():
    f = mesh.uniform(2, 4)
    p = assemble.Problem(f, "stokes_a", 2)
    L = _ls(p)
    assert L.levels == []
    rng = np.random.default_rng(0)
    b = rng.uniform(-1, 1, p.dofs.n_dofs) * p.dofs.free
    ref = L.base(b)                                  # the base problem is the same problem
    got = L(b)
    fr = p.dofs.free
    assert np.abs(got[fr] - ref[fr]).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("smoother", [("chebyshev", 3), ("jacobi", 2)])
def test_cycle_is_symmetric(smoother):
    f = _ball(2, 2, 2)
    p = assemble.Problem(f, "stokes_a", 2)
    L = _ls(p, smoother)
    free = p.dofs.free_ids
    M = np.zeros((len(free), len(free)))
    for j, g in enumerate(free):
        e = np.zeros(p.dofs.n_dofs)
        e[g] = 1.0
        M[:, j] = L(e)[free]
    assert np.abs(M - M.T).max() <= 1e-10 * np.abs(M).max()
    # positive definite on the free DoFs (a preconditioner for an SPD operator)
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


@pytest.mark.parametrize("dim,n,levels,k", [(2, 4, 2, 2), (3, 2, 2, 2)])
def test_fgmres_iterations_similar_to_global_coarsening(dim, n, levels, k):
    f = _ball(dim, n, levels)
    p = assemble.Problem(f, "stokes_a", k)
    A = p.assemble()
    rng = np.random.default_rng(3)
    xs = p.dofs.set_hanging(rng.uniform(-1, 1, p.dofs.n_dofs))   # Dirichlet values nonzero too
    b = A @ xs
    L = _ls(p)
    x_ls, it_ls, res_ls = solvers.fgmres(A, b, L, tol=1e-10)
    gc = solvers.hierarchy(f, "stokes_a", k)
    V = solvers.VCycle(gc, _bounds([(lv.A, lv.dinv) for lv in gc[:-1]]), ("chebyshev", 3))
    x_gc, it_gc, res_gc = solvers.fgmres(A, b, V, tol=1e-10)
    assert res_ls <= 1e-10 and res_gc <= 1e-10
    assert np.abs(x_ls - xs).max() <= 1e-7 * np.abs(xs).max()
    assert it_ls <= it_gc + 4 and it_ls <= 25


# -- the level recursion with rediscretised level operators (stabilised NS) --------------------------
@pytest.mark.parametrize("dim,n,levels,k", [(2, 4, 2, 2), (3, 2, 1, 2), (2, 3, 2, 1)])
def test_level_recursion_equals_subspace_correction_for_the_vector_laplacian(dim, n, levels, k):
    """Rediscretised level operators equal the Galerkin ones here, so the recursion the library runs
    (defects to owners, residual edge rows restricted, edge held at zero) is the subspace correction."""
    f = _ball(dim, n, levels)
    p = assemble.Problem(f, "stokes_a", k, nu=0.8)
    S = _ls(p)
    R = ls.LocalSmoothingLevels(p, [lv.lmax for lv in S.levels], [lv.lmax for lv in S.base_levels[:-1]],
                                ("chebyshev", 3), nu=0.8)
    b = np.random.default_rng(1).uniform(-1, 1, p.dofs.n_dofs)     # constrained entries nonzero too
    exp = S(b)
    assert np.abs(R(b) - exp).max() <= 1e-12 * np.abs(exp).max()


def _relaxation_lmax(A, dinv):
    """lmax with 2 / (lmax / 20 + lmax) = the weight minimising max |1 - w theta| over the eigenvalues
    theta of D^-1 A with |theta| >= rho / 2 (exact spectrum, small problems)."""
    th = np.linalg.eigvals((dinv[:, None] * A.toarray()))
    rho = np.abs(th).max()
    S_ = th[np.abs(th) >= 0.5 * rho]
    ws = np.linspace(1e-4, 2.0 / np.abs(S_).min(), 20001)
    w = ws[np.argmin(np.abs(1 - ws[:, None] * S_[None, :]).max(axis=1))]
    return 2.0 / (1.05 * w)


@pytest.mark.parametrize("k,nu", [(2, 1e-2), (1, 1e-2), (2, 0.2)])
def test_stabilised_ns_local_smoothing_converges(k, nu):
    """Section 5 / Tables 3-4: local smoothing of the stabilised operator (rediscretised levels,
    Dirichlet conditions for u and p on refinement edges) makes FGMRES converge, and global
    coarsening needs no more iterations (the paper's slight advantage for global coarsening; on
    these small 2D meshes, where edge DoFs are a large share, the gap is larger: 11-13 against
    4-7)."""
    f = _ball(2, 4, 2)
    params = dict(nu=nu, dt=1e-2)
    p = assemble.Problem(f, "stab_ns", k, **params)
    A = p.assemble()
    sm = ("jacobi", 5)
    tmp = ls.LocalSmoothingLevels(p, [1.0] * f.max_level, [1.0] * 8, sm, **params)
    lm_ls = [_relaxation_lmax(lv.op, lv.dinv) for lv in tmp.levels]
    lm_b = [_relaxation_lmax(lv.A, lv.dinv) for lv in tmp.base_levels[:-1]]
    R = ls.LocalSmoothingLevels(p, lm_ls, lm_b, sm, **params)
    gc = solvers.hierarchy(f, "stab_ns", k, **params)
    V = solvers.VCycle(gc, [_relaxation_lmax(lv.A, lv.dinv) for lv in gc[:-1]], sm)
    rng = np.random.default_rng(4)
    xs = p.dofs.set_hanging(rng.uniform(-1, 1, p.dofs.n_dofs))
    b = A @ xs
    proj = p.project_pressure_mean
    x_ls, it_ls, res_ls = solvers.fgmres(A, proj(b), R, tol=1e-10, project=proj)
    x_gc, it_gc, res_gc = solvers.fgmres(A, proj(b), V, tol=1e-10, project=proj)
    assert res_ls <= 1e-10 and res_gc <= 1e-10
    assert np.abs(proj(x_ls - xs)).max() <= 1e-6 * np.abs(xs).max()
    assert it_ls <= 15 and it_gc <= it_ls, (it_ls, it_gc)
