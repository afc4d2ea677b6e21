"""Pins of the oracle's element matrices and assembled operators.

Each check uses something the oracle does not compute the same way:
textbook values, tensor-product identities, closed-form integrals,
symmetry / null-space invariants, exact reproduction of polynomial
solutions and observed convergence rates."""
import numpy as np
import pytest
import sympy as sy

from oracle import assemble, fe, forms, mesh


def test_q1_laplacian_textbook():
    # unit square, Q1: diagonal 2/3, edge neighbours -1/6, opposite corner -1/3
    K = forms.vector_laplacian(2, 1, 1.0, [1.0])[0][:4, :4]
    expect = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6.0
    assert np.allclose(K, expect, atol=1e-15)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_tensor_identity_3d(k):
    # K_3d = K1 x M1 x M1 + M1 x K1 x M1 + M1 x M1 x K1 (x fastest index = last kron factor)
    K1 = forms.vector_laplacian(1, k, 1.0, [1.0])[0]
    M1 = forms.scalar_mass(1, k, k + 1, [1.0])[0]
    expect = np.kron(np.kron(M1, M1), K1) + np.kron(np.kron(M1, K1), M1) + np.kron(np.kron(K1, M1), M1)
    nb = (k + 1) ** 3
    K3 = forms.vector_laplacian(3, k, 1.0, [1.0])[0][:nb, :nb]
    assert np.allclose(K3, expect, atol=1e-13)
    # 1D closed form for k = 1: [[1,-1],[-1,1]] and [[1/3,1/6],[1/6,1/3]]
    if k == 1:
        assert np.allclose(K1[:2, :2], [[1, -1], [-1, 1]])
        assert np.allclose(M1, [[1 / 3, 1 / 6], [1 / 6, 1 / 3]])


@pytest.mark.parametrize("dim,k,h", [(2, 2, 0.5), (3, 3, 0.25)])
def test_mass_totals(dim, k, h):
    M = forms.scalar_mass(dim, k, k + 1, [h])[0]
    assert abs(M.sum() - h ** dim) < 1e-14
    # row sums = integral of each basis function = product of 1D GLL-basis integrals
    x, w = fe.gauss(k + 1)
    val, _, _ = fe.basis_1d(fe.gll_points(k), x)
    int1 = val @ w * h
    ni = fe.tensor_index(dim, k + 1)
    assert np.allclose(M.sum(1), np.prod(int1[ni], axis=1), atol=1e-15)


def _ball_forest(dim=3, n=2, levels=1):
    return mesh.refine_ball(mesh.uniform(dim, n), (0.3, 0.3, 0.3), 0.3, levels)


@pytest.mark.parametrize("dim,k,refined", [(2, 2, False), (2, 3, True), (3, 2, True)])
def test_stokes_symmetry_and_nullspace(dim, k, refined):
    f = _ball_forest(dim, 2, 1) if refined else mesh.uniform(dim, 3)
    p = assemble.Problem(f, "stokes", k, nu=0.7)
    A = p.assemble()
    assert abs(A - A.T).max() < 1e-13
    e = np.zeros(p.dofs.n_dofs)
    e[p.pressure_dofs()] = 1.0
    assert np.abs(A @ e).max() < 1e-13
    if refined:
        assert p.dofs.hanging.any()


def _bubble(dim):
    def u(x):
        v = np.prod(x * (1 - x), axis=1)
        return np.stack([v] * dim, axis=1)
    # closed form of int |grad v|^2 for v = prod x(1-x): dim * (1/3) * (1/30)^(dim-1)
    return u, dim * (1 / 3) * (1 / 30) ** (dim - 1)


@pytest.mark.parametrize("dim,k", [(2, 2), (3, 2), (2, 4)])
def test_energy_closed_form_on_hanging_mesh(dim, k):
    f = _ball_forest(dim, 2, 1)
    nu = 1.3
    p = assemble.Problem(f, "stokes_a", k, nu=nu)
    A = p.assemble()
    u, e1 = _bubble(dim)
    x = p.dofs.interpolate(u)
    x[p.dofs.constrained] = 0.0          # A ignores constrained entries on free rows
    energy = x @ (A @ x)
    assert abs(energy - nu * dim * e1) < 1e-12 * max(1, energy)


@pytest.mark.parametrize("dim,k", [(2, 2), (3, 3)])
def test_hanging_weights_reproduce_polynomials(dim, k):
    f = _ball_forest(dim, 2, 1)
    ns = mesh.NodeSet(f, k)
    assert len(ns.hanging) > 0
    rng = np.random.default_rng(0)
    coef = rng.uniform(-1, 1, (k + 1,) * dim)

    def poly(x):  # a global Q_k polynomial
        out = np.zeros(len(x))
        for idx in np.ndindex(*coef.shape):
            out += coef[idx] * np.prod([x[:, d] ** idx[d] for d in range(dim)], axis=0)
        return out

    v = poly(ns.x)
    for g, masters in ns.hanging.items():
        assert abs(v[g] - sum(w * v[m] for m, w in masters)) < 1e-12


def test_uniform_node_counts():
    for dim, n, k in [(2, 16, 2), (3, 4, 2), (3, 3, 3), (2, 5, 4)]:
        ns = mesh.NodeSet(mesh.uniform(dim, n), k)
        assert ns.n_nodes == (k * n + 1) ** dim
        assert len(ns.hanging) == 0


# -- manufactured exactness ---------------------------------------------------------
def _manufactured(dim, nu):
    if dim == 2:
        u = lambda x: np.stack([x[:, 0] ** 2, -2 * x[:, 0] * x[:, 1]], axis=1)
        p = lambda x: x[:, 0] + x[:, 1] - 1
        f = lambda x: np.stack([np.full(len(x), 1 - 2 * nu), np.ones(len(x))], axis=1)
    else:
        u = lambda x: np.stack([x[:, 1] ** 2 + x[:, 2], x[:, 2] ** 2 + x[:, 0], x[:, 0] ** 2 + x[:, 1]], axis=1)
        p = lambda x: x[:, 0] + x[:, 1] + x[:, 2] - 1.5
        f = lambda x: np.full((len(x), 3), 1 - 2 * nu)
    return u, p, f


@pytest.mark.parametrize("dim,n,refined", [(2, 4, False), (2, 2, True), (3, 2, False), (3, 2, True)])
def test_stokes_manufactured_exact(dim, n, refined):
    nu = 1.0 if dim == 2 else 0.5
    f = _ball_forest(dim, n, 1) if refined else mesh.uniform(dim, n)
    prob = assemble.Problem(f, "stokes", 2, nu=nu)
    u, p, fr = _manufactured(dim, nu)
    F = assemble.load_vector(prob, fr)
    b = assemble.dirichlet_system(prob, F, u)
    x = assemble.solve_direct(prob, b)
    full = assemble.complete_solution(prob, x, u)
    exact = prob.dofs.interpolate(lambda X: np.concatenate([u(X), p(X)[:, None]], axis=1))
    ids = prob.pressure_dofs()
    pres = np.zeros(prob.dofs.n_dofs, dtype=bool)
    pres[prob.dofs.offsets[1]:] = True
    err_u = np.abs(full - exact)[~pres].max()
    dp = (full - exact)[pres]
    err_p = np.abs(dp - dp.mean()).max()
    assert err_u < 1e-10 and err_p < 1e-9, (err_u, err_p)


@pytest.mark.slow
def test_stokes_convergence_rates_2d():
    X, Y = sy.symbols("x y")
    psi = sy.sin(sy.pi * X) ** 2 * sy.sin(sy.pi * Y) ** 2
    ue = [sy.diff(psi, Y), -sy.diff(psi, X)]
    pe = sy.cos(sy.pi * X) * sy.cos(sy.pi * Y)
    nu = 1.0
    fe_ = [-nu * (sy.diff(ue[i], X, 2) + sy.diff(ue[i], Y, 2)) + sy.diff(pe, [X, Y][i]) for i in range(2)]
    lu = [sy.lambdify((X, Y), e, "numpy") for e in ue]
    lp = sy.lambdify((X, Y), pe, "numpy")
    lf = [sy.lambdify((X, Y), e, "numpy") for e in fe_]
    uf = lambda x: np.stack([lu[i](x[:, 0], x[:, 1]) * np.ones(len(x)) for i in range(2)], axis=1)
    ff = lambda x: np.stack([lf[i](x[:, 0], x[:, 1]) * np.ones(len(x)) for i in range(2)], axis=1)
    errs = []
    for n in (4, 8, 16):
        prob = assemble.Problem(mesh.uniform(2, n), "stokes", 2, nu=nu)
        F = assemble.load_vector(prob, ff)
        b = assemble.dirichlet_system(prob, F, uf)
        x = assemble.complete_solution(prob, assemble.solve_direct(prob, b), uf)
        # L2 errors with a 6-point Gauss rule per direction
        phi_u, _, _, w, xq = fe.reference_tables(2, 2, 6)
        phi_p, _, _, _, _ = fe.reference_tables(2, 1, 6)
        h = prob.forest.h()
        xg = prob.forest.origin()[:, None, :] + h[:, None, None] * xq[None]
        d = prob.dofs
        eu = ep = 0.0
        nsu, nsp = d.nodesets
        pvals = x[d.offsets[1]:][nsp.cell_nodes]            # (nc, nbp)
        ph = np.einsum("qb,cb->cq", phi_p, pvals)
        pex = lp(xg[..., 0], xg[..., 1])
        W = w[None] * h[:, None] ** 2
        pm = (W * (ph - pex)).sum() / W.sum()
        ep = np.sqrt((W * (ph - pex - pm) ** 2).sum())
        for c in range(2):
            uv = x[c * nsu.n_nodes + nsu.cell_nodes]
            uh = np.einsum("qb,cb->cq", phi_u, uv)
            eu += (W * (uh - lu[c](xg[..., 0], xg[..., 1])) ** 2).sum()
        errs.append((np.sqrt(eu), ep))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert rates[-1, 0] > 2.8 and rates[-1, 1] > 1.8, rates


# -- stabilised Navier--Stokes -------------------------------------------------------
def _frozen_loc(dim, k, h, fun, x0=None):
    ni = fe.tensor_index(dim, k + 1)
    x0 = np.zeros(dim) if x0 is None else x0
    X = x0[None] + h * fe.gll_points(k)[ni]
    v = fun(X)
    return v[:, :dim].T[None], v[:, dim][None]


@pytest.mark.parametrize("dim,k", [(2, 2), (3, 1), (3, 2)])
def test_stab_ns_reduces_to_equal_order_stokes(dim, k):
    h = 0.25
    ub, pb = _frozen_loc(dim, k, h, forms.taylor_green(dim))
    K = forms.stabilized_ns(dim, k, [h], 0 * ub, 0 * pb, 0.3, np.inf, terms=0)[0]
    S = forms.stokes_taylor_hood(dim, k, 0.3, [h], div_sign=1.0, kp=k)[0]
    assert np.allclose(K, S, atol=1e-14)


@pytest.mark.parametrize("dim,k", [(2, 2), (3, 2)])
def test_pspg_block_is_tau_times_pressure_laplacian(dim, k):
    h, nu = 0.125, 0.02
    ub, pb = _frozen_loc(dim, k, h, forms.taylor_green(dim))
    K = forms.stabilized_ns(dim, k, [h], 0 * ub, 0 * pb, nu, np.inf)[0]
    nb = (k + 1) ** dim
    tau = h ** 2 / (12 * nu)                     # closed form of the formula for u = 0, dt = inf
    L = forms.vector_laplacian(dim, k, 1.0, [h])[0][:nb, :nb]
    assert np.allclose(K[dim * nb:, dim * nb:], tau * L, rtol=1e-12, atol=1e-15)


def test_mass_and_newton_terms_in_isolation():
    dim, k, h, dt = 3, 2, 0.25, 0.01
    nb = (k + 1) ** dim
    M = forms.scalar_mass(dim, k, k + 1, [h])[0]
    ub, pb = _frozen_loc(dim, k, h, forms.taylor_green(dim))
    base = forms.stabilized_ns(dim, k, [h], ub, pb, 0.1, dt, terms=0)[0]
    Km = forms.stabilized_ns(dim, k, [h], ub, pb, 0.1, dt, terms=forms.TERM_MASS)[0] - base
    for i in range(dim):
        assert np.allclose(Km[i * nb:(i + 1) * nb, i * nb:(i + 1) * nb], 1.5 / dt * M, rtol=1e-13, atol=1e-16)
    # Newton term with a linear frozen field (exactly interpolated): grad ub constant
    G = np.array([[0.3, -1.0, 0.2], [0.5, 0.1, 0.0], [0.0, 0.7, -0.4]])
    lin = lambda x: np.concatenate([x @ G.T, np.zeros((len(x), 1))], axis=1)
    ub, pb = _frozen_loc(dim, k, h, lin, x0=np.array([0.25, 0.5, 0.0]))
    base = forms.stabilized_ns(dim, k, [h], ub, pb, 0.1, dt, terms=0)[0]
    Kn = forms.stabilized_ns(dim, k, [h], ub, pb, 0.1, dt, terms=forms.TERM_NEWTON)[0] - base
    for i in range(dim):
        for j in range(dim):
            assert np.allclose(Kn[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb], G[i, j] * M, atol=1e-14)


def test_convection_is_skew_on_interior_dofs():
    f = mesh.uniform(2, 4)
    const = lambda x: np.concatenate([np.tile([0.7, -0.4], (len(x), 1)), np.zeros((len(x), 1))], axis=1)
    p0 = assemble.Problem(f, "stab_ns", 2, nu=0.1, dt=np.inf, terms=0, frozen=const)
    p1 = assemble.Problem(f, "stab_ns", 2, nu=0.1, dt=np.inf, terms=forms.TERM_CONV, frozen=const)
    C = (p1.assemble_K() - p0.assemble_K()).toarray()
    free = p0.dofs.free.copy()
    free[p0.dofs.offsets[1]:] = False           # velocity rows/cols only
    Cf = C[np.ix_(free, free)]
    assert np.abs(Cf + Cf.T).max() < 1e-13 and np.abs(Cf).max() > 1e-3


@pytest.mark.parametrize("newton", [False, True])
@pytest.mark.parametrize("dim", [2, 3])
def test_stab_ns_strong_consistency(dim, newton):
    """A polynomial, divergence-free (u, p) in Q_2 Q_2 is reproduced exactly: the
    operator applied to its interpolant equals the load assembled from the
    pointwise residual f = L(u, p) (Galerkin and stabilisation parts)."""
    nu, dt, k = 0.05, 0.1, 2
    n = 2
    f = mesh.uniform(dim, n)
    terms = forms.TERMS_ALL if newton else forms.TERMS_ALL & ~(forms.TERM_NEWTON | forms.TERM_SUPG_NEWTON)
    prob = assemble.Problem(f, "stab_ns", k, nu=nu, dt=dt, terms=terms)
    if dim == 2:
        ufun = lambda x: np.stack([x[:, 0] ** 2, -2 * x[:, 0] * x[:, 1]], axis=1)
        gradu = lambda x: np.stack([np.stack([2 * x[:, 0], 0 * x[:, 0]], 1),
                                    np.stack([-2 * x[:, 1], -2 * x[:, 0]], 1)], 1)
        lapu = lambda x: np.stack([2 + 0 * x[:, 0], 0 * x[:, 0]], 1)
        pfun = lambda x: x[:, 0] * x[:, 1] - 0.25
        gradp = lambda x: np.stack([x[:, 1], x[:, 0]], 1)
    else:
        ufun = lambda x: np.stack([x[:, 1] ** 2 + x[:, 2], x[:, 2] ** 2 + x[:, 0], x[:, 0] ** 2 + x[:, 1]], 1)
        z = lambda x: 0 * x[:, 0]
        gradu = lambda x: np.stack([np.stack([z(x), 2 * x[:, 1], 1 + z(x)], 1),
                                    np.stack([1 + z(x), z(x), 2 * x[:, 2]], 1),
                                    np.stack([2 * x[:, 0], 1 + z(x), z(x)], 1)], 1)
        lapu = lambda x: np.full((len(x), 3), 2.0)
        pfun = lambda x: x[:, 0] * x[:, 1] * x[:, 2] - 0.125
        gradp = lambda x: np.stack([x[:, 1] * x[:, 2], x[:, 0] * x[:, 2], x[:, 0] * x[:, 1]], 1)
    cm = 1.5 / dt
    # frozen state at the Gauss points from the oracle's own interpolant (same on both sides)
    t = forms.CellTables(dim, k, k + 1, f.h())
    ns = prob.dofs.nodesets[0]
    ub_loc = np.transpose(prob.ub_nodes[ns.cell_nodes], (0, 2, 1))
    pb_loc = prob.pb_nodes[ns.cell_nodes]
    U, G, LU, GP = forms.frozen_at_qp(t, ub_loc, pb_loc)
    xq = f.origin()[:, None, :] + f.h()[:, None, None] * t.xq[None]
    X = xq.reshape(-1, dim)
    sh = xq.shape[:2]
    uq, gq, lq, gpq = (ufun(X).reshape(*sh, dim), gradu(X).reshape(*sh, dim, dim),
                       lapu(X).reshape(*sh, dim), gradp(X).reshape(*sh, dim))
    # pointwise linearised residual of the exact polynomial solution
    fq = cm * uq + np.einsum("cqj,cqij->cqi", U, gq) + gpq - nu * lq
    if newton:
        fq += np.einsum("cqj,cqij->cqi", uq, G)
    tau = forms.tau_formula(np.linalg.norm(U, axis=2), f.h()[:, None], nu, dt)
    Rbar = np.einsum("cqj,cqij->cqi", U, G) + GP - nu * LU
    W = t.JxW
    # load: (f, v) + tau (f, ub.grad v) [+ tau (Rbar, u.grad v)] + tau (f, grad q)
    Ug = np.einsum("cqd,cqbd->cqb", U, t.grad)
    nb = t.nb
    loc = np.zeros((f.n_cells, (dim + 1) * nb))
    for i in range(dim):
        loc[:, i * nb:(i + 1) * nb] = (np.einsum("cq,cq,qb->cb", W, fq[..., i], t.phi)
                                       + np.einsum("cq,cq,cqb->cb", W * tau, fq[..., i], Ug))
        if newton:
            loc[:, i * nb:(i + 1) * nb] += np.einsum("cq,cq,cqj,cqbj->cb", W * tau, Rbar[..., i], uq, t.grad)
    loc[:, dim * nb:] = np.einsum("cq,cqi,cqbi->cb", W * tau, fq, t.grad)
    F = np.zeros(prob.dofs.n_dofs)
    np.add.at(F, prob.cell_dofs, loc)
    x = prob.dofs.interpolate(lambda X: np.concatenate([ufun(X), pfun(X)[:, None]], axis=1))
    K = prob.assemble_K()
    free = prob.dofs.free
    r = (K @ x - F)[free]
    assert np.abs(r).max() < 1e-11 * max(1.0, np.abs(F).max()), np.abs(r).max()


# ---- the stabilisation parameter (reading of Section 5's delta_1: Tezduyar's tau) -------------------
# Each limit is the published asymptotic behaviour of the parameter (a time-step, an advective and a
# viscous time scale); the hand values fix how the three combine.  None of the expected numbers is
# computed by the oracle.
TAU_LIMITS = [
    # (|u|, h, nu, dt, expected tau, which term dominates)
    (0.0, 1.0, 1e-12, 1e-6, 0.5e-6, "transient: tau -> dt / 2"),
    (1e6, 1.0, 1e-12, np.inf, 0.5e-6, "advective: tau -> h / (2 |u|)"),
    (0.0, 0.1, 1.0, np.inf, 0.01 / 12.0, "viscous: tau -> h^2 / (12 nu)"),
]
TAU_HAND = [
    # (|u|, h, nu, dt, sum of the three squares worked out by hand)
    (1.5, 1.0, 1.0 / 12.0, 0.5, 16.0 + 9.0 + 1.0),                # 4^2 + 3^2 + 9 (1/3)^2
    (3.0, 0.5, 0.25, 0.2, 100.0 + 144.0 + 144.0),                 # 10^2 + 12^2 + 9 * 4^2
    (0.0, 0.125, 0.02, 0.01, 40000.0 + 0.0 + 235.9296),           # 200^2 + 0 + 9 * 5.12^2
    (2.0, 0.25, 1e-3, 0.05, 1600.0 + 256.0 + 0.036864),           # 40^2 + 16^2 + 9 * 0.064^2
]


def _check_tau(tau_fn):
    for u, h, nu, dt, expect, what in TAU_LIMITS:
        got = tau_fn(u, h, nu, dt)
        assert abs(got - expect) <= 1e-9 * expect, (what, got, expect)
    for u, h, nu, dt, s in TAU_HAND:
        got = tau_fn(u, h, nu, dt)
        assert abs(got - 1.0 / np.sqrt(s)) <= 1e-13 / np.sqrt(s), (u, h, nu, dt, got)


def test_tau_limits_and_hand_values():
    _check_tau(forms.tau_formula)


def test_tau_pin_catches_a_wrong_factor():
    """The pin fails for the plausible misreadings of each term (planted in copies of the formula,
    on the CPU): 1/dt instead of 2/dt, |u|/h instead of 2|u|/h, a missing 9, the sum of the
    inverses instead of the inverse root of the sum of squares."""
    inf = np.isfinite
    wrong = [
        lambda u, h, nu, dt: 1 / np.sqrt((1 / dt if inf(dt) else 0) ** 2 + (2 * u / h) ** 2 + 9 * (4 * nu / h ** 2) ** 2),
        lambda u, h, nu, dt: 1 / np.sqrt((2 / dt if inf(dt) else 0) ** 2 + (u / h) ** 2 + 9 * (4 * nu / h ** 2) ** 2),
        lambda u, h, nu, dt: 1 / np.sqrt((2 / dt if inf(dt) else 0) ** 2 + (2 * u / h) ** 2 + (4 * nu / h ** 2) ** 2),
        lambda u, h, nu, dt: 1 / ((2 / dt if inf(dt) else 0) + 2 * u / h + 12 * nu / h ** 2),
    ]
    for fn in wrong:
        with pytest.raises(AssertionError):
            _check_tau(fn)
