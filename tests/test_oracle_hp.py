"""Pins of the oracle's hp-adaptive spaces and hp-multigrid (Section 3).

* With one degree everywhere the hp space, its constraints and its operator are the oracle's
  standard ones.
* Conformity, checked independently of the constraint construction: for random free values, the
  traces of the two cells on every shared face piece agree (h- and p-interfaces, 2D and 3D).
* Dimension: the number of free DoFs equals the dimension of the conforming space computed by brute
  force (rank of the continuity and boundary conditions on the broken space).
* The interpolant of a polynomial of the lowest degree present lies in the space, and its energy is
  the closed-form nu * int |grad u|^2.
* hp transfers are exact for polynomials of the coarse space.
* hp-multigrid (degrees lowered one by one, then h) as an FGMRES preconditioner converges.
* The configuration the construction does not cover is rejected.
"""
import numpy as np
import pytest

from oracle import assemble, fe, hp, mesh, solvers


def _ball(dim, n, levels):
    return mesh.refine_ball(mesh.uniform(dim, n), (0.3, 0.35, 0.4), 0.3, levels)


def _degrees(f, base, vary=True):
    """base + refinement level (+ parity of the root cell's x index): finer cells never have a lower
    degree than a coarser neighbour, and same-level neighbours may differ by one."""
    lev = f.cells[:, 0]
    root_x = f.cells[:, 1] >> lev
    return base + lev + ((root_x % 2) if vary else 0)


def _face_pieces(f):
    """(A, B, points) for every pair of cells sharing a piece of a face: GLL points of degree 5 on
    the piece (enough to identify traces of degree <= 5)."""
    N, cell_at = f.lattice()
    dim = f.dim
    h = f.h()
    org = f.origin()
    out = []
    x5 = fe.gll_points(5)
    for a in range(f.n_cells):
        for d in range(dim):
            for side in (0, 1):
                plane = org[a, d] + side * h[a]
                if plane <= 1e-12 or plane >= 1 - 1e-12:
                    continue
                # lattice cells just across the face
                lo = np.rint(org[a] * N).astype(int)
                hi = np.rint((org[a] + h[a]) * N).astype(int)
                sl = [slice(lo[j], hi[j]) for j in range(dim)]
                q = int(round(plane * N))
                sl[d] = slice(q, q + 1) if side else slice(q - 1, q)
                for b in np.unique(cell_at[tuple(sl)]):
                    # shared piece: intersection of the two face boxes
                    lo_s = np.maximum(org[a], org[b])
                    hi_s = np.minimum(org[a] + h[a], org[b] + h[b])
                    tang = [j for j in range(dim) if j != d]
                    grids = np.meshgrid(*[lo_s[j] + (hi_s[j] - lo_s[j]) * x5 for j in tang], indexing="ij")
                    pts = np.zeros((grids[0].size, dim))
                    for j, g in zip(tang, grids):
                        pts[:, j] = g.ravel()
                    pts[:, d] = plane
                    out.append((a, int(b), pts))
    return out


def test_uniform_degree_is_the_standard_space():
    for dim, n, levels, k in [(2, 3, 2, 2), (2, 2, 1, 3), (3, 2, 1, 2)]:
        f = _ball(dim, n, levels)
        H = hp.HpProblem(f, np.full(f.n_cells, k), "stokes_a", nu=0.6)
        S = assemble.Problem(f, "stokes_a", k, nu=0.6)
        xh, fh = H.dofs.support_points()
        xs, fs = S.dofs.support_points()
        key = {(tuple(np.rint(x * 2 ** 30).astype(np.int64)), c): i for i, (x, c) in enumerate(zip(xs, fs))}
        perm = np.array([key[(tuple(np.rint(x * 2 ** 30).astype(np.int64)), c)] for x, c in zip(xh, fh)])
        assert len(perm) == len(xs) and len(set(perm.tolist())) == len(perm)
        assert np.array_equal(H.dofs.constrained, S.dofs.constrained[perm])
        Ah, As = H.assemble(), S.assemble()[perm][:, perm]
        assert abs(Ah - As).max() <= 1e-13 * abs(As).max()


@pytest.mark.parametrize("dim,n,levels,base", [(2, 3, 2, 1), (2, 4, 1, 2), (3, 2, 1, 1), (3, 3, 1, 2)])
def test_traces_agree_on_every_interface(dim, n, levels, base):
    f = _ball(dim, n, levels)
    deg = _degrees(f, base)
    assert len(np.unique(deg)) >= 2
    P = hp.HpProblem(f, deg, "stokes_a")
    d = P.dofs
    assert d.hanging.any()
    rng = np.random.default_rng(1)
    x = d.distribute(rng.uniform(-1, 1, d.n_dofs))
    pieces = _face_pieces(f)
    p_faces = sum(1 for a, b, _ in pieces if deg[a] != deg[b] and f.cells[a, 0] == f.cells[b, 0])
    h_faces = sum(1 for a, b, _ in pieces if f.cells[a, 0] != f.cells[b, 0])
    assert p_faces > 0 and h_faces > 0
    worst = 0.0
    for a, b, pts in pieces:
        for comp in range(dim):
            ua = P.evaluate_in(x, pts, np.full(len(pts), a), 0, comp)
            ub = P.evaluate_in(x, pts, np.full(len(pts), b), 0, comp)
            worst = max(worst, np.abs(ua - ub).max())
    assert worst <= 1e-12


@pytest.mark.parametrize("dim,n,levels,base", [(2, 2, 1, 1), (2, 3, 1, 2), (3, 2, 1, 1)])
def test_dimension_equals_brute_force_rank(dim, n, levels, base):
    f = _ball(dim, n, levels)
    deg = _degrees(f, base)
    ns = hp.HpNodeSet(f, deg)
    free = ~ns.boundary
    free[list(ns.hanging)] = False
    # broken space: every cell's own nodal values; continuity on every shared face piece and zero
    # boundary traces as linear conditions
    offs = np.cumsum([0] + [(int(k) + 1) ** dim for k in deg])
    rows = []
    h, org = f.h(), f.origin()

    def basis(c, pts):
        xi = np.clip((pts - org[c]) / h[c], 0.0, 1.0)
        return fe.eval_basis_at(dim, int(deg[c]), xi)

    for a, b, pts in _face_pieces(f):
        G = np.zeros((len(pts), offs[-1]))
        G[:, offs[a]:offs[a + 1]] = basis(a, pts)
        G[:, offs[b]:offs[b + 1]] -= basis(b, pts)
        rows.append(G)
    for c in range(f.n_cells):                       # boundary nodes of every cell vanish
        loc = fe.tensor_index(dim, int(deg[c]) + 1)
        on = ((loc == 0) & (org[c] <= 1e-12)[None]) | ((loc == deg[c]) & (org[c] + h[c] >= 1 - 1e-12)[None])
        for i in np.nonzero(on.any(axis=1))[0]:
            r = np.zeros((1, offs[-1]))
            r[0, offs[c] + i] = 1.0
            rows.append(r)
    G = np.concatenate(rows)
    dim_space = offs[-1] - np.linalg.matrix_rank(G, tol=1e-9)
    assert dim_space == int(free.sum())


@pytest.mark.parametrize("dim,n,levels", [(2, 3, 1), (3, 2, 1)])
def test_polynomial_energy(dim, n, levels):
    f = _ball(dim, n, levels)
    deg = _degrees(f, 2)                             # lowest degree 2: x(1-x) y(1-y) ... is in the space
    nu = 0.7
    P = hp.HpProblem(f, deg, "stokes_a", nu=nu)

    def u(x):
        phi = np.prod(x * (1 - x), axis=1)
        return np.stack([(c + 1) * phi for c in range(dim)], axis=1)

    xv = P.dofs.interpolate(u)
    assert np.abs(P.dofs.distribute(xv) - xv).max() <= 1e-14
    energy = xv @ (P.assemble_K() @ xv)              # = x_free^T (C^T K C) x_free
    free = P.dofs.free_ids
    A = P.assemble()
    assert abs(xv[free] @ (A[free][:, free] @ xv[free]) - energy) <= 1e-12 * energy
    one_d = {2: 1.0 / 90.0 * 2, 3: 3 * (1.0 / 3.0) * (1.0 / 30.0) ** 2}[dim]   # int |grad phi|^2
    exact = nu * one_d * sum((c + 1) ** 2 for c in range(dim))
    assert abs(energy - exact) <= 1e-12 * exact


def test_transfers_exact_for_coarse_polynomials():
    f = _ball(2, 3, 1)
    deg = _degrees(f, 3)                             # degrees 3..5 -> 2..4 on the next level
    levels = hp.hierarchy(f, deg)
    fine, coarse = levels[0].problem, levels[1].problem
    assert (coarse.degrees == np.maximum(deg - 1, 1)).all()

    def u(x):
        phi = np.prod(x * (1 - x), axis=1)
        return np.stack([phi, -2.0 * phi], axis=1)     # degree 2: in the coarse space (degrees >= 2)

    got = levels[0].P @ coarse.dofs.interpolate(u)
    exp = fine.dofs.interpolate(u) * fine.dofs.free
    assert np.abs(got - exp).max() <= 1e-13
    # restriction is the transpose
    assert (levels[0].P.T - levels[0].P.T.tocsr()).nnz == 0


@pytest.mark.parametrize("dim,n,levels,base", [(2, 4, 1, 2), (3, 2, 1, 2)])
def test_hp_multigrid_preconditioner_converges(dim, n, levels, base):
    f = _ball(dim, n, levels)
    deg = _degrees(f, base)
    lv = hp.hierarchy(f, deg)
    assert lv[0].problem.degrees.max() >= 3 and lv[-1].problem.forest.n <= 2
    lmax = [1.2 * solvers.power_lmax(l.A, l.dinv, iterations=60) for l in lv[:-1]]
    V = solvers.VCycle(lv, lmax, ("chebyshev", 5))
    A = lv[0].A
    rng = np.random.default_rng(2)
    d = lv[0].problem.dofs
    xs = rng.uniform(-1, 1, d.n_dofs) * d.free
    x, its, res = solvers.fgmres(A, A @ xs, V, tol=1e-10)
    assert res <= 1e-10 and its <= 30
    assert np.abs(x - xs).max() <= 1e-7


def test_coarse_higher_degree_across_a_hanging_face_is_rejected():
    f = _ball(2, 3, 1)
    deg = 3 - f.cells[:, 0]                          # coarse cells 3, refined cells 2
    with pytest.raises(NotImplementedError):
        hp.HpNodeSet(f, deg)


def test_taylor_hood_uniform_degree_is_the_standard_operator():
    f = _ball(2, 3, 1)
    H = hp.HpProblem(f, np.full(f.n_cells, 3), "stokes", nu=0.8)
    S = assemble.Problem(f, "stokes", 3, nu=0.8)
    xh, fh = H.dofs.support_points()
    xs, fs = S.dofs.support_points()
    key = {(tuple(np.rint(x * 2 ** 30).astype(np.int64)), c): i for i, (x, c) in enumerate(zip(xs, fs))}
    perm = np.array([key[(tuple(np.rint(x * 2 ** 30).astype(np.int64)), c)] for x, c in zip(xh, fh)])
    assert np.array_equal(H.dofs.constrained, S.dofs.constrained[perm])
    Ah, As = H.assemble(), S.assemble()[perm][:, perm]
    assert abs(Ah - As).max() <= 1e-13 * abs(As).max()


def test_taylor_hood_hp_energy_closed_form():
    """u = (phi, 2 phi), phi = x(1-x)y(1-y), p = x - 1/2 on an hp mesh with velocity degrees 2..4
    (pressure 1..3): x^T A x = nu int |grad u|^2 - 2 int p div u = nu / 9 + 1/18."""
    f = _ball(2, 3, 1)
    deg = _degrees(f, 2)
    nu = 0.6
    P = hp.HpProblem(f, deg, "stokes", nu=nu)
    d = P.dofs

    def fields(x):
        phi = np.prod(x * (1 - x), axis=1)
        return np.stack([phi, 2 * phi, x[:, 0] - 0.5], axis=1)

    xv = d.interpolate(fields)
    assert np.abs(d.distribute(xv) - xv).max() <= 1e-14
    energy = xv @ (P.assemble_K() @ xv)
    exact = nu / 9.0 + 1.0 / 18.0
    assert abs(energy - exact) <= 1e-12 * exact
    # the pressure space is conforming across every interface too
    rng = np.random.default_rng(5)
    x = d.distribute(rng.uniform(-1, 1, d.n_dofs))
    worst = 0.0
    for a, b, pts in _face_pieces(f):
        pa = P.evaluate_in(x, pts, np.full(len(pts), a), 1, 0)
        pb = P.evaluate_in(x, pts, np.full(len(pts), b), 1, 0)
        worst = max(worst, np.abs(pa - pb).max())
    assert worst <= 1e-12


# -- the elimination rule: every configuration, including the combined h+p face ----------------------
@pytest.mark.parametrize("dim,n,levels,base", [(2, 3, 1, 1), (2, 3, 2, 1), (2, 2, 1, 2), (3, 2, 1, 1)])
def test_elimination_reproduces_the_dominance_rule(dim, n, levels, base):
    """Two independent constructions of the same space: local dominance and global elimination in
    the preference order (coarser, lower degree, node id) give the same slaves and the same weights
    on the free masters."""
    f = _ball(dim, n, levels)
    deg = _degrees(f, base)
    a = hp.HpNodeSet(f, deg)
    b = hp.HpNodeSet(f, deg, "elimination")
    # elimination keeps boundary nodes out of the unknowns (they are zero): compare interior slaves
    # and their free masters
    assert {g for g in a.hanging if not a.boundary[g]} == set(b.hanging)
    for g, masters in b.hanging.items():
        ref = {m: w for m, w in a.hanging[g] if not a.boundary[m]}
        got = dict(masters)
        assert not any(b.boundary[m] for m in got)
        assert max(abs(ref.get(m, 0.0) - got.get(m, 0.0)) for m in set(ref) | set(got)) <= 1e-12


def _combined(f, kind):
    lev = f.cells[:, 0]
    return {"3-2": 3 - lev, "4-2": 4 - 2 * lev}[kind]


@pytest.mark.parametrize("dim,n,levels,base", [(2, 3, 1, 1), (2, 3, 2, 2), (3, 2, 1, 1)])
def test_elimination_without_dirichlet_reproduces_every_constraint(dim, n, levels, base):
    """A field without boundary conditions (the Taylor--Hood pressure): every node is an unknown,
    and elimination gives every slave of the local rule, boundary ones included, with all weights."""
    f = _ball(dim, n, levels)
    deg = _degrees(f, base)
    a = hp.HpNodeSet(f, deg)
    b = hp.HpNodeSet(f, deg, "elimination", dirichlet=False)
    assert set(a.hanging) == set(b.hanging)
    if dim == 3:
        assert any(a.boundary[g] for g in a.hanging)     # the ball reaches the boundary there
    for g, masters in b.hanging.items():
        ref, got = dict(a.hanging[g]), dict(masters)     # the local rule may list zero weights
        assert max(abs(ref.get(m, 0.0) - got.get(m, 0.0)) for m in set(ref) | set(got)) <= 1e-12


@pytest.mark.parametrize("dim,n,kind", [(2, 3, "3-2"), (2, 4, "4-2"), (3, 2, "3-2")])
def test_combined_faces_conforming_with_the_right_dimension(dim, n, kind):
    """A hanging face whose coarse cell has the higher degree: traces agree on every interface and
    the number of free DoFs is the brute-force dimension of the conforming space."""
    f = _ball(dim, n, 1)
    deg = _combined(f, kind)
    with pytest.raises(NotImplementedError):
        hp.HpNodeSet(f, deg)
    P = hp.HpProblem(f, deg, "stokes_a", rule="elimination")
    d = P.dofs
    x = d.distribute(np.random.default_rng(2).uniform(-1, 1, d.n_dofs))
    worst = 0.0
    for a, b, pts in _face_pieces(f):
        ua = P.evaluate_in(x, pts, np.full(len(pts), a), 0, 0)
        ub = P.evaluate_in(x, pts, np.full(len(pts), b), 0, 0)
        worst = max(worst, np.abs(ua - ub).max())
    assert worst <= 1e-10
    if dim == 2:
        ns = d.nodesets[0]
        free = ~ns.boundary
        free[list(ns.hanging)] = False
        offs = np.cumsum([0] + [(int(k) + 1) ** dim for k in deg])
        h, org = f.h(), f.origin()
        rows = []
        for a, b, pts in _face_pieces(f):
            G = np.zeros((len(pts), offs[-1]))
            for c, sgn in ((a, 1.0), (b, -1.0)):
                G[:, offs[c]:offs[c + 1]] += sgn * fe.eval_basis_at(dim, int(deg[c]), np.clip((pts - org[c]) / h[c], 0, 1))
            rows.append(G)
        for c in range(f.n_cells):
            loc = fe.tensor_index(dim, int(deg[c]) + 1)
            on = ((loc == 0) & (org[c] <= 1e-12)[None]) | ((loc == deg[c]) & (org[c] + h[c] >= 1 - 1e-12)[None])
            for i in np.nonzero(on.any(axis=1))[0]:
                r = np.zeros((1, offs[-1]))
                r[0, offs[c] + i] = 1.0
                rows.append(r)
        G = np.concatenate(rows)
        assert offs[-1] - np.linalg.matrix_rank(G, tol=1e-9) == int(free.sum())


def test_combined_faces_energy_closed_form():
    f = _ball(2, 3, 1)
    nu = 0.7
    P = hp.HpProblem(f, _combined(f, "3-2"), "stokes_a", nu=nu, rule="elimination")

    def u(x):
        phi = np.prod(x * (1 - x), axis=1)
        return np.stack([phi, 2 * phi], axis=1)

    xv = P.dofs.interpolate(u)
    assert np.abs(P.dofs.distribute(xv) - xv).max() <= 1e-12
    energy = xv @ (P.assemble_K() @ xv)
    exact = nu * (1.0 / 45.0) * 5
    assert abs(energy - exact) <= 1e-11 * exact


def test_combined_faces_raise_the_jacobi_eigenvalue():
    """Section 3: eliminating the constrained unknowns of a combined h+p face leaves ill-conditioned
    relations between the remaining ones, visible in the eigenvalue estimate of the Jacobi-
    preconditioned A block (Fig. 3): lambda_max(D^-1 A) clearly above its value on the same mesh
    without combined faces.  The constraints being local, the rise does not grow with the mesh."""
    def lmax(f, deg, rule):
        P = hp.HpProblem(f, deg, "stokes_a", rule=rule)
        A = P.assemble()
        d = P.dofs.free
        Af = A[d][:, d].toarray()
        return np.abs(np.linalg.eigvals(Af / np.diag(Af)[:, None])).max()
    ratios = []
    for n in (3, 5):
        f = _ball(2, n, 1)
        plain = lmax(f, 2 + f.cells[:, 0], "dominance")
        combined = lmax(f, 3 - f.cells[:, 0], "elimination")
        assert plain < 2.0
        ratios.append(combined / plain)
    assert min(ratios) > 1.2 and abs(ratios[1] - ratios[0]) < 0.05


@pytest.mark.parametrize("dim,n,kind", [(2, 8, "3-2"), (2, 6, "4-2"), (3, 3, "3-2")])
def test_elimination_constraints_are_local(dim, n, kind):
    """Within equal (level, degree) the preference takes vertices before edge, then face interiors,
    so a slave's masters lie in the coarse cell of its face: bounded in number and in distance,
    whatever the size of the refined region."""
    f = _ball(dim, n, 1)
    ns = hp.HpNodeSet(f, _combined(f, kind), "elimination")
    h0 = 1.0 / n
    for g, masters in ns.hanging.items():
        assert len(masters) <= (4 if dim == 2 else 16)
        assert max(np.abs(ns.x[m] - ns.x[g]).max() for m, _ in masters) <= h0 + 1e-12
        assert max(abs(w) for _, w in masters) <= 2.0


def test_taylor_hood_on_combined_faces():
    """Velocity degree 3 on the coarse cells and 2 on the refined ones (pressure 2 and 1): both fields
    conforming across every interface, and the energy of u = (phi, 2 phi), p = x - 1/2 is
    nu / 9 + 1/18 as on any conforming space that holds them."""
    f = _ball(2, 3, 1)
    deg = _combined(f, "3-2")
    nu = 0.6
    P = hp.HpProblem(f, deg, "stokes", nu=nu, rule="elimination")
    d = P.dofs

    def fields(x):
        phi = np.prod(x * (1 - x), axis=1)
        return np.stack([phi, 2 * phi, x[:, 0] - 0.5], axis=1)

    xv = d.interpolate(fields)
    assert np.abs(d.distribute(xv) - xv).max() <= 1e-12
    energy = xv @ (P.assemble_K() @ xv)
    exact = nu / 9.0 + 1.0 / 18.0
    assert abs(energy - exact) <= 1e-11 * exact
    x = d.distribute(np.random.default_rng(6).uniform(-1, 1, d.n_dofs))
    worst = 0.0
    for a, b, pts in _face_pieces(f):
        for field in (0, 1):
            va = P.evaluate_in(x, pts, np.full(len(pts), a), field, 0)
            vb = P.evaluate_in(x, pts, np.full(len(pts), b), field, 0)
            worst = max(worst, np.abs(va - vb).max())
    assert worst <= 1e-10


def test_pressure_mass_uniform_degree_is_the_standard_one():
    f = _ball(2, 3, 1)
    H = hp.HpProblem(f, np.full(f.n_cells, 3), "pmass")
    S = assemble.Problem(f, "pmass", 2)
    xh, _ = H.dofs.support_points()
    xs, _ = S.dofs.support_points()
    key = {tuple(np.rint(x * 2 ** 30).astype(np.int64)): i for i, x in enumerate(xs)}
    perm = np.array([key[tuple(np.rint(x * 2 ** 30).astype(np.int64))] for x in xh])
    assert np.array_equal(H.dofs.constrained, S.dofs.constrained[perm])
    Ah, As = H.assemble(), S.assemble()[perm][:, perm]
    assert abs(Ah - As).max() <= 1e-15 * abs(As).max()


@pytest.mark.parametrize("rule,degf", [("dominance", lambda f: _degrees(f, 2)),
                                       ("elimination", lambda f: _combined(f, "3-2"))])
@pytest.mark.parametrize("dim", [2, 3])
def test_pressure_mass_closed_forms(dim, rule, degf):
    """Pressure degrees 1..3 (or combined faces): int 1 = 1 and int (x - 1/2)^2 = 1/12 over the
    unit square/cube, both functions being in every pressure space."""
    f = _ball(dim, 3 if dim == 2 else 2, 1)
    P = hp.HpProblem(f, degf(f), "pmass", rule=rule)
    M = P.assemble_K()
    one = P.dofs.interpolate(lambda x: np.ones((len(x), 1)))
    lin = P.dofs.interpolate(lambda x: (x[:, :1] - 0.5))
    for v in (one, lin):
        assert np.abs(P.dofs.distribute(v) - v).max() <= 1e-12
    assert abs(one @ M @ one - 1.0) <= 1e-13
    assert abs(lin @ M @ lin - 1.0 / 12.0) <= 1e-13


# -- Section 3's blended smoother: point Jacobi with additive Schwarz blocks on combined faces -------
def test_asm_without_combined_faces_is_point_jacobi():
    f = _ball(2, 4, 1)
    deg = 2 + f.cells[:, 0]
    P = hp.HpProblem(f, deg, "stokes_a")
    assert hp.combined_faces(P) == [] and hp.asm_blocks(P) == []
    lv = hp.hierarchy(f, deg, smoother="asm")
    assert all(isinstance(l.dinv, np.ndarray) for l in lv)


def test_asm_blocks_lie_on_combined_faces():
    f = _ball(2, 4, 1)
    deg = _combined(f, "3-2")
    P = hp.HpProblem(f, deg, "stokes_a", rule="elimination")
    faces = hp.combined_faces(P)
    blocks = hp.asm_blocks(P)
    assert len(faces) > 0 and len(blocks) == len(faces)
    d = P.dofs
    ns = d.nodesets[0]
    h, org = f.h(), f.origin()
    for (c, ax, side), B in zip(faces, blocks):
        assert f.cells[c, 0] == 0 and deg[c] == 3                  # the coarse, higher-degree side
        assert np.all(d.free[B])
        g = (B - d.offsets[0]) % ns.n_nodes
        assert np.all(np.abs(ns.x[g, ax] - (org[c, ax] + side * h[c])) <= 1e-12)
        # every component of every node of the block
        assert len(B) == 2 * len(np.unique(g))


def test_asm_preconditioner_is_spd_and_exact_on_one_block():
    f = _ball(2, 3, 1)
    P = hp.HpProblem(f, _combined(f, "3-2"), "stokes_a", rule="elimination")
    A = P.assemble()
    free = np.nonzero(P.dofs.free)[0]
    J = hp.JacobiASM(A, hp.asm_blocks(P))
    E = np.eye(A.shape[0])[:, free]
    Pm = np.stack([J(e) for e in E.T], axis=1)[free]
    assert np.abs(Pm - Pm.T).max() <= 1e-12 * np.abs(Pm).max()
    assert np.linalg.eigvalsh(0.5 * (Pm + Pm.T)).min() > 0
    whole = hp.JacobiASM(A, [free])
    Af = A[free][:, free].toarray()
    r = np.random.default_rng(0).uniform(-1, 1, A.shape[0])
    assert np.abs(whole(r)[free] - np.linalg.solve(Af, r[free])).max() <= 1e-12 * np.abs(r).max() * np.linalg.cond(Af)


@pytest.mark.parametrize("dim,n,kind", [(2, 8, "3-2"), (3, 2, "3-2")])
def test_hp_multigrid_with_jacobi_asm_converges(dim, n, kind):
    f = _ball(dim, n, 1)
    lv = hp.hierarchy(f, _combined(f, kind), rule="elimination", smoother="asm")
    assert any(isinstance(l.dinv, hp.JacobiASM) for l in lv)
    lmax = [1.2 * solvers.power_lmax(l.A, l.dinv, iterations=60) for l in lv[:-1]]
    V = solvers.VCycle(lv, lmax, ("chebyshev", 5))
    A = lv[0].A
    d = lv[0].problem.dofs
    xs = np.random.default_rng(2).uniform(-1, 1, d.n_dofs) * d.free
    x, its, res = solvers.fgmres(A, A @ xs, V, tol=1e-10)
    assert res <= 1e-10 and its <= 12
    assert np.abs(x - xs).max() <= 1e-7
