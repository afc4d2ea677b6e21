"""Local-smoothing (LS) multigrid on locally refined meshes (Section 2).

Oracle (test infrastructure only), float64, assembled sparse matrices.

Section 2 contrasts two ways of building the levels of a geometric hierarchy
on a locally refined mesh.  Global coarsening smooths on the whole domain and
resolves hanging nodes on every level (``solvers.hierarchy``).  Local
smoothing takes as level l the cells of refinement level l only -- the part
Omega_l of the domain refined at least l times -- smooths there with
homogeneous Dirichlet conditions on the internal boundary of Omega_l (the
refinement edge), and goes on to the next coarser part.

Written here as what that method is: a multiplicative subspace correction
over the level spaces
    V_l = { level-l finite-element functions on Omega_l that vanish on the
            refinement edge and on the Dirichlet boundary },   l = L, ..., 1,
and V_0, the finite-element space of the unrefined base mesh.  Every V_l lies
in the fine (hanging-node conforming) space V; ``level_prolongation`` gives
its embedding P_l (nodal interpolation at the free fine DoFs).  One cycle:
  pre-smoothing  l = L .. 1 : x_l = S_l(P_l^T r) from zero,  x += P_l x_l,
  level 0                   : one global-coarsening V-cycle of the base
                              hierarchy on P_0^T r,           x += P_0 x_0,
  post-smoothing l = 1 .. L : d_l = S_l(P_l^T r) from zero,  x += P_l d_l,
with r = b - A x updated after every correction and S_l the level smoother
(Chebyshev or relaxation around point Jacobi, ``solvers``) on
A_l = P_l^T A P_l, extended by identity rows on the level's edge and boundary
nodes.  The constrained (Dirichlet and hanging) rows of A are identity rows
and lie outside every level space: the cycle inverts them exactly, x = b on
those rows.  For the vector Laplacian the Galerkin product equals the operator
assembled on the level mesh with Dirichlet conditions on the refinement edge
(same bilinear form, exact quadrature); the tests pin that.

Readings: the paper does not say which levels carry the polynomial
coarsening.  Here the refined levels keep the fine degree k and the base
level is the first level of the base mesh's own global hierarchy (which
coarsens p and h in the order of Section 3 or 5).  LS levels exist for the
vector Laplacian (the Stokes A block) only: on the stabilised operator the
level operators would not be Galerkin products (tau depends on the cell size).
"""
import numpy as np
import scipy.sparse as sp

from . import assemble, fe, mesh, solvers, transfer


def level_cells(forest, l):
    """(m, dim) integer coordinates of the cells of refinement level l: the active cells of
    level l and the level-l ancestors of finer active cells."""
    c = forest.cells
    sel = c[:, 0] >= l
    crd = c[sel, 1:] >> (c[sel, 0] - l)[:, None]
    return np.unique(crd, axis=0)


class LevelSpace:
    """Q_k nodes of the level-l cells, numbered by their integer node index k * cell + slot.

    Attributes: ``cells`` (m, dim), ``idx`` (Nn, dim) node indices, ``x`` (Nn, dim) support
    points, ``cell_nodes`` (m, (k+1)^dim), ``edge`` (node on the refinement edge), ``boundary``
    (node on the domain boundary), ``interior`` (neither)."""

    def __init__(self, forest, l, k):
        dim = forest.dim
        self.dim, self.k, self.l = dim, k, l
        self.N = forest.n * 2 ** l                       # level-l cells per direction
        self.cells = level_cells(forest, l)
        loc = fe.tensor_index(dim, k + 1)
        keys = (k * self.cells[:, None, :] + loc[None, :, :]).reshape(-1, dim)
        uniq, inv = np.unique(keys, axis=0, return_inverse=True)
        self.idx = uniq
        self.cell_nodes = inv.reshape(len(self.cells), -1)
        self.n_nodes = len(uniq)
        xi = fe.gll_points(k)
        cell, slot = uniq // k, uniq % k
        top = cell == self.N                             # the last node of a line: slot k of N-1
        cell = np.where(top, self.N - 1, cell)
        slot = np.where(top, k, slot)
        self.x = (cell + xi[slot]) / self.N
        self.boundary = ((uniq == 0) | (uniq == k * self.N)).any(axis=1)
        # refinement edge: some level-l cell inside the domain whose closure holds the node is
        # not a cell of this level
        present = {tuple(c) for c in self.cells.tolist()}
        self.edge = np.zeros(self.n_nodes, dtype=bool)
        for g in range(self.n_nodes):
            choices = []
            for d in range(dim):
                i = int(uniq[g, d])
                choices.append((i // k - 1, i // k) if i % k == 0 else (i // k,))
            for cand in np.array(np.meshgrid(*choices, indexing="ij")).reshape(dim, -1).T:
                if ((cand >= 0) & (cand < self.N)).all() and tuple(cand.tolist()) not in present:
                    self.edge[g] = True
                    break
        self.interior = ~(self.edge | self.boundary)
        self._cell_of = {tuple(c): i for i, c in enumerate(self.cells.tolist())}

    def locate(self, x):
        """Id of a level cell whose closed box contains each point (npts, dim), -1 if none."""
        t = x * self.N
        lo = np.floor(t - 1e-9).astype(np.int64)
        hi = np.floor(t + 1e-9).astype(np.int64)
        out = -np.ones(len(x), dtype=np.int64)
        for sel in fe.tensor_index(self.dim, 2):
            cand = np.where(sel[None, :] == 0, lo, hi)
            for i in np.nonzero(out < 0)[0]:
                out[i] = self._cell_of.get(tuple(cand[i].tolist()), -1)
        return out


def level_prolongation(problem, space):
    """P_l: level vector (ncomp * Nn, component-major) -> fine DoF vector.  Column (c, g) is the
    level basis function of interior node g in component c, evaluated at every free fine DoF of
    component c (zero at constrained fine DoFs and for non-interior level nodes)."""
    d = problem.dofs
    ncomp, k, _ = d.fields[0]
    ns = d.nodesets[0]
    cells = space.locate(ns.x)
    inside = cells >= 0
    xi = ns.x[inside] * space.N - space.cells[cells[inside]]
    phi = fe.eval_basis_at(space.dim, k, np.clip(xi, 0.0, 1.0))    # (n_in, nb)
    lnodes = space.cell_nodes[cells[inside]]                          # (n_in, nb)
    keep = (np.abs(phi) > 1e-14) & space.interior[lnodes]
    fine_nodes = np.nonzero(inside)[0]
    rows, cols, vals = [], [], []
    for c in range(ncomp):
        rf = d.dof(0, c, fine_nodes)
        rows.append(np.repeat(rf[:, None], phi.shape[1], axis=1)[keep])
        cols.append((c * space.n_nodes + lnodes)[keep])
        vals.append(phi[keep])
    P = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(d.n_dofs, ncomp * space.n_nodes))
    P = sp.diags(d.free.astype(float)) @ P
    P = P.tocsr()
    P.eliminate_zeros()
    return P


class LsLevel:
    def __init__(self, problem, A, l):
        self.space = LevelSpace(problem.forest, l, problem.k)
        self.P = level_prolongation(problem, self.space)
        ncomp = problem.dofs.fields[0][0]
        inner = np.tile(self.space.interior, ncomp)
        self.A = (self.P.T @ A @ self.P + sp.diags((~inner).astype(float))).tocsr()
        self.dinv = 1.0 / self.A.diagonal()
        self.lmax = None


class LocalSmoothing:
    """The LS V-cycle of a 'stokes_a' problem on a locally refined forest.

    ``lmax_ls[l - 1]`` is the smoother bound of level l (l = 1..L); the base level's
    global-coarsening hierarchy gets ``lmax_base`` (one per level but its coarsest)."""

    def __init__(self, problem, lmax_ls, lmax_base, smoother=("chebyshev", 5), stop_n=2, order="p_then_h"):
        assert problem.kind == "stokes_a"
        self.problem = problem
        self.A = problem.assemble()
        forest = problem.forest
        self.L = forest.max_level
        self.levels = [LsLevel(problem, self.A, l) for l in range(1, self.L + 1)]
        for lv, lm in zip(self.levels, lmax_ls):
            lv.lmax = lm
        self.smoother = smoother
        base = mesh.uniform(forest.dim, forest.n)
        self.base_levels = solvers.hierarchy(base, "stokes_a", problem.k, order=order, stop_n=stop_n,
                                             nu=problem.nu)
        self.base = solvers.VCycle(self.base_levels, lmax_base, smoother)
        self.P0 = transfer.prolongation(self.base_levels[0].problem, problem)

    def _smooth(self, lv, b):
        kind, deg = self.smoother
        x0 = np.zeros_like(b)
        if kind == "chebyshev":
            return solvers.chebyshev(lv.A, lv.dinv, b, x0, deg, lv.lmax, x_is_zero=True)
        return solvers.jacobi_relaxation(lv.A, lv.dinv, b, x0, deg, lv.lmax)

    def __call__(self, b):
        A = self.A
        x = np.zeros_like(b)
        r = b.copy()
        for lv in reversed(self.levels):                  # pre-smoothing, finest part first
            x = x + lv.P @ self._smooth(lv, lv.P.T @ r)
            r = b - A @ x
        x = x + self.P0 @ self.base(self.P0.T @ r)       # the base mesh's V-cycle
        r = b - A @ x
        for lv in self.levels:                            # post-smoothing, coarsest part first
            x = x + lv.P @ self._smooth(lv, lv.P.T @ r)
            r = b - A @ x
        con = self.problem.dofs.constrained               # identity rows of A
        x[con] = b[con]
        return x


# -- the level recursion with rediscretised level operators ---------------------------------------
class _RLevel:
    """Level l >= 1 in the numbering of the uniform level-l mesh: its operator assembled on the
    level-l cells only, with the domain boundary (velocity) constrained ('full') and with the
    refinement edge constrained too, every component ('op'); identity rows outside Omega_l."""

    def __init__(self, forest, l, kind, k, params):
        dim = forest.dim
        self.U = assemble.Problem(mesh.uniform(dim, forest.n * 2 ** l), kind, k, **params)
        U = self.U
        sp_ = LevelSpace(forest, l, k)
        nsU = U.dofs.nodesets[0]
        key = {tuple(np.rint(x * 2 ** 30).astype(np.int64)): g for g, x in enumerate(nsU.x)}
        inside = np.zeros(nsU.n_nodes, dtype=bool)
        edge = np.zeros(nsU.n_nodes, dtype=bool)
        for x, e in zip(sp_.x, sp_.edge):
            g = key[tuple(np.rint(x * 2 ** 30).astype(np.int64))]
            inside[g] = True
            edge[g] |= e
        present = {tuple(c) for c in sp_.cells.tolist()}
        cells = np.array([i for i, c in enumerate(U.forest.cells[:, 1:].tolist()) if tuple(c) in present])
        Ke = U.element_matrices(cells)
        cd = U.cell_dofs[cells]
        n = U.dofs.n_dofs
        K = sp.csr_matrix((Ke.ravel(), (np.repeat(cd[:, :, None], cd.shape[1], 2).ravel(),
                                        np.repeat(cd[:, None, :], cd.shape[1], 1).ravel())), shape=(n, n))
        d = U.dofs
        node_of = np.concatenate([np.arange(d.nodesets[f].n_nodes) for f, (nc, _, _) in enumerate(d.fields)
                                  for _ in range(nc)])
        outside = ~inside[node_of]
        self.inside = ~outside
        full_c = d.dirichlet | outside
        op_c = full_c | edge[node_of]

        def constrain(c):
            D = sp.diags((~c).astype(float))
            return (D @ K @ D + sp.diags(c.astype(float))).tocsr()

        self.full, self.op = constrain(full_c), constrain(op_c)
        self.op_c, self.full_c = op_c, full_c
        self.dinv = 1.0 / self.op.diagonal()
        self.lmax = None
        self.P = None                                 # from the next coarser uniform level


class LocalSmoothingLevels:
    """The local-smoothing cycle as a level recursion with rediscretised level operators (the form a
    stabilised operator needs: tau depends on the cell size, so level operators are not Galerkin
    products).  For 'stokes_a' it equals ``LocalSmoothing`` (pinned).  Each free fine DoF is owned by
    the coarsest level among the active cells holding it; its defect is copied there, and the result
    is copied back from there; constrained fine rows return b.  Level 0 is the base mesh's
    global-coarsening hierarchy (``solvers.hierarchy``, the kind's default order)."""

    def __init__(self, problem, lmax_ls, lmax_base, smoother=("chebyshev", 5), stop_n=2, **params):
        from . import transfer
        self.problem = problem
        f, kind, k = problem.forest, problem.kind, problem.k
        self.L = f.max_level
        self.levels = [_RLevel(f, l, kind, k, params) for l in range(1, self.L + 1)]
        for lv, lm in zip(self.levels, lmax_ls):
            lv.lmax = lm
        self.smoother = smoother
        self.base_levels = solvers.hierarchy(mesh.uniform(f.dim, f.n), kind, k, stop_n=stop_n, **params)
        self.base = solvers.VCycle(self.base_levels, lmax_base, smoother)
        uni = [self.base_levels[0].problem] + [lv.U for lv in self.levels]
        for l, lv in enumerate(self.levels):
            lv.P = transfer.prolongation(uni[l], uni[l + 1])
        # owners: fine free DoF -> (level, DoF of that level's uniform numbering)
        d = problem.dofs
        xs, fid = d.support_points()
        ns = d.nodesets[0]
        owner_node = ns.owner_level
        node_of = np.concatenate([np.arange(d.nodesets[f_].n_nodes) for f_, (nc, _, _) in enumerate(d.fields)
                                  for _ in range(nc)])
        self.copies = []
        for l in range(self.L + 1):
            Ud = uni[l].dofs
            xu, fu = Ud.support_points()
            key = {(tuple(np.rint(x * 2 ** 30).astype(np.int64)), c): i for i, (x, c) in enumerate(zip(xu, fu))}
            pairs = [(g, key[(tuple(np.rint(xs[g] * 2 ** 30).astype(np.int64)), fid[g])])
                     for g in np.nonzero(d.free)[0] if owner_node[node_of[g]] == l]
            self.copies.append(np.array(pairs, dtype=np.int64).reshape(-1, 2))

    def _smooth(self, lv, b):
        kind, deg = self.smoother
        x0 = np.zeros_like(b)
        if kind == "chebyshev":
            return solvers.chebyshev(lv.op, lv.dinv, b, x0, deg, lv.lmax, x_is_zero=True)
        return solvers.jacobi_relaxation(lv.op, lv.dinv, b, x0, deg, lv.lmax)

    def __call__(self, b):
        uni_n = [self.base_levels[0].A.shape[0]] + [lv.U.dofs.n_dofs for lv in self.levels]
        B = []
        for l in range(self.L + 1):
            v = np.zeros(uni_n[l])
            c = self.copies[l]
            v[c[:, 1]] = b[c[:, 0]]
            B.append(v)
        X = [None] * (self.L + 1)
        for l in range(self.L, 0, -1):                  # down: smooth, residual with edge rows, restrict
            lv = self.levels[l - 1]
            z = B[l].copy()
            z[lv.op_c] = 0.0
            X[l] = self._smooth(lv, z)
            r = (B[l] - lv.full @ X[l]) * lv.inside
            cst = lv.P.T @ r
            below_c = self.levels[l - 2].full_c if l >= 2 else self.base_levels[0].problem.dofs.constrained
            cst[below_c] = 0.0
            B[l - 1] = B[l - 1] + cst
        X[0] = self.base(B[0])
        for l in range(1, self.L + 1):                  # up: prolongate, residual, smooth the correction
            lv = self.levels[l - 1]
            X[l] = X[l] + (lv.P @ X[l - 1]) * lv.inside
            r = B[l] - lv.full @ X[l]
            r[lv.op_c] = 0.0
            X[l] = X[l] + self._smooth(lv, r)
        x = np.zeros_like(b)
        for l in range(self.L + 1):
            c = self.copies[l]
            x[c[:, 0]] = X[l][c[:, 1]]
        con = self.problem.dofs.constrained
        x[con] = b[con]
        return x
