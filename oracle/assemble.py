"""Global assembly of the constrained operators.

Oracle (test infrastructure only).  For a DoF handler with constraint matrix
C (all DoFs <- free DoFs) and an assembled matrix K over all DoFs, the
operator is A = C^T K C on the free DoFs and the identity on every
constrained (Dirichlet or hanging) DoF; vmult(x) = A x ignores the
constrained entries of x on the free rows.  Restriction by the transpose of
the interpolation, Eq. 4, is what makes C^T appear on the test side.
"""
import numpy as np
import scipy.sparse as sp

from . import forms, mesh


class Problem:
    """One operator on one mesh: kind in {'stokes', 'stokes_a', 'stab_ns', 'pmass'}.

    Parameters mirror the paper's problem statement: viscosity nu, velocity
    degree k (Taylor--Hood pressure k-1; stabilised NS equal order k), time
    step dt and term flags for the stabilised operator, and the frozen state
    (Taylor--Green by default)."""

    def __init__(self, forest, kind, k, nu=1.0, dt=np.inf, terms=forms.TERMS_ALL,
                 div_sign=None, frozen=None, alpha=1.5):
        self.forest, self.kind, self.k, self.nu, self.dt, self.terms = forest, kind, k, nu, dt, terms
        self.alpha = alpha
        self.g_nodes = None
        dim = forest.dim
        self.dim = dim
        if kind == "stokes":
            fields = [(dim, k, True), (1, k - 1, False)]
            self.div_sign = -1.0 if div_sign is None else div_sign
        elif kind == "stokes_a":
            fields = [(dim, k, True)]
        elif kind == "stab_ns":
            fields = [(dim, k, True), (1, k, False)]
            self.div_sign = 1.0 if div_sign is None else div_sign
        elif kind == "pmass":
            fields = [(1, k, False)]
        else:
            raise ValueError(kind)
        self.dofs = mesh.DofHandler(forest, fields)
        self.cell_dofs = self.dofs.cell_dofs()
        if kind == "stab_ns":
            if frozen is None:
                frozen = forms.taylor_green(dim)
            # nodal interpolant of the frozen state on the Q_k nodes
            ns = self.dofs.nodesets[0]
            vals = frozen(ns.x)                                  # (Nn, dim+1)
            self.ub_nodes = vals[:, :dim]
            self.pb_nodes = vals[:, dim]

    # -- element matrices ------------------------------------------------------
    def element_matrices(self, cells):
        f = self.forest
        h = f.h()[cells]
        dim, k = self.dim, self.k
        if self.kind == "stokes":
            return forms.stokes_taylor_hood(dim, k, self.nu, h, self.div_sign)
        if self.kind == "stokes_a":
            return forms.vector_laplacian(dim, k, self.nu, h)
        if self.kind == "pmass":
            return forms.scalar_mass(dim, k, k + 1, h)
        ub, pb, gl = self._state_local(cells)
        return forms.stabilized_ns(dim, k, h, ub, pb, self.nu, self.dt, self.terms, self.div_sign,
                                   self.alpha, gl)

    # -- state of the stabilised NS problem (Section 5: Newton linearisation, BDF2) ----
    def _state_local(self, cells, nodes_u=None):
        ns = self.dofs.nodesets[0]
        cn = ns.cell_nodes[cells]                                # (nc, nb)
        ubn = self.ub_nodes if nodes_u is None else nodes_u
        ub = np.transpose(ubn[cn], (0, 2, 1))                    # (nc, dim, nb)
        pb = self.pb_nodes[cn]
        gl = None if self.g_nodes is None else np.transpose(self.g_nodes[cn], (0, 2, 1))
        return ub, pb, gl

    def _split(self, U):
        n = self.dofs.nodesets[0].n_nodes
        U = np.asarray(U, dtype=float)
        return U[: self.dim * n].reshape(self.dim, n).T.copy(), U[self.dim * n: (self.dim + 1) * n].copy()

    def state_vector(self):
        """The current state (u, p) as a vector in this problem's DoF order."""
        return np.concatenate([self.ub_nodes.T.ravel(), self.pb_nodes])

    def set_state(self, U, g=None):
        """State (u, p) from a DoF vector (constrained entries included as given); g: DoF vector
        whose velocity entries hold the explicit field g of ``forms.stabilized_ns_residual``."""
        self.ub_nodes, self.pb_nodes = self._split(U)
        self.g_nodes = None if g is None else self._split(g)[0]

    def set_dt(self, dt, alpha):
        self.dt, self.alpha = dt, alpha

    def residual(self, tau_state=None, chunk=512):
        """Nonlinear residual F(state) on the free rows (test functions C v), zero on constrained
        rows; tau_state: DoF vector whose velocity fixes tau (default: the state)."""
        d = self.dofs
        Fall = np.zeros(d.n_dofs)
        tu = None if tau_state is None else self._split(tau_state)[0]
        nc = self.forest.n_cells
        hh = self.forest.h()
        for s0 in range(0, nc, chunk):
            cells = np.arange(s0, min(nc, s0 + chunk))
            ub, pb, gl = self._state_local(cells)
            tl = None if tu is None else self._state_local(cells, tu)[0]
            Fe = forms.stabilized_ns_residual(self.dim, self.k, hh[cells], ub, pb, self.nu, self.dt, gl,
                                              self.div_sign, self.alpha, tl)
            np.add.at(Fall, self.cell_dofs[cells], Fe)
        F = np.zeros(d.n_dofs)
        F[d.free_ids] = d.C.T @ Fall
        return F

    # -- global matrices --------------------------------------------------------
    def assemble_K(self, chunk=512):
        """Unconstrained global matrix over all DoFs."""
        n = self.dofs.n_dofs
        rows, cols, vals = [], [], []
        nc = self.forest.n_cells
        for s in range(0, nc, chunk):
            cells = np.arange(s, min(nc, s + chunk))
            Ke = self.element_matrices(cells)
            cd = self.cell_dofs[cells]
            rows.append(np.repeat(cd[:, :, None], cd.shape[1], axis=2).ravel())
            cols.append(np.repeat(cd[:, None, :], cd.shape[1], axis=1).ravel())
            vals.append(Ke.ravel())
        K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
        K.sum_duplicates()
        return K

    def assemble(self):
        """The constrained operator A over all DoFs (identity rows on constrained DoFs)."""
        K = self.assemble_K()
        d = self.dofs
        C = d.C
        Af = (C.T @ K @ C).tocsr()                               # free x free
        P = sp.csr_matrix((np.ones(len(d.free_ids)), (d.free_ids, np.arange(len(d.free_ids)))),
                          shape=(d.n_dofs, len(d.free_ids)))
        I_c = sp.diags(d.constrained.astype(float))
        A = (P @ Af @ P.T + I_c).tocsr()
        A.sum_duplicates()
        return A

    def vmult(self, x, A=None):
        A = self.assemble() if A is None else A
        return A @ x

    # -- row sampling -------------------------------------------------------------
    def sampled_rows(self, rows, x):
        """(A x)[rows] without assembling A, from the cells touching each needed DoF.

        For a free DoF r: (C^T K C x)_r = y_r + sum over hanging DoFs h with master
        r of w_hr y_h, where y = K (C x); each y_i is summed over the cells that
        contain DoF i.  Constrained rows return x_r."""
        d = self.dofs
        xc = d.distribute(x)                                     # C x (constraints resolved)
        # masters -> list of (hanging dof, weight)
        Ccsc = d.C.tocsc()
        free_col = -np.ones(d.n_dofs, dtype=np.int64)
        free_col[d.free_ids] = np.arange(len(d.free_ids))
        # inverse map dof -> cells containing it
        cd = self.cell_dofs
        order = np.argsort(cd.ravel(), kind="stable")
        sorted_dofs = cd.ravel()[order]
        out = np.empty(len(rows))
        cache = {}
        for t, r in enumerate(rows):
            if d.constrained[r]:
                out[t] = x[r]
                continue
            col = free_col[r]
            lo, hi = Ccsc.indptr[col], Ccsc.indptr[col + 1]
            terms = list(zip(Ccsc.indices[lo:hi], Ccsc.data[lo:hi]))   # (dof i, weight) incl. (r, 1)
            acc = 0.0
            for i, w in terms:
                a, b = np.searchsorted(sorted_dofs, [i, i + 1])
                for flat in order[a:b]:
                    cell, loc = divmod(int(flat), cd.shape[1])
                    if cell not in cache:
                        cache[cell] = self.element_matrices(np.array([cell]))[0]
                    acc += w * cache[cell][loc] @ xc[cd[cell]]
            out[t] = acc
        return out

    def diagonal(self, A=None):
        A = self.assemble() if A is None else A
        return A.diagonal()

    def pressure_dofs(self):
        """Free pressure DoFs (for the constant-pressure null space)."""
        d = self.dofs
        if self.kind not in ("stokes", "stab_ns"):
            return np.zeros(0, dtype=np.int64)
        P = d.offsets[-1]
        ids = np.arange(P, d.n_dofs)
        return ids[d.free[ids]]

    def project_pressure_mean(self, x):
        """Remove the l2 mean of the free pressure DoFs (null-space projection)."""
        ids = self.pressure_dofs()
        y = np.array(x, dtype=float, copy=True)
        if len(ids):
            y[ids] -= y[ids].mean()
        return y


def load_vector(problem, f):
    """Velocity load (f, v) for f(x) -> (npts, dim), Gauss quadrature with q = k_u + 1."""
    dof = problem.dofs
    dim, k = problem.dim, problem.k
    t = forms.CellTables(dim, k, k + 1, problem.forest.h())
    x0 = problem.forest.origin()
    h = problem.forest.h()
    xq = x0[:, None, :] + h[:, None, None] * t.xq[None]          # (nc, nq, dim)
    fq = f(xq.reshape(-1, dim)).reshape(xq.shape[0], xq.shape[1], dim)
    F = np.zeros(dof.n_dofs)
    ns = dof.nodesets[0]
    for c in range(dim):
        loc = np.einsum("cq,qb,cq->cb", t.JxW, t.phi, fq[:, :, c])
        np.add.at(F, dof.offsets[0] + c * ns.n_nodes + ns.cell_nodes, loc)
    return F


def lifting(problem, g):
    """Vector z with the boundary values g (npts -> (npts, dim)) on Dirichlet DoFs, the
    inhomogeneous part of each hanging constraint (weights times boundary masters) on
    hanging DoFs and zero elsewhere, so that the full solution is C x_free + z."""
    d = problem.dofs
    ns = d.nodesets[0]
    gv = g(ns.x)
    z = np.zeros(d.n_dofs)
    for c in range(problem.dim):
        base = d.offsets[0] + c * ns.n_nodes
        bnd = np.nonzero(ns.boundary)[0]
        z[base + bnd] = gv[bnd, c]
        for h_, masters in ns.hanging.items():
            if d.dirichlet[base + h_]:
                continue
            z[base + h_] = sum(w * gv[m, c] for m, w in masters if ns.boundary[m])
    return z


def dirichlet_system(problem, F, g):
    """Right-hand side b of A x = b for the problem with load F and boundary values g:
    free rows C^T (F - K z), Dirichlet rows g, hanging rows 0.  The full solution is
    recovered with ``complete_solution``."""
    d = problem.dofs
    K = problem.assemble_K()
    z = lifting(problem, g)
    bfree = d.C.T @ (F - K @ z)
    b = np.zeros(d.n_dofs)
    b[d.free_ids] = bfree
    b[d.dirichlet] = z[d.dirichlet]
    return b


def complete_solution(problem, x, g):
    """Full vector from a solution of A x = b: hanging DoFs from all masters (free and boundary)."""
    d = problem.dofs
    return d.C @ x[d.free_ids] + lifting(problem, g)


def solve_direct(problem, b, A=None):
    """Direct solve of A x = b; a constant-pressure null space is fixed by zero l2 pressure mean
    (bordered system)."""
    import scipy.sparse.linalg as spla
    A = problem.assemble() if A is None else A
    ids = problem.pressure_dofs()
    if len(ids) == 0:
        return spla.spsolve(A.tocsc(), b)
    n = A.shape[0]
    e = sp.csr_matrix((np.ones(len(ids)), (ids, np.zeros(len(ids), dtype=np.int64))), shape=(n, 1))
    Ab = sp.bmat([[A, e], [e.T, None]]).tocsc()
    bb = np.concatenate([problem.project_pressure_mean(b), [0.0]])
    return spla.spsolve(Ab, bb)[:n]
