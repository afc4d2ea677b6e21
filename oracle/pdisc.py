"""Stokes with a discontinuous pressure: Q_k^dim / P^disc_{k-1} (the spatial pair of Section 4).

Oracle (test infrastructure only), float64, assembled sparse matrices.

* Velocity: Q_k with the hanging-node and Dirichlet constraints of ``mesh.DofHandler``.
* Pressure: on every cell the polynomials of total degree <= k - 1 in the cell's centred, scaled
  coordinates s = (x - x_c) / h, monomial basis s^a (|a| <= k - 1, graded order); no continuity
  and no constraints.  With all-Dirichlet velocity the constant pressure -- 1 in every cell's
  constant mode, 0 elsewhere -- is the null direction.
* Operator: nu (grad u, grad v) - (p, div v) - (div u, q), the symmetric form of Eq. 5; Gauss
  quadrature with k + 1 points per direction.
* Pressure transfers: L2 projection of the coarse pressure onto every fine cell's polynomials
  (exact when the coarse cell contains the fine one and for degree steps on one mesh).
"""
import numpy as np
import scipy.sparse as sp

from . import assemble, fe, forms, mesh, transfer


def exponents(dim, kp):
    """Multi-indices of total degree <= kp, graded (constant first)."""
    out = []
    for tot in range(kp + 1):
        if dim == 2:
            out += [(a, tot - a) for a in range(tot, -1, -1)]
        else:
            out += [(a, b, tot - a - b) for a in range(tot, -1, -1) for b in range(tot - a, -1, -1)]
    return np.array(out, dtype=np.int64)


def monomials(exps, s):
    """(npts, nm) values of s^a at points s (npts, dim)."""
    return np.prod(s[:, None, :] ** exps[None, :, :], axis=2)


class _Dofs:
    """DoF view of the velocity-pressure vector: velocity block (constraints of the velocity
    DofHandler), then the pressure coefficients cell by cell (all free)."""

    def __init__(self, vel, n_p):
        nv = vel.n_dofs
        self.vel, self.nv = vel, nv
        self.n_dofs = nv + n_p
        self.constrained = np.concatenate([vel.constrained, np.zeros(n_p, dtype=bool)])
        self.hanging = np.concatenate([vel.hanging, np.zeros(n_p, dtype=bool)])
        self.free = ~self.constrained
        self.free_ids = np.nonzero(self.free)[0]
        Cv = vel.C
        self.C = sp.block_diag([Cv, sp.identity(n_p)]).tocsr()

    def distribute(self, x):
        return self.C @ x[self.free_ids]


class StokesPdisc:
    def __init__(self, forest, k, nu=1.0):
        assert k >= 1
        self.forest, self.k, self.nu, self.dim = forest, k, nu, forest.dim
        self.kind = "stokes_pdisc"
        dim = forest.dim
        self.vel = mesh.DofHandler(forest, [(dim, k, True)])
        self.exps = exponents(dim, k - 1)
        self.npc = len(self.exps)
        nc = forest.n_cells
        self.dofs = _Dofs(self.vel, nc * self.npc)
        self.p_offset = self.vel.n_dofs
        self.cell_dofs = np.concatenate(
            [self.vel.cell_dofs(), self.p_offset + np.arange(nc)[:, None] * self.npc + np.arange(self.npc)[None, :]],
            axis=1)

    def _tables(self):
        t = forms.CellTables(self.dim, self.k, self.k + 1, self.forest.h())
        s = t.xq - 0.5                                  # centred, scaled cell coordinates
        return t, monomials(self.exps, s)               # pressure values (nq, npc), h-independent

    def assemble_K(self):
        dim, k, nc = self.dim, self.k, self.forest.n_cells
        t, pq = self._tables()
        nb = t.nb
        lap = self.nu * np.einsum("cq,cqad,cqbd->cab", t.JxW, t.grad, t.grad)
        n = dim * nb + self.npc
        Ke = np.zeros((nc, n, n))
        P = dim * nb
        for i in range(dim):
            Ke[:, i * nb:(i + 1) * nb, i * nb:(i + 1) * nb] = lap
            b = -np.einsum("cq,cqa,qb->cab", t.JxW, t.grad[..., i], pq)     # -(p, d_i v)
            Ke[:, i * nb:(i + 1) * nb, P:] = b
            Ke[:, P:, i * nb:(i + 1) * nb] = np.transpose(b, (0, 2, 1))       # -(d_i u, q)
        cd = self.cell_dofs
        rows = np.repeat(cd[:, :, None], n, axis=2).ravel()
        cols = np.repeat(cd[:, None, :], n, axis=1).ravel()
        K = sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(self.dofs.n_dofs,) * 2)
        K.sum_duplicates()
        return K

    def assemble(self):
        """A = C^T K C on the free DoFs, identity rows on the constrained (velocity) DoFs."""
        d = self.dofs
        K = self.assemble_K()
        Af = (d.C.T @ K @ d.C).tocsr()
        Pm = sp.csr_matrix((np.ones(len(d.free_ids)), (d.free_ids, np.arange(len(d.free_ids)))),
                           shape=(d.n_dofs, len(d.free_ids)))
        A = (Pm @ Af @ Pm.T + sp.diags(d.constrained.astype(float))).tocsr()
        A.sum_duplicates()
        return A

    def velocity_mass(self):
        """Velocity mass on the free velocity rows (constraints resolved), zero elsewhere."""
        dim, k = self.dim, self.k
        Me = forms.scalar_mass(dim, k, k + 1, self.forest.h())
        nb = Me.shape[1]
        ns = self.vel.nodesets[0]
        rows, cols, vals = [], [], []
        for comp in range(dim):
            cd = comp * ns.n_nodes + ns.cell_nodes
            rows.append(np.repeat(cd[:, :, None], nb, axis=2).ravel())
            cols.append(np.repeat(cd[:, None, :], nb, axis=1).ravel())
            vals.append(Me.ravel())
        n = self.dofs.n_dofs
        K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
        d = self.dofs
        Mf = (d.C.T @ K @ d.C).tocsr()
        Pm = sp.csr_matrix((np.ones(len(d.free_ids)), (d.free_ids, np.arange(len(d.free_ids)))),
                           shape=(n, len(d.free_ids)))
        return (Pm @ Mf @ Pm.T).tocsr()

    def pressure_null(self):
        """The constant pressure: 1 in every cell's constant mode."""
        e = np.zeros(self.dofs.n_dofs)
        e[self.p_offset + np.arange(self.forest.n_cells) * self.npc] = 1.0
        return e

    def pressure_at(self, x, pts):
        """The pressure of x at physical points (each in the cell holding it)."""
        N, cell_at = self.forest.lattice()
        idx = np.clip(np.floor(pts * N + 1e-9).astype(np.int64), 0, N - 1)
        cells = cell_at[tuple(idx[:, d] for d in range(self.dim))]
        h = self.forest.h()[cells]
        s = (pts - self.forest.origin()[cells]) / h[:, None] - 0.5
        vals = monomials(self.exps, s)
        coef = x[self.p_offset + cells[:, None] * self.npc + np.arange(self.npc)[None, :]]
        return (vals * coef).sum(axis=1)

    def project_pressure(self, func):
        """Per-cell L2 projection of func(points) -> (npts,) onto the pressure space (coefficients)."""
        out = np.zeros(self.forest.n_cells * self.npc)
        xg, wg = fe.gauss(self.k + 1)
        qi = fe.tensor_index(self.dim, self.k + 1)
        xi = xg[qi]
        w = np.prod(wg[qi], axis=1)
        V = monomials(self.exps, xi - 0.5)
        Mref = V.T @ (w[:, None] * V)
        h, org = self.forest.h(), self.forest.origin()
        for c in range(self.forest.n_cells):
            pts = org[c] + xi * h[c]
            out[c * self.npc:(c + 1) * self.npc] = np.linalg.solve(Mref, V.T @ (w * func(pts)))
        return out


def prolongation(coarse, fine):
    """P (n_fine x n_coarse) between StokesPdisc problems: velocity by interpolation of the coarse
    finite-element function at the free fine DoFs (Eq. 4), pressure by L2 projection onto every
    fine cell (coarse pressure evaluated in the coarse cell holding each quadrature point)."""
    pv = transfer.prolongation(assemble.Problem(coarse.forest, "stokes_a", coarse.k),
                               assemble.Problem(fine.forest, "stokes_a", fine.k))
    # pressure: fine cell coefficients = Mref^{-1} V^T W (coarse pressure at the fine quadrature points)
    q = max(fine.k, coarse.k) + 1
    xg, wg = fe.gauss(q)
    qi = fe.tensor_index(fine.dim, q)
    xi = xg[qi]
    w = np.prod(wg[qi], axis=1)
    Vf = monomials(fine.exps, xi - 0.5)
    proj = np.linalg.solve(Vf.T @ (w[:, None] * Vf), Vf.T * w[None, :])     # (npf, nq)
    N, cell_at = coarse.forest.lattice()
    hf, of = fine.forest.h(), fine.forest.origin()
    hc, oc = coarse.forest.h(), coarse.forest.origin()
    rows, cols, vals = [], [], []
    for c in range(fine.forest.n_cells):
        pts = of[c] + xi * hf[c]
        idx = np.clip(np.floor(pts * N + 1e-9).astype(np.int64), 0, N - 1)
        cc = cell_at[tuple(idx[:, d] for d in range(fine.dim))]
        for cp in np.unique(cc):
            sel = cc == cp
            Vc = np.zeros((len(pts), coarse.npc))
            Vc[sel] = monomials(coarse.exps, (pts[sel] - oc[cp]) / hc[cp] - 0.5)
            blk = proj @ Vc                                                  # (npf, npc)
            for a in range(fine.npc):
                for b in range(coarse.npc):
                    if abs(blk[a, b]) > 1e-15:
                        rows.append(fine.p_offset + c * fine.npc + a)
                        cols.append(coarse.p_offset + cp * coarse.npc + b)
                        vals.append(blk[a, b])
    pp = sp.csr_matrix((vals, (rows, cols)), shape=(fine.dofs.n_dofs, coarse.dofs.n_dofs))
    P = sp.lil_matrix((fine.dofs.n_dofs, coarse.dofs.n_dofs))
    P[:fine.p_offset, :coarse.p_offset] = pv
    return (P.tocsr() + pp).tocsr()
