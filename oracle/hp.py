"""hp-adaptive continuous finite elements and hp-multigrid (Section 3, Exp. 1).

Oracle (test infrastructure only), float64, assembled sparse matrices.

Section 3 solves the stationary Stokes equations on meshes refined both in the cell size h and in
the polynomial degree p of every cell, with Taylor--Hood elements (velocity Q_k, pressure
Q_{k-1}, k per cell), the block preconditioner of Eq. 5, and one V-cycle of hp-multigrid for the
A block: the degree of every cell is lowered one by one until all cells are linear, then global
coarsening follows; hanging-node constraints of hp-discretisations are resolved on every level.

Readings of the paper:
* Conformity (the paper cites the standard hp constraint algorithm without restating it): a node
  is constrained when some cell whose closed box contains it does not have it as a node and
  dominates every cell that does -- it is coarser, or of the same level and of lower degree.  The
  node then takes that cell's finite-element function at its position (its degree-k_X basis over
  its own nodes); chains are resolved transitively; Dirichlet nodes are fixed to zero and take
  precedence.  This gives a conforming space whenever no hanging face has a coarse neighbour of
  higher degree than the fine cells on it (the tests check continuity across every interface and
  the dimension against a brute-force rank).  The opposite configuration -- the combined h+p face
  where the paper's Jacobi+ASM smoother places its blocks -- needs both sides constrained to the
  lower degree; the local rule rejects it (NotImplementedError).
* The same space by elimination (rule 'elimination'), for every configuration including the
  combined face: the continuity conditions on every shared face piece, as linear equations in the
  unknown node values, brought to reduced row echelon form with the columns ordered from the least
  to the most preferred node (coarser, then lower degree, then vertices before edge, face and cell
  interiors, then node id), so that the slaves are the least preferred nodes.  The entity order
  is what the standard construction does face by face (the vertex and edge values of the coarse
  face are kept): without it, ties broken by node id alone let a shared vertex become a slave and
  the constraints chain along the whole refinement interface.  Where the local rule applies it
  gives the same interior slaves and the same weights on the free masters.  With combined faces
  the Jacobi-preconditioned A block has a larger largest eigenvalue (the ill-conditioned relations
  between the remaining unknowns that Section 3 gives as the reason for the ASM blend).
* Degrees: cell-wise k_c in 1..4 for the vector Laplacian; Taylor--Hood needs k_c >= 2 (pressure
  k_c - 1 >= 1).  Quadrature per cell: Gauss with k_c + 1 points per direction.
* p-coarsening ("decreased one by one until ... all linear elements"): k_c -> max(k_c - 1, 1) on
  every cell per level; then the global-coarsening h-levels of ``solvers.coarse_forests`` with
  linear elements.  Transfers: interpolation of the coarse finite-element function at the free
  fine DoFs, restriction its transpose (Eq. 4).
"""
import numpy as np
import scipy.sparse as sp

from . import fe, forms, mesh, solvers


class HpNodeSet:
    """Nodes of a forest with a degree per cell, identified exactly, with h/p constraints.

    Attributes: ``x`` (Nn, dim) support points, ``lat`` positions in finest-lattice units,
    ``cell_nodes`` list of node-id arrays (one per cell, (k_c+1)^dim, lexicographic),
    ``boundary`` (Nn,), ``hanging`` dict node -> [(master, weight)] (masters unconstrained)."""

    def __init__(self, forest, degrees, rule="dominance", dirichlet=True):
        """rule: 'dominance' (the local rule of the module docstring) or 'elimination' (every
        configuration, including a hanging face whose coarse cell has the higher degree: continuity
        on every shared face piece as linear conditions, eliminated in the preference order
        coarser -> lower degree -> lower entity dimension -> node id; the least preferred nodes
        become the slaves).
        dirichlet (elimination only): boundary values are fixed to zero and are not unknowns;
        without it (a field with no boundary condition, the Taylor--Hood pressure) every node is
        an unknown."""
        dim = forest.dim
        self.forest, self.dim = forest, dim
        self.rule = rule
        self.fixed_boundary = dirichlet
        self.degrees = np.asarray(degrees, dtype=np.int64)
        assert self.degrees.shape == (forest.n_cells,) and self.degrees.min() >= 1
        L = forest.max_level
        N = forest.n * 2 ** L
        self.N_lattice = N
        kmax = int(self.degrees.max())
        lev = forest.cells[:, 0]
        scale = 2 ** (L - lev)
        keys, lats, owners = [], [], []
        for c in range(forest.n_cells):
            k = int(self.degrees[c])
            xi = fe.gll_points(k)
            rational = np.isclose(xi, 0.0) | np.isclose(xi, 1.0) | np.isclose(xi, 0.5)
            loc = fe.tensor_index(dim, k + 1)
            cc = forest.cells[c, 1:]
            kk = np.empty((len(loc), dim), dtype=np.int64)
            for d in range(dim):
                a = loc[:, d]
                rkey = 2 * cc[d] * scale[c] + np.rint(2 * xi[a] * scale[c]).astype(np.int64)
                # irrational positions: unique per (level, cell coordinate, degree, slot)
                ikey = -1 - ((((lev[c] * (N + 1)) + cc[d]) * (kmax + 1) + k) * (kmax + 1) + a)
                kk[:, d] = np.where(rational[a], rkey, ikey)
            keys.append(kk)
            lats.append((cc[None, :] + xi[loc]) * scale[c])
            owners.append(np.full(len(loc), c))
        flat = np.concatenate(keys)
        uniq, inv = np.unique(flat, axis=0, return_inverse=True)
        inv = inv.ravel()
        self.n_nodes = uniq.shape[0]
        self.lat = np.empty((self.n_nodes, dim))
        self.lat[inv] = np.concatenate(lats)
        self.x = self.lat / N
        self.boundary = ((self.lat <= 1e-12) | (self.lat >= N - 1e-12)).any(axis=1)
        offs = np.cumsum([0] + [len(k_) for k_ in keys])
        self.cell_nodes = [inv[offs[c]:offs[c + 1]] for c in range(forest.n_cells)]
        # the cells owning each node; the dominating (level, degree) among them
        own_c = np.concatenate(owners)
        self.owners = [[] for _ in range(self.n_nodes)]
        for g, c in zip(inv, own_c):
            self.owners[g].append(int(c))
        self.dom = [min((int(lev[c]), int(self.degrees[c])) for c in cs) for cs in self.owners]
        if rule == "elimination":
            self._eliminate()
        else:
            self._find_constraints()

    def _touching(self):
        """(Nn, 2^dim) ids of the cells whose closed box holds each node."""
        _, cell_at = self.forest.lattice()
        N = self.N_lattice
        lo = np.clip(np.floor(self.lat - 1e-9).astype(np.int64), 0, N - 1)
        hi = np.clip(np.floor(self.lat + 1e-9).astype(np.int64), 0, N - 1)
        out = []
        for sel in fe.tensor_index(self.dim, 2):
            idx = tuple(np.where(sel[d] == 0, lo[:, d], hi[:, d]) for d in range(self.dim))
            out.append(cell_at[idx])
        return np.stack(out, axis=1)

    def _weights_in_cell(self, cid, g):
        L = self.forest.max_level
        row = self.forest.cells[cid]
        s = 2.0 ** (L - row[0])
        xi = (self.lat[g] - row[1:] * s) / s
        vals = fe.eval_basis_at(self.dim, int(self.degrees[cid]), xi[None, :])[0]
        return [(int(self.cell_nodes[cid][b]), float(w)) for b, w in enumerate(vals) if abs(w) > 1e-13]

    def _find_constraints(self):
        lev = self.forest.cells[:, 0]
        touching = self._touching()
        direct = {}
        for g in range(self.n_nodes):
            best = None
            for cid in sorted(set(touching[g].tolist())):
                if cid in self.owners[g]:
                    continue
                key = (int(lev[cid]), int(self.degrees[cid]))
                if key < self.dom[g] and (best is None or key < best[0]):
                    best = (key, cid)
            if best is None:
                continue
            (lx, kx), cid = best
            if lx < self.dom[g][0]:
                # h-hanging: every fine cell owning the node must be of degree >= the coarse one
                if kx > min(int(self.degrees[c]) for c in self.owners[g]):
                    raise NotImplementedError("a hanging face whose coarse cell has a higher degree than the fine cell")
            direct[g] = self._weights_in_cell(cid, g)
        resolved = {}

        def resolve(g, depth=0):
            if g in resolved:
                return resolved[g]
            assert depth < 32, "constraint cycle"
            out = {}
            for m, w in direct[g]:
                if m in direct:
                    for mm, ww in resolve(m, depth + 1):
                        out[mm] = out.get(mm, 0.0) + w * ww
                else:
                    out[m] = out.get(m, 0.0) + w
            resolved[g] = sorted(out.items())
            return resolved[g]

        self.hanging = {g: resolve(g) for g in direct}


    def _face_pieces(self):
        """(A, B, points) for every pair of cells sharing a piece of a face, with GLL points of
        degree kmax + 1 on the piece (enough to identify the traces)."""
        f = self.forest
        N, cell_at = f.lattice()
        dim, h, org = self.dim, f.h(), f.origin()
        xs = fe.gll_points(int(self.degrees.max()) + 1)
        out = []
        for a in range(f.n_cells):
            for d in range(dim):
                for side in (0, 1):
                    plane = org[a, d] + side * h[a]
                    if plane <= 1e-12 or plane >= 1 - 1e-12:
                        continue
                    lo = np.rint(org[a] * N).astype(int)
                    hi = np.rint((org[a] + h[a]) * N).astype(int)
                    sl = [slice(lo[j], hi[j]) for j in range(dim)]
                    q = int(round(plane * N))
                    sl[d] = slice(q, q + 1) if side else slice(q - 1, q)
                    for b in np.unique(cell_at[tuple(sl)]):
                        if b < a and f.cells[b, 0] == f.cells[a, 0]:
                            continue                     # same-level pairs once
                        lo_s = np.maximum(org[a], org[b])
                        hi_s = np.minimum(org[a] + h[a], org[b] + h[b])
                        tang = [j for j in range(dim) if j != d]
                        grids = np.meshgrid(*[lo_s[j] + (hi_s[j] - lo_s[j]) * xs for j in tang], indexing="ij")
                        pts = np.zeros((grids[0].size, dim))
                        for j, g in zip(tang, grids):
                            pts[:, j] = g.ravel()
                        pts[:, d] = plane
                        out.append((a, int(b), pts))
        return out

    def _entity(self, g):
        """Dimension of the entity a node is interior to in a dominating owner cell: 0 vertex, 1
        edge, 2 face, 3 cell (the number of local coordinates strictly between 0 and k)."""
        lev = self.forest.cells[:, 0]
        for c in self.owners[g]:
            if (int(lev[c]), int(self.degrees[c])) == self.dom[g]:
                k = int(self.degrees[c])
                i = int(np.nonzero(self.cell_nodes[c] == g)[0][0])
                a = [(i // (k + 1) ** d) % (k + 1) for d in range(self.dim)]
                return sum(1 for v in a if 0 < v < k)
        raise AssertionError("node without a dominating owner")

    def _eliminate(self):
        """Constraints by elimination (rule 'elimination'): the continuity conditions G u = 0 on the
        unknown node values, reduced to row echelon form with the columns in reverse preference order,
        so that every pivot (slave) is as little preferred as possible; slave = -sum of its row's
        free entries.  With fixed_boundary the boundary nodes are zero and are not unknowns."""
        f, dim = self.forest, self.dim
        lev = f.cells[:, 0]
        h, org = f.h(), f.origin()
        var = np.nonzero(~self.boundary)[0] if self.fixed_boundary else np.arange(self.n_nodes)
        col_of = -np.ones(self.n_nodes, dtype=np.int64)
        pref = sorted(var.tolist(), key=lambda g: (self.dom[g][0], self.dom[g][1], self._entity(g), g))
        order = pref[::-1]                                 # least preferred first: pivots land there
        for j, g in enumerate(order):
            col_of[g] = j
        rows = []
        for a, b, pts in self._face_pieces():
            G = np.zeros((len(pts), len(order)))
            for c, sgn in ((a, 1.0), (b, -1.0)):
                xi = np.clip((pts - org[c]) / h[c], 0.0, 1.0)
                phi = fe.eval_basis_at(dim, int(self.degrees[c]), xi)
                for bb, g in enumerate(self.cell_nodes[c]):
                    if col_of[g] >= 0:
                        G[:, col_of[g]] += sgn * phi[:, bb]
            rows.append(G)
        G = np.concatenate(rows) if rows else np.zeros((0, len(order)))
        # reduced row echelon form (Gauss--Jordan, largest entry in the pivot column)
        R = G.copy()
        piv_cols, r = [], 0
        tol = 1e-10 * max(1.0, np.abs(R).max() if R.size else 1.0)
        for j in range(R.shape[1]):
            if r >= R.shape[0]:
                break
            i = r + int(np.argmax(np.abs(R[r:, j])))
            if abs(R[i, j]) <= tol:
                continue
            R[[r, i]] = R[[i, r]]
            R[r] /= R[r, j]
            others = np.nonzero(np.abs(R[:, j]) > 0)[0]
            for i2 in others:
                if i2 != r:
                    R[i2] -= R[i2, j] * R[r]
            piv_cols.append(j)
            r += 1
        R = R[:r]
        R[np.abs(R) < 1e-13] = 0.0
        pivots = set(piv_cols)
        self.hanging = {}
        for i, j in enumerate(piv_cols):
            g = order[j]
            masters = [(order[q], -float(R[i, q])) for q in np.nonzero(R[i])[0] if q not in pivots]
            self.hanging[int(g)] = sorted((int(m), w) for m, w in masters)


class HpDofHandler:
    """DoFs of fields on an hp forest: ``fields`` = [(n_components, degree_shift, dirichlet)], the
    field's degree on cell c being degrees[c] - degree_shift.  Numbering: field by field, component
    by component, node by node (as ``mesh.DofHandler``)."""

    def __init__(self, forest, degrees, fields, rule="dominance"):
        self.forest, self.dim = forest, forest.dim
        self.degrees = np.asarray(degrees, dtype=np.int64)
        self.fields = fields
        self.nodesets, self.offsets = [], []
        off = 0
        for nc, shift, dbc in fields:
            ns = HpNodeSet(forest, self.degrees - shift, rule, dirichlet=dbc)
            self.nodesets.append(ns)
            self.offsets.append(off)
            off += nc * ns.n_nodes
        self.n_dofs = off
        n = off
        dirichlet = np.zeros(n, dtype=bool)
        hanging = np.zeros(n, dtype=bool)
        for f, (nc, _, dbc) in enumerate(fields):
            ns = self.nodesets[f]
            for c in range(nc):
                base = self.offsets[f] + c * ns.n_nodes
                if dbc:
                    dirichlet[base + np.nonzero(ns.boundary)[0]] = True
                for g in ns.hanging:
                    hanging[base + g] = True
        hanging &= ~dirichlet
        self.dirichlet, self.hanging = dirichlet, hanging
        self.constrained = dirichlet | hanging
        self.free = ~self.constrained
        self.free_ids = np.nonzero(self.free)[0]
        col = -np.ones(n, dtype=np.int64)
        col[self.free_ids] = np.arange(len(self.free_ids))
        rows, cols, vals = list(self.free_ids), list(col[self.free_ids]), [1.0] * len(self.free_ids)
        for f, (nc, _, dbc) in enumerate(fields):
            ns = self.nodesets[f]
            for c in range(nc):
                base = self.offsets[f] + c * ns.n_nodes
                for g, masters in ns.hanging.items():
                    if dirichlet[base + g]:
                        continue
                    for m, w in masters:
                        if self.free[base + m]:
                            rows.append(base + g)
                            cols.append(col[base + m])
                            vals.append(w)
        self.C = sp.csr_matrix((vals, (rows, cols)), shape=(n, len(self.free_ids)))

    def distribute(self, x):
        """Hanging entries from their masters, Dirichlet entries zero."""
        return self.C @ x[self.free_ids]

    def cell_dofs(self, c):
        """Global DoFs of cell c in cell-local order (field, component, node)."""
        parts = []
        for f, (nc, _, _) in enumerate(self.fields):
            ns = self.nodesets[f]
            for comp in range(nc):
                parts.append(self.offsets[f] + comp * ns.n_nodes + ns.cell_nodes[c])
        return np.concatenate(parts)

    def support_points(self):
        xs, fid = [], []
        base = 0
        for f, (nc, _, _) in enumerate(self.fields):
            ns = self.nodesets[f]
            for comp in range(nc):
                xs.append(ns.x)
                fid.append(np.full(ns.n_nodes, base + comp))
            base += nc
        return np.concatenate(xs), np.concatenate(fid)

    def interpolate(self, func):
        xs, fid = self.support_points()
        vals = func(xs)
        return vals[np.arange(len(fid)), fid]


class HpProblem:
    """Operator on an hp forest: kind 'stokes_a' (vector Laplacian nu (grad u, grad v)), 'stokes'
    (Taylor--Hood, symmetric form of Eq. 5) or 'pmass' (the mass matrix of the Taylor--Hood pressure
    space, degree k_c - 1 per cell, no boundary conditions: the Schur-complement approximation of
    Eq. 5 up to the factor 1/nu).  ``degrees`` are the velocity degrees in every case."""

    def __init__(self, forest, degrees, kind, nu=1.0, rule="dominance"):
        dim = forest.dim
        self.forest, self.kind, self.nu, self.dim = forest, kind, nu, dim
        self.degrees = np.asarray(degrees, dtype=np.int64)
        if kind == "stokes_a":
            fields = [(dim, 0, True)]
        elif kind == "stokes":
            assert self.degrees.min() >= 2, "Taylor--Hood needs velocity degree >= 2"
            fields = [(dim, 0, True), (1, 1, False)]
        elif kind == "pmass":
            assert self.degrees.min() >= 2, "Taylor--Hood needs velocity degree >= 2"
            fields = [(1, 1, False)]
        else:
            raise ValueError(kind)
        self.dofs = HpDofHandler(forest, self.degrees, fields, rule)

    def assemble_K(self):
        d = self.dofs
        h = self.forest.h()
        rows, cols, vals = [], [], []
        for k in np.unique(self.degrees):
            cells = np.nonzero(self.degrees == k)[0]
            if self.kind == "stokes_a":
                Ke = forms.vector_laplacian(self.dim, int(k), self.nu, h[cells])
            elif self.kind == "pmass":
                Ke = forms.scalar_mass(self.dim, int(k) - 1, int(k), h[cells])
            else:
                Ke = forms.stokes_taylor_hood(self.dim, int(k), self.nu, h[cells], -1.0)
            cd = np.stack([d.cell_dofs(c) for c in cells])
            rows.append(np.repeat(cd[:, :, None], cd.shape[1], axis=2).ravel())
            cols.append(np.repeat(cd[:, None, :], cd.shape[1], axis=1).ravel())
            vals.append(Ke.ravel())
        K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(d.n_dofs, d.n_dofs))
        K.sum_duplicates()
        return K

    def assemble(self):
        """A = C^T K C on the free DoFs, identity rows on the constrained ones."""
        K = self.assemble_K()
        d = self.dofs
        Af = (d.C.T @ K @ d.C).tocsr()
        P = sp.csr_matrix((np.ones(len(d.free_ids)), (d.free_ids, np.arange(len(d.free_ids)))),
                          shape=(d.n_dofs, len(d.free_ids)))
        A = (P @ Af @ P.T + sp.diags(d.constrained.astype(float))).tocsr()
        A.sum_duplicates()
        return A

    def pressure_dofs(self):
        d = self.dofs
        if self.kind != "stokes":
            return np.zeros(0, dtype=np.int64)
        ids = np.arange(d.offsets[-1], d.n_dofs)
        return ids[d.free[ids]]

    def evaluate(self, x, pts, field=0, comp=0):
        """The finite-element function of DoF vector x (constraints distributed) at points, each
        evaluated in a cell whose closed box holds it."""
        d = self.dofs
        ns = d.nodesets[field]
        N, cell_at = self.forest.lattice()
        idx = np.clip(np.floor(pts * N + 1e-9).astype(np.int64), 0, N - 1)
        cells = cell_at[tuple(idx[:, j] for j in range(self.dim))]
        return self.evaluate_in(x, pts, cells, field, comp)

    def evaluate_in(self, x, pts, cells, field=0, comp=0):
        """The finite-element function of x at pts, evaluated in the given cells."""
        d = self.dofs
        ns = d.nodesets[field]
        shift = d.fields[field][1]
        h = self.forest.h()[cells]
        xi = np.clip((pts - self.forest.origin()[cells]) / h[:, None], 0.0, 1.0)
        out = np.empty(len(pts))
        base = d.offsets[field] + comp * ns.n_nodes
        for c in np.unique(cells):
            sel = np.nonzero(cells == c)[0]
            phi = fe.eval_basis_at(self.dim, int(self.degrees[c]) - shift, xi[sel])
            out[sel] = phi @ x[base + ns.cell_nodes[c]]
        return out


def prolongation(coarse, fine):
    """P (n_fine x n_coarse): the coarse hp function (constraints resolved) at the free fine DoFs."""
    dc, df = coarse.dofs, fine.dofs
    rows, cols, vals = [], [], []
    N, cell_at = coarse.forest.lattice()
    for f, ((ncc, sc, _), (ncf, sf, _)) in enumerate(zip(dc.fields, df.fields)):
        assert ncc == ncf
        nsc, nsf = dc.nodesets[f], df.nodesets[f]
        idx = np.clip(np.floor(nsf.x * N + 1e-9).astype(np.int64), 0, N - 1)
        cells = cell_at[tuple(idx[:, d] for d in range(coarse.dim))]
        h = coarse.forest.h()[cells]
        xi = np.clip((nsf.x - coarse.forest.origin()[cells]) / h[:, None], 0.0, 1.0)
        for g in range(nsf.n_nodes):
            c = cells[g]
            phi = fe.eval_basis_at(coarse.dim, int(coarse.degrees[c]) - sc, xi[g][None, :])[0]
            keep = np.abs(phi) > 1e-14
            for comp in range(ncc):
                rows.extend([df.offsets[f] + comp * nsf.n_nodes + g] * int(keep.sum()))
                cols.extend((dc.offsets[f] + comp * nsc.n_nodes + nsc.cell_nodes[c][keep]).tolist())
                vals.extend(phi[keep].tolist())
    interp = sp.csr_matrix((vals, (rows, cols)), shape=(df.n_dofs, dc.n_dofs))
    sel = sp.csr_matrix((np.ones(len(dc.free_ids)), (np.arange(len(dc.free_ids)), dc.free_ids)),
                        shape=(len(dc.free_ids), dc.n_dofs))
    P = (sp.diags(df.free.astype(float)) @ interp @ dc.C @ sel).tocsr()
    P.eliminate_zeros()
    return P


class Level:
    def __init__(self, problem):
        self.problem = problem
        self.A = problem.assemble()
        self.dinv = 1.0 / self.A.diagonal()
        self.P = None
        self.lmax = None


def combined_faces(problem):
    """(coarse cell, axis, side) of every cell face whose neighbours across it are finer and of lower
    degree: the faces, h-refined on one side and p-refined on the other, where Section 3 places the
    blocks of its additive Schwarz smoother."""
    f = problem.forest
    deg = problem.degrees
    lev = f.cells[:, 0]
    h, org = f.h(), f.origin()
    out = set()
    for a, b, pts in problem.dofs.nodesets[0]._face_pieces():
        if lev[a] == lev[b]:
            continue
        c, fc = (a, b) if lev[a] < lev[b] else (b, a)
        if deg[c] <= deg[fc]:
            continue
        for ax in range(f.dim):
            if np.all(np.abs(pts[:, ax] - pts[0, ax]) <= 1e-12):
                out.add((int(c), ax, int(round((pts[0, ax] - org[c, ax]) / h[c]))))
    return sorted(out)


def asm_blocks(problem):
    """Blocks of the additive Schwarz part of Section 3's smoother: for every combined face, the free
    velocity unknowns (all components together) whose node lies on the closed face of its coarse
    cell.  Ascending DoF indices; faces without free unknowns give no block."""
    d = problem.dofs
    ns = d.nodesets[0]
    f = problem.forest
    h, org = f.h(), f.origin()
    blocks = []
    for c, ax, side in combined_faces(problem):
        plane = org[c, ax] + side * h[c]
        on = (np.abs(ns.x[:, ax] - plane) <= 1e-12) & np.all(
            (ns.x >= org[c] - 1e-12) & (ns.x <= org[c] + h[c] + 1e-12), axis=1)
        nodes = np.nonzero(on)[0]
        idx = np.array([d.offsets[0] + comp * ns.n_nodes + g for comp in range(f.dim) for g in nodes], dtype=np.int64)
        idx = np.sort(idx[d.free[idx]])
        if len(idx):
            blocks.append(idx)
    return blocks


class JacobiASM:
    """The smoother's preconditioner blending additive Schwarz and point Jacobi (Section 3):
    P^{-1} r = sum over blocks B of R_B^T A_BB^{-1} R_B r (summed where blocks overlap) plus
    r_i / A_ii on the unknowns in no block."""

    def __init__(self, A, blocks):
        A = A.tocsr()
        self.blocks = blocks
        self.dinv = 1.0 / A.diagonal()
        self.in_block = np.zeros(A.shape[0], dtype=bool)
        self.inv = []
        for B in blocks:
            self.in_block[B] = True
            self.inv.append(np.linalg.inv(A[B][:, B].toarray()))

    def __call__(self, r):
        z = np.where(self.in_block, 0.0, self.dinv * r)
        for B, Bi in zip(self.blocks, self.inv):
            z[B] += Bi @ r[B]
        return z


def hierarchy(forest, degrees, nu=1.0, stop_n=2, rule="dominance", smoother="jacobi"):
    """hp-multigrid levels of the A block (finest first): every cell's degree lowered by one per
    level until all cells are linear, then global coarsening with linear elements.  rule: the
    constraint construction of every level (``HpNodeSet``).  smoother: 'jacobi' (every level's
    ``dinv`` is the diagonal inverse) or 'asm' (levels with combined faces get ``JacobiASM``)."""
    degrees = np.asarray(degrees, dtype=np.int64)
    seq = [(forest, degrees)]
    while seq[-1][1].max() > 1:
        seq.append((forest, np.maximum(seq[-1][1] - 1, 1)))
    for f in solvers.coarse_forests(forest, stop_n)[1:]:
        seq.append((f, np.ones(f.n_cells, dtype=np.int64)))
    levels = [Level(HpProblem(f, d, "stokes_a", nu, rule=rule)) for f, d in seq]
    for l in range(len(levels) - 1):
        levels[l].P = prolongation(levels[l + 1].problem, levels[l].problem)
    if smoother == "asm":
        for lv in levels[:-1]:
            blocks = asm_blocks(lv.problem)
            if blocks:
                lv.dinv = JacobiASM(lv.A, blocks)
    return levels


def degrees_by_position(forest, func):
    """Degree of every cell from a function of the cell centre (ncells, dim) -> int array."""
    return np.asarray(func(forest.centres()), dtype=np.int64)
