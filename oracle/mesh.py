"""Forests of axis-aligned cells, node identification and constraints.

Oracle (test infrastructure only).  Meshes are forests over an n^dim grid of
root cells on the unit square/cube; a cell is (level, integer coordinates at
that level) and has edge length 1 / (n 2^level).

Readings of the paper (Section 2 and the configurations built here):
* Local refinement (global-coarsening hierarchies, Section 2): root cells whose
  centre lies strictly inside a ball are refined, then level-1 cells with the
  same property, and so on for the requested number of levels; afterwards a
  2:1 closure refines every cell that touches (face, edge or vertex) a cell
  two or more levels finer, until no such cell remains.
* A coarser global-coarsening level is obtained by replacing the cells of the
  finest level by their parents; a uniform mesh with n root cells per
  direction coarsens to the uniform mesh with ceil(n/2) (nested for even n,
  non-nested for odd n: Section 2 lists non-nested multigrid among the
  supported hierarchies, and its transfer is the same interpolation).
* Hanging nodes (Section 2, "resolution of (hanging-node) constraints"): a
  node that lies in the closure of a coarser active cell without being a node
  of that cell takes the value of the coarser cell's finite-element function
  at its position.  Chains are resolved transitively.  Dirichlet (boundary)
  velocity nodes take precedence and are fixed to zero.
"""
import numpy as np
import scipy.sparse as sp

from . import fe


class Forest:
    """Active cells of a forest: array ``cells`` (Nc, 1+dim) = [level, c_0, .., c_{dim-1}]."""

    def __init__(self, dim, n, cells):
        self.dim, self.n = dim, n
        cells = np.asarray(cells, dtype=np.int64).reshape(-1, 1 + dim)
        # canonical order: by level, then lexicographic coordinates (z slowest)
        keys = [cells[:, 1 + d] for d in range(dim)] + [cells[:, 0]]
        self.cells = cells[np.lexsort(keys)]

    @property
    def n_cells(self):
        return self.cells.shape[0]

    @property
    def max_level(self):
        return int(self.cells[:, 0].max())

    def h(self):
        """Edge length of every cell."""
        return 1.0 / (self.n * 2.0 ** self.cells[:, 0])

    def origin(self):
        """Lower corner of every cell."""
        return self.cells[:, 1:] * self.h()[:, None]

    def centres(self):
        return self.origin() + 0.5 * self.h()[:, None]

    def lattice(self, L=None):
        """Map from the finest-level lattice (N = n 2^L cells per direction) to cell ids.

        Returns (N, cell_at) where cell_at has shape (N,)*dim (index order [x, y, z])."""
        L = self.max_level if L is None else L
        N = self.n * 2 ** L
        cell_at = -np.ones((N,) * self.dim, dtype=np.int64)
        for cid, row in enumerate(self.cells):
            l = row[0]
            s = 2 ** (L - l)
            sl = tuple(slice(row[1 + d] * s, (row[1 + d] + 1) * s) for d in range(self.dim))
            cell_at[sl] = cid
        assert (cell_at >= 0).all(), "cells do not cover the domain"
        return N, cell_at

    def refine(self, mask):
        """Replace the masked cells by their 2^dim children."""
        mask = np.asarray(mask, dtype=bool)
        keep = self.cells[~mask]
        par = self.cells[mask]
        kids = []
        for off in fe.tensor_index(self.dim, 2):
            ch = par.copy()
            ch[:, 0] += 1
            ch[:, 1:] = 2 * par[:, 1:] + off[None, :]
            kids.append(ch)
        return Forest(self.dim, self.n, np.concatenate([keep] + kids, axis=0))

    def coarsen_finest(self):
        """One global-coarsening step: the finest-level cells are replaced by their parents;
        a uniform forest with n root cells becomes the uniform forest with ceil(n/2)."""
        L = self.max_level
        if L == 0:
            if self.n < 2:
                raise ValueError("cannot coarsen a single cell")
            return uniform(self.dim, (self.n + 1) // 2)
        fine = self.cells[self.cells[:, 0] == L]
        keep = self.cells[self.cells[:, 0] != L]
        par = np.unique(np.concatenate([[[L - 1]] * len(fine), fine[:, 1:] // 2], axis=1), axis=0)
        assert len(par) * 2 ** self.dim == len(fine), "finest level is not made of complete sibling groups"
        return Forest(self.dim, self.n, np.concatenate([keep, par], axis=0))


def uniform(dim, n):
    """Uniform mesh of n^dim cells on the unit square/cube."""
    idx = fe.tensor_index(dim, n)
    return Forest(dim, n, np.concatenate([np.zeros((len(idx), 1), dtype=np.int64), idx], axis=1))


def _max_neighbour_level(forest):
    """For every cell, the largest level among the cells touching its closure."""
    N, cell_at = forest.lattice()
    lev = forest.cells[:, 0][cell_at]
    dil = lev.copy()
    pad = np.pad(lev, 1, mode="constant", constant_values=-1)
    for off in fe.tensor_index(forest.dim, 3):
        sl = tuple(slice(o, o + N) for o in off)
        dil = np.maximum(dil, pad[sl])
    out = np.full(forest.n_cells, -1, dtype=np.int64)
    np.maximum.at(out, cell_at.ravel(), dil.ravel())
    return out


def balance(forest):
    """2:1 closure over faces, edges and vertices."""
    while True:
        need = _max_neighbour_level(forest) >= forest.cells[:, 0] + 2
        if not need.any():
            return forest
        forest = forest.refine(need)


def refine_ball(forest, centre, radius, levels):
    """Refine cells with centre strictly inside the ball, level by level, then 2:1 closure."""
    c = np.asarray(centre, dtype=float)[: forest.dim]
    for lev in range(levels):
        inside = (np.linalg.norm(forest.centres() - c[None, :], axis=1) < radius) & (forest.cells[:, 0] == lev)
        forest = forest.refine(inside)
    return balance(forest)


def is_balanced(forest):
    return bool((_max_neighbour_level(forest) <= forest.cells[:, 0] + 1).all())


class NodeSet:
    """Q_k nodes of a forest, identified exactly, with hanging-node constraints.

    Attributes
      x          (Nn, dim) support-point coordinates
      lat        (Nn, dim) positions in finest-lattice units (float)
      cell_nodes (Nc, (k+1)^dim) node ids of every cell, lexicographic local order
      boundary   (Nn,) node lies on the domain boundary
      hanging    dict node -> list of (master node, weight), masters unconstrained
    """

    def __init__(self, forest, k):
        self.forest, self.k, self.dim = forest, k, forest.dim
        dim = forest.dim
        L = forest.max_level
        N = forest.n * 2 ** L
        self.N_lattice = N
        xi = fe.gll_points(k)
        rational = np.isclose(xi, 0.0) | np.isclose(xi, 1.0) | np.isclose(xi, 0.5)
        loc = fe.tensor_index(dim, k + 1)                  # (nb, dim)
        lev = forest.cells[:, 0]
        scale = 2 ** (L - lev)                             # lattice cells per cell edge
        keys = np.empty((forest.n_cells, loc.shape[0], dim), dtype=np.int64)
        lat = np.empty((forest.n_cells, loc.shape[0], dim))
        for d in range(dim):
            c = forest.cells[:, 1 + d]
            a = loc[:, d]
            lat[:, :, d] = (c[:, None] + xi[a][None, :]) * scale[:, None]
            # rational positions: integer key in half-lattice units; irrational: unique negative code
            rkey = 2 * c[:, None] * scale[:, None] + np.rint(2 * xi[a][None, :] * scale[:, None]).astype(np.int64)
            ikey = -1 - (((lev[:, None] * (N + 1)) + c[:, None]) * (k + 1) + a[None, :])
            keys[:, :, d] = np.where(rational[a][None, :], rkey, ikey)
        flat = keys.reshape(-1, dim)
        uniq, inv = np.unique(flat, axis=0, return_inverse=True)
        self.n_nodes = uniq.shape[0]
        self.cell_nodes = inv.reshape(forest.n_cells, -1)
        self.lat = np.empty((self.n_nodes, dim))
        self.lat[inv.ravel()] = lat.reshape(-1, dim)
        self.x = self.lat / N
        self.boundary = ((self.lat <= 1e-12) | (self.lat >= N - 1e-12)).any(axis=1)
        self.owner_level = np.full(self.n_nodes, np.iinfo(np.int64).max)
        np.minimum.at(self.owner_level, self.cell_nodes.ravel(), np.repeat(lev, loc.shape[0]))
        self._find_hanging(N)

    def _find_hanging(self, N):
        forest, dim, k = self.forest, self.dim, self.k
        _, cell_at = forest.lattice()
        # the lattice cells whose closed box contains a node: floor(p -+ eps) per direction
        lo = np.clip(np.floor(self.lat - 1e-9).astype(np.int64), 0, N - 1)
        hi = np.clip(np.floor(self.lat + 1e-9).astype(np.int64), 0, N - 1)
        touching = []
        for sel in fe.tensor_index(dim, 2):
            idx = tuple(np.where(sel[d] == 0, lo[:, d], hi[:, d]) for d in range(dim))
            touching.append(cell_at[idx])
        touching = np.stack(touching, axis=1)                      # (Nn, 2^dim) cell ids
        coarsest = forest.cells[:, 0][touching].min(axis=1)
        direct = {}
        for g in np.nonzero(coarsest < self.owner_level)[0]:
            for cid in sorted(set(touching[g].tolist())):
                if forest.cells[cid, 0] < self.owner_level[g] and not (self.cell_nodes[cid] == g).any():
                    direct[int(g)] = self._weights_in_cell(cid, g)
                    break
        # resolve chains transitively
        resolved = {}

        def resolve(g, depth=0):
            if g in resolved:
                return resolved[g]
            assert depth < 16, "constraint cycle"
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

    def _weights_in_cell(self, cid, g):
        """Weights of the coarse cell's nodes that reproduce its FE function at node g."""
        forest = self.forest
        L = forest.max_level
        row = forest.cells[cid]
        s = 2.0 ** (L - row[0])
        xi = (self.lat[g] - row[1:] * s) / s
        vals = fe.eval_basis_at(self.dim, self.k, xi[None, :])[0]
        out = []
        for b, w in enumerate(vals):
            if abs(w) > 1e-13:
                out.append((int(self.cell_nodes[cid, b]), float(w)))
        return out


class DofHandler:
    """Global DoFs of a list of fields on one forest.

    ``fields`` is a list of (n_components, degree, dirichlet_on_boundary).
    Oracle numbering: field by field, component by component, node by node.
    Cell-local ordering: the same (field, component, local node)."""

    def __init__(self, forest, fields):
        self.forest, self.dim = forest, forest.dim
        self.fields = fields
        self.nodesets, self.offsets = [], []
        off = 0
        cache = {}
        for nc, k, _ in fields:
            if k not in cache:
                cache[k] = NodeSet(forest, k)
            ns = cache[k]
            self.nodesets.append(ns)
            self.offsets.append(off)
            off += nc * ns.n_nodes
        self.n_dofs = off
        self._build_constraints()

    def set_hanging(self, x):
        """Copy of x with every hanging (non-Dirichlet) entry replaced by the weighted sum of its
        masters' entries (free and boundary masters alike)."""
        y = np.array(x, dtype=float, copy=True)
        for f, (nc, k, dbc) in enumerate(self.fields):
            ns = self.nodesets[f]
            for c in range(nc):
                base = self.offsets[f] + c * ns.n_nodes
                for g, masters in ns.hanging.items():
                    if not self.dirichlet[base + g]:
                        y[base + g] = sum(w * y[base + m] for m, w in masters)
        return y

    def dof(self, f, comp, node):
        return self.offsets[f] + comp * self.nodesets[f].n_nodes + node

    def cell_dofs(self):
        """(Nc, n_local) global DoFs of every cell in cell-local order."""
        parts = []
        for f, (nc, k, _) in enumerate(self.fields):
            ns = self.nodesets[f]
            for c in range(nc):
                parts.append(self.offsets[f] + c * ns.n_nodes + ns.cell_nodes)
        return np.concatenate(parts, axis=1)

    def support_points(self):
        """(n_dofs, dim) coordinates, (n_dofs,) field id (0..dim-1 velocity comps, dim pressure)."""
        xs, fid = [], []
        comp_base = 0
        for f, (nc, k, _) in enumerate(self.fields):
            ns = self.nodesets[f]
            for c in range(nc):
                xs.append(ns.x)
                fid.append(np.full(ns.n_nodes, comp_base + c))
            comp_base += nc
        return np.concatenate(xs), np.concatenate(fid)

    def _build_constraints(self):
        n = self.n_dofs
        dirichlet = np.zeros(n, dtype=bool)
        hanging = np.zeros(n, dtype=bool)
        for f, (nc, k, dbc) in enumerate(self.fields):
            ns = self.nodesets[f]
            for c in range(nc):
                base = self.offsets[f] + c * ns.n_nodes
                if dbc:
                    dirichlet[base + np.nonzero(ns.boundary)[0]] = True
                for g in ns.hanging:
                    hanging[base + g] = True
        hanging &= ~dirichlet                     # Dirichlet takes precedence
        self.dirichlet, self.hanging = dirichlet, hanging
        self.constrained = dirichlet | hanging
        self.free = ~self.constrained
        free_ids = np.nonzero(self.free)[0]
        self.free_ids = free_ids
        col = -np.ones(n, dtype=np.int64)
        col[free_ids] = np.arange(len(free_ids))
        rows, cols, vals = list(free_ids), list(col[free_ids]), [1.0] * len(free_ids)
        for f, (nc, k, dbc) in enumerate(self.fields):
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
                        else:
                            assert dirichlet[base + m], "master must be free or Dirichlet"
        # C maps free DoFs to all DoFs: x_all = C x_free
        self.C = sp.csr_matrix((vals, (rows, cols)), shape=(n, len(free_ids)))

    def distribute(self, x):
        """Set hanging entries from their masters and Dirichlet entries to zero."""
        return self.C @ x[self.free_ids]

    def interpolate(self, func):
        """Nodal interpolant of func(x) -> (npts, n_total_components) into the DoF vector."""
        xs, fid = self.support_points()
        vals = func(xs)
        return vals[np.arange(len(fid)), fid]
