"""Intergrid transfer by interpolation (Eq. 4), h and p alike.

Oracle (test infrastructure only).  The prolongation P maps a coarse vector
to the fine space: its constrained entries are first resolved (hanging nodes
from their masters, Dirichlet to zero), the coarse finite-element function is
evaluated at the support point of every free fine DoF, and constrained fine
DoFs get zero.  Restriction is the transpose (Eq. 4: "the restriction
operator is defined by the transpose").  This single definition covers
geometric (coarse mesh -> refined mesh, same degree) and polynomial (same
mesh, lower degree -> higher degree) transfers.
"""
import numpy as np
import scipy.sparse as sp

from . import fe


def _locate(forest, x):
    """Id of a cell of ``forest`` whose closed box contains each point x (npts, dim)."""
    N, cell_at = forest.lattice()
    idx = np.clip(np.floor(x * N + 1e-9).astype(np.int64), 0, N - 1)
    return cell_at[tuple(idx[:, d] for d in range(forest.dim))]


def prolongation(coarse, fine):
    """Sparse P (n_fine x n_coarse) between two assemble.Problem objects of the same kind."""
    dc, df = coarse.dofs, fine.dofs
    assert len(dc.fields) == len(df.fields)
    rows, cols, vals = [], [], []
    for f, ((ncc, kc, _), (ncf, kf, _)) in enumerate(zip(dc.fields, df.fields)):
        assert ncc == ncf
        nsc, nsf = dc.nodesets[f], df.nodesets[f]
        cells = _locate(coarse.forest, nsf.x)
        h = coarse.forest.h()[cells]
        x0 = coarse.forest.origin()[cells]
        xi = (nsf.x - x0) / h[:, None]
        xi = np.clip(xi, 0.0, 1.0)
        phi = fe.eval_basis_at(coarse.dim, kc, xi)                   # (Nn_f, nb_c)
        cn = nsc.cell_nodes[cells]                                    # (Nn_f, nb_c)
        for c in range(ncc):
            rf = df.offsets[f] + c * nsf.n_nodes + np.arange(nsf.n_nodes)
            cc = dc.offsets[f] + c * nsc.n_nodes + cn
            keep = np.abs(phi) > 1e-14
            rows.append(np.repeat(rf[:, None], phi.shape[1], axis=1)[keep])
            cols.append(cc[keep])
            vals.append(phi[keep])
    interp = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                           shape=(df.n_dofs, dc.n_dofs))
    # resolve coarse constraints: x_all = C_c x_free, with x_free the free entries of x
    sel = sp.csr_matrix((np.ones(len(dc.free_ids)), (np.arange(len(dc.free_ids)), dc.free_ids)),
                        shape=(len(dc.free_ids), dc.n_dofs))
    P = sp.diags(df.free.astype(float)) @ interp @ dc.C @ sel
    P = P.tocsr()
    P.eliminate_zeros()
    return P
