"""Space-time finite elements for the transient Stokes equations (Section 4).

Oracle (test infrastructure only), float64, assembled sparse matrices.

Section 4 discretises each time slab I_n = (t_{n-1}, t_n], tau_n = t_n - t_{n-1}, with a Q-stage
variational time discretisation and collects the stage values of the spatial vector in stage-major
order, x_n = (x_{n,1}, ..., x_{n,Q}).  On the slab the system is the Kronecker operator
    (A_Q (x) M + tau M_Q (x) A) x_n = F_n + (m_Q (x) M) u_{n-1},
and, after mass scaling with M_Q^{-1} (x) I, the operator of Eq. 6:
    K = G_Q (x) M + tau I_Q (x) A,   G_Q = M_Q^{-1} A_Q,
with M the Stokes block mass (velocity mass, zero pressure block) and A the Stokes operator.

Readings of the paper (it cites the temporal matrices without restating them):
* Time discretisation: DG(r), Q = r + 1, with the Lagrange basis phi_i at the Q right Gauss--Radau
  points of the slab (the last point is the slab's end, so the value handed to the next slab is
  the last stage).  On the reference slab [0, 1]:
      M_Q[j, i] = int phi_i phi_j,   A_Q[j, i] = int phi_i' phi_j + phi_i(0) phi_j(0),   m_Q[j] = phi_j(0)
  (time derivative, upwind jump at the slab's start, and the previous slab's end value).  This is
  the Q-stage Radau IIA method; its stability function is the (r, r+1) Pade approximant of exp.
* Space: Taylor--Hood Q_k / Q_{k-1} (the paper uses Q_k / P^disc_{k-1} and states that other
  inf-sup stable pairs work the same way).
* Time transfers between DG(r_c) and DG(r_f) on one slab: interpolation of the coarse temporal
  polynomial at the fine temporal nodes; restriction its transpose; space-time transfers are the
  tensor products P_tau (x) P_h (Section 4).
"""
import numpy as np
import scipy.sparse as sp
from numpy.polynomial import legendre as Leg

from . import assemble, fe, forms


def radau_right(Q):
    """The Q right Gauss--Radau points on [0, 1] (the last one is 1)."""
    if Q == 1:
        return np.array([1.0])
    # roots of P_Q - P_{Q-1} on [-1, 1]
    c = np.zeros(Q + 1)
    c[Q] = 1.0
    c[Q - 1] = -1.0
    x = np.sort(Leg.legroots(c).real)
    t = 0.5 * (x + 1.0)
    t[-1] = 1.0
    return t


def temporal_matrices(r):
    """(nodes, M_Q, A_Q, m_Q) of DG(r) on the reference slab [0, 1]."""
    Q = r + 1
    t = radau_right(Q)
    xg, wg = fe.gauss(Q + 1)                       # exact for degree 2Q + 1
    phi = np.array([[fe.lagrange_value(t, i, s) for s in xg] for i in range(Q)])          # (Q, ng)
    dphi = np.array([[_lagrange_deriv(t, i, s) for s in xg] for i in range(Q)])
    M = np.einsum("ig,jg,g->ji", phi, phi, wg)
    phi0 = np.array([fe.lagrange_value(t, i, 0.0) for i in range(Q)])
    A = np.einsum("ig,jg,g->ji", dphi, phi, wg) + np.outer(phi0, phi0)
    return t, M, A, phi0


def _lagrange_deriv(nodes, a, x):
    """Derivative of the Lagrange polynomial a of the nodes at x (product rule)."""
    s = 0.0
    for m in range(len(nodes)):
        if m == a:
            continue
        term = 1.0 / (nodes[a] - nodes[m])
        for q in range(len(nodes)):
            if q != a and q != m:
                term *= (x - nodes[q]) / (nodes[a] - nodes[q])
        s += term
    return s


def time_prolongation(rc, rf):
    """P_tau (Q_f x Q_c): the coarse DG(rc) temporal polynomial at the fine DG(rf) nodes."""
    tc = radau_right(rc + 1)
    tf = radau_right(rf + 1)
    return np.array([[fe.lagrange_value(tc, j, s) for j in range(rc + 1)] for s in tf])


class SpaceTimeStokes:
    """One slab of the transient Stokes equations: Taylor--Hood Q_k/Q_{k-1} on a forest, DG(r) in
    time.  Vectors are stage-major: Q blocks of the spatial Stokes vector."""

    def __init__(self, forest, k, r, nu=1.0, tau=0.1):
        self.space = assemble.Problem(forest, "stokes", k, nu=nu)
        self.r, self.Q, self.tau, self.nu = r, r + 1, tau, nu
        self.nodes, self.M_Q, self.A_Q, self.m_Q = temporal_matrices(r)
        self.G_Q = np.linalg.solve(self.M_Q, self.A_Q)
        self.A = self.space.assemble()                    # Stokes operator, identity constrained rows
        self.M = self._velocity_mass()
        self.n = self.A.shape[0]

    def _velocity_mass(self):
        """Stokes block mass: the velocity mass on the free velocity rows, zero elsewhere."""
        sp_ = self.space
        d = sp_.dofs
        dim, k = sp_.dim, sp_.k
        h = sp_.forest.h()
        Me = forms.scalar_mass(dim, k, k + 1, h)          # (nc, nb, nb)
        nb = Me.shape[1]
        ns = d.nodesets[0]
        rows, cols, vals = [], [], []
        for comp in range(dim):
            cd = d.offsets[0] + comp * ns.n_nodes + ns.cell_nodes        # (nc, nb)
            rows.append(np.repeat(cd[:, :, None], nb, axis=2).ravel())
            cols.append(np.repeat(cd[:, None, :], nb, axis=1).ravel())
            vals.append(Me.ravel())
        K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(d.n_dofs, d.n_dofs))
        Mf = (d.C.T @ K @ d.C).tocsr()
        P = sp.csr_matrix((np.ones(len(d.free_ids)), (d.free_ids, np.arange(len(d.free_ids)))),
                          shape=(d.n_dofs, len(d.free_ids)))
        return (P @ Mf @ P.T).tocsr()

    def operator(self):
        """K = G_Q (x) M + tau I_Q (x) A, with identity rows for constrained spatial entries."""
        Q = self.Q
        K = sp.kron(sp.csr_matrix(self.G_Q), self.M) + self.tau * sp.kron(sp.identity(Q), self.A)
        return K.tocsr()

    def rhs(self, f, u_prev, t0=0.0):
        """Mass-scaled right-hand side (M_Q^{-1} (x) I)(F + (m_Q (x) M) u_prev) on the free rows, for a
        spatial load f(t) -> vector (Gauss quadrature in time with Q + 2 points) and the previous
        slab's end value u_prev; constrained rows are zero (see ``set_constrained``)."""
        Q, tau = self.Q, self.tau
        xg, wg = fe.gauss(Q + 2)
        phi = np.array([[fe.lagrange_value(self.nodes, j, s) for s in xg] for j in range(Q)])
        F = np.zeros((Q, self.n))
        for g, (s, w) in enumerate(zip(xg, wg)):
            fv = f(t0 + s * tau)
            for j in range(Q):
                F[j] += tau * w * phi[j, g] * fv
        B = F + np.outer(self.m_Q, self.M @ u_prev)
        out = np.linalg.solve(self.M_Q, B)                # mass scaling, stage by stage
        out[:, self.space.dofs.constrained] = 0.0
        return out.ravel()

    def set_constrained(self, b, stage_values):
        """Constrained rows of K are tau times identity rows: b's constrained entries of stage q become
        tau * stage_values[q] (prescribed values of those entries)."""
        con = self.space.dofs.constrained
        bb = b.reshape(self.Q, self.n)
        for q in range(self.Q):
            bb[q, con] = self.tau * stage_values[q][con]
        return bb.ravel()
