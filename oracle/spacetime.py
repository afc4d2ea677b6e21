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

    def __init__(self, forest, k, r, nu=1.0, tau=0.1, pressure="continuous"):
        """pressure: 'continuous' (Taylor--Hood Q_k/Q_{k-1}) or 'disc' (Q_k/P^disc_{k-1})."""
        from . import pdisc
        self.pressure = pressure
        if pressure == "disc":
            self.space = pdisc.StokesPdisc(forest, k, nu=nu)
        else:
            self.space = assemble.Problem(forest, "stokes", k, nu=nu)
        self.r, self.Q, self.tau, self.nu = r, r + 1, tau, nu
        self.nodes, self.M_Q, self.A_Q, self.m_Q = temporal_matrices(r)
        self.G_Q = np.linalg.solve(self.M_Q, self.A_Q)
        self.A = self.space.assemble()                    # Stokes operator, identity constrained rows
        self.M = self.space.velocity_mass() if pressure == "disc" else self._velocity_mass()
        self.n = self.A.shape[0]

    def pressure_null(self):
        """The constant pressure of one stage (null direction of A with all-Dirichlet velocity)."""
        if self.pressure == "disc":
            return self.space.pressure_null()
        e = np.zeros(self.n)
        e[self.space.pressure_dofs()] = 1.0
        return e

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


# -- space-time multigrid (hp-STMG, Section 4) ----------------------------------------------------
class StLevel:
    """One level: the slab operator, the transfer from the next coarser level, and the patches of the
    space-time Schwarz smoother over all stages of the slab -- 'cell': one spatial cell (its free
    velocity and pressure DoFs); 'vertex': the cells around one mesh vertex (the free DoFs whose
    node lies inside that star, i.e. every cell holding the node is in the star)."""

    def __init__(self, forest, k, r, nu, tau, patch="vertex", pressure="continuous"):
        self.k, self.r = k, r
        self.st = SpaceTimeStokes(forest, k, r, nu=nu, tau=tau, pressure=pressure)
        self.K = self.st.operator()
        self.P = None
        st = self.st
        d = st.space.dofs
        cd = st.space.cell_dofs                                  # (nc, n_local)
        n, Q = st.n, st.Q
        self.patches, self.inv = [], []
        mult = np.zeros(Q * n)
        Kd = self.K.tocsr()
        for loc in _patch_dofs(st.space, patch):
            idx = (np.arange(Q)[:, None] * n + loc[None, :]).ravel()
            Kp = Kd[idx][:, idx].toarray()
            self.patches.append(idx)
            try:
                self.inv.append(np.linalg.inv(Kp))
            except np.linalg.LinAlgError:      # a patch holding every pressure DoF: constant pressure null
                self.inv.append(np.linalg.pinv(Kp))
            mult[idx] += 1.0
        self.weight = np.where(mult > 0, 1.0 / np.maximum(mult, 1.0), 0.0)
        con = np.zeros((Q, n), dtype=bool)
        con[:, d.constrained] = True
        self.con = con.ravel()

    def schwarz(self, r):
        """Weighted additive Schwarz: sum of the patch solves, each entry divided by the number of
        patches that hold it; constrained rows (tau times identity) solved exactly."""
        z = np.zeros_like(r)
        for idx, Ki in zip(self.patches, self.inv):
            z[idx] += Ki @ r[idx]
        z *= self.weight
        z[self.con] = r[self.con] / self.st.tau
        return z


def _patch_dofs(problem, patch):
    """Free DoFs of every smoother patch (arrays of spatial DoF indices)."""
    d = problem.dofs
    cd = problem.cell_dofs
    if patch == "cell":
        return [np.unique(cd[c][d.free[cd[c]]]) for c in range(cd.shape[0])]
    # vertex stars: cells holding each vertex of the mesh (vertices = nodes of the Q1 space)
    f = problem.forest
    dim = f.dim
    corners = fe.tensor_index(dim, 2)
    h, org = f.h(), f.origin()
    key = lambda x: tuple(np.rint(np.asarray(x) * 2 ** 30).astype(np.int64))
    star = {}
    for c in range(f.n_cells):
        for cr in corners:
            star.setdefault(key(org[c] + cr * h[c]), []).append(c)
    # cells holding each DoF
    holders = [set() for _ in range(d.n_dofs)]
    for c in range(f.n_cells):
        for g in cd[c]:
            holders[g].add(c)
    out = []
    for cells in star.values():
        cs = set(cells)
        loc = sorted({g for c in cells for g in cd[c] if d.free[g] and holders[g] <= cs})
        if loc:
            out.append(np.array(loc))
    return out


def _star_covers_all(forest):
    """Whether some vertex star (the cells having one vertex as a corner) holds every cell."""
    corners = fe.tensor_index(forest.dim, 2)
    h, org = forest.h(), forest.origin()
    count = {}
    for c in range(forest.n_cells):
        for cr in corners:
            key = tuple(np.rint((org[c] + cr * h[c]) * 2 ** 30).astype(np.int64))
            count[key] = count.get(key, 0) + 1
    return max(count.values()) == forest.n_cells


def stmg_levels(forest, k, r, nu=1.0, tau=0.1, stop_n=2, patch=None, pressure="disc"):
    """Levels finest first.  Section 4's rules -- coarsen in space before time (R1), and in each of
    them polynomially before geometrically (R2: p before h, the temporal degree before tau) -- give:
    the spatial degree halved (k >= 2 kept: Q2 is the lowest stable velocity for both pairs), then
    global h-coarsening in space down to stop_n, then the temporal degree halved (DG(r) ->
    DG(r // 2)) on the coarsest mesh; no geometric coarsening in time (time-marching).  Temporal
    steps are left out when a vertex star of the coarsest mesh holds every cell (with vertex-star
    patches that patch would hold every unknown and be singular); the coarsest level is then solved
    at the fine temporal degree.  Patches: one cell for the discontinuous pressure (the paper's pair:
    every pressure DoF belongs to one cell), vertex stars for the continuous one (a cell patch would
    cut the pressure coupling; a vertex star of a discontinuous pressure holds a pressure constant as
    a local null mode)."""
    if patch is None:
        patch = "cell" if pressure == "disc" else "vertex"
    from . import solvers, transfer
    seq = [(forest, k, r)]
    while seq[-1][1] > 2:
        seq.append((forest, max(2, seq[-1][1] // 2), seq[-1][2]))
    for fc in solvers.coarse_forests(forest, stop_n)[1:]:
        seq.append((fc, seq[-1][1], seq[-1][2]))
    if not (patch == "vertex" and _star_covers_all(seq[-1][0])):
        while seq[-1][2] > 0:
            seq.append((seq[-1][0], seq[-1][1], seq[-1][2] // 2))
    levels = [StLevel(f, kk, rr, nu, tau, patch, pressure) for f, kk, rr in seq]
    for l in range(len(levels) - 1):
        fine, coarse = levels[l], levels[l + 1]
        if fine.r != coarse.r:                                   # temporal p-step: P_tau (x) I
            Pt = time_prolongation(coarse.r, fine.r)
            fine.P = sp.kron(sp.csr_matrix(Pt), sp.identity(fine.st.n)).tocsr()
        else:                                                     # spatial step: I_Q (x) P_h
            if pressure == "disc":
                from . import pdisc
                Ph = pdisc.prolongation(coarse.st.space, fine.st.space)
            else:
                Ph = transfer.prolongation(coarse.st.space, fine.st.space)
            fine.P = sp.kron(sp.identity(fine.st.Q), Ph).tocsr()
    return levels


class STMG:
    """One V-cycle of space-time multigrid: `nu_s` damped weighted Schwarz steps (damping omega)
    before and after the coarse correction, a direct solve on the coarsest level (least squares: the
    pressure constant of every stage is a null direction).

    Readings (the paper gives neither the damping nor the number of steps): omega = 0.7, nu_s = 4;
    patches as chosen by ``stmg_levels``.  Undamped, the weighted additive Schwarz iteration has spectral radius
    about 1.8 on Taylor--Hood; with Taylor--Hood's continuous pressure, cell patches (the paper's
    choice for a discontinuous pressure) need omega <= 0.5 and give iteration counts that grow
    under refinement, vertex stars do far less so."""

    def __init__(self, levels, nu_s=4, omega=0.7):
        self.levels, self.nu_s, self.omega = levels, nu_s, omega
        # pseudo-inverse with an explicit cutoff: the null singular values (one constant pressure per
        # stage) come out of the SVD at 1e-19..1e-15 relative, above numpy's default cutoff in some
        # builds, while the smallest non-null ones sit near 1e-5 relative
        self.coarse = np.linalg.pinv(levels[-1].K.toarray(), rcond=1e-10)

    def __call__(self, b, l=0):
        lv = self.levels[l]
        if l == len(self.levels) - 1:
            return self.coarse @ b
        x = np.zeros_like(b)
        for _ in range(self.nu_s):
            x = x + self.omega * lv.schwarz(b - lv.K @ x)
        xc = self(lv.P.T @ (b - lv.K @ x), l + 1)
        x = x + lv.P @ xc
        for _ in range(self.nu_s):
            x = x + self.omega * lv.schwarz(b - lv.K @ x)
        return x

    def project(self, v):
        """Remove the constant pressure of every stage (the null space of K and K^T)."""
        lv = self.levels[0]
        e = lv.st.pressure_null()
        out = np.array(v, dtype=float, copy=True).reshape(lv.st.Q, lv.st.n)
        for q in range(lv.st.Q):
            out[q] -= (out[q] @ e) / (e @ e) * e
        return out.ravel()
