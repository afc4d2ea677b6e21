"""Element matrices by direct quadrature (no sum factorisation).

Oracle (test infrastructure only).  Every basis function's value, gradient
and Laplacian is evaluated at every Gauss point of an axis-aligned cell
x = x0 + h * xi, so grad = grad_xi / h, Laplacian = sum of second reference
derivatives / h^2 and the quadrature weight is w * h^dim.

Cell-local DoF order: field by field, component by component, node by node
(lexicographic, x fastest).

Forms (symbols as in the paper):
* vector Laplacian (the A block of Eq. 5):  nu (grad u, grad v)
* Stokes, Eq. 1 with Taylor--Hood Q_k / Q_{k-1}:
      nu (grad u, grad v) - (p, div v) + s (div u, q)
  s = +1 is Eq. 1 as printed; s = -1 gives the symmetric form of Eq. 5
  ([[A, B], [B^T, 0]]), which is the default reading for Stokes.
* pressure mass (p, q) on the pressure space (Schur complement of Eq. 5).
* stabilised Navier--Stokes, Eq. 3 with the SUPG and PSPG terms of Section 5
  and BDF2 in time, linearised by Newton's method at a frozen state (ub, pb)
  with the stabilisation parameter tau frozen:
      Galerkin:  (c_m du + ub.grad du + du.grad ub, v) + nu (grad du, grad v)
                 - (dp, div v) + s (div du, q)
      SUPG:      tau (Rlin, ub.grad v) + tau (Rbar, du.grad v)
      PSPG:      tau (Rlin, grad q)
  with c_m = 3/(2 dt) (BDF2, constant step, history equal to the frozen
  state), Rlin = c_m du + ub.grad du + du.grad ub + grad dp - nu lap du,
  Rbar = ub.grad ub + grad pb - nu lap ub and
  tau = [(2/dt)^2 + (2|ub|/h)^2 + 9 (4 nu / h^2)^2]^(-1/2) (Tezduyar), h the
  cell edge length.  s = +1 (Eq. 3 as printed).
"""
import numpy as np

from . import fe

TERM_MASS = 1
TERM_CONV = 2
TERM_NEWTON = 4
TERM_SUPG = 8
TERM_SUPG_NEWTON = 16
TERM_PSPG = 32
TERM_STRONG_VISC = 64
TERMS_ALL = 127


def tau_formula(unorm, h, nu, dt):
    """Tezduyar's stabilisation parameter; dt = inf drops the transient part."""
    inv_dt = 0.0 if not np.isfinite(dt) else 1.0 / dt
    return 1.0 / np.sqrt((2.0 * inv_dt) ** 2 + (2.0 * unorm / h) ** 2 + 9.0 * (4.0 * nu / h ** 2) ** 2)


class CellTables:
    """Physical basis tables of Q_k at the q^dim Gauss points of cells of edge h."""

    def __init__(self, dim, k, q, h):
        phi, dphi, d2phi, w, xq = fe.reference_tables(dim, k, q)
        h = np.asarray(h, dtype=float).reshape(-1)
        self.dim, self.k, self.q = dim, k, q
        self.phi = phi                                              # (nq, nb)
        self.grad = dphi[None] / h[:, None, None, None]             # (nc, nq, nb, dim)
        self.lap = d2phi.sum(axis=2)[None] / h[:, None, None] ** 2  # (nc, nq, nb)
        self.JxW = w[None, :] * h[:, None] ** dim                   # (nc, nq)
        self.xq = xq
        self.nb = phi.shape[1]


def vector_laplacian(dim, k, nu, h):
    """(nc, dim*nb, dim*nb) element matrices of nu (grad u, grad v)."""
    t = CellTables(dim, k, k + 1, h)
    lap = nu * np.einsum("cq,cqad,cqbd->cab", t.JxW, t.grad, t.grad)
    nc, nb = lap.shape[0], t.nb
    out = np.zeros((nc, dim * nb, dim * nb))
    for c in range(dim):
        out[:, c * nb:(c + 1) * nb, c * nb:(c + 1) * nb] = lap
    return out


def scalar_mass(dim, k, q, h):
    """(nc, nb, nb) element mass matrices (phi_b, phi_a) with q^dim Gauss points."""
    t = CellTables(dim, k, q, h)
    return np.einsum("cq,qa,qb->cab", t.JxW, t.phi, t.phi)


def stokes_taylor_hood(dim, k, nu, h, div_sign=-1.0, kp=None):
    """(nc, n, n) element matrices of Eq. 1 on Q_k^dim / Q_kp (Taylor--Hood: kp = k-1),
    n = dim*nb_u + nb_p."""
    kp = k - 1 if kp is None else kp
    tu = CellTables(dim, k, k + 1, h)
    tp = CellTables(dim, kp, k + 1, h)
    nbu, nbp = tu.nb, tp.nb
    nc = tu.JxW.shape[0]
    n = dim * nbu + nbp
    out = np.zeros((nc, n, n))
    lap = nu * np.einsum("cq,cqad,cqbd->cab", tu.JxW, tu.grad, tu.grad)
    P = dim * nbu
    for i in range(dim):
        out[:, i * nbu:(i + 1) * nbu, i * nbu:(i + 1) * nbu] = lap
        # -(p, d_i v): test velocity component i, trial pressure
        b = -np.einsum("cq,cqa,qb->cab", tu.JxW, tu.grad[..., i], tp.phi)
        out[:, i * nbu:(i + 1) * nbu, P:] = b
        # s (d_i u, q): test pressure, trial velocity component i
        out[:, P:, i * nbu:(i + 1) * nbu] = div_sign * np.einsum("cq,qa,cqb->cab", tu.JxW, tp.phi, tu.grad[..., i])
    return out


def frozen_at_qp(t, ub_loc, pb_loc):
    """Frozen state at the Gauss points from cell-local nodal values.

    ub_loc (nc, dim, nb), pb_loc (nc, nb).  Returns U (nc,nq,dim),
    G (nc,nq,dim,dim) with G[..., i, j] = d_j ub_i, lap U (nc,nq,dim), grad pb (nc,nq,dim)."""
    U = np.einsum("qb,cib->cqi", t.phi, ub_loc)
    G = np.einsum("cqbj,cib->cqij", t.grad, ub_loc)
    LU = np.einsum("cqb,cib->cqi", t.lap, ub_loc)
    GP = np.einsum("cqbj,cb->cqj", t.grad, pb_loc)
    return U, G, LU, GP


def stabilized_ns(dim, k, h, ub_loc, pb_loc, nu, dt, terms=TERMS_ALL, div_sign=1.0, alpha=1.5, g_loc=None):
    """(nc, n, n) Newton-linearised SUPG/PSPG BDF2 element matrices on Q_k^dim Q_k, n = (dim+1) nb.

    Local order: velocity components 0..dim-1 then pressure, each over the nb nodes.
    g_loc (nc, dim, nb): nodal explicit part of the time derivative and forcing (see
    ``stabilized_ns_residual``); it enters Rbar as c_m ub + g.  Without it the frozen state's
    history equals the state, so the time derivative in Rbar vanishes."""
    t = CellTables(dim, k, k + 1, h)
    h = np.asarray(h, dtype=float).reshape(-1)
    nb = t.nb
    nc = t.JxW.shape[0]
    m = 1.0 if terms & TERM_MASS else 0.0
    cv = 1.0 if terms & TERM_CONV else 0.0
    nw = 1.0 if terms & TERM_NEWTON else 0.0
    su = 1.0 if terms & TERM_SUPG else 0.0
    sn = 1.0 if terms & TERM_SUPG_NEWTON else 0.0
    ps = 1.0 if terms & TERM_PSPG else 0.0
    lv = 1.0 if terms & TERM_STRONG_VISC else 0.0
    cm = alpha / dt if np.isfinite(dt) else 0.0

    U, G, LU, GP = frozen_at_qp(t, ub_loc, pb_loc)
    tau = tau_formula(np.linalg.norm(U, axis=2), h[:, None], nu, dt)      # (nc, nq)
    Rbar = np.einsum("cqj,cqij->cqi", U, G) + GP - nu * LU                # (nc, nq, dim)
    if g_loc is not None:
        Rbar = Rbar + cm * U + np.einsum("qb,cib->cqi", t.phi, g_loc)
    W = t.JxW
    phi, g, lap = t.phi, t.grad, t.lap
    Ug = np.einsum("cqd,cqbd->cqb", U, g)                                 # ub . grad phi_b
    # scalar (component-diagonal) part of Rlin for a velocity trial function
    S = m * cm * phi[None] + cv * Ug - lv * nu * lap                      # (nc, nq, nb)

    n = (dim + 1) * nb
    K = np.zeros((nc, n, n))
    P = dim * nb
    mass = np.einsum("cq,qa,qb->cab", W, phi, phi)
    conv = np.einsum("cq,qa,cqb->cab", W, phi, Ug)
    visc = nu * np.einsum("cq,cqad,cqbd->cab", W, g, g)
    supg_S = np.einsum("cq,cqa,cqb->cab", W * tau, Ug, S)                  # tau (S_b, ub.grad phi_a)
    for i in range(dim):
        for j in range(dim):
            blk = nw * np.einsum("cq,qa,qb,cq->cab", W, phi, phi, G[:, :, i, j])
            blk += su * nw * np.einsum("cq,cqa,qb,cq->cab", W * tau, Ug, phi, G[:, :, i, j])
            blk += sn * np.einsum("cq,cq,qb,cqa->cab", W * tau, Rbar[:, :, i], phi, g[:, :, :, j])
            if i == j:
                blk += m * cm * mass + cv * conv + visc + su * supg_S
            K[:, i * nb:(i + 1) * nb, j * nb:(j + 1) * nb] = blk
        # test velocity i, trial pressure: -(dp, d_i v) + tau (d_i dp, ub.grad v)
        K[:, i * nb:(i + 1) * nb, P:] = (-np.einsum("cq,cqa,qb->cab", W, g[..., i], phi)
                                         + su * np.einsum("cq,cqa,cqb->cab", W * tau, Ug, g[..., i]))
    for j in range(dim):
        # test pressure, trial velocity j: s (d_j du_j, q) + tau (Rlin, grad q)
        blk = div_sign * np.einsum("cq,qa,cqb->cab", W, phi, g[..., j])
        blk += ps * np.einsum("cq,cqa,cqb->cab", W * tau, g[..., j], S)
        blk += ps * nw * np.einsum("cq,cqai,cqi,qb->cab", W * tau, g, G[:, :, :, j], phi)
        K[:, P:, j * nb:(j + 1) * nb] = blk
    K[:, P:, P:] = ps * np.einsum("cq,cqad,cqbd->cab", W * tau, g, g)
    return K


def stabilized_ns_residual(dim, k, h, u_loc, p_loc, nu, dt, g_loc=None, div_sign=1.0, alpha=1.5, tau_u_loc=None):
    """(nc, (dim+1) nb) element residual vectors of the SUPG/PSPG BDF discretisation of the
    incompressible Navier--Stokes equations (Section 5) at the discrete state (u, p).

    The time derivative at t^{n+1} is (alpha u + sum_j beta_j u^{n-j}) / dt; its explicit part
    and the forcing are passed as one nodal field g = sum_j beta_j u^{n-j} / dt - f_h, so that the
    strong momentum residual is R = c_m u + g + u.grad u + grad p - nu lap u, c_m = alpha / dt
    (g absent: R without the time derivative, as for the frozen state).  Residual, per test
    function (v, q):
      (c_m u + g + u.grad u, v) + nu (grad u, grad v) - (p, div v) + (tau R, u.grad v)
      + s (div u, q) + (tau R, grad q),
    with tau (Tezduyar) from |u| at the point, or from the field tau_u_loc when given (tau frozen
    at another state: the Jacobian of this residual at that state is the linearised operator)."""
    t = CellTables(dim, k, k + 1, h)
    h = np.asarray(h, dtype=float).reshape(-1)
    nb = t.nb
    nc = t.JxW.shape[0]
    cm = alpha / dt if np.isfinite(dt) else 0.0
    U, G, LU, GP = frozen_at_qp(t, u_loc, p_loc)
    P = np.einsum("qb,cb->cq", t.phi, p_loc)
    if g_loc is None:
        Tt = np.zeros_like(U)
    else:
        Tt = cm * U + np.einsum("qb,cib->cqi", t.phi, g_loc)
    conv = np.einsum("cqj,cqij->cqi", U, G)
    R = Tt + conv + GP - nu * LU
    Ut = U if tau_u_loc is None else np.einsum("qb,cib->cqi", t.phi, tau_u_loc)
    tau = tau_formula(np.linalg.norm(Ut, axis=2), h[:, None], nu, dt)
    W = t.JxW
    phi, g = t.phi, t.grad
    Ug = np.einsum("cqd,cqbd->cqb", U, g)                                 # u . grad phi_a
    F = np.zeros((nc, (dim + 1) * nb))
    for i in range(dim):
        Fi = np.einsum("cq,cq,qa->ca", W, Tt[:, :, i] + conv[:, :, i], phi)
        Fi += nu * np.einsum("cq,cqd,cqad->ca", W, G[:, :, i, :], g)
        Fi -= np.einsum("cq,cq,cqa->ca", W, P, g[..., i])
        Fi += np.einsum("cq,cq,cqa->ca", W * tau, R[:, :, i], Ug)
        F[:, i * nb:(i + 1) * nb] = Fi
    div = np.einsum("cqii->cq", G)
    F[:, dim * nb:] = (div_sign * np.einsum("cq,cq,qa->ca", W, div, phi)
                       + np.einsum("cq,cqd,cqad->ca", W * tau, R, g))
    return F


def taylor_green(dim):
    """Frozen Taylor--Green state (u_1..u_dim, p) as a function of points (npts, dim)."""
    tp = 2.0 * np.pi

    def f(x):
        out = np.zeros((x.shape[0], dim + 1))
        if dim == 3:
            X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
            out[:, 0] = np.sin(tp * X) * np.cos(tp * Y) * np.cos(tp * Z)
            out[:, 1] = -np.cos(tp * X) * np.sin(tp * Y) * np.cos(tp * Z)
            out[:, 2] = 0.0
            out[:, 3] = (np.cos(2 * tp * X) + np.cos(2 * tp * Y)) * (np.cos(2 * tp * Z) + 2.0) / 16.0
        else:
            X, Y = x[:, 0], x[:, 1]
            out[:, 0] = np.sin(tp * X) * np.cos(tp * Y)
            out[:, 1] = -np.cos(tp * X) * np.sin(tp * Y)
            out[:, 2] = (np.cos(2 * tp * X) + np.cos(2 * tp * Y)) / 16.0
        return out

    return f
