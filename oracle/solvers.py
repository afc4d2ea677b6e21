"""Smoothers, V-cycle, FGMRES and the block-triangular Stokes preconditioner.

Oracle (test infrastructure only), written plainly on assembled sparse
matrices in float64.

Readings of the paper (Sections 2, 3 and 5):
* Chebyshev smoothing around point Jacobi (Section 3, degree 5; degree 3 for
  the stabilised operator here): the three-term recurrence of Saad,
  "Iterative Methods for Sparse Linear Systems", Alg. 12.1, applied to
  D^{-1} A with theta = (lmax + lmin)/2, delta = (lmax - lmin)/2.  The degree
  is the number of operator applications (one fewer from a zero start).
  lmin = lmax / 20.
* Relaxation around point Jacobi (Section 5, Exp. 3): x <- x + w D^{-1} (b - A x)
  with w = 2 / (lmin + lmax).
* Hierarchy: uniform meshes coarsen n -> ceil(n/2) while n > 2 (non-nested
  for odd n, Section 2); the coarsest level is therefore tiny.
* Coarse solver: direct (dense) solve; a pressure null space (constant
  pressure with all-Dirichlet velocity) is removed by adding e e^T, e the
  normalised indicator of the free pressure DoFs.
* V-cycle (Section 3: A^{-1} ~ one V-cycle): pre-smooth from zero, residual,
  restrict (transpose of the prolongation), recurse, prolongate-add,
  post-smooth.
* FGMRES(m) (Section 3): right-preconditioned flexible GMRES, restart m,
  classical Gram--Schmidt applied twice, Givens rotations, zero start; stop
  when ||b - A x|| <= tol ||b||, the true residual being recomputed at every
  restart.  With a pressure null space, b and every preconditioned vector are
  projected to zero l2 pressure mean.
* Block-triangular preconditioner of Eq. 5 with S ~ nu^{-1} M_p:
  z_p = -nu M_p^{-1} r_p by a fixed number (10) of Jacobi-preconditioned CG
  steps from zero, z_u = V-cycle(A, r_u - B z_p).
"""
import numpy as np
import scipy.sparse as sp

from . import assemble, mesh, transfer


# -- smoothers -------------------------------------------------------------------
def _prec(dinv):
    """The smoother's preconditioner: a diagonal inverse (array, applied pointwise) or a callable."""
    return dinv if callable(dinv) else (lambda r: dinv * r)


def chebyshev(A, dinv, b, x, degree, lmax, lmin=None, x_is_zero=False):
    P = _prec(dinv)
    lmin = lmax / 20.0 if lmin is None else lmin
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    x = np.array(x, dtype=float, copy=True)
    r = b.copy() if x_is_zero else b - A @ x
    d = P(r) / theta
    x += d
    rho_old = 1.0 / sigma
    for _ in range(1, degree):
        r = b - A @ x
        rho = 1.0 / (2.0 * sigma - rho_old)
        d = rho * rho_old * d + (2.0 * rho / delta) * P(r)
        x += d
        rho_old = rho
    return x


def jacobi_relaxation(A, dinv, b, x, iterations, lmax, lmin=None):
    P = _prec(dinv)
    lmin = lmax / 20.0 if lmin is None else lmin
    omega = 2.0 / (lmin + lmax)
    x = np.array(x, dtype=float, copy=True)
    for _ in range(iterations):
        x += omega * P(b - A @ x)
    return x


def cg_jacobi_fixed(M, dinv, b, iterations):
    """Fixed number of Jacobi-preconditioned CG steps from zero."""
    x = np.zeros_like(b)
    r = b.copy()
    z = dinv * r
    p = z.copy()
    rz = r @ z
    for _ in range(iterations):
        if rz == 0.0:
            break
        q = M @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        z = dinv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x


# -- hierarchy -------------------------------------------------------------------
def coarse_forests(forest, stop_n=2):
    """Global-coarsening sequence of meshes, finest first; uniform meshes are
    coarsened to ceil(n/2) cells per direction while n > stop_n."""
    out = [forest]
    f = forest
    while True:
        if f.max_level == 0 and f.n <= stop_n:
            break
        f = f.coarsen_finest()
        out.append(f)
    return out


class Level:
    def __init__(self, problem):
        self.problem = problem
        self.A = problem.assemble()
        self.dinv = 1.0 / self.A.diagonal()
        self.P = None            # prolongation from the next coarser level to this one
        self.lmax = None


def hierarchy(forest, kind, k, order=None, stop_n=2, **params):
    """Levels (finest first).  Stokes A block: p-coarsening to k = 1 first, then h
    (Section 3).  Stabilised NS: h-coarsening first, then p (Section 5)."""
    if order is None:
        order = "h_then_p" if kind == "stab_ns" else "p_then_h"
    seq = []
    if order == "p_then_h":
        for kk in range(k, 0, -1):
            seq.append((forest, kk))
        for f in coarse_forests(forest, stop_n)[1:]:
            seq.append((f, 1))
    else:
        fs = coarse_forests(forest, stop_n)
        for f in fs:
            seq.append((f, k))
        for kk in range(k - 1, 0, -1):
            seq.append((fs[-1], kk))
    levels = [Level(assemble.Problem(f, kind, kk, **params)) for f, kk in seq]
    for l in range(len(levels) - 1):
        levels[l].P = transfer.prolongation(levels[l + 1].problem, levels[l].problem)
    return levels


def coarse_matrix(problem, A):
    """Dense coarse matrix, regularised by e e^T when the pressure is only fixed up to a constant."""
    Ad = A.toarray()
    ids = problem.pressure_dofs()
    if len(ids):
        e = np.zeros(A.shape[0])
        e[ids] = 1.0 / np.sqrt(len(ids))
        Ad = Ad + np.outer(e, e)
    return Ad


class VCycle:
    """Smoother per level: ('chebyshev', degree) or ('jacobi', iterations); lmax per level given."""

    def __init__(self, levels, lmax, smoother=("chebyshev", 5)):
        self.levels = levels
        for lv, lm in zip(levels[:-1], lmax):
            lv.lmax = lm
        self.smoother = smoother
        self.coarse = np.linalg.inv(coarse_matrix(levels[-1].problem, levels[-1].A))

    def smooth(self, lv, b, x, x_is_zero):
        kind, deg = self.smoother
        if kind == "chebyshev":
            return chebyshev(lv.A, lv.dinv, b, x, deg, lv.lmax, x_is_zero=x_is_zero)
        return jacobi_relaxation(lv.A, lv.dinv, b, x, deg, lv.lmax)

    def __call__(self, b, l=0):
        lv = self.levels[l]
        if l == len(self.levels) - 1:
            return self.coarse @ b
        x = self.smooth(lv, b, np.zeros_like(b), True)
        r = b - lv.A @ x
        xc = self(lv.P.T @ r, l + 1)
        x = x + lv.P @ xc
        return self.smooth(lv, b, x, False)


# -- Krylov --------------------------------------------------------------------------
def fgmres(A, b, M, tol=1e-8, restart=30, maxit=1000, project=None):
    """Flexible GMRES with right preconditioning M (callable); returns (x, iterations, relres)."""
    proj = (lambda v: v) if project is None else project
    b = proj(b)
    n = b.shape[0]
    x = np.zeros(n)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    r = b - A @ x
    it = 0
    while True:
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm or it >= maxit:
            return x, it, beta / bnorm
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(restart):
            Z[j] = proj(M(V[j]))
            w = A @ Z[j]
            h1 = V[: j + 1] @ w
            w = w - V[: j + 1].T @ h1
            h2 = V[: j + 1] @ w
            w = w - V[: j + 1].T @ h2
            H[: j + 1, j] = h1 + h2
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_done = j + 1
            if abs(g[j + 1]) <= tol * bnorm or it >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + Z[:j_done].T @ y
        r = b - A @ x


class StokesBlockPreconditioner:
    """Eq. 5: z_p = -nu M_p^{-1} r_p (10 Jacobi-CG steps), z_u = V-cycle(r_u - B z_p)."""

    def __init__(self, stokes_problem, A_stokes, vcycle_a, pmass_A, cg_iterations=10):
        self.sp = stokes_problem
        self.A = A_stokes
        self.vc = vcycle_a
        self.Mp = pmass_A
        self.dinv_p = 1.0 / pmass_A.diagonal()
        self.nu = stokes_problem.nu
        self.nu_dofs = stokes_problem.dofs.offsets[1]
        self.cg_iterations = cg_iterations

    def __call__(self, r):
        nu_dofs = self.nu_dofs
        rp = r[nu_dofs:]
        zp = -self.nu * cg_jacobi_fixed(self.Mp, self.dinv_p, rp, self.cg_iterations)
        full = np.zeros_like(r)
        full[nu_dofs:] = zp
        Bz = (self.A @ full)[:nu_dofs]
        zu = self.vc(r[:nu_dofs] - Bz)
        return np.concatenate([zu, zp])


def power_lmax(A, dinv, iterations=200, seed=1):
    """Largest eigenvalue magnitude of P^{-1} A by power iteration (P^{-1} a diagonal inverse or a
    callable; for oracle self-tests)."""
    P = _prec(dinv)
    rng = np.random.default_rng(seed)
    v = rng.uniform(-1, 1, A.shape[0])
    lam = 0.0
    for _ in range(iterations):
        w = P(A @ v)
        lam = np.linalg.norm(w) / np.linalg.norm(v)
        v = w / np.linalg.norm(w)
    return lam
