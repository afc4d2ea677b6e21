"""Newton's method and variable-step BDF2 for the stabilised Navier--Stokes problem.

Oracle (test infrastructure only), written plainly on assembled matrices in float64.

Readings of the paper (Section 5: BDF2 in time, the nonlinear system linearised by Newton's
method, each linear system solved by FGMRES preconditioned by the monolithic multigrid):
* Newton with tau frozen at the current iterate: J(U_k) dU = -F(U_k), U_{k+1} = U_k + dU, where
  F is ``forms.stabilized_ns_residual`` and J the linearised operator at the state U_k (all
  terms).  Here the linear systems are solved directly (the oracle checks the nonlinear
  iteration, not the Krylov solver).  Stop when ||F(U_k)|| <= max(atol, rtol ||F(U_0)||).
* Constrained entries: the increments vanish on Dirichlet and hanging rows; the hanging entries
  of the state follow their masters after every update; the pressure increment has zero mean.
* Variable-step BDF2 with ratio w = dt_n / dt_{n-1}:
    u'(t_{n+1}) ~ [ (1+2w)/(1+w) u^{n+1} - (1+w) u^n + w^2/(1+w) u^{n-1} ] / dt_n,
  i.e. alpha = (1+2w)/(1+w) and the explicit field g = [-(1+w) u^n + w^2/(1+w) u^{n-1}] / dt_n
  - f_h(t_{n+1}); w = 0 is BDF1 (implicit Euler).  The forcing enters through its nodal
  interpolant f_h.
* Time-step control by a CFL number: dt = CFL h_min / max_nodes |u|.
"""
import numpy as np

from . import assemble


def newton(problem, U0, g=None, rtol=1e-10, atol=1e-13, maxit=15):
    """Solve F(U) = 0 from U0; returns (U, residual norms per iterate)."""
    d = problem.dofs
    U = d.set_hanging(np.asarray(U0, dtype=float))
    hist = []
    for it in range(maxit + 1):
        problem.set_state(U, g)
        F = problem.residual()
        r = float(np.linalg.norm(F))
        hist.append(r)
        if r <= max(atol, rtol * hist[0]) or it == maxit:
            break
        dU = assemble.solve_direct(problem, -F, problem.assemble())
        dU[d.constrained] = 0.0
        U = d.set_hanging(U + dU)
    return U, hist


def bdf_coefficients(dt, omega):
    """(alpha, beta_n, beta_nm1): u' ~ (alpha u^{n+1} + beta_n u^n + beta_nm1 u^{n-1}) / dt."""
    if omega == 0.0:
        return 1.0, -1.0, 0.0
    return (1.0 + 2.0 * omega) / (1.0 + omega), -(1.0 + omega), omega * omega / (1.0 + omega)


def explicit_field(u_n, u_nm1, dt, omega, forcing=None):
    """g = (beta_n u^n + beta_nm1 u^{n-1}) / dt - f_h (DoF vectors; pressure entries unused)."""
    _, bn, bnm1 = bdf_coefficients(dt, omega)
    g = bn * np.asarray(u_n, dtype=float) / dt
    if bnm1 != 0.0:
        g = g + bnm1 * np.asarray(u_nm1, dtype=float) / dt
    if forcing is not None:
        g = g - forcing
    return g


def bdf_step(problem, u_n, u_nm1, dt, omega, guess, forcing=None, **newton_kw):
    """One BDF step: the state at t_{n+1} from u^n, u^{n-1} (omega = dt_n / dt_{n-1}, 0: BDF1).
    ``guess`` carries the Dirichlet values at t_{n+1}; returns (U, residual norms)."""
    alpha, _, _ = bdf_coefficients(dt, omega)
    problem.set_dt(dt, alpha)
    g = explicit_field(u_n, u_nm1, dt, omega, forcing)
    return newton(problem, guess, g, **newton_kw)


def cfl_dt(problem, U, cfl):
    """dt = cfl * h_min / max over velocity nodes of |u|."""
    n = problem.dofs.nodesets[0].n_nodes
    u = np.asarray(U, dtype=float)[: problem.dim * n].reshape(problem.dim, n)
    umax = float(np.sqrt((u * u).sum(axis=0)).max())
    return cfl * float(problem.forest.h().min()) / umax
