"""Thin Python layer over the C ABI (names follow include/mfns.h).

Torch tensors supply device memory and streams; every step of the path runs
in libmfns.so.  There is no CPU fallback: without the built library or a GPU
these calls raise.
"""
import ctypes as C

import numpy as np
import torch

from . import _lib as L


def _ptr(t):
    if not t.is_cuda:
        raise ValueError("vectors must be CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("vectors must be contiguous")
    return C.c_void_p(t.data_ptr())


def _vec(t, n=None, dtype=None, name="vector"):
    """Device pointer of a contiguous CUDA tensor after checking its length and dtype against what
    the call expects (the library checks the length again; the dtype it cannot see)."""
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} entries, expected {n}")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} is {t.dtype}, expected {dtype}")
    return _ptr(t)


def _prec_of(t):
    if t.dtype == torch.float64:
        return L.FP64
    if t.dtype == torch.float32:
        return L.FP32
    raise ValueError(f"vectors must be float64 or float32, got {t.dtype}")


def _f64(*ts):
    for t in ts:
        if t is not None and t.dtype != torch.float64:
            raise ValueError("state, explicit field, forcing and solution vectors must be float64")


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _dtype(prec):
    return torch.float64 if prec == L.FP64 else torch.float32


class Context:
    def __init__(self, device=0, hbm_budget_bytes=0):
        self.lib = L.load()
        h = C.c_void_p()
        L.check(self.lib.mfns_ctx_create(device, hbm_budget_bytes, C.byref(h)))
        self.h = h
        self.device = device

    def set_batching(self, enable):
        """Batched preconditioners in mfns_batch_step (default on)."""
        L.check(self.lib.mfns_ctx_set_batching(self.h, int(bool(enable))))

    def memory(self):
        u, p = C.c_size_t(), C.c_size_t()
        L.check(self.lib.mfns_ctx_memory(self.h, C.byref(u), C.byref(p)))
        return u.value, p.value

    def close(self):
        if self.h:
            self.lib.mfns_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    def __init__(self, ctx, dim, n):
        self.lib = ctx.lib
        h = C.c_void_p()
        L.check(self.lib.mfns_mesh_uniform(ctx.h, dim, n, C.byref(h)))
        self.h = h
        self.dim, self.n = dim, n

    def refine_ball(self, centre, radius, levels):
        c = (C.c_double * 3)(*[float(v) for v in (list(centre) + [0.0, 0.0, 0.0])[:3]])
        L.check(self.lib.mfns_mesh_refine_ball(self.h, c, float(radius), int(levels)))
        return self

    def info(self):
        n, l = C.c_int64(), C.c_int()
        L.check(self.lib.mfns_mesh_info(self.h, C.byref(n), C.byref(l)))
        return n.value, l.value

    def cells(self):
        """(n_cells, 4) int32: level, x, y, z of every active cell in the canonical order."""
        n = C.c_int64()
        L.check(self.lib.mfns_mesh_cells(self.h, None, 0, C.byref(n)))
        out = np.zeros((n.value, 4), dtype=np.int32)
        L.check(self.lib.mfns_mesh_cells(self.h, out.ctypes.data_as(C.c_void_p), n.value, C.byref(n)))
        return out

    def close(self):
        if self.h:
            self.lib.mfns_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_desc(kind, degree, nu=1.0, dt=0.0, terms=0, div_sign=0.0, smoother=0, smoother_degree=0,
              mg_order=0, mg_precision=L.FP64, coarse_stop_n=0, fgmres_restart=0, tol=0.0, maxit=0,
              cg_iterations=0, lambda_max=0.0, recompute_frozen=0, fused_smoother=0, hierarchy=0):
    return L.ProblemDesc(kind, degree, nu, dt, terms, div_sign, smoother, smoother_degree, mg_order,
                         mg_precision, coarse_stop_n, fgmres_restart, tol, maxit, cg_iterations, lambda_max,
                         recompute_frozen, int(bool(fused_smoother)), int(hierarchy))


class Problem:
    def __init__(self, ctx, mesh, degrees=None, **desc):
        """degrees: optional per-cell degree (order of Mesh.cells()) for an hp problem."""
        self.ctx = ctx
        self.lib = ctx.lib
        self.desc = make_desc(**desc)
        h = C.c_void_p()
        if degrees is None:
            L.check(self.lib.mfns_problem_create(ctx.h, mesh.h, C.byref(self.desc), C.byref(h)))
        else:
            deg = np.ascontiguousarray(degrees, dtype=np.int32)
            L.check(self.lib.mfns_problem_create_hp(ctx.h, mesh.h, C.byref(self.desc),
                                                    deg.ctypes.data_as(C.c_void_p), len(deg), C.byref(h)))
        self.h = h
        self.info = self.get_info()

    def get_info(self):
        inf = L.Info()
        L.check(self.lib.mfns_problem_info(self.h, C.byref(inf)))
        return inf

    def n_dofs(self, which=L.OP_SYSTEM):
        if which == L.OP_SYSTEM:
            return self.info.n_dofs
        if which == L.OP_PMASS:
            return self.info.n_dofs - self.info.n_velocity_dofs
        return self.info.level_dofs[which]

    def support_points(self, which=L.OP_SYSTEM):
        n = self.n_dofs(which)
        xyz = np.zeros((n, 3))
        field = np.zeros(n, dtype=np.int32)
        L.check(self.lib.mfns_dof_support_points(self.h, which, xyz.ctypes.data_as(C.c_void_p),
                                                 field.ctypes.data_as(C.c_void_p)))
        return xyz[:, : self.info.dim], field

    def constrained(self, which=L.OP_SYSTEM):
        n = C.c_int64()
        L.check(self.lib.mfns_constrained_dofs(self.h, which, None, 0, C.byref(n)))
        idx = np.zeros(n.value, dtype=np.int64)
        L.check(self.lib.mfns_constrained_dofs(self.h, which, idx.ctypes.data_as(C.c_void_p), n.value,
                                               C.byref(n)))
        return idx

    def set_lambda_max(self, level, lmax):
        L.check(self.lib.mfns_set_lambda_max(self.h, level, float(lmax)))
        self.info = self.get_info()

    def vector(self, which=L.OP_SYSTEM, prec=L.FP64, device="cuda"):
        return torch.zeros(self.n_dofs(which), dtype=_dtype(prec), device=device)

    def vmult(self, src, dst, which=L.OP_SYSTEM, prec=None, stream=None):
        prec = _prec_of(src) if prec is None else prec
        n, dt = self.n_dofs(which), _dtype(prec)
        L.check(self.lib.mfns_vmult(self.h, which, prec, _vec(src, n, dt, "src"), _vec(dst, n, dt, "dst"), n,
                                    _stream(stream)))
        return dst

    def vmult_host(self, srcs, dsts, which=L.OP_SYSTEM, stream=None):
        """dsts[i] = A srcs[i] for contiguous HOST (CPU) tensors of one dtype (page-locked for
        asynchronous copies): the library stages, applies and reads back, pipelined; the results
        are written when `stream` reaches the end of the call."""
        if len(srcs) != len(dsts) or not srcs:
            raise ValueError("srcs and dsts: equal, nonzero counts")
        prec = _prec_of(srcs[0])
        n, dt = self.n_dofs(which), _dtype(prec)
        for t in list(srcs) + list(dsts):
            if t.is_cuda or not t.is_contiguous():
                raise ValueError("host vectors: contiguous CPU tensors")
            if t.numel() != n or t.dtype != dt:
                raise ValueError(f"host vector: {t.numel()} entries of {t.dtype}, expected {n} of {dt}")
        sp = (C.c_void_p * len(srcs))(*[t.data_ptr() for t in srcs])
        dp = (C.c_void_p * len(dsts))(*[t.data_ptr() for t in dsts])
        L.check(self.lib.mfns_vmult_host(self.h, which, prec, sp, dp, len(srcs), n, _stream(stream)))
        return dsts

    def diagonal(self, diag, which=L.OP_SYSTEM, stream=None):
        prec = _prec_of(diag)
        n = self.n_dofs(which)
        L.check(self.lib.mfns_diagonal(self.h, which, prec, _vec(diag, n, name="diag"), n, _stream(stream)))
        return diag

    def kernel_timing(self, mode, which=L.OP_SYSTEM):
        """mode 1: reset+enable, 0: disable, 2: read -> (total kernel ms, launches)."""
        ms, n = C.c_double(), C.c_int64()
        L.check(self.lib.mfns_kernel_timing(self.h, which, mode, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def apply_constraints(self, x, which=L.OP_SYSTEM, stream=None):
        prec = _prec_of(x)
        n = self.n_dofs(which)
        L.check(self.lib.mfns_apply_constraints(self.h, which, prec, _vec(x, n, name="x"), n, _stream(stream)))
        return x

    def smooth(self, level, b, x, x_is_zero=False, stream=None):
        prec = _prec_of(b)
        n, dt = b.numel(), b.dtype          # the library checks n against the level's length
        L.check(self.lib.mfns_smooth(self.h, level, prec, _vec(b, n, dt, "b"), _vec(x, n, dt, "x"), n,
                                     int(bool(x_is_zero)), _stream(stream)))
        return x

    def prolongate_add(self, level, coarse, fine, stream=None):
        prec = _prec_of(coarse)
        nc, nf, dt = self.info.level_dofs[level + 1], self.info.level_dofs[level], coarse.dtype
        L.check(self.lib.mfns_prolongate_add(self.h, level, prec, _vec(coarse, nc, dt, "coarse"), nc,
                                             _vec(fine, nf, dt, "fine"), nf, _stream(stream)))
        return fine

    def restrict(self, level, fine, coarse, stream=None):
        prec = _prec_of(fine)
        nc, nf, dt = self.info.level_dofs[level + 1], self.info.level_dofs[level], fine.dtype
        L.check(self.lib.mfns_restrict(self.h, level, prec, _vec(fine, nf, dt, "fine"), nf,
                                       _vec(coarse, nc, dt, "coarse"), nc, _stream(stream)))
        return coarse

    def vcycle(self, b, x, stream=None):
        """x = V-cycle(b); b and x have info.cycle_dofs entries (the fine operator of the multigrid)."""
        prec = _prec_of(b)
        n, dt = self.info.cycle_dofs, b.dtype
        L.check(self.lib.mfns_vcycle(self.h, prec, _vec(b, n, dt, "b"), _vec(x, n, dt, "x"), n, _stream(stream)))
        return x

    def solve(self, b, x, stream=None, raise_on_nonconvergence=True):
        si = L.SolveInfo()
        n, f64 = self.info.n_dofs, torch.float64
        code = self.lib.mfns_solve(self.h, _vec(b, n, f64, "b"), _vec(x, n, f64, "x"), n, C.byref(si),
                                   _stream(stream))
        if code != L.OK and (code != L.ERR_NOT_CONVERGED or raise_on_nonconvergence):
            L.check(code)
        return si

    # -- nonlinear / time-dependent stabilised NS (Section 5) --------------------------------
    def set_state(self, dt, alpha, state, explicit_field=None, stream=None):
        """Linearisation state (FP64 system vector), dt, BDF coefficient alpha and the explicit field g."""
        _f64(state, explicit_field)
        n = self.info.n_dofs
        g = None if explicit_field is None else _vec(explicit_field, n, name="explicit_field")
        L.check(self.lib.mfns_set_state(self.h, float(dt), float(alpha), _vec(state, n, name="state"), g, n,
                                        _stream(stream)))

    def residual(self, dst, stream=None):
        prec = _prec_of(dst)
        n = self.info.n_dofs
        L.check(self.lib.mfns_residual(self.h, prec, _vec(dst, n, name="dst"), n, _stream(stream)))
        return dst

    def bdf_step(self, u, u_n, u_nm1=None, forcing=None, dt=0.0, omega=1.0, rtol=1e-8, atol=0.0, lin_tol=1e-4,
                 max_newton=10, extrapolate=False, stream=None, raise_on_nonconvergence=True):
        """One BDF step (omega = dt_n / dt_{n-1}, 0: BDF1) by Newton-FGMRES; u: guess in, solution out."""
        _f64(u, u_n, u_nm1, forcing)
        desc = L.NewtonDesc(dt=float(dt), omega=float(omega), rtol=float(rtol), atol=float(atol),
                            lin_tol=float(lin_tol), max_newton=int(max_newton), extrapolate=int(bool(extrapolate)))
        info = L.NewtonInfo()
        n = self.info.n_dofs
        opt = lambda t, nm: None if t is None else _vec(t, n, name=nm)
        code = self.lib.mfns_bdf_step(self.h, C.byref(desc), _vec(u_n, n, name="u_n"), opt(u_nm1, "u_nm1"),
                                      opt(forcing, "forcing"), _vec(u, n, name="u"), n, C.byref(info),
                                      _stream(stream))
        if code != L.OK and (code != L.ERR_NOT_CONVERGED or raise_on_nonconvergence):
            L.check(code)
        return info

    def max_velocity(self, u, stream=None):
        _f64(u)
        out = C.c_double()
        n = self.info.n_dofs
        L.check(self.lib.mfns_max_velocity(self.h, _vec(u, n, name="u"), n, C.byref(out), _stream(stream)))
        return out.value

    def solve_begin(self, b, x, stream=None):
        n, f64 = self.info.n_dofs, torch.float64
        L.check(self.lib.mfns_solve_begin(self.h, _vec(b, n, f64, "b"), _vec(x, n, f64, "x"), n, _stream(stream)))

    def solve_status(self):
        si = L.SolveInfo()
        L.check(self.lib.mfns_solve_status(self.h, C.byref(si)))
        return si

    def close(self):
        if self.h:
            self.lib.mfns_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_step(problems):
    """One FGMRES iteration for every running solve of `problems`; returns the running flags."""
    n = len(problems)
    arr = (C.c_void_p * n)(*[p.h for p in problems])
    run = (C.c_int * n)()
    L.check(L.load().mfns_batch_step(arr, n, run))
    return [bool(v) for v in run]


def batch_vcycle(problems, bs, xs, stream=None):
    """One batched V-cycle (zero start) per problem: x_i = V-cycle_i(b_i), shared launches per level."""
    n = len(problems)
    prec = _prec_of(bs[0])
    dt = bs[0].dtype
    lens = [p.info.cycle_dofs for p in problems]
    arr = (C.c_void_p * n)(*[p.h for p in problems])
    bp = (C.c_void_p * n)(*[_vec(b, m, dt, "b").value for b, m in zip(bs, lens)])
    xp = (C.c_void_p * n)(*[_vec(x, m, dt, "x").value for x, m in zip(xs, lens)])
    ln = (C.c_int64 * n)(*lens)
    L.check(L.load().mfns_batch_vcycle(arr, n, prec, bp, xp, ln, _stream(stream)))
    return xs


def temporal_matrices(r):
    """DG(r) reference-slab matrices (host, no device): (nodes, m_Q, M_Q, A_Q, G_Q)."""
    Q = r + 1
    out = [np.zeros(Q), np.zeros(Q), np.zeros((Q, Q)), np.zeros((Q, Q)), np.zeros((Q, Q))]
    L.check(L.load().mfns_spacetime_temporal(r, *[a.ctypes.data_as(C.c_void_p) for a in out]))
    return tuple(out)


class SpaceTime:
    """One time slab (Section 4) on the Taylor--Hood space of a Stokes problem: DG(r) in time,
    stage-major vectors of length Q * n."""

    def __init__(self, problem, r, tau, _handle=None, _lib=None):
        self.problem = problem                       # kept alive: the slab refers to it
        self.lib = problem.lib if problem is not None else _lib
        h = C.c_void_p()
        if _handle is None:
            L.check(self.lib.mfns_spacetime_create(problem.h, r, tau, C.byref(h)))
        else:
            h = _handle
        self.h = h
        Q, n = C.c_int(), C.c_int64()
        self.nodes = np.zeros(r + 1)
        self.G = np.zeros((r + 1, r + 1))
        L.check(self.lib.mfns_spacetime_info(h, C.byref(Q), C.byref(n), self.nodes.ctypes.data_as(C.c_void_p),
                                             self.G.ctypes.data_as(C.c_void_p)))
        self.Q, self.n = Q.value, n.value

    @classmethod
    def pdisc(cls, ctx, mesh, k, nu, r, tau):
        """A slab on the Q_k / P^disc_{k-1} pair (uniform meshes, FP64); owns its spatial operators."""
        h = C.c_void_p()
        L.check(ctx.lib.mfns_spacetime_create_pdisc(ctx.h, mesh.h, k, nu, r, tau, C.byref(h)))
        return cls(None, r, tau, _handle=h, _lib=ctx.lib)

    def support_points(self):
        xyz = np.zeros((self.n, 3))
        fld = np.zeros(self.n, dtype=np.int32)
        L.check(self.lib.mfns_spacetime_support_points(self.h, xyz.ctypes.data_as(C.c_void_p),
                                                       fld.ctypes.data_as(C.c_void_p)))
        return xyz, fld

    def vmult(self, src, dst, stream=None):
        prec = _prec_of(src)
        n = self.Q * self.n
        L.check(self.lib.mfns_spacetime_vmult(self.h, prec, _vec(src, n, src.dtype, "src"),
                                              _vec(dst, n, src.dtype, "dst"), n, _stream(stream)))
        return dst

    # -- space-time multigrid (FP64 vectors; patch inverses FP64 or FP32) ----------------------
    def mg_build(self, nu_s=4, omega=0.7, coarse_n=2, inverse_precision=0, stream=None):
        """inverse_precision: 0 = FP64 Schwarz patch inverses, 1 = FP32 (stored and applied)."""
        L.check(self.lib.mfns_spacetime_mg_build(self.h, nu_s, omega, coarse_n, inverse_precision,
                                                 _stream(stream)))
        nl = C.c_int()
        L.check(self.lib.mfns_spacetime_mg_level(self.h, -1, C.byref(nl), None, None, None))
        self.mg_levels = []
        for l in range(nl.value):
            k, r, n = C.c_int(), C.c_int(), C.c_int64()
            L.check(self.lib.mfns_spacetime_mg_level(self.h, l, None, C.byref(k), C.byref(r), C.byref(n)))
            self.mg_levels.append((k.value, r.value, n.value))
        return self.mg_levels

    def mg_support_points(self, level):
        n = self.mg_levels[level][2]
        xyz = np.zeros((n, 3))
        fld = np.zeros(n, dtype=np.int32)
        L.check(self.lib.mfns_spacetime_mg_support_points(self.h, level, xyz.ctypes.data_as(C.c_void_p),
                                                          fld.ctypes.data_as(C.c_void_p)))
        return xyz, fld

    def mg_apply(self, level, what, src, dst, stream=None):
        """what: 0 operator, 1 Schwarz smoother, 2 prolongate-add (src coarse), 3 restrict (dst coarse)."""
        f64 = torch.float64
        L.check(self.lib.mfns_spacetime_mg_apply(self.h, level, what, _vec(src, dtype=f64, name="src"), src.numel(),
                                                 _vec(dst, dtype=f64, name="dst"), dst.numel(), _stream(stream)))
        return dst

    def vcycle(self, b, x, stream=None):
        n, f64 = self.Q * self.n, torch.float64
        L.check(self.lib.mfns_spacetime_vcycle(self.h, _vec(b, n, f64, "b"), _vec(x, n, f64, "x"), n,
                                               _stream(stream)))
        return x

    def mg_smoother_bytes(self, level):
        """(bytes of the level's Schwarz patch inverses, number of patches)."""
        nb, npat = C.c_int64(), C.c_int64()
        L.check(self.lib.mfns_spacetime_mg_smoother_bytes(self.h, level, C.byref(nb), C.byref(npat)))
        return nb.value, npat.value

    def solve(self, b, x, tol=1e-10, maxit=200, stream=None, raise_on_nonconvergence=True):
        """FGMRES preconditioned by the space-time V-cycle; returns (iterations, relres)."""
        its, rel, conv = C.c_int(), C.c_double(), C.c_int()
        n, f64 = self.Q * self.n, torch.float64
        code = self.lib.mfns_spacetime_solve(self.h, _vec(b, n, f64, "b"), _vec(x, n, f64, "x"), n, tol, maxit,
                                             C.byref(its), C.byref(rel), C.byref(conv), _stream(stream))
        if code != L.OK and (code != L.ERR_NOT_CONVERGED or raise_on_nonconvergence):
            L.check(code)
        return its.value, rel.value

    def close(self):
        if self.h:
            self.lib.mfns_spacetime_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
