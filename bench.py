#!/usr/bin/env python
"""Benchmark of the matrix-free stabilised Navier--Stokes operator (GB300).

Workload (one step): one application of the Newton-linearised SUPG/PSPG BDF2
Navier--Stokes operator, equal-order Q2Q2 on a uniform 64^3 hexahedral mesh of
the unit cube (129^3 nodes x 4 fields = 8,586,756 DoFs), nu = 1e-2, dt = 1e-2,
frozen Taylor--Green state, on a seeded U(-1,1) vector; FP32 arithmetic.
Alongside: the FP64 apply, a degree-3 Chebyshev--Jacobi sweep and an FP32
V-cycle of the same problem, the end-to-end apply through the public API with
host buffers, clocks, the roofline of the cell kernel and the CPU oracle.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n 64]
Multi-GPU (torchrun): every rank runs an independent replica (no collective on
the data path); value = DoFs processed by all ranks / max time over ranks.
"""
import argparse
import datetime
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DoF/s stab-NS Q2 vmult; solves/s + p50/p99 latency, FP32-MG vs FP64 @1e-8"
UNIT = "DoF/s"
FLOP_PER_CELL = 17000.0          # algorithmic flops per Q2Q2 cell apply, frozen point values precomputed
FQ_BYTES_PER_CELL_F32 = 16 * 27 * 4  # precomputed frozen point data read per cell (u, grad u, Rbar, tau)
FP32_LANES, N_SM, SM_MHZ_MAX = 128, 152, 2070.0
CPU_SAMPLE_N = 12                # oracle sample: 12^3 cells of the same operator
HEADLINE_N = 64                  # the headline workload: 64^3 cells


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=HEADLINE_N)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--vmult-only", action="store_true", help="time only the FP32 apply (profiling runs)")
    ap.add_argument("--no-solves", action="store_true", help="skip the solve and serving sections")
    ap.add_argument("--serve-requests", type=int, default=32, help="requests of the bounded serving stream")
    ap.add_argument("--section", default=None, choices=["solves", "transient", "serving", "hp", "spacetime",
                                                        "next_rows"],
                    help="run one section of the line alone and print its JSON (used in child processes)")
    return ap.parse_args()


def max_over_ranks(values, world, device):
    """Every timing entry maximised over the ranks (the job takes as long as its slowest replica);
    a no-op for one rank.  device: where the reduction runs (CUDA under nccl, CPU under gloo)."""
    t = torch_mod().tensor(values, device=device, dtype=torch_mod().float64)
    if world > 1:
        torch_mod().distributed.all_reduce(t, op=torch_mod().distributed.ReduceOp.MAX)
    return t.tolist()


def whole_job_rate(units_per_rank, world, ms):
    """Whole-job throughput: the units all replicas processed per second of the slowest one."""
    return world * units_per_rank / (ms * 1e-3)


def torch_mod():
    import torch
    return torch


def dist_setup(gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi sampler during the timed region: rows stamped before mark() (the sampler's start-up,
    an idle GPU) are left out of the figures."""

    TS_FMT = "%Y/%m/%d %H:%M:%S.%f"

    def __init__(self, device):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.t_mark = None
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(device), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.p = None

    def wait_ready(self, timeout_s=5.0):
        """Return once the sampler has written its first sample (at most timeout_s): nvidia-smi
        takes a moment to start, longer than the short timed regions that follow."""
        if self.p is None:
            return
        t0 = time.time()
        while time.time() - t0 < timeout_s and self.p.poll() is None:
            if os.path.getsize(self.f.name) > 0:
                return
            time.sleep(0.02)

    def mark(self):
        """Start of the timed region: earlier rows are not counted."""
        self.t_mark = datetime.datetime.now()

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            if self.t_mark is not None:
                try:
                    if datetime.datetime.strptime(parts[0], self.TS_FMT) < self.t_mark:
                        continue
                except ValueError:
                    pass  # an unexpected stamp format: the row counts
            try:
                sm.append(float(parts[2]))
                mx.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[6:10]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_src_hash():
    h = hashlib.sha256()
    for f in ("op_apply.cuh", "op_kernel.cuh", "op_launch.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2603_29621_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic():
    """DRAM bytes per launch of the FP32 structured cell kernel from the committed ncu summary,
    or None when the kernel sources changed since the capture."""
    path = os.path.join(ROOT, "profiles", "op_kernel_stabns_q2_fp32.md")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != kernel_src_hash():
        return None
    try:
        return float(vals["dram_bytes_per_full_launch"])
    except (KeyError, ValueError):
        return None


def _cpu_model():
    """The host CPU's model string (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


class OracleSpmv:
    """The oracle's vmult (its assembled CSR matrix, scipy's product) over row blocks on `threads`
    host threads (scipy's sparse product releases the GIL): the arithmetic is the oracle's, only
    the rows are split between cores."""

    def __init__(self, n_cells=CPU_SAMPLE_N):
        from concurrent.futures import ThreadPoolExecutor

        from oracle import assemble, mesh
        from paper_2603_29621_gb300 import inputs

        t0 = time.perf_counter()
        op = assemble.Problem(mesh.uniform(3, n_cells), "stab_ns", 2, nu=1e-2, dt=1e-2)
        self.A = op.assemble().tocsr()
        self.t_asm = time.perf_counter() - t0
        self.n_cells = n_cells
        self.x = inputs.uniform_vector(self.A.shape[0])
        self.y = np.empty_like(self.x)
        self._pool = ThreadPoolExecutor
        self.threads = 1
        self.set_threads(1)

    def set_threads(self, t):
        n = self.A.shape[0]
        self.threads = t
        self.bounds = np.linspace(0, n, t + 1).astype(np.int64)
        self.blocks = [self.A[self.bounds[i]:self.bounds[i + 1]] for i in range(t)]
        self.pool = self._pool(t)

    def _job(self, i):
        self.y[self.bounds[i]:self.bounds[i + 1]] = self.blocks[i] @ self.x

    def __call__(self):
        list(self.pool.map(self._job, range(self.threads)))

    def rate(self, seconds):
        """(DoF/s, products, seconds) of back-to-back products for about `seconds`."""
        self()
        reps, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < seconds:
            self()
            reps += 1
        dt = time.perf_counter() - t0
        return self.A.shape[0] * reps / dt, reps, dt

    def sample(self):
        return (f"oracle vmult (assembled CSR, scipy product over row blocks) on {self.n_cells}^3 Q2Q2 cells "
                f"of the same operator ({self.A.shape[0]} DoFs, {self.A.nnz} nnz)")


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(seconds=8.0):
    """The oracle on all host cores and on one core, on a 12^3-cell sample of the same operator."""
    o = OracleSpmv()
    cores = host_cores()
    v1, r1, t1 = o.rate(seconds / 2)
    o.set_threads(cores)
    vn, rn, tn = o.rate(seconds / 2)
    return {"value": vn, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (o.sample() + f"; {rn} products in {tn:.1f} s on {cores} threads; assembly "
                       f"{o.t_asm:.1f} s not timed"),
            "cpu_model": _cpu_model(), "nproc": os.cpu_count(),
            "one_core": {"value": v1, "unit": UNIT, "products": r1, "seconds": t1}}


def solve_section(api, L, inputs, torch, tol_ns=1e-13, tol_stokes=1e-14):
    """Config 4 (stabilised NS 48^3 Q2Q2, three viscosities) and config 3 (Stokes Q2/Q1 on the
    ball-refined 32^3 mesh): FGMRES in FP64 with FP64 or FP32 multigrid; iterations, solve time
    and error against the manufactured discrete solution x* (smooth fields sampled at the
    support points, b = A x*)."""
    ctx = api.Context(torch.cuda.current_device())
    out = {"stab_ns_48": [], "stokes_ball_32": [], "stokes_ball_32_ls": []}

    def one(kind, n, k, nu, dt, mgp, ball, tol, hierarchy=0):  # -> (record, solution, pressure mean removed)
        m = api.Mesh(ctx, 3, n)
        if ball:
            m.refine_ball(*ball)
        t0 = time.perf_counter()
        p = api.Problem(ctx, m, kind=kind, degree=k, nu=nu, dt=dt, mg_precision=mgp, tol=tol, maxit=300,
                        hierarchy=hierarchy)
        setup = time.perf_counter() - t0
        xyz, fld = p.support_points()
        xs = torch.tensor(inputs.smooth_solution(xyz, fld, 3, nu if kind == L.STOKES else 1.0), device="cuda")
        b = torch.empty_like(xs)
        p.vmult(xs, b)
        x = torch.zeros_like(xs)
        p.solve(b, x, raise_on_nonconvergence=False)           # warm-up (graph capture)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = p.solve(b, x, raise_on_nonconvergence=False)
        torch.cuda.synchronize()
        dt_solve = time.perf_counter() - t0
        ps = slice(p.info.n_velocity_dofs, None) if kind == L.STOKES else slice(3, None, 4)
        d = x - xs
        d[ps] -= d[ps].mean()
        xr = xs.clone()
        xr[ps] -= xr[ps].mean()
        err = float(torch.linalg.norm(d) / torch.linalg.norm(xr))
        r = {"mg": "fp32" if mgp else "fp64", "hierarchy": "local_smoothing" if hierarchy else "global_coarsening",
             "nu": nu, "dofs": p.info.n_dofs, "cells": p.info.n_cells,
             "levels": p.info.n_levels, "iterations": info.iterations, "rel_residual": info.rel_residual,
             "converged": bool(info.converged), "solve_s": dt_solve, "setup_s": setup, "error_vs_xstar": err,
             # the single-device counterpart of the paper's load metrics: the work on every level
             "level_cells": [int(p.info.level_cells[i]) for i in range(p.info.n_levels)],
             "level_dofs": [int(p.info.level_dofs[i]) for i in range(p.info.n_levels)]}
        try:  # one multigrid cycle in the preconditioner's precision (device time, warm)
            vb = torch.tensor(inputs.uniform_vector(int(p.info.cycle_dofs), seed=6), device="cuda",
                              dtype=torch.float32 if mgp == L.FP32 else torch.float64)
            vx = torch.zeros_like(vb)
            for _ in range(3):
                p.vcycle(vb, vx)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(10):
                p.vcycle(vb, vx)
            e1.record()
            e1.synchronize()
            r["cycle_ms"] = e0.elapsed_time(e1) / 10
        except Exception as e:  # noqa: BLE001
            r["cycle_ms_error"] = f"{type(e).__name__}: {e}"

        if mgp == L.FP32 and not hierarchy:  # the system operator's apply (indexed cells, hanging nodes)
            for prec, vec in (("fp64", xs), ("fp32", xs.float())):
                out_v = torch.empty_like(vec)
                for _ in range(3):
                    p.vmult(vec, out_v)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(10):
                    p.vmult(vec, out_v)
                e1.record()
                e1.synchronize()
                r[f"vmult_{prec}_dofs_per_s_l2_warm"] = p.info.n_dofs / (e0.elapsed_time(e1) / 10 * 1e-3)
        xa = x.clone()
        xa[ps] -= xa[ps].mean()
        p.close()
        m.close()
        return r, xa

    def pair(key, *a, hierarchy=0):
        r64, x64 = one(*a[:5], L.FP64, *a[5:], hierarchy=hierarchy)
        r32, x32 = one(*a[:5], L.FP32, *a[5:], hierarchy=hierarchy)
        r32["rel_diff_vs_fp64_mg"] = float(torch.linalg.norm(x32 - x64) / torch.linalg.norm(x64))
        out[key] += [r64, r32]
        return x64

    for nu in (1e-1, 1e-2, 1e-3):
        pair("stab_ns_48", L.STAB_NS, 48, 2, nu, 1e-2, None, tol_ns)
    ball = ((0.5, 0.5, 0.5), 0.25, 2)
    x_gc = pair("stokes_ball_32", L.STOKES, 32, 2, 1.0, 0.0, ball, tol_stokes)
    # Section 2: local smoothing (levels = refinement levels, Dirichlet conditions on the refinement
    # edge) against global coarsening on the same problem
    x_ls = pair("stokes_ball_32_ls", L.STOKES, 32, 2, 1.0, 0.0, ball, tol_stokes, hierarchy=L.LOCAL_SMOOTHING)
    out["stokes_ball_32_ls"][0]["rel_diff_vs_global_coarsening"] = float(
        torch.linalg.norm(x_ls - x_gc) / torch.linalg.norm(x_gc))
    gc, lsr = out["stokes_ball_32"], out["stokes_ball_32_ls"]
    out["stokes_ball_32_ls_vs_gc"] = {
        r["mg"]: {"iterations_gc": g["iterations"], "iterations_ls": r["iterations"],
                  "solve_s_gc": g["solve_s"], "solve_s_ls": r["solve_s"]} for g, r in zip(gc, lsr)}
    for key in [k for k in out if isinstance(out[k], list)]:
        r64 = [r for r in out[key] if r["mg"] == "fp64"]
        r32 = [r for r in out[key] if r["mg"] == "fp32"]
        out[key + "_fp32_speedup"] = sum(r["solve_s"] for r in r64) / max(sum(r["solve_s"] for r in r32), 1e-12)
    ctx.close()
    return out


def hp_section(api, L, inputs, torch):
    """Section 3 (hp-adaptivity): the vector Laplacian on the ball-refined 16^3 mesh with a degree per
    cell (2 + refinement level + parity of the root cell's x index: 2..4, never lower on the fine side
    of a hanging face), hp-multigrid (every degree lowered by one per level, then h) in FP32 inside
    FP64 FGMRES, beside the same mesh with degree 2 everywhere.  Errors are recorded, not raised:
    this section runs last."""
    out = {}
    ctx = None
    try:
        ctx = api.Context(torch.cuda.current_device())
        for name, use_hp in (("hp_degrees_2_to_4", True), ("uniform_degree_2", False)):
            m = api.Mesh(ctx, 3, 16)
            m.refine_ball((0.5, 0.5, 0.5), 0.25, 1)
            cells = m.cells()
            deg = (2 + cells[:, 0] + ((cells[:, 1] >> cells[:, 0]) % 2)).astype(np.int32)
            desc = dict(kind=L.STOKES_A, nu=1.0, tol=1e-10, mg_precision=L.FP32, maxit=200)
            t0 = time.perf_counter()
            if use_hp:
                p = api.Problem(ctx, m, degrees=deg, degree=int(deg.max()), **desc)
            else:
                p = api.Problem(ctx, m, degree=2, **desc)
            setup = time.perf_counter() - t0
            xyz, fld = p.support_points()
            xs = torch.tensor(inputs.smooth_solution(xyz, fld, 3), device="cuda")
            b = torch.empty_like(xs)
            p.vmult(xs, b)
            x = torch.zeros_like(xs)
            p.solve(b, x, raise_on_nonconvergence=False)            # warm-up (graph capture)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = p.solve(b, x, raise_on_nonconvergence=False)
            torch.cuda.synchronize()
            out[name] = {"dofs": p.info.n_dofs, "cells": p.info.n_cells, "levels": p.info.n_levels,
                         "degrees": [int(deg.min()), int(deg.max())] if use_hp else [2, 2],
                         "iterations": info.iterations, "converged": bool(info.converged),
                         "rel_residual": info.rel_residual, "solve_s": time.perf_counter() - t0, "setup_s": setup,
                         "error_vs_xstar": float(torch.linalg.norm(x - xs) / torch.linalg.norm(xs))}
            p.close()
            m.close()
    except Exception as e:  # noqa: BLE001 -- reported in the JSON line
        out["error"] = f"{type(e).__name__}: {e}"
    try:
        if ctx is not None:
            ctx.close()
    except Exception as e:  # noqa: BLE001
        out.setdefault("error", f"{type(e).__name__}: {e}")
    return out


def _guarded_solve(api, L, inputs, torch, ctx, build, pslice):
    """Set up with build(), solve a manufactured discrete solution twice (warm-up, timed) and report
    iterations, time and the error against x* with the pressure mean removed (pslice)."""
    t0 = time.perf_counter()
    p, m = build()
    setup = time.perf_counter() - t0
    xyz, fld = p.support_points()
    xs = torch.tensor(inputs.smooth_solution(xyz, fld, 3), device="cuda")
    b = torch.empty_like(xs)
    p.vmult(xs, b)
    x = torch.zeros_like(xs)
    p.solve(b, x, raise_on_nonconvergence=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = p.solve(b, x, raise_on_nonconvergence=False)
    torch.cuda.synchronize()
    dt_solve = time.perf_counter() - t0
    ps = pslice(p)
    d = x - xs
    d[ps] -= d[ps].mean()
    xr = xs.clone()
    xr[ps] -= xr[ps].mean()
    r = {"dofs": p.info.n_dofs, "cells": p.info.n_cells, "levels": p.info.n_levels, "iterations": info.iterations,
         "rel_residual": info.rel_residual, "converged": bool(info.converged), "solve_s": dt_solve,
         "setup_s": setup, "error_vs_xstar": float(torch.linalg.norm(d) / torch.linalg.norm(xr)),
         "level_cells": [int(p.info.level_cells[i]) for i in range(p.info.n_levels)]}
    p.close()
    m.close()
    return r


def next_rows_section(api, L, inputs, torch):
    """Section 2's local smoothing for Section 5's stabilised operator (Q2Q2, nu = 1e-2, dt = 1e-2) on
    the ball-refined 24^3 mesh (two levels) beside global coarsening, and Section 3's hp Taylor--Hood Stokes
    (velocity degrees 2..4 per cell, pressure one lower) on the ball-refined 16^3 mesh; FP32
    multigrid inside FP64 FGMRES.  Errors are recorded per row, not raised: this section runs last."""
    out = {}
    ctx = None
    try:
        ctx = api.Context(torch.cuda.current_device())
    except Exception as e:  # noqa: BLE001
        return {"error": f"{type(e).__name__}: {e}"}
    for name, hierarchy in (("global_coarsening", L.GLOBAL_COARSENING), ("local_smoothing", L.LOCAL_SMOOTHING)):
        def build(h=hierarchy):
            m = api.Mesh(ctx, 3, 24)
            m.refine_ball((0.5, 0.5, 0.5), 0.25, 2)
            p = api.Problem(ctx, m, kind=L.STAB_NS, degree=2, nu=1e-2, dt=1e-2, mg_precision=L.FP32, tol=1e-10,
                            maxit=300, hierarchy=h)
            return p, m
        try:
            out["stab_ns_ball_24_" + name] = _guarded_solve(api, L, inputs, torch, ctx, build,
                                                             lambda p: slice(3, None, 4))
        except Exception as e:  # noqa: BLE001
            out["stab_ns_ball_24_" + name] = {"error": f"{type(e).__name__}: {e}"}

    def build_hp():
        m = api.Mesh(ctx, 3, 16)
        m.refine_ball((0.5, 0.5, 0.5), 0.25, 1)
        cells = m.cells()
        deg = (2 + cells[:, 0] + ((cells[:, 1] >> cells[:, 0]) % 2)).astype(np.int32)
        p = api.Problem(ctx, m, degrees=deg, kind=L.STOKES, degree=int(deg.max()), nu=1.0, mg_precision=L.FP32,
                        tol=1e-10, maxit=300)
        return p, m
    try:
        out["hp_taylor_hood_ball_16"] = _guarded_solve(api, L, inputs, torch, ctx, build_hp,
                                                       lambda p: slice(p.info.n_velocity_dofs, None))
    except Exception as e:  # noqa: BLE001
        out["hp_taylor_hood_ball_16"] = {"error": f"{type(e).__name__}: {e}"}
    try:
        ctx.close()
    except Exception as e:  # noqa: BLE001
        out.setdefault("error", f"{type(e).__name__}: {e}")
    return out


def _schwarz_rate(st, torch):
    """Device time of one Schwarz application on the finest space-time level and the achieved rate
    of reading its patch inverses (the patch solve's algorithmic bytes), GB/s."""
    nbytes, npatch = st.mg_smoother_bytes(0)
    N = st.Q * st.n
    r = torch.rand(N, dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    for _ in range(3):
        st.mg_apply(0, 1, r, z)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        st.mg_apply(0, 1, r, z)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / 10
    return {"patches": npatch, "inverse_bytes": nbytes, "ms": ms, "inverse_gbs": nbytes / (ms * 1e-3) / 1e9}


def spacetime_section(api, L, inputs, torch):
    """Section 4 (space-time): the slab operator K = G_Q (x) M + tau I_Q (x) A of DG(1) in time on the
    Taylor--Hood Q2/Q1 space of the unit cube with 32^3 cells (one product, FP64 and FP32), and
    FGMRES preconditioned by the space-time multigrid (vertex-star Schwarz, nu_s = 4, omega = 0.7)
    on 8^3 cells, tau = 0.05, for a manufactured slab solution, with FP64 and with FP32 patch
    inverses; one Schwarz application on 16^3 cells with each.  Errors are recorded, not raised:
    this section runs last."""
    out = {}
    ctx = None
    try:
        ctx = api.Context(torch.cuda.current_device())
        m = api.Mesh(ctx, 3, 32)
        p = api.Problem(ctx, m, kind=L.STOKES, degree=2, nu=1.0, lambda_max=1.0)
        st = api.SpaceTime(p, 1, 0.05)
        N = st.Q * st.n
        for dt, name in ((torch.float64, "fp64"), (torch.float32, "fp32")):
            x = torch.tensor(inputs.uniform_vector(N, seed=1), device="cuda", dtype=dt)
            y = torch.empty_like(x)
            for _ in range(3):
                st.vmult(x, y)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 10
            e0.record()
            for _ in range(reps):
                st.vmult(x, y)
            e1.record()
            torch.cuda.synchronize()
            out.setdefault("slab_vmult_32cube_dg1", {"entries": N, "cells": 32 ** 3})[name + "_ms"] = \
                e0.elapsed_time(e1) / reps
        st.close()
        p.close()
        m.close()
        m = api.Mesh(ctx, 3, 8)
        p = api.Problem(ctx, m, kind=L.STOKES, degree=2, nu=1.0, lambda_max=1.0)
        st = api.SpaceTime(p, 1, 0.05)
        t0 = time.perf_counter()
        levels = st.mg_build(nu_s=4, omega=0.7)
        setup = time.perf_counter() - t0
        xyz, fld = p.support_points()
        one = inputs.smooth_solution(xyz, fld, 3)
        xs_np = np.concatenate([(1.0 + 0.5 * q) * one for q in range(st.Q)])
        pres = fld == 3
        for q in range(st.Q):                                       # no constant pressure per stage
            blk = xs_np[q * st.n:(q + 1) * st.n]
            blk[pres] -= blk[pres].mean()
        xs = torch.tensor(xs_np, device="cuda")
        b = torch.empty_like(xs)
        st.vmult(xs, b)
        x = torch.zeros_like(xs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its, rel = st.solve(b, x, tol=1e-10, maxit=200, raise_on_nonconvergence=False)
        torch.cuda.synchronize()
        out["stmg_solve_8cube_dg1"] = {"entries": st.Q * st.n, "levels": [list(l) for l in levels],
                                       "setup_s": setup, "iterations": its, "rel_residual": rel,
                                       "solve_s": time.perf_counter() - t0,
                                       "error_vs_xstar": float(torch.linalg.norm(x - xs) / torch.linalg.norm(xs)),
                                       "schwarz_level0": _schwarz_rate(st, torch)}
        # the same solve with FP32 patch inverses (stored and applied in FP32, the rest FP64)
        st.mg_build(nu_s=4, omega=0.7, inverse_precision=1)
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its, rel = st.solve(b, x, tol=1e-10, maxit=200, raise_on_nonconvergence=False)
        torch.cuda.synchronize()
        out["stmg_solve_8cube_dg1"]["fp32_inverses"] = {
            "iterations": its, "rel_residual": rel, "solve_s": time.perf_counter() - t0,
            "error_vs_xstar": float(torch.linalg.norm(x - xs) / torch.linalg.norm(xs)),
            "schwarz_level0": _schwarz_rate(st, torch)}
        st.close()
        p.close()
        m.close()
        # the Schwarz application where its patch inverses outgrow the L2: 16^3 cells, FP64 and FP32
        m = api.Mesh(ctx, 3, 16)
        p = api.Problem(ctx, m, kind=L.STOKES, degree=2, nu=1.0, lambda_max=1.0)
        st = api.SpaceTime(p, 1, 0.05)
        row = {"entries": st.Q * st.n}
        for prec, name in ((0, "fp64_inverses"), (1, "fp32_inverses")):
            t0 = time.perf_counter()
            st.mg_build(nu_s=4, omega=0.7, inverse_precision=prec)
            row[name] = dict(_schwarz_rate(st, torch), setup_s=time.perf_counter() - t0)
        out["schwarz_16cube_dg1"] = row
        st.close()
        p.close()
        m.close()
    except Exception as e:  # noqa: BLE001 -- reported in the JSON line
        out["error"] = f"{type(e).__name__}: {e}"
    try:
        # the paper's pair Q2/P1^disc with DG(1), cell patches, on 8^3 cells
        m = api.Mesh(ctx, 3, 8)
        st = api.SpaceTime.pdisc(ctx, m, 2, 1.0, 1, 0.05)
        t0 = time.perf_counter()
        levels = st.mg_build(nu_s=4, omega=0.7)
        setup = time.perf_counter() - t0
        xs = torch.tensor(inputs.uniform_vector(st.Q * st.n, seed=4), device="cuda")
        b = torch.empty_like(xs)
        st.vmult(xs, b)
        x = torch.zeros_like(xs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its, rel = st.solve(b, x, tol=1e-10, maxit=200, raise_on_nonconvergence=False)
        torch.cuda.synchronize()
        out["stmg_solve_pdisc_8cube_dg1"] = {"entries": st.Q * st.n, "levels": [list(l) for l in levels],
                                             "setup_s": setup, "iterations": its, "rel_residual": rel,
                                             "solve_s": time.perf_counter() - t0,
                                             "schwarz_level0": _schwarz_rate(st, torch)}
        st.close()
        m.close()
    except Exception as e:  # noqa: BLE001
        out["pdisc_error"] = f"{type(e).__name__}: {e}"
    try:
        if ctx is not None:
            ctx.close()
    except Exception as e:  # noqa: BLE001
        out.setdefault("error", f"{type(e).__name__}: {e}")
    return out


def serving_section(api, L, torch, count):
    """Config 5, bounded: a seeded Poisson stream of `count` requests (n in 8..48, k in 1..3, nu
    log-uniform in [1e-3, 1], Stokes / stabilised NS 50/50, b = A x*), offered at 0.8 x the measured
    single-stream throughput, served with FP32 and with FP64 multigrid; with FP32 multigrid also at
    0.5 x and 1.2 x that rate."""
    from paper_2603_29621_gb300 import serve
    ctx = api.Context(torch.cuda.current_device(), hbm_budget_bytes=150 * 1024 ** 3)
    probe = serve.poisson_stream(6, rate=1.0, seed=3)
    serve.solve_alone(ctx, probe[0])                        # first use in this process: not timed
    t0 = time.perf_counter()
    for req in probe:
        serve.solve_alone(ctx, req)
    mu = len(probe) / (time.perf_counter() - t0)          # single-stream solves/s incl. set-up
    rate = 0.8 * mu
    reqs = serve.poisson_stream(count, rate=rate)
    out = {"requests": count, "offered_rate_per_s": rate, "single_stream_solves_per_s": mu}
    sols = {}
    for name, mgp in (("fp64_mg", L.FP64), ("fp32_mg", L.FP32)):
        srv = serve.Server(ctx, max_active=16, mg_precision=mgp)
        recs, summary = srv.run(reqs, realtime=True, keep_solutions=True)
        srv.close()
        out[name] = summary
        sols[name] = {r["rid"]: (r["x"], r["kind"], r["dofs"]) for r in recs if "x" in r}
    diffs = []
    for rid, (x32, kind, n) in sols["fp32_mg"].items():
        x64 = sols["fp64_mg"][rid][0]
        diffs.append(float(np.linalg.norm(x32 - x64) / np.linalg.norm(x64)))
    out["fp32_vs_fp64_max_rel_diff"] = max(diffs) if diffs else None
    out["fp32_vs_fp64_throughput"] = out["fp32_mg"]["solves_per_s"] / max(out["fp64_mg"]["solves_per_s"], 1e-12)
    # the same stream offered at 0.5 x and 1.2 x the single-stream rate (FP32 multigrid)
    out["load_sweep_fp32_mg"] = {}
    for f in (0.5, 1.2):
        srv = serve.Server(ctx, max_active=16, mg_precision=L.FP32)
        summ = srv.run(serve.poisson_stream(count, rate=f * mu), realtime=True)[1]
        srv.close()
        out["load_sweep_fp32_mg"][f"{f}x"] = dict(summ, offered_rate_per_s=f * mu)
    # saturated burst (all requests at once, n in 8..32): batched preconditioners (one V-cycle launch
    # per level and colour over all active problems) against every problem on its own stream
    burst = serve.poisson_stream(max(8, count // 2), rate=1e4, seed=4, n_range=(8, 32))
    for name, on in (("burst_fp32_batched", True), ("burst_fp32_per_problem", False)):
        ctx.set_batching(on)
        srv = serve.Server(ctx, max_active=16, mg_precision=L.FP32)
        out[name] = srv.run(burst, realtime=True)[1]
        srv.close()
    ctx.set_batching(True)
    out["burst_batched_speedup"] = (out["burst_fp32_batched"]["solves_per_s"]
                                    / max(out["burst_fp32_per_problem"]["solves_per_s"], 1e-12))
    ctx.close()
    return out


def transient_section(api, L, inputs, torch, n=48, steps=4, cfl=0.5, nu=1e-2):
    """Time stepping of the stabilised NS problem on n^3 Q2Q2 cells (Section 5): Taylor--Green
    initial state (its boundary values kept as Dirichlet data), one BDF1 step, then variable-step
    BDF2 with dt = cfl h / max|u|; every step solved by Newton-FGMRES with the multigrid at the
    current state (inexact Newton: FGMRES to 1e-4, Newton to a 1e-8 residual reduction)."""
    ctx = api.Context(torch.cuda.current_device())
    out = {"cells": n ** 3, "steps": steps, "cfl": cfl, "nu": nu}
    finals = {}
    for name, mgp in (("fp64_mg", L.FP64), ("fp32_mg", L.FP32)):
        m = api.Mesh(ctx, 3, n)
        t0 = time.perf_counter()
        p = api.Problem(ctx, m, kind=L.STAB_NS, degree=2, nu=nu, dt=1e-2, mg_precision=mgp, maxit=200)
        setup = time.perf_counter() - t0
        xyz, fld = p.support_points()
        u_n = torch.tensor(inputs.taylor_green_state(xyz, fld, 3), device="cuda")
        u_nm1 = None
        h = 1.0 / n
        dt_old = None
        recs = []
        torch.cuda.synchronize()
        t_all = time.perf_counter()
        for s in range(steps):
            dt = cfl * h / p.max_velocity(u_n)
            om = 0.0 if dt_old is None else dt / dt_old
            u = u_n.clone()
            info = p.bdf_step(u, u_n, u_nm1, dt=dt, omega=om, rtol=1e-8, lin_tol=1e-4, max_newton=8,
                              extrapolate=u_nm1 is not None, raise_on_nonconvergence=False)
            recs.append({"dt": dt, "omega": om, "newton": info.newton_iterations, "fgmres": info.linear_iterations,
                         "residual_reduction": info.residual / max(info.residual0, 1e-300),
                         "converged": bool(info.converged), "seconds": info.seconds})
            u_nm1, u_n, dt_old = u_n, u, dt
        torch.cuda.synchronize()
        total = time.perf_counter() - t_all
        later = recs[1:] if len(recs) > 1 else recs
        out[name] = {"dofs": p.info.n_dofs, "levels": p.info.n_levels, "setup_s": setup, "total_s": total,
                     "s_per_step_after_first": sum(r["seconds"] for r in later) / len(later),
                     "dof_steps_per_s": p.info.n_dofs * steps / total, "steps": recs}
        xf = u_n.clone()
        xf[3::4] -= xf[3::4].mean()
        finals[name] = xf
        p.close()
        m.close()
    out["fp32_mg_speedup"] = out["fp64_mg"]["total_s"] / max(out["fp32_mg"]["total_s"], 1e-12)
    out["fp32_vs_fp64_final_state_rel_diff"] = float(torch.linalg.norm(finals["fp32_mg"] - finals["fp64_mg"])
                                                     / torch.linalg.norm(finals["fp64_mg"]))
    ctx.close()
    return out


def headline_config(n, world):
    """The workload of the headline line (both arms print it): the 64^3 stabilised Q2Q2 product."""
    return {"workload": f"stab-NS Q2Q2 vmult, uniform {n}^3 hex unit cube, nu=1e-2, dt=1e-2 (BDF2), "
                        "Taylor-Green frozen state, seeded U(-1,1) input",
            "n_cells": n ** 3, "n_dofs": 4 * (2 * n + 1) ** 3, "parallelism": f"replicas x{world}",
            "l2": "flushed between timed steps (512 MiB write)"}


def run_reference(args, world, rank):
    """The oracle (the reference arm: a plain assembled-matrix program written from the paper) on the
    host's cores, on a bounded 12^3 sample of the headline workload; rank 0 only."""
    if rank != 0:
        return
    o = OracleSpmv()
    cores = host_cores()
    o.set_threads(cores)
    for _ in range(args.warmup):
        o()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o()
    dt = time.perf_counter() - t0
    val = o.A.shape[0] * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": headline_config(args.n, world),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": o.sample() + f" per step (a bounded sample of the {args.n}^3 workload; "
                                                    "rates per DoF compared)",
                             "cpu_model": _cpu_model(), "nproc": os.cpu_count()},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


SECTIONS = ("solves", "transient", "serving", "hp", "spacetime", "next_rows")
SECTION_TIMEOUT_S = {"solves": 420, "transient": 240, "serving": 420, "hp": 240, "spacetime": 240, "next_rows": 300}


def run_section(name, args):
    """One section of the line in a child process: a failure there (an exception, a CUDA error that
    poisons the context, a timeout) is recorded in the line and cannot take the headline with it."""
    cmd = [sys.executable, os.path.abspath(__file__), "--section", name, "--serve-requests",
           str(args.serve_requests)]
    t0 = time.perf_counter()
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=SECTION_TIMEOUT_S[name])
    except subprocess.TimeoutExpired:
        return {"error": f"timed out after {SECTION_TIMEOUT_S[name]} s"}
    wall = time.perf_counter() - t0
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    if r.returncode != 0 or not lines:
        return {"error": f"exit {r.returncode}: " + (r.stderr.strip().splitlines() or ["no output"])[-1][:400],
                "wall_s": wall}
    try:
        out = json.loads(lines[-1])
    except ValueError as e:
        return {"error": f"unparsable section output: {e}", "wall_s": wall}
    out["wall_s"] = wall
    return out


def section_main(args):
    import torch

    import __graft_entry__ as g
    from paper_2603_29621_gb300 import _lib as L
    from paper_2603_29621_gb300 import api, inputs

    torch.cuda.set_device(0)
    g.build()
    name = args.section
    if name == "solves":
        out = solve_section(api, L, inputs, torch)
    elif name == "transient":
        out = transient_section(api, L, inputs, torch)
    elif name == "serving":
        out = serving_section(api, L, torch, args.serve_requests)
    elif name == "hp":
        out = hp_section(api, L, inputs, torch)
    elif name == "spacetime":
        out = spacetime_section(api, L, inputs, torch)
    elif name == "next_rows":
        out = next_rows_section(api, L, inputs, torch)
    else:
        raise SystemExit(f"unknown section {name}")
    print(json.dumps(out), flush=True)


def run_ours(args, world, rank, local):
    import torch

    import __graft_entry__ as g
    from paper_2603_29621_gb300 import _lib as L
    from paper_2603_29621_gb300 import api, inputs

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    g.build()
    dev = torch.device("cuda", local)
    ctx = api.Context(local)
    n = args.n
    m = api.Mesh(ctx, 3, n)
    prob = api.Problem(ctx, m, kind=L.STAB_NS, degree=2, nu=1e-2, dt=1e-2, smoother=1, smoother_degree=3,
                       mg_precision=L.FP32)
    ndof = prob.info.n_dofs
    ncell = prob.info.n_cells
    nodes = ndof // 4
    x64 = torch.tensor(inputs.uniform_vector(ndof), device=dev)
    src32, src64 = x64.float(), x64
    dst32, dst64 = torch.empty_like(src32), torch.empty_like(src64)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    def timed(fn, steps, warmup, nvtx=None):
        for _ in range(warmup):
            fn()
        barrier()
        if nvtx:  # lets a profiler select the timed launches (ncu --nvtx --nvtx-include)
            torch.cuda.nvtx.range_push(nvtx)
        total = 0.0
        for s in range(steps):
            flush.fill_(float(s))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        if nvtx:
            torch.cuda.nvtx.range_pop()
        barrier()
        return total / steps  # ms per step

    # ---- headline: FP32 vmult as a user runs it (later colours overlap the previous colour's tail)
    # clocks sampled over the headline, the per-launch pass and the end-to-end passes (the headline
    # alone lasts a few milliseconds, shorter than the sampling period)
    clocks = Clocks(local)
    clocks.wait_ready()
    clocks.mark()
    ms32 = timed(lambda: prob.vmult(src32, dst32), args.steps, args.warmup, nvtx="timed_vmult_fp32")
    # ---- the cell kernel's colour launches one by one, each bracketed by CUDA events on the
    # launching stream (the events serialise the launches): the per-launch roofline figure
    prob.kernel_timing(1)
    timed(lambda: prob.vmult(src32, dst32), args.steps, args.warmup)
    kms, klaunch = prob.kernel_timing(2)
    prob.kernel_timing(0)
    # the warm-up launches were recorded as well: the average over all recorded launches
    avg_launch_ms = kms / max(klaunch, 1)
    launches_per_step = klaunch // (args.steps + args.warmup)
    if args.vmult_only:
        clocks.stop()
        if rank == 0:
            print(json.dumps({"vmult_fp32_ms": ms32, "dofs_per_s": world * ndof / (ms32 * 1e-3),
                              "avg_launch_ms": avg_launch_ms, "launches_per_step": launches_per_step}))
        return
    # ---- end to end through the public API with host buffers (pinned), every step
    h_src = torch.empty(ndof, dtype=torch.float32, pin_memory=True)
    h_src.copy_(src32.cpu())
    h_dst = torch.empty(ndof, dtype=torch.float32, pin_memory=True)

    # end to end through the C ABI with HOST buffers (mfns_vmult_host: the library copies each
    # step's input in, applies and reads the result back): one vector per call, each call serial
    ms_e2e_serial = timed(lambda: prob.vmult_host([h_src], [h_dst]), args.steps, args.warmup)

    # the same stream of steps handed to the library in one call: it pipelines the copy of step
    # i+1's input and the read-back of step i-1's result with step i's apply (two staging sets)
    h_dst2 = torch.empty(ndof, dtype=torch.float32, pin_memory=True)

    def e2e_pipelined(steps):
        barrier()
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        prob.vmult_host([h_src] * steps, [(h_dst, h_dst2)[i % 2] for i in range(steps)])
        e1.record(stream)
        e1.synchronize()
        barrier()
        return e0.elapsed_time(e1) / steps

    e2e_pipelined(args.warmup)
    ms_e2e = e2e_pipelined(args.steps)
    clk = clocks.stop()
    # ---- max over ranks
    ms32, ms_e2e, ms_e2e_serial = max_over_ranks([ms32, ms_e2e, ms_e2e_serial], world, dev)
    extra = {}
    if rank == 0:
        # ---- FP64 vmult, Chebyshev-3 sweep, V-cycle (FP32), each recorded, none can end the run
        def guarded(key, fn):
            try:
                extra[key] = fn()
            except Exception as e:  # noqa: BLE001 -- reported in the JSON line
                extra[key] = {"error": f"{type(e).__name__}: {e}"}

        steps_s = max(3, args.steps // 4)
        guarded("fp64", lambda: (lambda ms: {"value": world * ndof / (ms * 1e-3), "unit": UNIT,
                                             "ms_per_apply": ms})(
            timed(lambda: prob.vmult(src64, dst64), steps_s, 3)))
        b32 = src32.clone()
        xs = torch.zeros_like(b32)

        def cheb():
            ms = timed(lambda: prob.smooth(0, b32, xs, x_is_zero=False), max(3, args.steps // 2), 3,
                       nvtx="timed_cheb")
            return {"ms_per_sweep": ms, "dofs_per_s": world * ndof / (ms * 1e-3)}

        def vcyc():
            assert prob.info.cycle_dofs == ndof
            return {"ms": timed(lambda: prob.vcycle(b32, xs), steps_s, 3, nvtx="timed_vcycle_fp32"),
                    "levels": prob.info.n_levels}

        guarded("chebyshev3_fp32", cheb)
        guarded("vcycle_fp32", vcyc)

        def fused():
            pf = api.Problem(ctx, m, kind=L.STAB_NS, degree=2, nu=1e-2, dt=1e-2, smoother=1, smoother_degree=3,
                             mg_precision=L.FP32, fused_smoother=1)
            try:
                for lvl in range(prob.info.n_levels - 1):
                    pf.set_lambda_max(lvl, prob.info.lambda_max[lvl])
                return {"ms_per_sweep": timed(lambda: pf.smooth(0, b32, xs, x_is_zero=False),
                                              max(3, args.steps // 2), 3, nvtx="timed_cheb_fused"),
                        "vcycle_ms": timed(lambda: pf.vcycle(b32, xs), steps_s, 3)}
            finally:
                pf.close()

        guarded("fused_smoother_fp32", fused)
    prob.close()
    m.close()
    ctx.close()
    del flush
    torch.cuda.empty_cache()
    if rank != 0:
        return
    value = whole_job_rate(ndof, world, ms32)
    cells_per_launch = ncell / launches_per_step if launches_per_step else ncell
    peak_alu = N_SM * FP32_LANES * 2 * SM_MHZ_MAX * 1e6 / 1e12    # TFLOP/s
    achieved_alu = FLOP_PER_CELL * cells_per_launch / (avg_launch_ms * 1e-3) / 1e12
    traffic = ncu_traffic()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    # algorithmic bytes of one apply: src and dst (4 fields each) and the frozen state (u, p: 4
    # fields) once per node, FP32 -- 12 x 2,146,689 x 4 B = 103.0 MB at 64^3; a colour launch
    # processes 1/launches_per_step of the cells and is charged that share
    alg_bytes = 12 * nodes * 4
    bytes_launch = alg_bytes * cells_per_launch / ncell
    achieved = bytes_launch / (avg_launch_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": headline_config(n, world),
        "clocks": clk,
        # per step: the clearing kernel (which also writes the identity rows) and the colour launches
        "gpu_launches": (launches_per_step + 1) * args.steps,
        "e2e": {"value": whole_job_rate(ndof, world, ms_e2e), "unit": UNIT, "h2d_bytes_per_step": ndof * 4,
                "d2h_bytes_per_step": ndof * 4, "ms_per_step": ms_e2e,
                "how": "C ABI with HOST buffers: one mfns_vmult_host call for all timed steps (pinned "
                       "host vectors); every step's input is copied in and its result read back, the "
                       "library pipelining step i+1's input copy and step i-1's read-back with step i's "
                       "apply over two staging sets; bound by the host link (both directions at once)",
                "serial": {"value": whole_job_rate(ndof, world, ms_e2e_serial), "ms_per_step": ms_e2e_serial,
                           "how": "one mfns_vmult_host call per step: copy in, apply, copy out"}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy, burst), of measured",
                     "kernel": "op_kernel<3,2,STAB_NS,float,structured> (one colour launch)",
                     "alg_bytes_per_apply": alg_bytes, "alg_bytes_per_launch": bytes_launch,
                     "alg_bytes_rule": "12 fields (src 4, dst 4, frozen u,p 4) x nodes x 4 B",
                     "cells_per_launch": cells_per_launch, "avg_launch_ms": avg_launch_ms,
                     "avg_launch_note": "launches timed one by one (events serialise them); in the "
                                        "headline apply later colours overlap the previous colour's tail",
                     "launches_per_apply": launches_per_step,
                     "whole_apply": {"achieved_gbs": alg_bytes / (ms32 * 1e-3) / 1e9,
                                     "frac": alg_bytes / (ms32 * 1e-3) / 1e9 / hbm_peak},
                     "alu": {"achieved_tflops": achieved_alu, "peak_tflops": peak_alu,
                             "frac": achieved_alu / peak_alu, "flop_per_cell": FLOP_PER_CELL,
                             "peak_rule": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"},
                     "ridge_flop_per_byte": peak_alu * 1e12 / (hbm_peak * 1e9),
                     "intensity_flop_per_byte": FLOP_PER_CELL * ncell / alg_bytes,
                     "with_point_data": {"note": "bytes the kernel reads by design: src, dst and the "
                                                 "precomputed frozen point block (1,728 B per cell)",
                                         "bytes_per_launch": (8 * nodes * 4 * cells_per_launch / ncell
                                                              + cells_per_launch * FQ_BYTES_PER_CELL_F32),
                                         "achieved_gbs": (8 * nodes * 4 * cells_per_launch / ncell
                                                          + cells_per_launch * FQ_BYTES_PER_CELL_F32)
                                         / (avg_launch_ms * 1e-3) / 1e9}},
    }
    line.update(extra)
    if world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline()
        except Exception as e:  # noqa: BLE001
            line["cpu_baseline"] = {"error": f"{type(e).__name__}: {e}", "kind": "oracle"}
    if world == 1 and not args.no_solves:
        t0 = time.perf_counter()
        for name in SECTIONS:
            line[name] = run_section(name, args)
        line["sections_wall_s"] = time.perf_counter() - t0
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.section:
        section_main(args)
        return
    world, rank, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
