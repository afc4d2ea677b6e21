"""Continuous-batching serving of Stokes / stabilised Navier--Stokes solves on one GPU.

Requests arrive as a seeded Poisson stream; each is a solve on a uniform cube
(n^3 cells, degree k, viscosity nu, kind Stokes Q_{k+1}/Q_k or stabilised NS
Q_kQ_k) with a manufactured right-hand side b = A x*.  The loop

* admits arrived requests while slots and the context's HBM budget allow
  (problem set-up runs in a worker thread, so set-up overlaps device work),
* advances every active solve by one FGMRES iteration per round with
  mfns_batch_step (each request on its own CUDA stream, one host
  synchronisation per round for all of them),
* retires finished requests, freeing their slot and memory at once,

and reports solves/s, p50/p99 latency (completion - arrival) and the error of
every result against x*.  All solver work runs in libmfns; torch only holds
vectors and streams, and computes the error metric of finished results.
"""
import concurrent.futures as cf
import dataclasses
import math
import time

import numpy as np
import torch

from . import _lib as L
from . import api, inputs


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the stream
    kind: int               # L.STOKES or L.STAB_NS
    n: int
    k: int                  # stabilised NS: Q_kQ_k; Stokes: Q_{k+1}/Q_k
    nu: float
    seed: int


def poisson_stream(count, rate, seed=inputs.SEED_SERVE, n_range=(8, 48), degrees=(1, 2, 3), nu_range=(1e-3, 1.0)):
    """Seeded request stream: exponential inter-arrival times of mean 1/rate, n uniform in
    n_range, k uniform in degrees, nu log-uniform in nu_range, kinds 50/50."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        kind = L.STOKES if rng.random() < 0.5 else L.STAB_NS
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        k = int(rng.choice(degrees))
        nu = float(math.exp(rng.uniform(math.log(nu_range[0]), math.log(nu_range[1]))))
        out.append(Request(i, t, kind, n, k, nu, 1000 + i))
    return out


@dataclasses.dataclass
class Active:
    req: Request
    prob: object
    b: torch.Tensor
    x: torch.Tensor
    xstar: torch.Tensor
    stream: torch.cuda.Stream
    admitted: float


def _degree(req):
    return req.k + 1 if req.kind == L.STOKES else req.k


def _manufactured(prob, req):
    """x* ~ U(-1,1) (seeded per request); for Stokes the pressure entries are scaled by nu,
    the pressure scale of nu (grad u, grad v) - (p, div v)."""
    xstar = torch.tensor(inputs.uniform_vector(prob.info.n_dofs, seed=req.seed), device="cuda")
    if req.kind == L.STOKES:
        xstar[prob.info.n_velocity_dofs:] *= req.nu
    return xstar


def _pressure_slice(prob, req):
    """Entries of the pressure (null-space) component: Stokes block, or every (dim+1)-th entry."""
    if req.kind == L.STOKES:
        return slice(prob.info.n_velocity_dofs, prob.info.n_dofs)
    return slice(3, prob.info.n_dofs, 4)


class Server:
    def __init__(self, ctx, max_active=16, mg_precision=L.FP32, tol=1e-12, setup_workers=2, dt=1e-2):
        self.ctx = ctx
        self.max_active = max_active
        self.mg_precision = mg_precision
        self.tol = tol
        self.dt = dt
        self.pool = cf.ThreadPoolExecutor(setup_workers)

    def _setup(self, req):
        """Create the problem and its right-hand side (worker thread)."""
        stream = torch.cuda.Stream()
        m = api.Mesh(self.ctx, 3, req.n)
        prob = api.Problem(self.ctx, m, kind=req.kind, degree=_degree(req), nu=req.nu,
                           dt=self.dt if req.kind == L.STAB_NS else 0.0, mg_precision=self.mg_precision,
                           tol=self.tol, maxit=300)
        m.close()
        with torch.cuda.stream(stream):
            xstar = _manufactured(prob, req)
            b = torch.empty_like(xstar)
            prob.vmult(xstar, b, stream=stream)
            x = torch.zeros_like(xstar)
        prob.solve_begin(b, x, stream=stream)
        return prob, b, x, xstar, stream

    def _error(self, a):
        """||x - x*|| / ||x*|| with the pressure mean (null space) removed from both."""
        with torch.cuda.stream(a.stream):
            ps = _pressure_slice(a.prob, a.req)
            d = a.x - a.xstar
            d[ps] -= d[ps].mean()
            xs = a.xstar.clone()
            xs[ps] -= xs[ps].mean()
            return float(torch.linalg.norm(d) / torch.linalg.norm(xs))

    def run(self, requests, realtime=True, keep_solutions=False):
        """Serve the stream; returns per-request records and summary statistics.
        realtime=False replays arrivals on a simulated clock (no sleeping while idle);
        keep_solutions=True stores each solution (host copy) in its record."""
        future = sorted(requests, key=lambda r: r.arrival)
        waiting = []                      # arrived, not yet admitted (FIFO)
        active, setups, records = [], [], []
        t0 = time.perf_counter()
        offset = 0.0                      # simulated clock: skipped idle time
        fi = 0
        rounds = 0
        budget_blocked = False

        def now():
            return time.perf_counter() - t0 + offset

        while fi < len(future) or waiting or active or setups:
            t = now()
            while fi < len(future) and future[fi].arrival <= t:
                waiting.append(future[fi])
                fi += 1
            # admission: start set-ups while slots (and memory) are free
            while waiting and not budget_blocked and len(active) + len(setups) < self.max_active:
                req = waiting.pop(0)
                setups.append((req, self.pool.submit(self._setup, req)))
            still = []
            for req, fut in setups:
                if not fut.done():
                    still.append((req, fut))
                    continue
                try:
                    prob, b, x, xs, st = fut.result()
                    active.append(Active(req, prob, b, x, xs, st, now()))
                except L.MfnsError as e:
                    if e.code != L.ERR_BUDGET:
                        raise
                    if not active and len(still) == 0:
                        # nothing will release memory: the request alone exceeds the budget
                        records.append({"rid": req.rid, "kind": req.kind, "n": req.n, "k": req.k, "nu": req.nu,
                                        "arrival": req.arrival, "rejected": "exceeds the HBM budget alone",
                                        "converged": False, "latency": now() - req.arrival, "completed": now(),
                                        "iterations": 0, "error": float("inf")})
                        continue
                    waiting.insert(0, req)       # retry once memory has been released
                    budget_blocked = True
            setups = still
            if active:
                running = api.batch_step([a.prob for a in active])
                rounds += 1
                keep = []
                for a, run in zip(active, running):
                    if run:
                        keep.append(a)
                        continue
                    a.stream.synchronize()
                    st = a.prob.solve_status()
                    done = now()
                    records.append({"rid": a.req.rid, "kind": a.req.kind, "n": a.req.n, "k": a.req.k, "nu": a.req.nu,
                                    "dofs": a.prob.info.n_dofs, "arrival": a.req.arrival, "admitted": a.admitted,
                                    "completed": done, "latency": done - a.req.arrival,
                                    "iterations": st.iterations, "rel_residual": st.rel_residual,
                                    "converged": bool(st.converged), "error": self._error(a)})
                    if keep_solutions:
                        xs = a.x.clone()
                        ps = _pressure_slice(a.prob, a.req)
                        xs[ps] -= xs[ps].mean()      # the pressure is fixed up to a constant
                        records[-1]["x"] = xs.cpu().numpy()
                    a.prob.close()
                    budget_blocked = False
                active = keep
            elif setups:
                time.sleep(0.0005)
            elif fi < len(future) and not waiting:
                gap = future[fi].arrival - now()
                if gap > 0:
                    if realtime:
                        time.sleep(gap)
                    else:
                        offset += gap
        lat = np.array([r["latency"] for r in records])
        span = max(r["completed"] for r in records) - min(r["arrival"] for r in records) if records else 0.0
        summary = {"requests": len(records), "solves_per_s": len(records) / span if span > 0 else 0.0,
                   "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
                   "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
                   "max_error": max(r["error"] for r in records) if records else None,
                   "all_converged": all(r["converged"] for r in records), "rounds": rounds,
                   "makespan_s": span}
        conv = sorted(r["error"] for r in records if r["converged"])
        summary["not_converged"] = [{k: r[k] for k in ("rid", "kind", "n", "k", "nu") if k in r}
                                    for r in records if not r["converged"]]
        summary["error_converged_p50"] = float(np.percentile(conv, 50)) if conv else None
        summary["error_converged_p99"] = float(np.percentile(conv, 99)) if conv else None
        summary["error_converged_max"] = conv[-1] if conv else None
        return records, summary

    def close(self):
        self.pool.shutdown(wait=True)


def solve_alone(ctx, req, mg_precision=L.FP32, tol=1e-12, dt=1e-2):
    """The same request solved on its own with mfns_solve (reference for the mixed results);
    returns (solution with the pressure mean removed, solve info)."""
    m = api.Mesh(ctx, 3, req.n)
    prob = api.Problem(ctx, m, kind=req.kind, degree=_degree(req), nu=req.nu,
                       dt=dt if req.kind == L.STAB_NS else 0.0, mg_precision=mg_precision, tol=tol, maxit=300)
    xstar = _manufactured(prob, req)
    b = torch.empty_like(xstar)
    prob.vmult(xstar, b)
    x = torch.zeros_like(xstar)
    info = prob.solve(b, x, raise_on_nonconvergence=False)
    ps = _pressure_slice(prob, req)
    x[ps] -= x[ps].mean()          # the pressure is fixed up to a constant (as in the records)
    torch.cuda.synchronize()
    return x, info
