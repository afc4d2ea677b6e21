"""Continuous batching: batched FGMRES rounds and the serving loop, through the C ABI.

A result must not depend on what else is in the batch: every request of a
mixed stream is compared with the same request solved alone (mfns_solve);
problems are independent and every reduction has a fixed order, so the
results agree to round-off (bound 1e-12 relative; in practice identical)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2603_29621_gb300 import api
    return api.Context(0)


def test_batch_step_matches_single_solves(ctx):
    from paper_2603_29621_gb300 import _lib as L
    from paper_2603_29621_gb300 import api, inputs
    cases = [(L.STAB_NS, 6, 2, 1e-2), (L.STOKES, 4, 3, 0.3), (L.STAB_NS, 8, 1, 1e-3), (L.STOKES, 6, 2, 1.0)]
    probs, xs, bs, streams = [], [], [], []
    for i, (kind, n, k, nu) in enumerate(cases):
        m = api.Mesh(ctx, 3, n)
        p = api.Problem(ctx, m, kind=kind, degree=k, nu=nu, dt=1e-2 if kind == L.STAB_NS else 0.0,
                        mg_precision=L.FP32, tol=1e-11)
        st = torch.cuda.Stream()
        b = torch.tensor(inputs.uniform_vector(p.info.n_dofs, seed=60 + i), device="cuda")
        x = torch.zeros_like(b)
        p.solve_begin(b, x, stream=st)
        probs.append(p), xs.append(x), bs.append(b), streams.append(st)
    running = [True] * len(probs)
    rounds = 0
    while any(running):
        running = api.batch_step(probs)
        rounds += 1
        assert rounds < 400
    torch.cuda.synchronize()
    for p, x, b in zip(probs, xs, bs):
        st = p.solve_status()
        assert st.converged and st.rel_residual <= 1e-11
        x1 = torch.zeros_like(b)
        info = p.solve(b, x1)
        torch.cuda.synchronize()
        assert info.iterations == st.iterations
        assert torch.equal(x, x1) or float((x - x1).norm() / x1.norm()) <= 1e-12


def test_serving_results_same_alone_and_in_the_mix(ctx):
    from paper_2603_29621_gb300 import _lib as L
    from paper_2603_29621_gb300 import serve
    reqs = serve.poisson_stream(10, rate=200.0, n_range=(4, 10), seed=5)
    srv = serve.Server(ctx, max_active=4, tol=1e-12)
    records, summary = srv.run(reqs, realtime=True, keep_solutions=True)
    srv.close()
    assert summary["requests"] == len(reqs) and summary["all_converged"]
    assert summary["max_error"] <= 1e-8, summary
    byid = {r["rid"]: r for r in records}
    # admission overlapped: more than one request was active in some rounds
    assert summary["rounds"] < sum(r["iterations"] for r in records)
    for req in reqs:
        x_alone, info = serve.solve_alone(ctx, req, tol=1e-12)   # pressure mean removed, like the records
        x_mix = byid[req.rid]["x"]
        xa = x_alone.cpu().numpy()
        assert info.iterations == byid[req.rid]["iterations"]
        assert np.array_equal(xa, x_mix) or np.linalg.norm(xa - x_mix) <= 1e-12 * np.linalg.norm(xa)


def test_serving_respects_the_hbm_budget():
    from paper_2603_29621_gb300 import api, serve
    small = api.Context(0, hbm_budget_bytes=400 * 1024 * 1024)
    reqs = serve.poisson_stream(6, rate=1000.0, n_range=(8, 12), degrees=(2,), seed=9)
    srv = serve.Server(small, max_active=6, tol=1e-10)
    records, summary = srv.run(reqs, realtime=False)
    srv.close()
    used, peak = small.memory()
    assert summary["requests"] == 6 and summary["all_converged"]
    assert peak <= 400 * 1024 * 1024 and used == 0
