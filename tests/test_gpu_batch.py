"""Batched multi-problem V-cycles (one launch per level and colour over uneven problems).

The batched V-cycle must give, for every problem, exactly (bitwise) what the problem's own
V-cycle gives: each block of a multi-problem launch reads its problem's fields from a descriptor
table and performs the per-cell arithmetic of a single-problem launch in the same order.  The
batch mixes dimensions, degrees, operators, mesh sizes (different hierarchy depths, odd sizes
with non-nested coarsening) and multigrid precisions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2603_29621_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

# (kind, dim, n, k, physics)
MIX = [
    ("stab_ns", 3, 6, 2, dict(nu=1e-2, dt=1e-2)),
    ("stab_ns", 3, 4, 2, dict(nu=1e-1, dt=5e-2)),
    ("stab_ns", 3, 5, 1, dict(nu=1e-2, dt=1e-2)),
    ("stab_ns", 3, 3, 3, dict(nu=1e-3, dt=1e-2)),
    ("stab_ns", 2, 9, 3, dict(nu=1e-2, dt=1e-2)),
    ("stokes_a", 3, 4, 2, dict(nu=1.0)),
    ("stokes_a", 3, 7, 3, dict(nu=0.5)),
    ("stokes_a", 2, 8, 2, dict(nu=1.0)),
]


@pytest.fixture(scope="module")
def ctx():
    from paper_2603_29621_gb300 import api
    return api.Context(0)


def _problems(ctx, mgp):
    from paper_2603_29621_gb300 import _lib as L, api
    kinds = {"stab_ns": L.STAB_NS, "stokes_a": L.STOKES_A}
    out = []
    for kind, dim, n, k, phys in MIX:
        m = api.Mesh(ctx, dim, n)
        out.append((api.Problem(ctx, m, kind=kinds[kind], degree=k, mg_precision=mgp, **phys), m))
    return out


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_batched_vcycle_equals_single_vcycles(ctx, prec):
    from paper_2603_29621_gb300 import api
    pm = _problems(ctx, prec)
    probs = [p for p, _ in pm]
    dt = torch.float64 if prec == 0 else torch.float32
    bs = [torch.tensor(inputs.uniform_vector(p.info.n_dofs, seed=40 + i), device="cuda", dtype=dt)
          for i, p in enumerate(probs)]
    depth = {p.info.n_levels for p in probs}
    assert len(depth) >= 3  # hierarchies of different depth share the batch
    single = []
    for p, b in zip(probs, bs):
        x = torch.zeros_like(b)
        p.vcycle(b, x)
        single.append(x)
    xs = [torch.full_like(b, 3.0) for b in bs]
    api.batch_vcycle(probs, bs, xs)
    torch.cuda.synchronize()
    for i, (a, b) in enumerate(zip(xs, single)):
        assert torch.equal(a, b), (MIX[i], float((a - b).abs().max()))
    # a second batched call (plans rebuilt) gives the same again
    xs2 = [torch.zeros_like(b) for b in bs]
    api.batch_vcycle(probs, bs, xs2)
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(xs2, single))


def test_batched_vcycle_rejects_unsupported(ctx):
    from paper_2603_29621_gb300 import _lib as L, api
    m = api.Mesh(ctx, 3, 2)
    m.refine_ball((0.3, 0.3, 0.3), 0.3, 1)
    p_ref = api.Problem(ctx, m, kind=L.STOKES_A, degree=2, nu=1.0)
    m2 = api.Mesh(ctx, 3, 4)
    p_uni = api.Problem(ctx, m2, kind=L.STOKES_A, degree=2, nu=1.0)
    b = [torch.zeros(p.info.n_dofs, device="cuda", dtype=torch.float64) for p in (p_uni, p_ref)]
    x = [torch.zeros_like(v) for v in b]
    with pytest.raises(L.MfnsError) as e:
        api.batch_vcycle([p_uni, p_ref], b, x)
    assert e.value.code == L.ERR_UNSUPPORTED


def test_batch_step_uses_batched_preconditioners_and_matches_solo(ctx):
    """mfns_batch_step with several stab-NS / vector-Laplacian problems (batched preconditioner
    graph) reproduces each problem's own solve bitwise."""
    from paper_2603_29621_gb300 import api
    pm = _problems(ctx, 1)
    probs = [p for p, _ in pm]
    bs = [torch.tensor(inputs.uniform_vector(p.info.n_dofs, seed=60 + i), device="cuda") for i, p in enumerate(probs)]
    solo = []
    for p, b in zip(probs, bs):
        x = torch.zeros_like(b)
        p.solve(b, x, raise_on_nonconvergence=False)
        solo.append((x, p.solve_status().iterations))
    xs = [torch.zeros_like(b) for b in bs]
    streams = [torch.cuda.Stream() for _ in probs]
    for p, b, x, st in zip(probs, bs, xs, streams):
        p.solve_begin(b, x, stream=st)
    running = [True] * len(probs)
    rounds = 0
    while any(running):
        running = api.batch_step(probs)
        rounds += 1
        assert rounds < 2000
    torch.cuda.synchronize()
    for i, (p, x) in enumerate(zip(probs, xs)):
        assert p.solve_status().iterations == solo[i][1]
        assert torch.equal(x, solo[i][0]), (MIX[i], float((x - solo[i][0]).abs().max()))
