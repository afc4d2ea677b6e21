"""GPU operator parity against the oracle, through the C ABI.

Each case builds the same mesh on both sides, maps the library's DoF order to
the oracle's by (support point, field), applies the matrix-free operator to a
seeded U(-1,1) vector and compares with the oracle's assembled A = C^T K C (+) I
element by element: relative l2 error <= 1e-12 in FP64 (the accuracy target of the path) and
<= 2e-5 in FP32 (single-precision round-off of a ~10^3-term sum per entry)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import assemble, mesh  # noqa: E402
from paper_2603_29621_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

KINDS = {"stokes": 0, "stokes_a": 1, "stab_ns": 2, "pmass": 3}
TOL = {0: 1e-12, 1: 2e-5}


@pytest.fixture(scope="module")
def ctx():
    from paper_2603_29621_gb300 import api
    return api.Context(0)


def _make(ctx, kind, dim, n, k, refine, **phys):
    from paper_2603_29621_gb300 import api
    m = api.Mesh(ctx, dim, n)
    f = mesh.uniform(dim, n)
    if refine:
        m.refine_ball(refine[0], refine[1], refine[2])
        f = mesh.refine_ball(f, refine[0], refine[1], refine[2])
    prob = api.Problem(ctx, m, kind=KINDS[kind], degree=k, lambda_max=1.0, **phys)
    oprob = assemble.Problem(f, kind, k, nu=phys.get("nu", 1.0), dt=phys.get("dt", 0) or np.inf,
                             terms=phys.get("terms", 127) or 127)
    xg, fg = prob.support_points()
    xo, fo = oprob.dofs.support_points()
    if kind == "pmass":  # the library labels the single pressure-like field with index dim
        fo = fo + dim
    perm = inputs.match_dofs(xg, fg, xo, fo)
    return prob, oprob, perm


def _vmult(prob, perm, x, prec, which=-1):
    xd = np.empty_like(x)
    xd[perm] = x
    dt = torch.float64 if prec == 0 else torch.float32
    src = torch.tensor(xd, device="cuda", dtype=dt)
    dst = torch.full_like(src, 7.0)
    prob.vmult(src, dst, which=which)
    torch.cuda.synchronize()
    return dst.double().cpu().numpy()[perm]


BALL = ((0.3, 0.3, 0.3), 0.3, 1)
CASES = [
    # kind, dim, n, k, refine, physics
    ("stab_ns", 3, 2, 2, None, dict(nu=1e-2, dt=1e-2)),
    ("stab_ns", 3, 3, 1, None, dict(nu=1e-1, dt=5e-2)),
    ("stab_ns", 3, 2, 3, None, dict(nu=1e-3, dt=1e-2)),
    ("stab_ns", 2, 4, 2, None, dict(nu=1e-2, dt=1e-2)),
    ("stab_ns", 2, 3, 4, None, dict(nu=2e-2, dt=0.0)),
    ("stab_ns", 3, 2, 2, BALL, dict(nu=1e-2, dt=1e-2)),
    ("stab_ns", 2, 2, 3, BALL, dict(nu=1e-2, dt=1e-1)),
    ("stokes", 2, 4, 2, None, dict(nu=1.0)),
    ("stokes", 3, 2, 2, None, dict(nu=0.5)),
    ("stokes", 3, 2, 3, None, dict(nu=1.0)),
    ("stokes", 2, 2, 4, None, dict(nu=1.0)),
    ("stokes", 3, 2, 2, BALL, dict(nu=1.0)),
    ("stokes", 2, 2, 3, BALL, dict(nu=1.0)),
    ("stokes_a", 3, 3, 1, None, dict(nu=1.0)),
    ("stokes_a", 3, 2, 4, None, dict(nu=2.0)),
    ("stokes_a", 3, 2, 2, BALL, dict(nu=1.0)),
    ("stokes_a", 2, 4, 3, BALL, dict(nu=1.0)),
    ("pmass", 3, 3, 1, None, dict(nu=1.0)),
    ("pmass", 2, 2, 3, BALL, dict(nu=1.0)),
    # edge cases: one cell (seven empty colours), odd n (colours of unequal size, ragged last
    # blocks in every colour launch), a level of many blocks
    ("stab_ns", 3, 1, 2, None, dict(nu=1e-2, dt=1e-2)),
    ("stab_ns", 3, 5, 2, None, dict(nu=1e-2, dt=1e-2)),
    ("stab_ns", 3, 7, 2, None, dict(nu=5e-3, dt=2e-2)),
    ("stab_ns", 2, 1, 2, None, dict(nu=1e-2, dt=1e-2)),
    ("stokes_a", 3, 1, 2, None, dict(nu=1.0)),
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[1]}d-n{c[2]}-k{c[3]}-{'ball' if c[4] else 'uni'}")
def test_vmult_matches_oracle(ctx, case, prec):
    kind, dim, n, k, refine, phys = case
    prob, oprob, perm = _make(ctx, kind, dim, n, k, refine, **phys)
    x = inputs.uniform_vector(len(perm))
    y = _vmult(prob, perm, x, prec)
    yo = oprob.vmult(x)
    rel = np.linalg.norm(y - yo) / np.linalg.norm(yo)
    assert rel <= TOL[prec], rel
    # constrained rows are identity
    c = oprob.dofs.constrained
    assert np.allclose(y[c], x[c], rtol=0, atol=1e-6 if prec else 0.0)


@pytest.mark.parametrize("case", [CASES[0], CASES[5], CASES[11], CASES[16]], ids=lambda c: f"{c[0]}-{c[1]}d")
def test_diagonal_matches_oracle(ctx, case):
    kind, dim, n, k, refine, phys = case
    prob, oprob, perm = _make(ctx, kind, dim, n, k, refine, **phys)
    d = torch.zeros(len(perm), dtype=torch.float64, device="cuda")
    prob.diagonal(d)
    torch.cuda.synchronize()
    dg = d.cpu().numpy()[perm]
    do = oprob.assemble().diagonal()
    assert np.abs(dg - do).max() <= 1e-12 * np.abs(do).max()


@pytest.mark.parametrize("case", [CASES[5], CASES[11], CASES[6]], ids=lambda c: f"{c[0]}-{c[1]}d")
def test_apply_constraints_matches_oracle(ctx, case):
    kind, dim, n, k, refine, phys = case
    prob, oprob, perm = _make(ctx, kind, dim, n, k, refine, **phys)
    x = inputs.uniform_vector(len(perm))
    xd = np.empty_like(x)
    xd[perm] = x
    t = torch.tensor(xd, device="cuda")
    prob.apply_constraints(t)
    torch.cuda.synchronize()
    y = t.cpu().numpy()[perm]
    d = oprob.dofs
    # oracle: hanging entries from all masters (free and boundary), other entries unchanged
    expect = x.copy()
    for f, (nc, kk, dbc) in enumerate(d.fields):
        ns = d.nodesets[f]
        for c in range(nc):
            base = d.offsets[f] + c * ns.n_nodes
            for g, masters in ns.hanging.items():
                if d.dirichlet[base + g]:
                    continue
                expect[base + g] = sum(w * x[base + m] for m, w in masters)
    assert np.abs(y - expect).max() < 1e-13


def test_wrong_vector_lengths_are_rejected_and_leave_the_runtime_clean(ctx):
    """Every vector crosses the C ABI with its length: a length other than the one the call expects
    is MFNS_ERR_ARG (nothing read or written), and no CUDA error is left pending for the caller's
    next call.  Local smoothing: the V-cycle takes vectors of cycle_dofs (the fine operator), not of
    level_dofs[0] (the finest refinement level)."""
    import ctypes as C
    from paper_2603_29621_gb300 import _lib as L, api
    lib = ctx.lib
    m = api.Mesh(ctx, 3, 2)
    prob = api.Problem(ctx, m, kind=L.STAB_NS, degree=2, nu=1e-2, dt=1e-2, lambda_max=1.0)
    n = prob.info.n_dofs
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    src = torch.rand(n + 8, dtype=torch.float64, device="cuda")
    dst = torch.full((n + 8,), 7.0, dtype=torch.float64, device="cuda")
    p = lambda t: C.c_void_p(t.data_ptr())
    assert lib.mfns_vmult(prob.h, L.OP_SYSTEM, L.FP64, p(src), p(dst), n - 1, s) == L.ERR_ARG
    assert b"expected" in lib.mfns_last_error()
    assert lib.mfns_vmult(prob.h, L.OP_SYSTEM, L.FP64, p(src), p(dst), n + 8, s) == L.ERR_ARG
    assert lib.mfns_vcycle(prob.h, L.FP64, p(src), p(dst), n + 1, s) == L.ERR_ARG
    assert lib.mfns_solve(prob.h, p(src), p(dst), n - 4, None, s) == L.ERR_ARG
    assert lib.mfns_smooth(prob.h, 0, L.FP64, p(src), p(dst), n + 1, 0, s) == L.ERR_ARG
    nc = prob.info.level_dofs[1]
    assert lib.mfns_prolongate_add(prob.h, 0, L.FP64, p(src), nc + 1, p(dst), n, s) == L.ERR_ARG
    assert lib.mfns_restrict(prob.h, 0, L.FP64, p(src), n, p(dst), nc - 1, s) == L.ERR_ARG
    torch.cuda.synchronize()
    assert bool((dst == 7.0).all())                      # nothing written
    y = src.clone() * 2                                  # the caller's runtime has no pending error
    torch.cuda.synchronize()
    assert float(y.sum()) > 0
    with pytest.raises(ValueError):
        prob.vmult(src, dst)                             # the binding checks before calling in
    # local smoothing: vcycle vectors have cycle_dofs entries
    m2 = api.Mesh(ctx, 2, 4)
    m2.refine_ball((0.3, 0.35, 0.4), 0.3, 1)
    pl = api.Problem(ctx, m2, kind=L.STOKES_A, degree=2, hierarchy=L.LOCAL_SMOOTHING, lambda_max=1.0)
    assert pl.info.cycle_dofs == pl.info.n_dofs != pl.info.level_dofs[0]
    short = torch.zeros(pl.info.level_dofs[0], dtype=torch.float64, device="cuda")
    assert lib.mfns_vcycle(pl.h, L.FP64, p(short), p(torch.zeros_like(short)), short.numel(), s) == L.ERR_ARG
    b = torch.rand(pl.info.cycle_dofs, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    pl.vcycle(b, x)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(x).all()) and float(x.abs().max()) > 0


@pytest.mark.parametrize("prec", [0, 1])
def test_vmult_host_equals_device_product(ctx, prec):
    """mfns_vmult_host (host vectors in and out, copies and products pipelined over two staging
    sets): every result is bitwise the device product of its input -- four vectors (both staging
    sets used twice, one source listed twice), a second call reusing the staging, and pageable host
    memory; wrong lengths and counts are rejected without touching memory."""
    import ctypes as C
    from paper_2603_29621_gb300 import _lib as L, api
    m = api.Mesh(ctx, 3, 3)
    prob = api.Problem(ctx, m, kind=L.STAB_NS, degree=2, nu=1e-2, dt=1e-2, lambda_max=1.0)
    n = prob.info.n_dofs
    dt = torch.float64 if prec == 0 else torch.float32
    hs = [torch.tensor(inputs.uniform_vector(n, seed=20 + i), dtype=dt).pin_memory() for i in range(3)]
    srcs = [hs[0], hs[1], hs[2], hs[0]]
    dsts = [torch.full((n,), 7.0, dtype=dt).pin_memory() for _ in srcs]
    refs = []
    for s_ in srcs:
        r = torch.empty(n, dtype=dt, device="cuda")
        prob.vmult(s_.cuda(), r)
        refs.append(r)
    torch.cuda.synchronize()
    refs = [r.cpu() for r in refs]
    for _ in range(2):
        for d_ in dsts:
            d_.fill_(7.0)
        prob.vmult_host(srcs, dsts)
        torch.cuda.synchronize()
        for d_, r in zip(dsts, refs):
            assert torch.equal(d_, r)
    pageable = torch.empty(n, dtype=dt)
    prob.vmult_host([hs[1].clone()], [pageable])
    torch.cuda.synchronize()
    assert torch.equal(pageable, refs[1])
    lib = ctx.lib
    sp = (C.c_void_p * 1)(hs[0].data_ptr())
    dp = (C.c_void_p * 1)(dsts[0].data_ptr())
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    before = dsts[0].clone()
    assert lib.mfns_vmult_host(prob.h, L.OP_SYSTEM, prec, sp, dp, 1, n + 1, s) == L.ERR_ARG
    assert lib.mfns_vmult_host(prob.h, L.OP_SYSTEM, prec, sp, dp, 0, n, s) == L.ERR_ARG
    torch.cuda.synchronize()
    assert torch.equal(dsts[0], before)
    with pytest.raises(ValueError):
        prob.vmult_host([hs[0].cuda()], [dsts[0]])
