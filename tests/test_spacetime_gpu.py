"""The space-time slab operator (Section 4, Eq. 6) on the GPU against the oracle, through the C ABI.

K = G_Q (x) M + tau I_Q (x) A on stage-major vectors, Taylor--Hood in space (uniform meshes and a
ball-refined mesh with hanging nodes), DG(r) in time on right Radau points, r = 0..3: every entry
of K x agrees with the oracle's assembled Kronecker operator to 1e-12 relative (FP64) and 1e-5 in
the 2-norm (FP32)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mesh, spacetime  # noqa: E402
from paper_2603_29621_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu
CENTRE = (0.3, 0.35, 0.4)


@pytest.fixture(scope="module")
def ctx():
    from paper_2603_29621_gb300 import api
    return api.Context(0)


CASES = [(2, 4, False, 2, 1), (2, 3, True, 2, 2), (2, 4, False, 3, 0), (3, 2, False, 2, 1), (3, 2, True, 2, 3),
         (3, 2, False, 3, 1)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}d-n{c[1]}-{'ball' if c[2] else 'uni'}-k{c[3]}-r{c[4]}")
def test_slab_operator_matches_oracle(ctx, case):
    from paper_2603_29621_gb300 import _lib as L, api
    dim, n, ball, k, r = case
    nu, tau = 0.8, 0.3
    f = mesh.uniform(dim, n)
    m = api.Mesh(ctx, dim, n)
    if ball:
        f = mesh.refine_ball(f, CENTRE, 0.3, 1)
        m.refine_ball(CENTRE, 0.3, 1)
    prob = api.Problem(ctx, m, kind=L.STOKES, degree=k, nu=nu, lambda_max=1.0)
    st = api.SpaceTime(prob, r, tau)
    ost = spacetime.SpaceTimeStokes(f, k, r, nu=nu, tau=tau, pressure="continuous")
    assert st.Q == ost.Q and st.n == ost.n
    assert np.abs(st.nodes - ost.nodes).max() <= 1e-14
    assert np.abs(st.G - ost.G_Q).max() <= 1e-12 * np.abs(ost.G_Q).max()
    K = ost.operator()
    xg, fg = prob.support_points()
    xo, fo = ost.space.dofs.support_points()
    perm = inputs.match_dofs(xg, fg, xo, fo)                 # library entry of oracle entry i
    full = (np.arange(st.Q)[:, None] * st.n + perm[None, :]).ravel()
    x = inputs.uniform_vector(st.Q * st.n, seed=11)
    exp = K @ x
    for dtype, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        xd = np.empty_like(x)
        xd[full] = x
        src = torch.tensor(xd, device="cuda", dtype=dtype)
        dst = torch.full_like(src, 7.0)
        st.vmult(src, dst)
        torch.cuda.synchronize()
        got = dst.double().cpu().numpy()[full]
        if dtype == torch.float64:
            assert np.abs(got - exp).max() <= tol * np.abs(exp).max()
        else:
            assert np.linalg.norm(got - exp) <= tol * np.linalg.norm(exp)


def test_slab_rejects_other_problems(ctx):
    from paper_2603_29621_gb300 import _lib as L, api
    m = api.Mesh(ctx, 2, 3)
    prob = api.Problem(ctx, m, kind=L.STOKES_A, degree=2, lambda_max=1.0)
    with pytest.raises(L.MfnsError) as e:
        api.SpaceTime(prob, 1, 0.1)
    assert e.value.code == L.ERR_UNSUPPORTED
