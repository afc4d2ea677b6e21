"""mfns_smooth_noalloc against mfns_smooth, through the C ABI.

The no-allocation smoother serves callers that may not allocate device memory
when they call in (for example while a stream is captured, or under a no-malloc
policy after start-up); it keeps its scratch in a fixed device array of the
library.  It must produce what mfns_smooth produces, call after call (the shared
array keeps the previous call's contents), and refuse levels larger than that
array.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _smooth_both(lib, prob, level, b, x0, zero, dtype):
    xa = x0.clone()
    xb = x0.clone()
    prec = 0 if dtype == torch.float64 else 1
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    from paper_2603_29621_gb300 import _lib as L
    n = b.numel()
    L.check(lib.mfns_smooth(prob.h, level, prec, C.c_void_p(b.data_ptr()), C.c_void_p(xa.data_ptr()), n, int(zero),
                            s))
    L.check(lib.mfns_smooth_noalloc(prob.h, level, prec, C.c_void_p(b.data_ptr()), C.c_void_p(xb.data_ptr()), n,
                                    int(zero), s))
    torch.cuda.synchronize()
    return xa.double().cpu().numpy(), xb.double().cpu().numpy()


@pytest.mark.parametrize("smoother", [1, 2])  # Chebyshev, Jacobi relaxation
def test_noalloc_smoother_matches_mfns_smooth(smoother):
    from paper_2603_29621_gb300 import _lib as L
    from paper_2603_29621_gb300 import api, inputs

    ctx = api.Context(0)
    m = api.Mesh(ctx, 3, 4)
    prob = api.Problem(ctx, m, kind=L.STAB_NS, degree=2, nu=1e-2, dt=1e-2, smoother=smoother, smoother_degree=3)
    lib = ctx.lib
    for dtype, tol in ((torch.float64, 1e-11), (torch.float32, 1e-5)):
        for level in (0, 1):
            n = prob.n_dofs(level)
            # two calls in a row with different inputs: the second sees the first call's scratch contents
            for call, zero in enumerate((False, True)):
                b = torch.tensor(inputs.uniform_vector(n, seed=40 + call), device="cuda", dtype=dtype)
                x0 = torch.tensor(inputs.uniform_vector(n, seed=50 + call), device="cuda", dtype=dtype)
                if zero:
                    x0.zero_()
                ref, got = _smooth_both(lib, prob, level, b, x0, zero, dtype)
                err = np.abs(got - ref).max() / np.abs(ref).max()
                assert err <= tol, (dtype, level, call, err)


def test_noalloc_smoother_rejects_levels_beyond_its_scratch():
    from paper_2603_29621_gb300 import _lib as L
    from paper_2603_29621_gb300 import api

    ctx = api.Context(0)
    m = api.Mesh(ctx, 3, 32)
    prob = api.Problem(ctx, m, kind=L.STAB_NS, degree=2, nu=1e-2, dt=1e-2, lambda_max=2.0)
    n = prob.n_dofs(0)
    assert n > (1 << 20)
    b = torch.zeros(n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    code = ctx.lib.mfns_smooth_noalloc(prob.h, 0, 0, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), n, 0,
                                       C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == L.ERR_ARG
    assert b"at most 1048576" in ctx.lib.mfns_last_error()
