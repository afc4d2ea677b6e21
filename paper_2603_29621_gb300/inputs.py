"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws random numbers and maps vectors between the library's
DoF order and another order by support-point coordinates; it holds none of the
method's arithmetic.
"""
import numpy as np

SEED_SRC = 0      # source vectors
SEED_LAMBDA = 1   # eigenvalue-estimate start vectors (inside the library)
SEED_SERVE = 2    # serving request stream


def uniform_vector(n, seed=SEED_SRC, low=-1.0, high=1.0):
    """PCG64 U(low, high) vector of length n (float64)."""
    return np.random.default_rng(seed).uniform(low, high, n)


def match_dofs(xa, fa, xb, fb, digits=9):
    """Permutation perm with (xa[perm[i]], fa[perm[i]]) == (xb[i], fb[i]) (coordinates rounded to
    `digits` decimals); both sides are sorted by the integer key (coordinates, field) and paired."""
    xa, xb = np.asarray(xa, dtype=float), np.asarray(xb, dtype=float)

    def keys(x, f):
        q = np.rint(np.round(x, digits) * 10.0 ** digits).astype(np.int64)
        return np.column_stack([q, np.asarray(f, dtype=np.int64)])

    ka, kb = keys(xa, fa), keys(xb, fb)
    if ka.shape != kb.shape:
        raise ValueError("the two DoF sets differ in size")
    oa = np.lexsort(ka.T[::-1])
    ob = np.lexsort(kb.T[::-1])
    sa, sb = ka[oa], kb[ob]
    if len(sa) > 1 and np.any(np.all(sa[1:] == sa[:-1], axis=1)):
        raise ValueError("duplicate support points")
    if not np.array_equal(sa, sb):
        raise ValueError("the two DoF sets have different support points")
    perm = np.empty(len(kb), dtype=np.int64)
    perm[ob] = oa
    return perm


def smooth_solution(xyz, field, dim, pressure_scale=1.0):
    """Smooth manufactured discrete solution x* sampled at support points (xyz, field):
    velocity component c = (1 + c/2) sin(pi x) sin(pi y) [sin(pi z)] + c x y / 4,
    pressure = pressure_scale * cos(pi x) cos(2 pi y) [cos(pi z)]."""
    x, y = xyz[:, 0], xyz[:, 1]
    z = xyz[:, 2] if dim == 3 else np.zeros_like(x)
    sz = np.sin(np.pi * z) if dim == 3 else 1.0
    cz = np.cos(np.pi * z) if dim == 3 else 1.0
    out = np.empty(len(field))
    for c in range(dim):
        sel = field == c
        out[sel] = ((1 + 0.5 * c) * np.sin(np.pi * x) * np.sin(np.pi * y) * sz + 0.25 * c * x * y)[sel]
    sel = field == dim
    out[sel] = (pressure_scale * np.cos(np.pi * x) * np.cos(2 * np.pi * y) * cz)[sel]
    return out


def taylor_green_state(xyz, field, dim):
    """Initial condition sampled at support points (xyz, field): the Taylor--Green field
    u = (sin 2 pi x cos 2 pi y cos 2 pi z, -cos 2 pi x sin 2 pi y cos 2 pi z, 0),
    p = (cos 4 pi x + cos 4 pi y)(cos 4 pi z + 2) / 16 (2D: without the z factors)."""
    tp = 2.0 * np.pi
    x, y = xyz[:, 0], xyz[:, 1]
    cz = np.cos(tp * xyz[:, 2]) if dim == 3 else 1.0
    pz = (np.cos(2 * tp * xyz[:, 2]) + 2.0) if dim == 3 else 1.0
    vals = [np.sin(tp * x) * np.cos(tp * y) * cz, -np.cos(tp * x) * np.sin(tp * y) * cz]
    if dim == 3:
        vals.append(np.zeros_like(x))
    vals.append((np.cos(2 * tp * x) + np.cos(2 * tp * y)) * pz / 16.0)
    out = np.empty(len(field))
    for c in range(dim + 1):
        sel = field == c
        out[sel] = vals[c][sel]
    return out
