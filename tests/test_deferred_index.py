"""Index arithmetic of the deferred product of a uniform 3D level (host-side model, CPU).

The deferred launch spans every colour (blockIdx.y = colour) with the block count of the largest
colour; each team decomposes its cell index as the colour launches do, and a colour with no cell
(one cell per direction) returns before touching memory.  The gather pass finds, for every node of
the (k n + 1)^3 lattice, its cells colour by colour.  This model of both checks that every cell is
processed exactly once, that no lane's cell position or per-cell buffer entry leaves its range,
and that the gather's cells of a node, with their positions and local slots, are exactly the cells
whose closed box holds the node (brute force)."""
import itertools

import pytest


def _check(n, K, warps=4, CPW=3):
    nb1 = K + 1; NB = nb1 ** 3
    off = []; o = 0; tot = []
    for c in range(8):
        m = [(n - ((c >> d) & 1) + 1) // 2 for d in range(3)]
        nc = m[0] * m[1] * m[2]; off.append(o); o += nc; tot.append(nc)
    ncells = o; assert ncells == n ** 3
    cpb = warps * CPW
    gx = (max(tot) + cpb - 1) // cpb
    seen = {}
    for c in range(8):
        bits = [(c >> d) & 1 for d in range(3)]
        m = [(n - bits[d] + 1) // 2 for d in range(3)]
        total = m[0] * m[1] * m[2]
        for bx in range(gx):
            for w in range(warps):
                for team in range(CPW):
                    t = bx * cpb + w * CPW + team
                    if total == 0:
                        continue          # the block returns before touching memory
                    valid = t < total
                    tt = t if valid else total - 1
                    cc = [2 * (tt % m[0]) + bits[0], 2 * ((tt // m[0]) % m[1]) + bits[1], 2 * (tt // (m[0] * m[1])) + bits[2]]
                    assert all(0 <= x < n for x in cc), (n, K, c, t, cc)
                    pos = off[c] + tt
                    assert 0 <= pos < ncells
                    assert (pos * NB + NB - 1) * 4 + 3 < ncells * NB * 4
                    if valid:
                        assert pos not in seen
                        seen[pos] = tuple(cc)
    assert len(seen) == ncells
    # gather: every node's cells, by colour, must be the kernel's (position, slot)
    M = K * n + 1
    for i in itertools.product(range(M), repeat=3):
        cells = []
        for c in range(8):
            cd = []; loc = []; ok = True
            for d in range(3):
                b = (c >> d) & 1; q, r = divmod(i[d], K)
                if r != 0: cell = q; ok &= (cell & 1) == b
                elif (q & 1) == b: cell = q; ok &= q < n
                else: cell = q - 1; ok &= q >= 1
                cd.append(cell); loc.append(i[d] - K * cell)
            if not ok: continue
            m0 = (n - (c & 1) + 1) // 2; m1 = (n - ((c >> 1) & 1) + 1) // 2
            pos = off[c] + (cd[0] >> 1) + m0 * ((cd[1] >> 1) + m1 * (cd[2] >> 1))
            assert seen[pos] == tuple(cd), (n, K, i, c)
            assert all(0 <= l <= K for l in loc)
            cells.append(tuple(cd))
        # brute force: the cells whose closed box holds the node
        brute = {cx for cx in itertools.product(range(n), repeat=3) if all(K * cx[d] <= i[d] <= K * (cx[d] + 1) for d in range(3))}
        assert set(cells) == brute and len(cells) == len(brute), (n, K, i)


@pytest.mark.parametrize("K", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7])
def test_deferred_launch_and_gather_indexing(n, K):
    _check(n, K)
