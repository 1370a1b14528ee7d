"""CPU checks of index arithmetic that the fused cluster solver relies on.

The fused cluster solver (hh_fused.cuh) splits Omega_B into slabs of z planes
over the blocks of a cluster and gathers spectrum columns from all of them;
the same formulas, restated here, must visit every element of the
six-component half spectrum exactly once, stay inside the owner's slab, and
address every voxel of a block's planes exactly once.
"""

import numpy as np
import pytest


def fused_cols(nz):
    return 2 if nz >= 128 else max(2, min(16, 256 // nz))


def _check_cluster(nx, ny, nz, C, threads=256):
    nxh, RP, zper = nx // 2 + 1, (nx + 2) | 1, (nz + C - 1) // C
    zc = [min(nz, min(r * zper, nz) + zper) - min(r * zper, nz) for r in range(C)]
    assert sum(zc) == nz
    W = fused_cols(nz)
    hit = np.zeros((C, zper * 3 * ny * RP), dtype=np.int64)
    J = ny * nxh
    for rank in range(C):
        jb, je = J * rank // C, J * (rank + 1) // C
        for j0 in range(jb, je, W):
            Wc = min(W, je - j0)
            e = np.arange(6 * nz * Wc)
            jl, cz = e % Wc, e // Wc
            c, z = cz // nz, cz % nz
            j = j0 + jl
            ky, kx = j // nxh, j % nxh
            ow, zl = z // zper, z % zper
            off = ((zl * 3 + (c >> 1)) * ny + ky) * RP + (c & 1) * nxh + kx
            assert (ow < C).all() and (zl < np.array(zc)[ow]).all() and (off < zper * 3 * ny * RP).all()
            np.add.at(hit, (ow, off), 1)
    want = np.zeros_like(hit)
    for ow in range(C):
        for zl in range(zc[ow]):
            for c2 in range(3):
                for ky in range(ny):
                    b = ((zl * 3 + c2) * ny + ky) * RP
                    want[ow, b:b + 2 * nxh] = 1
    assert np.array_equal(hit, want)
    # voxel phases: v -> (plane, y, x) of the block's planes
    for rank in range(C):
        v = np.arange(zc[rank] * nx * ny)
        zl, rem = v // (nx * ny), v % (nx * ny)
        y, x = rem // nx, rem % nx
        so = (zl * 3 * ny + y) * RP + x
        assert (so + 2 * ny * RP < zc[rank] * 3 * ny * RP).all()
        assert len(set(zip(zl.tolist(), y.tolist(), x.tolist()))) == len(v)


@pytest.mark.parametrize("shape", [(16, 16, 16), (26, 18, 18), (48, 32, 32), (17, 13, 7), (40, 40, 9), (40, 40, 5),
                                   (12, 12, 12), (33, 20, 3)])
@pytest.mark.parametrize("C", [1, 2, 4, 8])
def test_fused_cluster_index_maps(shape, C):
    nx, ny, nz = shape
    if C > nz:
        pytest.skip("a cluster never has more blocks than planes")
    _check_cluster(nx, ny, nz, C)


# ------------------------------------------------ division-free index walks
# The plane and column passes walk e = tid, tid + S, ... (S = 256 threads)
# through row-major index spaces without dividing after the first position
# (Walk2: e = hi * W + lo; Walk3: e = (a * B + b) * W + lo). These mirror the
# device structs step for step and check them against divmod over every
# extent the passes use.

def _walk2(e0, S, W):
    hi, lo = divmod(e0, W)
    dhi, dlo = divmod(S, W)
    while True:
        yield hi, lo
        lo += dlo
        hi += dhi
        if lo >= W:
            lo -= W
            hi += 1


def _walk3(e0, S, W, B):
    row, lo = divmod(e0, W)
    a, b = divmod(row, B)
    dhi, dlo = divmod(S, W)
    da0, db0 = divmod(dhi, B)
    da1, db1 = divmod(dhi + 1, B)
    while True:
        yield a, b, lo
        lo += dlo
        da, db = da0, db0
        if lo >= W:
            lo -= W
            da, db = da1, db1
        b += db
        a += da
        if b >= B:
            b -= B
            a += 1


def test_walk2_matches_divmod():
    S = 256
    for W in list(range(1, 50)) + [64, 96, 128, 255, 256, 257, 300]:
        n = 6 * 48 * W
        for tid in range(0, S, 7):
            g = _walk2(tid, S, W)
            for e in range(tid, n, S):
                assert next(g) == divmod(e, W), (W, tid, e)


def test_walk3_matches_divmod():
    S = 256
    for W in range(1, 26):          # nxh of edges 1..48
        for B in range(1, 50):      # ny
            n = 6 * B * W
            for tid in (0, 1, 37, 128, 255):
                g = _walk3(tid, S, W, B)
                for e in range(tid, n, S):
                    row, lo = divmod(e, W)
                    assert next(g) == (*divmod(row, B), lo), (W, B, tid, e)
