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
