"""CPU checks of index arithmetic that the CUDA kernels rely on.

FDiv (hh_fftcore.cuh) replaces integer division in the transforms' index
arithmetic by a product with a single-precision reciprocal and one
correction step; the argument in its comment (exact for 0 <= n < 2^22) is
checked here exhaustively for a range of divisors, with numpy's IEEE
single-precision arithmetic standing in for the device's.

The fused cluster solver (hh_fused.cuh) splits Omega_B into slabs of z planes
over the blocks of a cluster and gathers spectrum columns through offset
tables; the same formulas, restated here, must visit every element of the
six-component half spectrum exactly once, stay inside the owner's slab, and
walk every voxel of a block's planes exactly once.
"""

import numpy as np
import pytest


def fdiv(n, d):
    r = np.float32(1.0) / np.float32(d)
    q = (n.astype(np.float32) * r).astype(np.int64)
    rem = n - q * d
    return q + (rem >= d).astype(np.int64) - (rem < 0).astype(np.int64)


def test_reciprocal_quotient_is_exact_below_2_pow_22():
    n = np.arange(0, 1 << 22, dtype=np.int64)
    for d in list(range(1, 130)) + [255, 256, 257, 1000, 1023, 1024, 4095, 65537, 1 << 20, 1 << 30]:
        assert np.array_equal(fdiv(n, d), n // d), d


def fused_cols(nz, tbytes):
    w = (512 // nz) // (tbytes // 4)
    return max(2, min(32, w))


def _check_cluster(nx, ny, nz, C, tbytes, threads=1024):
    nxh, RP, zper = nx // 2 + 1, (nx + 2) | 1, (nz + C - 1) // C
    zc = [min(nz, min(r * zper, nz) + zper) - min(r * zper, nz) for r in range(C)]
    assert sum(zc) == nz
    zo = []
    for t in range(6 * nz):
        c, z = divmod(t, nz)
        ow, zl = divmod(z, zper)
        zo.append(ow | ((((zl * 3 + (c >> 1)) * ny) * RP + (c & 1) * nxh) << 4))
    W = fused_cols(nz, tbytes)
    rs = threads // W
    hit = np.zeros((C, zper * 3 * ny * RP), dtype=np.int64)
    J = ny * nxh
    for rank in range(C):
        jb, je = J * rank // C, J * (rank + 1) // C
        for j0 in range(jb, je, W):
            Wc = min(W, je - j0)
            jj = np.arange(j0, j0 + Wc)
            co = (jj // nxh) * RP + jj % nxh
            for cz in range(6 * nz):  # every (component, plane) row is some thread's
                ow, off = zo[cz] & 15, (zo[cz] >> 4) + co
                assert ow < C and (off < zc[ow] * 3 * ny * RP).all() and cz * W + Wc <= W * 6 * nz
                np.add.at(hit[ow], off, 1)
            assert rs >= 1
    # exactly the spectrum positions: pair row (zl, c2, ky), halves (c & 1) * nxh + kx
    want = np.zeros_like(hit)
    for ow in range(C):
        for zl in range(zc[ow]):
            for c2 in range(3):
                for ky in range(ny):
                    b = ((zl * 3 + c2) * ny + ky) * RP
                    want[ow, b:b + 2 * nxh] = 1
    assert np.array_equal(hit, want)
    # row walk of the voxel phases
    for rank in range(C):
        rows, step, seen = zc[rank] * ny, threads // nx, 0
        for t in range(min(threads, step * nx)):
            x, row = t % nx, t // nx
            zl, y = divmod(row, ny)
            while row < rows:
                assert (zl, y) == divmod(row, ny)
                assert (zl * 3 * ny + y) * RP + x + 2 * ny * RP < zc[rank] * 3 * ny * RP
                seen += 1
                row += step
                y += step
                while y >= ny:
                    y -= ny
                    zl += 1
        assert seen == rows * nx


@pytest.mark.parametrize("shape", [(16, 16, 16), (26, 18, 18), (48, 32, 32), (17, 13, 7), (40, 40, 9), (40, 40, 5),
                                   (12, 12, 12), (33, 20, 3)])
@pytest.mark.parametrize("C", [1, 2, 4, 8])
@pytest.mark.parametrize("tbytes", [4, 8])
def test_fused_cluster_index_maps(shape, C, tbytes):
    nx, ny, nz = shape
    if C > nz:
        pytest.skip("a cluster never has more blocks than planes")
    _check_cluster(nx, ny, nz, C, tbytes)
