"""The benchmark's workload at its full size, in the benchmark's launch
configuration, against the FP64 oracle on sampled subimages and against
properties that hold at any size on every subimage.

Workload: the 512^3 overlapping-sphere sandstone (solid K = 37, G = 44 GPa;
pore 1e-4 GPa: contrast 4.4e5) cut into 27,000 uneven cores of edge 16/24/32
with buffers 0..8; one call homogenizes one tile of 180 cores (one z-slab by
six y-rows of the core grid) with FP32 fields, tol 1e-5 and coarse unit 8,
as every timed step does.

The oracle needs about a minute per subimage at this contrast, so it solves
four of the tile's subimages one by one, in a spawned process pool while the
GPU works: the smallest unbuffered core, the smallest buffered one, and the
smallest subimages whose core has a 24-voxel and a 32-voxel edge (the tile's
z-slab is 16 voxels high, so those cores are 24 x 16 x 16 and 32 x 16 x 16),
each to a relative residual of 1e-6 (oracle solves of the first sample
stopped at 1e-5 and at 1e-7 differ in K and G by a few 1e-7). The bar is the
benchmark's accuracy criterion against plain FP64: 0.5 % on K and G, and
0.5 % of the largest entry on C_R. Measured in the first version of this
test: the unbuffered 16^3 core agrees to 2e-6; the buffered 18^3 core, whose
FP32 true residual stalls at 1.8e-4 on one load case (the not-converged
warning), to 1.3e-3 in K, 1.3e-4 in G and 1.6e-3 on C_R.

The largest subimage of the tile (core 32 x 16 x 16, buffer 8: 48 x 32 x 32)
is too slow for a converged oracle solve; the whole tile is solved a second
time in the same launch configuration at a fixed 20 iterations, and that
subimage's C_R is compared with the oracle's 20 iterations to 2e-5 (the FP32
operator tolerance of the parity tests), as are the 24- and 32-edge samples.

Properties on all 180 subimages: every load case stopped below max_iter with
a true residual under 1e-3 (FP32 stalls a few load cases above tol at this
contrast, which ends them with the not-converged warning);
for unbuffered cores (C_R = <sigma> per unit load) the diagonal entries lie
between the Reuss and Voigt bounds of the core's own phase fractions and
sym(C_R) is positive definite (the conjugate-gradient iterates start at the
Voigt energy and decrease towards the exact one, which the Reuss bound
bounds from below; 1e-3 relative slack for the stopping tolerance); the
level-2 stiffness of the tile is symmetric positive definite.
"""

import multiprocessing as mp

import numpy as np
import pytest

import bench
from oracle import hh_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a CUDA device")
    from paper_2208_02320_gb300 import Context, _build
    _build.build()
    c = Context(0)
    yield c
    c.close()


def _oracle_job(img, box, ph, tol):
    """Arguments of one oracle solve of a buffered box (core = Omega_R)."""
    B = int(box[6])
    core = (slice(B, B + int(box[5])), slice(B, B + int(box[4])), slice(B, B + int(box[3])))
    return O.IsoMedium.from_labels(O.extract_box(img, box), ph), core, tol


def _bounds_diag(labels, ph):
    """Diagonal Voigt and Reuss stiffness entries (normal, shear) of the
    phase mixture of `labels`."""
    f = np.bincount(labels.ravel(), minlength=len(ph)) / labels.size
    K, G = ph[:, 0], ph[:, 1]
    KV, GV = f @ K, f @ G
    KR, GR = 1.0 / (f @ (1.0 / K)), 1.0 / (f @ (1.0 / G))
    return (KV + 4.0 * GV / 3.0, GV), (KR + 4.0 * GR / 3.0, GR)


def test_full_size_tile_against_oracle_and_bounds(ctx):
    img, ph, boxes, tiles = bench.workload(6)
    tile = tiles[0]
    assert len(tile) == 180 and img.shape == (512, 512, 512)
    sizes = (tile[:, 3:6] + 2 * tile[:, 6:7]).prod(axis=1)
    b0 = [i for i in range(len(tile)) if tile[i, 6] == 0]
    bb = [i for i in range(len(tile)) if tile[i, 6] > 0]
    e24 = [i for i in range(len(tile)) if tile[i, 3:6].max() == 24]
    e32 = [i for i in range(len(tile)) if tile[i, 3:6].max() == 32]
    sample = [min(b0, key=lambda i: sizes[i]), min(bb, key=lambda i: sizes[i]),
              min(e24, key=lambda i: sizes[i]), min(e32, key=lambda i: sizes[i])]
    big = int(np.argmax(sizes))
    assert (tile[big, 3:6] + 2 * tile[big, 6]).max() >= 40
    fixed = [big, sample[2], sample[3]]
    jobs = [_oracle_job(img, tile[k], ph, 1e-6) for k in sample]
    fjobs = [_oracle_job(img, tile[k], ph, 1e-6)[:2] + (1e-6, 20000, "component", 20) for k in fixed]
    with mp.get_context("spawn").Pool(len(jobs) + len(fjobs)) as pool:
        pending = pool.starmap_async(O.homogenize_box, jobs)
        fpending = pool.starmap_async(O.homogenize_box, fjobs)
        r = ctx.homogenize_partition(img, ph, tile, unit=8, precision="fp32", tol=1e-5)
        rf = ctx.solve_subimages(img, ph, tile, precision="fp32", fixed_iters=20)
        ref_C = [o["C"] for o in pending.get(timeout=1500)]
        fref_C = [o["C"] for o in fpending.get(timeout=1500)]

    # At contrast 4.4e5 the FP32 true residual of a few load cases stalls
    # above tol (3e-5 on the benchmark's tiles, 1.8e-4 on this one): those stop
    # with the not-converged warning (status 1, results filled), as every timed
    # step of the benchmark does. The bound only catches a divergence; the
    # accuracy is judged by the oracle samples below.
    print(f"status {r['status']}, resid_max {r['resid_max']:.2e}, iters_max {r['iters_max']}")
    assert r["status"] in (0, 1) and r["resid_max"] < 1e-3 and r["n_subimages"] == 180
    # a core without pore voxels has a zero right-hand side: 0 iterations
    assert (r["iters_boxes"] >= 0).all() and (r["iters_boxes"] < 20000).all()
    Ceff = 0.5 * (r["C"] + r["C"].T)
    assert np.abs(r["C"] - r["C"].T).max() <= 1e-3 * np.abs(Ceff).max()
    assert np.linalg.eigvalsh(Ceff).min() > 0.0

    # sampled subimages against the FP64 oracle
    errs = []
    for k, Cref in zip(sample, ref_C):
        got = r["C_boxes"][k]
        Kg, Gg = O.moduli_voigt(0.5 * (got + got.T))
        Kr, Gr = O.moduli_voigt(0.5 * (Cref + Cref.T))
        errs.append((abs(Kg - Kr) / Kr, abs(Gg - Gr) / Gr, np.abs(got - Cref).max() / np.abs(Cref).max()))
        print(f"box {k} {tile[k].tolist()}: K {Kg:.6f} vs {Kr:.6f}, G {Gg:.6f} vs {Gr:.6f}, "
              f"max|dC| / max|C| {errs[-1][2]:.2e}, iterations {r['iters_boxes'][k].tolist()}")

    # properties of every unbuffered core
    bad = []
    for k in b0:
        lab = O.extract_box(img, tile[k])
        (nV, sV), (nR, sR) = _bounds_diag(lab, ph)
        C = r["C_boxes"][k]
        d = np.diag(C)
        ok = ((d[:3] <= nV * (1 + 1e-3)).all() and (d[:3] >= nR * (1 - 1e-3)).all() and
              (d[3:] <= sV * (1 + 1e-3)).all() and (d[3:] >= sR * (1 - 1e-3)).all() and
              np.linalg.eigvalsh(0.5 * (C + C.T)).min() > 0.0)
        if not ok:
            bad.append(k)
            print(f"box {k}: diag {d}, Voigt {nV:.4f}/{sV:.4f}, Reuss {nR:.3e}/{sR:.3e}")
    print(f"{len(b0)} unbuffered cores checked against their bounds, {len(bad)} outside")

    # the largest subimage and the 24/32-edge samples at a fixed iteration count
    ferrs = []
    for k, Cref in zip(fixed, fref_C):
        ferrs.append(np.abs(rf["C"][k] - Cref).max() / np.abs(Cref).max())
        print(f"box {k} {tile[k].tolist()} (Omega_B {(tile[k, 3:6] + 2 * tile[k, 6]).tolist()}), 20 iterations: "
              f"max|dC| / max|C| {ferrs[-1]:.2e}")

    for (eK, eG, eC), k in zip(errs, sample):
        assert eK <= 5e-3 and eG <= 5e-3 and eC <= 5e-3, k
    for e, k in zip(ferrs, fixed):
        assert e < 2e-5, k
    assert not bad
