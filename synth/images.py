"""Seeded synthetic phase maps that stand in for the paper's micro-CT rocks.

The rocks of the paper (Berea, Castlegate, Fontainebleau; Section 2, Table 1)
are proprietary scans and are not available. These generators produce seeded
uint8 label images with the statistics the paper reports for them: porosity of
a few to a few tens of percent, correlation lengths of roughly ten voxels, and
isotropic structure. Every random number comes from the counter-based
SplitMix64 generator (Steele, Lea and Flood, 2014) so that a (seed, stream,
counter) triple always yields the same value.

Labels index a phase-moduli table of (K, G) pairs in GPa. The tables below are
the paper's quartz/pore pair (Section 2), its Appendix B pair, and the sets the
synthetic workloads use.
"""

from __future__ import annotations

import hashlib
import math

import numpy as np

# Phase tables: row = label, columns = (bulk modulus K, shear modulus G) in GPa.
# Quartz and pore as assigned in Section 2 (pore moduli replaced by 1e-5 GPa).
PHASES_QUARTZ_PORE_PAPER = np.array([[36.0, 45.0], [1e-5, 1e-5]])
# Appendix B: phase 1 ten times stiffer than phase 2.
PHASES_APPENDIX_B = np.array([[98.04, 37.59], [9.80, 3.76]])
# Synthetic workloads: solid grain and (near-)void pore.
PHASES_SOLID_PORE = np.array([[37.0, 44.0], [1e-4, 1e-4]])
# Three-phase sandstone: solid, clay, pore.
PHASES_SOLID_CLAY_PORE = np.array([[37.0, 44.0], [21.0, 7.0], [1e-4, 1e-4]])
# Carbonate: calcite, dolomite, pore.
PHASES_CARBONATE = np.array([[70.2, 29.0], [94.9, 45.0], [1e-4, 1e-4]])

_M64 = (1 << 64) - 1
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counters) -> np.ndarray:
    """SplitMix64 output for every counter value (uint64 array)."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _M64) + (c + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        z = z ^ (z >> np.uint64(31))
    return z


def _stream_seed(seed: int, stream: int) -> int:
    return int(splitmix64(seed, np.array([stream], dtype=np.uint64))[0])


def uniform01(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniform doubles in [0, 1) from stream `stream` of `seed` (53-bit)."""
    s = _stream_seed(seed, stream)
    z = splitmix64(s, np.arange(offset, offset + n, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal01(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n standard normals by the Box-Muller transform of two uniform streams."""
    u1 = uniform01(seed, 2 * stream, n, offset)
    u2 = uniform01(seed, 2 * stream + 1, n, offset)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


def gaussian_random_field(shape, ell: float, seed: int, stream: int = 0) -> np.ndarray:
    """Periodic Gaussian random field with covariance exp(-r^2 / (2 ell^2)).

    White noise is convolved (periodically) with a Gaussian kernel of width
    ell / sqrt(2); the convolution of that kernel with itself has the stated
    covariance. The result is normalised to zero mean and unit variance.
    """
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    w = normal01(seed, stream, n).reshape(shape)
    s2 = 0.5 * ell * ell
    grids = []
    for ax, L in enumerate(shape):
        d = np.arange(L, dtype=np.float64)
        d = np.minimum(d, L - d)  # periodic distance to the origin
        sh = [1] * len(shape)
        sh[ax] = L
        grids.append((d * d).reshape(sh))
    r2 = sum(grids)
    g = np.exp(-r2 / (2.0 * s2))
    axes = tuple(range(len(shape)))
    f = np.fft.irfftn(np.fft.rfftn(w, axes=axes) * np.fft.rfftn(g, axes=axes), s=shape, axes=axes)
    f -= f.mean()
    sd = f.std()
    return f / sd if sd > 0 else f


def threshold_bands(field: np.ndarray, fractions, labels, rest_label: int) -> np.ndarray:
    """Label the lowest-valued voxels band by band.

    The first round(fractions[0] * V) voxels in ascending order of `field`
    (ties broken by linear index) get labels[0], the next round(fractions[1] *
    V) get labels[1], and so on; all remaining voxels get `rest_label`.
    """
    flat = field.ravel()
    order = np.argsort(flat, kind="stable")
    out = np.full(flat.shape, rest_label, dtype=np.uint8)
    start = 0
    V = flat.size
    for f, lab in zip(fractions, labels):
        cnt = int(round(f * V))
        out[order[start:start + cnt]] = lab
        start += cnt
    return out.reshape(field.shape)


def grf_two_phase(n: int = 32, ell: float = 4.0, porosity: float = 0.20,
                  seed: int = 2208023201) -> np.ndarray:
    """Two-phase image (label 0 solid, label 1 pore) thresholded at a quantile."""
    f = gaussian_random_field((n, n, n), ell, seed)
    return threshold_bands(f, [porosity], [1], rest_label=0)


def grf_three_phase(n: int = 256, ell: float = 6.0, pore: float = 0.18, clay: float = 0.12,
                    seed: int = 2208023202) -> np.ndarray:
    """Three-phase image: lowest `pore` fraction -> label 2, next `clay` -> 1, rest -> 0."""
    f = gaussian_random_field((n, n, n), ell, seed)
    return threshold_bands(f, [pore, clay], [2, 1], rest_label=0)


def boolean_spheres(n: int = 512, median_radius: float = 10.0, sigma_log: float = 0.3,
                    porosity: float = 0.15, seed: int = 2208023203, batch: int = 4096) -> np.ndarray:
    """Periodic Boolean model of overlapping spherical grains.

    Sphere centres are uniform in the periodic box and radii are lognormal
    (median `median_radius`, log-standard deviation `sigma_log`). Spheres are
    added one at a time until the pore fraction drops to `porosity` or below;
    the sphere that crosses the threshold is kept. Voxel (i, j, k) with centre
    at integer coordinates is grain if it lies within some sphere. Labels: 0
    grain, 1 pore.
    """
    solid = np.zeros((n, n, n), dtype=bool)
    V = n ** 3
    target_solid = V - math.floor(porosity * V)
    covered = 0
    k = 0
    while covered < target_solid:
        cx = uniform01(seed, 0, batch, k) * n
        cy = uniform01(seed, 1, batch, k) * n
        cz = uniform01(seed, 2, batch, k) * n
        rr = median_radius * np.exp(sigma_log * normal01(seed, 3, batch, k))
        for i in range(batch):
            c = (cz[i], cy[i], cx[i])
            r = rr[i]
            R = int(math.ceil(r)) + 1
            idx = []
            d2 = []
            for ax in range(3):
                lo = int(math.floor(c[ax])) - R
                j = np.arange(lo, lo + 2 * R + 2)
                d = j - c[ax]
                sh = [1, 1, 1]
                sh[ax] = j.size
                d2.append((d * d).reshape(sh))
                idx.append(np.mod(j, n))
            inside = (d2[0] + d2[1] + d2[2]) <= r * r
            sub = solid[np.ix_(idx[0], idx[1], idx[2])]
            newly = inside & ~sub
            cnt = int(newly.sum())
            if cnt:
                solid[np.ix_(idx[0], idx[1], idx[2])] = sub | inside
                covered += cnt
            if covered >= target_solid:
                break
        k += batch
    return np.where(solid, 0, 1).astype(np.uint8)


def multiscale_carbonate(n: int = 1024, porosity: float = 0.22, seed: int = 2208023205) -> np.ndarray:
    """Two-scale carbonate-like image: labels 0 calcite, 1 dolomite, 2 pore.

    The pore indicator thresholds the sum of two equal-variance Gaussian random
    fields with correlation lengths 10 and 60 voxels at the `porosity`
    quantile. The solid is split 50/50 between calcite and dolomite by the
    median of a third, independent field with correlation length 60.
    """
    f = gaussian_random_field((n, n, n), 10.0, seed, 0) + gaussian_random_field((n, n, n), 60.0, seed, 1)
    pore = threshold_bands(f, [porosity], [1], rest_label=0).astype(bool)
    del f
    g = gaussian_random_field((n, n, n), 60.0, seed, 2)
    out = np.full((n, n, n), 2, dtype=np.uint8)
    solid_idx = np.flatnonzero(~pore.ravel())
    gs = g.ravel()[solid_idx]
    order = np.argsort(gs, kind="stable")
    half = solid_idx.size // 2
    flat = out.ravel()
    flat[solid_idx[order[:half]]] = 0
    flat[solid_idx[order[half:]]] = 1
    return out


def _shuffle(values, seed: int, stream: int):
    """Fisher-Yates shuffle driven by the counter-based stream."""
    v = list(values)
    u = uniform01(seed, stream, len(v))
    for i in range(len(v) - 1, 0, -1):
        j = int(u[i] * (i + 1))
        v[i], v[j] = v[j], v[i]
    return v


def uniform_partition(N: int, n: int, b: int) -> np.ndarray:
    """(N/n)^3 cubic cores of edge n, all with buffer width b.

    Returns an int32 array of rows (ox, oy, oz, nx, ny, nz, b) in z-major,
    then y, then x order of the cores (x fastest).
    """
    if N % n:
        raise ValueError("subimage edge must divide the image edge")
    m = N // n
    rows = [(i * n, j * n, k * n, n, n, n, b) for k in range(m) for j in range(m) for i in range(m)]
    return np.array(rows, dtype=np.int32).reshape(-1, 7)


def uneven_partition(N: int = 512, counts=((16, 27), (24, 2), (32, 1)), bmax: int = 8,
                     seed: int = 2208023203) -> np.ndarray:
    """Cut each axis into segments of the given lengths in a seeded order.

    Every axis gets the multiset of segment lengths in `counts` (length,
    multiplicity), shuffled independently per axis; the boxes are the products
    of one segment per axis. Each box draws its own buffer width uniformly from
    0..bmax. Returns int32 rows (ox, oy, oz, nx, ny, nz, b), x fastest.
    """
    segs = []
    for L, c in counts:
        segs += [L] * c
    if sum(segs) != N:
        raise ValueError("segment lengths must add up to N")
    axes = []
    for ax in range(3):
        s = _shuffle(segs, seed, 100 + ax)
        o = np.concatenate([[0], np.cumsum(s)[:-1]])
        axes.append((o, s))
    (ox, sx), (oy, sy), (oz, sz) = axes
    nb = len(sx) * len(sy) * len(sz)
    bw = np.floor(uniform01(seed, 200, nb) * (bmax + 1)).astype(np.int64)
    rows = []
    t = 0
    for k in range(len(sz)):
        for j in range(len(sy)):
            for i in range(len(sx)):
                rows.append((ox[i], oy[j], oz[k], sx[i], sy[j], sz[k], int(bw[t])))
                t += 1
    return np.array(rows, dtype=np.int32)


def laminate(shape, labels_along_z) -> np.ndarray:
    """Image whose label depends on z only: label of plane z is labels_along_z[z]."""
    nz, ny, nx = shape
    lab = np.asarray(labels_along_z, dtype=np.uint8)
    assert lab.size == nz
    return np.broadcast_to(lab[:, None, None], shape).copy()


def image_sha256(img: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(img).tobytes()).hexdigest()


def workload(name: str) -> dict:
    """The named synthetic workloads with their sizes, phases and partitions.

    grf32        two-phase 32^3 field (correlation length 4, porosity 0.20);
                 direct solve plus 8^3 cores with no buffer (4^3 coarse image).
    grf256       three-phase 256^3 field (correlation length 6); cores 16..128,
                 buffers 0/4/8.
    spheres512   512^3 overlapping-sphere sandstone (porosity 0.15) cut into
                 27,000 uneven cores of edge 16/24/32 with buffers 0..8 and an
                 8-voxel coarse unit (64^3 coarse image).
    carbonate1024 1024^3 two-scale carbonate, 64^3 cores with buffer 8.
    """
    if name == "grf32":
        return dict(name=name, image=grf_two_phase(), phases=PHASES_SOLID_PORE,
                    boxes=uniform_partition(32, 8, 0), unit=8, tol=1e-6)
    if name == "grf256":
        return dict(name=name, image=grf_three_phase(), phases=PHASES_SOLID_CLAY_PORE,
                    ns=(16, 32, 64, 128), bs=(0, 4, 8), tol=1e-6)
    if name == "spheres512":
        return dict(name=name, image=boolean_spheres(), phases=PHASES_SOLID_PORE,
                    boxes=uneven_partition(), unit=8, tol=1e-6)
    if name == "carbonate1024":
        return dict(name=name, image=multiscale_carbonate(), phases=PHASES_CARBONATE,
                    boxes=uniform_partition(1024, 64, 8), unit=64, tol=1e-6)
    raise KeyError(name)
