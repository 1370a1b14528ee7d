"""CPU checks of the schedule of the compiled-shape field kernels.

The compiled plane and column passes (csrc/hh_plane_ct.cuh) move the
six-component plane through shared memory in a fixed schedule: the first
pass of each two-pass transform in place per (line, t1) pair, the second
pass and the packed first pass of the inverse x transform in rounds of whole
lines, the unpack step in rounds of whole rows. Their index formulas are
restated here with numpy standing in for the register DFTs, and the schedule
is checked on every compiled shape: every access inside the block's plane
buffer, every pair of a pass taken exactly once, the positions a round reads
on lines that no other round touches, and the transforms equal to numpy's
FFT (forward: the half spectrum of the six real components; inverse: the
real components times the number of voxels of the plane).
"""

import os
import re

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2208_02320_gb300", "csrc")
NT = 256


def _read(name):
    return open(os.path.join(CSRC, name)).read()


def _split_table():
    text = _read("hh_fft2.cuh")
    body = text[text.index("#define HH_FFT2_TABLE"):text.index("// N1 of the two-pass plan")]
    return {int(n): int(a) for n, a, b in re.findall(r"X\((\d+), (\d+), (\d+)\)", body)}


SPLIT = _split_table()
CT = _read("hh_plane_ct.cuh")
STAGE = int(re.search(r"#define HH_CT_STAGE (\d+)", CT).group(1))


def _plane_groups():
    groups = {}
    for g in range(4):
        m = re.search(r"#define HH_CT_PLANES_%d\(X\)(.*?)\n(?!  X)" % g, CT, re.S)
        groups[g] = [tuple(map(int, t)) for t in re.findall(r"X\((\d+), (\d+)\)", m.group(1))]
    return groups


def _col_lengths():
    m = re.search(r"#define HH_CT_COL_LENGTHS\(X\)(.*?)\n(?!  X)", CT, re.S)
    return [int(t) for t in re.findall(r"X\((\d+)\)", m.group(1))]


PLANES = _plane_groups()
ALL_PLANES = [p for g in range(4) for p in PLANES[g]]


def cdiv(a, b):
    return (a + b - 1) // b


class Geo:
    def __init__(self, NL, LPG, GS, LS, ES):
        self.NL, self.LPG, self.GS, self.LS, self.ES = NL, LPG, GS, LS, ES

    def off(self, l):
        l = np.asarray(l)
        if self.LPG >= self.NL:
            return l * self.LS
        return (l // self.LPG) * self.GS + (l % self.LPG) * self.LS


def _dft(v, inv):
    # v: (..., R) -> R-point DFT along the last axis, forward exp(-2 pi i), inverse unnormalized exp(+)
    return np.fft.ifft(v, axis=-1) * v.shape[-1] if inv else np.fft.fft(v, axis=-1)


def pass1_local(S, N1, N2, inv, G, size):
    TOT = G.NL * N1
    p = np.arange(TOT)
    line, t1 = p % G.NL, p // G.NL
    o = G.off(line) + t1 * G.ES
    idx = o[:, None] + np.arange(N2)[None, :] * N1 * G.ES
    assert idx.min() >= 0 and idx.max() < size
    assert len(np.unique(idx)) == idx.size  # pairs touch disjoint positions
    v = _dft(S[idx], inv)
    w = np.exp((1j if inv else -1j) * 2 * np.pi * (t1[:, None] * np.arange(N2)[None, :]) / (N1 * N2))
    S[idx] = v * w  # written where read (k2 N1 + t1 for k2 < N2)


def pass_rounds(S, N1, N2, inv, G, kind, size, NXH=0):
    N = N1 * N2
    J = N2 if kind == "p2" else N1
    R = N1 if kind == "p2" else N2
    step = N2 if kind == "p2" else N1
    PMAX = max(1, STAGE // R)
    LPR0 = max(1, PMAX * NT // J)
    NR = cdiv(G.NL, LPR0)
    LPR = cdiv(G.NL, NR)
    IT = cdiv(LPR * J, NT)
    TOT = LPR * J
    lines_seen = []
    taken = np.zeros((G.NL, J), dtype=np.int64)
    for r in range(NR):
        p = np.arange(IT * NT)
        line = r * LPR + p % LPR
        jj = p // LPR
        ok = (p < TOT) & (line < G.NL)
        line, jj = line[ok], jj[ok]
        np.add.at(taken, (line, jj), 1)
        lo = G.off(line)
        if kind == "p2":
            ridx = lo[:, None] + (jj[:, None] * N1 + np.arange(N1)[None, :]) * G.ES
            v = _dft(S[ridx], inv)
            widx = (lo + jj * G.ES)[:, None] + np.arange(N1)[None, :] * step * G.ES
        else:
            assert G.ES == 1
            n = jj[:, None] + N1 * np.arange(N2)[None, :]
            low = n < NXH
            ia = np.where(low, n, N - n)
            A, B = S[lo[:, None] + ia], S[lo[:, None] + NXH + ia]
            A, B = np.where(low, A, np.conj(A)), np.where(low, B, np.conj(B))
            ridx = np.concatenate([lo[:, None] + ia, lo[:, None] + NXH + ia], axis=1)
            v = _dft(A + 1j * B, inv)
            w = np.exp((1j if inv else -1j) * 2 * np.pi * (jj[:, None] * np.arange(N2)[None, :]) / N)
            v = v * w
            widx = (lo + jj)[:, None] + np.arange(N2)[None, :] * step
        assert ridx.min() >= 0 and ridx.max() < size and widx.min() >= 0 and widx.max() < size
        assert len(np.unique(widx)) == widx.size
        # the round reads and writes only positions of its own lines
        rows = set(np.unique(line).tolist())
        assert not any(rows & s for s in lines_seen)
        lines_seen.append(rows)
        S[widx] = v  # after the round's barrier
    assert (taken == 1).all()


def fft_ct(S, N, inv, G, size):
    N1 = SPLIT[N]
    N2 = N // N1
    if N2 > 1:
        pass1_local(S, N1, N2, inv, G, size)
    pass_rounds(S, N1, N2, inv, G, "p2", size)


def fft_inv_packed_ct(S, N, G, size):
    N1 = SPLIT[N]
    N2 = N // N1
    assert N2 > 1
    pass_rounds(S, N1, N2, True, G, "packed", size, NXH=N // 2 + 1)
    pass_rounds(S, N1, N2, True, G, "p2", size)


def unpack_ct(S, NX, NROWS, RP, size):
    NXH = NX // 2 + 1
    EMAX = max(1, STAGE // 2)
    RPR0 = max(1, EMAX * NT // NXH)
    NR = cdiv(NROWS, RPR0)
    RPR = cdiv(NROWS, NR)
    IT = cdiv(RPR * NXH, NT)
    TOT = RPR * NXH
    for r in range(NR):
        e = np.arange(IT * NT)
        row, k = r * RPR + e // NXH, e % NXH
        ok = (e < TOT) & (row < NROWS)
        row, k = row[ok], k[ok]
        base = row * RP
        a, b = S[base + k], S[base + np.where(k == 0, 0, NX - k)]
        A = 0.5 * (a + np.conj(b))
        B = -0.5j * (a - np.conj(b))
        assert (base + k + NXH).max() < size
        S[base + k], S[base + k + NXH] = A, B


def _plane_geometry(NX, NY):
    NXH, RP = NX // 2 + 1, (NX + 2) | 1
    size = 3 * NY * RP
    gy = Geo(6 * NXH, 2 * NXH, NY * RP, 1, RP)
    gx = Geo(3 * NY, 1 << 30, 0, RP, 1)
    return NXH, RP, size, gx, gy


def _spec_pos(NX, NY):
    # (c, ky, kx) of every spectrum element the plane passes copy, in their e = ky * NXH + kx order
    NXH, RP = NX // 2 + 1, (NX + 2) | 1
    e = np.arange(NY * NXH)
    ky, kx = e // NXH, e % NXH
    return [((c >> 1) * NY + ky) * RP + (c & 1) * NXH + kx for c in range(6)], ky, kx


def test_compiled_plane_shapes_are_the_buffered_boxes_of_unit_cores():
    want = {(nx, ny) for nx in range(16, 49, 2) for ny in range(16, 49, 2) if abs(nx - ny) in (0, 8, 16)}
    assert set(ALL_PLANES) == want and len(ALL_PLANES) == len(want) == 61
    for g, shapes in PLANES.items():
        lo, hi = {0: (16, 22), 1: (24, 30), 2: (32, 38), 3: (40, 48)}[g]
        assert all(lo <= nx <= hi for nx, ny in shapes)
    assert _col_lengths() == list(range(16, 49, 2))
    assert all(n in SPLIT for n in range(16, 49, 2))


@pytest.mark.parametrize("shape", ALL_PLANES)
def test_plane_pass_schedule(shape):
    NX, NY = shape
    NXH, RP, size, gx, gy = _plane_geometry(NX, NY)
    rng = np.random.default_rng(NX * 64 + NY)
    s = rng.standard_normal((6, NY, NX))
    # forward: the voxel phase's pair rows, x transform, unpack, y transform
    S = np.full(size, np.nan, dtype=complex)
    v = np.arange(NX * NY)
    y, x = v // NX, v % NX
    for c2 in range(3):
        pos = (c2 * NY + y) * RP + x
        assert pos.max() < size
        S[pos] = s[2 * c2][y, x] + 1j * s[2 * c2 + 1][y, x]
    fft_ct(S, NX, False, gx, size)
    unpack_ct(S, NX, 3 * NY, RP, size)
    fft_ct(S, NY, False, gy, size)
    pos, ky, kx = _spec_pos(NX, NY)
    assert len(np.unique(np.concatenate(pos))) == 6 * NY * NXH
    for c in range(6):
        ref = np.fft.rfft2(s[c])  # axes (y, x): full ky, half kx, natural order
        got = S[pos[c]]
        assert np.abs(got - ref[ky, kx]).max() < 1e-9 * np.abs(ref).max(), c
    # inverse: spectrum copies, y transform, packed x transform, voxel phase
    T = np.full(size, np.nan, dtype=complex)
    for c in range(6):
        T[pos[c]] = np.fft.rfft2(s[c])[ky, kx]
    fft_ct(T, NY, True, gy, size)
    fft_inv_packed_ct(T, NX, gx, size)
    for c2 in range(3):
        z = T[(c2 * NY + y) * RP + x]
        assert np.abs(z.real - NX * NY * s[2 * c2][y, x]).max() < 1e-9 * NX * NY
        assert np.abs(z.imag - NX * NY * s[2 * c2 + 1][y, x]).max() < 1e-9 * NX * NY


@pytest.mark.parametrize("NZ", _col_lengths())
@pytest.mark.parametrize("CW", [16, 32])
def test_column_pass_schedule(NZ, CW):
    size = 6 * NZ * CW
    # copies: thread t keeps column jl = t % CW, rows cz = t / CW + i (NT / CW)
    ITL = cdiv(6 * NZ * CW, NT)
    hit = np.zeros(size, dtype=np.int64)
    for t in range(NT):
        jl, cz0 = t % CW, t // CW
        for i in range(ITL):
            cz = cz0 + i * (NT // CW)
            if (i + 1) * NT <= size or cz < 6 * NZ:
                hit[cz * CW + jl] += 1
    assert (hit == 1).all()
    # modes: every (kzp, jl) once
    ITM = cdiv(NZ * CW, NT)
    modes = [(t // CW + i * (NT // CW), t % CW) for t in range(NT) for i in range(ITM)
             if (i + 1) * NT <= NZ * CW or t // CW + i * (NT // CW) < NZ]
    assert sorted(modes) == [(k, j) for k in range(NZ) for j in range(CW)]
    rng = np.random.default_rng(NZ * 64 + CW)
    tile = rng.standard_normal(size) + 1j * rng.standard_normal(size)
    g = Geo(6 * CW, CW, NZ * CW, 1, CW)
    S = tile.copy()
    fft_ct(S, NZ, False, g, size)
    ref = np.fft.fft(tile.reshape(6, NZ, CW), axis=1).reshape(-1)
    assert np.abs(S - ref).max() < 1e-9 * np.abs(ref).max()
    fft_ct(S, NZ, True, g, size)
    assert np.abs(S - NZ * tile).max() < 1e-9 * NZ


PROG = r"""
#include "hh_device.cuh"
#include <cstdio>
int main() {
  for (int nx = 1; nx <= 64; ++nx)
    for (int ny = 1; ny <= 64; ++ny) {
      const int g = hh::ct_plane_group(nx, ny);
      if (g >= 0) std::printf("P %d %d %d\n", nx, ny, g);
    }
  for (int n = 1; n <= 64; ++n)
    if (hh::ct_col_length(n)) std::printf("Z %d\n", n);
  for (int cw = 1; cw <= 64; ++cw)
    if (hh::ct_width(cw)) std::printf("W %d\n", cw);
  return 0;
}
"""


def test_host_shape_codes_match_the_compiled_bodies(tmp_path):
    """The host's choice of compiled shapes (ct_plane_group, ct_col_length,
    ct_width, compiled as host code) names exactly the bodies the kernels'
    switches contain: a shape the host marks but no kernel compiles would be
    skipped by the kernel."""
    import shutil
    import subprocess
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("no nvcc")
    src = tmp_path / "codes.cu"
    src.write_text(PROG)
    exe = tmp_path / "codes"
    inc = os.path.join(os.path.dirname(CSRC), "..", "include")
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-I", inc, "-o", str(exe), str(src)], check=True,
                   capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    planes = {(int(a), int(b)): int(g) for t, a, b, g in (l.split() for l in out if l.startswith("P"))}
    assert planes == {p: g for g in range(4) for p in PLANES[g]}
    assert [int(l.split()[1]) for l in out if l.startswith("Z")] == _col_lengths()
    assert [int(l.split()[1]) for l in out if l.startswith("W")] == [16, 32]
    body = CT[CT.index("k_column_ct(KParams<T> P, int skip_mode)"):]
    assert re.findall(r"case N \* 64 \+ (\d+):", body) == ["16", "32"]
