"""Ensemble files (hh_surrogate_save / hh_surrogate_load): host-only calls,
run on the CPU. A round trip is bit-exact, the header fields are where the
documented format puts them, and every damaged file is refused."""

import os
import shutil
import struct

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def B():
    from paper_2208_02320_gb300 import _build
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc") and not os.path.exists(_build.LIB):
        pytest.skip("nvcc not available")
    _build.build()
    from paper_2208_02320_gb300 import binding
    binding.load()
    return binding


def _fnv1a64(data: bytes) -> int:
    # FNV-1a, 64-bit, from its published definition
    h = 0xCBF29CE484222325
    for b in data:
        h = ((h ^ b) * 0x100000001B3) & ((1 << 64) - 1)
    return h


def _ensemble(B, m, seed):
    n = B.load().hh_cnn_num_params()
    th = (synth.uniform01(seed, 0, m * n).reshape(m, n) - 0.5).astype(np.float32)
    th[0, :4] = [np.inf, -0.0, np.float32(1e-45), np.nan]  # bit patterns survive as they are
    return th


def test_round_trip_is_bit_exact(B, tmp_path):
    th = _ensemble(B, 3, 1)
    p = str(tmp_path / "ens.hhs")
    B.surrogate_save(p, th, 123.5)
    got, sc = B.surrogate_load(p)
    assert sc == 123.5 and got.shape == th.shape
    assert np.array_equal(got.view(np.uint32), th.view(np.uint32))


def test_documented_layout(B, tmp_path):
    th = _ensemble(B, 2, 2)
    p = str(tmp_path / "ens.hhs")
    B.surrogate_save(p, th, 100.0)
    raw = open(p, "rb").read()
    n = th.shape[1]
    assert raw[:8] == b"HHSURR01"
    ens, zero, n_params, scale, h = struct.unpack("<iiqdQ", raw[8:40])
    assert (ens, zero, n_params, scale) == (2, 0, n, 100.0)
    body = raw[40:]
    assert len(body) == 4 * 2 * n and body == th.astype("<f4").tobytes()
    assert h == _fnv1a64(body)


def test_damaged_files_are_refused(B, tmp_path):
    th = _ensemble(B, 2, 3)
    good = str(tmp_path / "good.hhs")
    B.surrogate_save(good, th, 100.0)
    raw = bytearray(open(good, "rb").read())
    cases = {
        "flipped parameter bit": raw[:100] + bytes([raw[100] ^ 1]) + raw[101:],
        "truncated": raw[:-4],
        "trailing byte": raw + b"\0",
        "wrong magic": b"HHSURR02" + raw[8:],
        "wrong n_params": raw[:16] + struct.pack("<q", th.shape[1] + 1) + raw[24:],
        "empty": b"",
    }
    for name, data in cases.items():
        p = str(tmp_path / "bad.hhs")
        open(p, "wb").write(bytes(data))
        with pytest.raises(B.HHError) as e:
            B.surrogate_load(p)
        assert e.value.status == B.HH_ERR_ARG, name
    with pytest.raises(B.HHError):
        B.surrogate_load(str(tmp_path / "missing.hhs"))


def test_argument_checks(B, tmp_path):
    import ctypes
    lib = B.load()
    th = _ensemble(B, 1, 4)
    p = str(tmp_path / "ens.hhs").encode()
    ptr = th.ctypes.data_as(ctypes.c_void_p)
    assert lib.hh_surrogate_save(p, ptr, 0, 100.0) == B.HH_ERR_ARG
    assert lib.hh_surrogate_save(p, ptr, 1, 0.0) == B.HH_ERR_ARG
    assert lib.hh_surrogate_save(p, ptr, 1, float("inf")) == B.HH_ERR_ARG
    assert lib.hh_surrogate_save(None, ptr, 1, 100.0) == B.HH_ERR_ARG
    assert lib.hh_surrogate_save(p, ptr, 1, 100.0) == B.HH_OK
    ens, sc = ctypes.c_int(), ctypes.c_double()
    # header query, then a buffer one float short
    assert lib.hh_surrogate_load(p, None, 0, ctypes.byref(ens), ctypes.byref(sc)) == B.HH_OK
    assert (ens.value, sc.value) == (1, 100.0)
    out = np.zeros(th.size, dtype=np.float32)
    assert lib.hh_surrogate_load(p, out.ctypes.data_as(ctypes.c_void_p), th.size - 1, ctypes.byref(ens),
                                 ctypes.byref(sc)) == B.HH_ERR_ARG
    assert b"capacity" in lib.hh_last_error(None)


def test_initial_parameters_match_the_oracle_initializer(B):
    """hh_cnn_init_params: He-uniform weights from the i-th SplitMix64 output of
    the seed (top 53 bits), biases zero, equal to the oracle's initializer fed
    with the same draws (up to FP32 rounding)."""
    from oracle import cnn_oracle as N
    for seed in (0, 2208, 2**64 - 3):
        got = B.cnn_init_params(seed)
        n = N.n_params()
        u = (synth.splitmix64(seed, np.arange(n, dtype=np.uint64)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        ref = N.init_params(u)
        assert got.shape == (n,) and got.dtype == np.float32
        assert np.array_equal(got, ref.astype(np.float32))
