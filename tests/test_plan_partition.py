"""Choice of subimage edge and buffer (hh_plan_partition, a host-only call)
against the oracle's enumeration, and the oracle pinned by what the error
and cost models fix without enumerating.

Models (Section 2: n >= 3 xi; Section 3, Eq. 2: (N/n)^3 solves of the
buffered box, each ~ (n + 2b)^a; Section 5: relative error c_b / n with one
constant per buffer width, Table fit_pad)."""

import os
import shutil

import numpy as np
import pytest

from oracle import hh_oracle as O


def _divisors(n):
    return [d for d in range(1, n + 1) if n % d == 0]


def test_largest_prime_factor():
    assert [O.largest_prime_factor(m) for m in (1, 2, 12, 31, 37, 74, 96, 2 * 3 * 29)] == [1, 2, 3, 31, 37, 37, 3, 29]


def test_no_buffer_closed_form():
    # one buffer width 0 and a > 3: the cost V n^(a-3) grows with n, so the
    # answer is the smallest common divisor n >= max(n_min, c / eps)
    for N, c, eps, n_min in ((900, 1.3, 0.005, 30), (512, 0.8, 0.02, 8), (240, 2.0, 0.5, 1)):
        n, b, err, cost, met, _ = O.plan_partition((N, N, N), n_min, [0], [c], 3.66, eps)
        want = min(d for d in _divisors(N) if d >= max(n_min, c / eps) and O.largest_prime_factor(d) <= 31)
        assert (n, b, met) == (want, 0, True)
        assert err == c / want
        assert np.isclose(cost, (N / want) ** 3 * want ** 3.66, rtol=1e-14)


def test_equal_constants_never_buffer():
    # a buffer that does not lower the constant only adds cost
    n, b, *_ = O.plan_partition((128, 128, 128), 1, [0, 4, 8], [1.0, 1.0, 1.0], 3.66, 0.05)
    assert (n, b) == (32, 0)


def test_table_fit_pad_bulk_b1():
    # Table fit_pad, rock B1, bulk modulus: M_inf 60.40, C = 78.71, 59.79,
    # 43.31 at buffers 0, 10, 20; N = 900, a = 3.66 (Section 3), target 0.5 %.
    # Smallest divisors of 900 meeting c / n <= 0.005: 300 (b 0, needs
    # n >= 260.6), 225 (b 10, n >= 198.0), 150 (b 20, n >= 143.4). Their costs
    # relative to (300, 0): (64/27)(245/300)^3.66 = 1.13 and
    # 8 (190/300)^3.66 = 1.50, so no buffer wins at this target.
    c = np.array([78.71, 59.79, 43.31]) / 60.40
    n, b, err, cost, met, table = O.plan_partition((900, 900, 900), 1, [0, 10, 20], c, 3.66, 0.005)
    assert (n, b, met) == (300, 0, True)
    best = {bb: min(t for t in table if t[1] == bb and t[2] <= 0.005) for bb in (0, 10, 20)}
    assert [best[bb][0] for bb in (0, 10, 20)] == [300, 225, 150]
    r10 = best[10][3] / best[0][3]
    r20 = best[20][3] / best[0][3]
    assert 1.12 < r10 < 1.14 and 1.49 < r20 < 1.51
    # with a steeper single-solve cost (a = 5) buffers pay: relative costs
    # (64/27)(245/300)^5 = 0.86 and 8 (190/300)^5 = 0.81
    n, b, *_ = O.plan_partition((900, 900, 900), 1, [0, 10, 20], c, 5.0, 0.005)
    assert (n, b) == (150, 20)


def test_unsupported_lengths_are_skipped():
    # 48 + 2 * 13 = 74 = 2 * 37: not an FFT length of the solver
    n, b, *_ = O.plan_partition((96, 96, 96), 1, [0, 13], [10.0, 0.1], 3.66, 0.25)
    assert (n, b) == (48, 0)
    _, _, _, _, _, table = O.plan_partition((96, 96, 96), 1, [13], [0.1], 3.66, 1.0)
    assert all(t[0] + 26 != 74 for t in table)


def test_target_unmet_returns_least_error():
    n, b, err, cost, met, _ = O.plan_partition((64, 64, 64), 1, [0, 2], [8.0, 4.0], 3.66, 1e-4)
    assert not met and (n, b) == (64, 2) and err == 4.0 / 64


@pytest.fixture(scope="module")
def B():
    from paper_2208_02320_gb300 import _build
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc") and not os.path.exists(_build.LIB):
        pytest.skip("nvcc not available")
    _build.build()
    from paper_2208_02320_gb300 import binding
    binding.load()
    return binding


def test_library_matches_oracle(B):
    rng = np.random.default_rng(2208)
    shapes = [(64, 64, 64), (96, 96, 96), (120, 90, 60), (900, 900, 900), (512, 512, 512), (74, 74, 74)]
    for trial in range(60):
        shape = shapes[trial % len(shapes)]
        nb = int(rng.integers(1, 5))
        bs = sorted(int(v) for v in rng.choice(np.arange(0, 21), size=nb, replace=False))
        c = rng.uniform(0.05, 3.0, size=nb)
        a = float(rng.uniform(3.05, 4.0))
        eps = float(10 ** rng.uniform(-3, -0.5))
        n_min = int(rng.integers(0, 40))
        try:
            want = O.plan_partition(shape, n_min, bs, c, a, eps)
        except ValueError:  # no candidate at all
            with pytest.raises(B.HHError) as e:
                B.plan_partition(shape, n_min, bs, c, a, eps)
            assert e.value.status == B.HH_ERR_ARG
            continue
        got = B.plan_partition(shape, n_min, bs, c, a, eps)
        assert (got["n"], got["b"], got["met"]) == (want[0], want[1], want[4]), (shape, n_min, bs, c, a, eps)
        assert got["err"] == want[2]
        assert np.isclose(got["cost"], want[3], rtol=1e-13)


def test_library_rejects_bad_arguments(B):
    for kw in (dict(bs=[-1], c_rel=[1.0]), dict(bs=[0], c_rel=[np.nan]), dict(bs=[0], c_rel=[-1.0]),
               dict(bs=[0], c_rel=[1.0], a=0.0), dict(bs=[0], c_rel=[1.0], eps=0.0)):
        args = dict(shape=(64, 64, 64), n_min=1, a=3.66, eps=0.01)
        args.update(kw)
        with pytest.raises(B.HHError) as e:
            B.plan_partition(**args)
        assert e.value.status == B.HH_ERR_ARG
    # n_min above every edge: no candidate
    with pytest.raises(B.HHError):
        B.plan_partition((64, 64, 64), 65, [0], [1.0], 3.66, 0.01)
