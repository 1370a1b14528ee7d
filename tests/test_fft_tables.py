"""Host-side checks of the FFT plan tables (no GPU).

The compile-time cosines and sines (csrc/hh_ctmath.h: octant reduction and
Taylor series) are compiled with the host compiler and compared with the C
library's long-double cos/sin; the two-pass split table (csrc/hh_fft2.cuh) is
checked for consistency: N = N1 N2 with N1 <= 23, N2 <= 16, and every length
that admits such a split is listed.
"""

import os
import re
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2208_02320_gb300", "csrc")

PROG = r"""
#include "hh_ctmath.h"
#include <cmath>
#include <cstdio>
static_assert(hh::ct_trig(1, 4, true) == 1.0 || hh::ct_trig(1, 4, true) > 0.9999999999999, "constexpr");
int main() {
  double worst = 0.0;
  for (int n = 1; n <= 256; ++n)
    for (int t = -n; t < 2 * n; ++t) {
      const long double a = 2.0L * 3.141592653589793238462643383279502884L * t / n;
      worst = std::fmax(worst, std::fabs((double)cosl(a) - hh::ct_trig(t, n, false)));
      worst = std::fmax(worst, std::fabs((double)sinl(a) - hh::ct_trig(t, n, true)));
    }
  std::printf("%.6e\n", worst);
  return 0;
}
"""


def test_compile_time_trig_matches_libm(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "ct.cpp"
    src.write_text(PROG)
    exe = tmp_path / "ct"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, "-o", str(exe), str(src)], check=True)
    worst = float(subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout)
    assert worst < 1e-15


def _table():
    text = open(os.path.join(CSRC, "hh_fft2.cuh")).read()
    body = text[text.index("#define HH_FFT2_TABLE"):text.index("// N1 of the two-pass plan")]
    return [tuple(map(int, m)) for m in re.findall(r"X\((\d+), (\d+), (\d+)\)", body)]


def _smooth23(n):
    for p in (2, 3, 5, 7, 11, 13, 17, 19, 23):
        while n % p == 0:
            n //= p
    return n == 1


def test_two_pass_split_table():
    tab = _table()
    lengths = [t[0] for t in tab]
    assert lengths == sorted(set(lengths))
    for n, n1, n2 in tab:
        assert n1 * n2 == n and n1 <= 23 and 1 <= n2 <= 16
        # most balanced split among the admissible ones
        best = min(max(a, n // a) for a in range(1, n + 1) if n % a == 0 and a <= 23 and n // a <= 16)
        assert max(n1, n2) == best
    for n in range(2, 129):
        has = any(n % a == 0 and a <= 23 and n // a <= 16 for a in range(1, n + 1))
        assert (n in lengths) == (has and _smooth23(n)), n
