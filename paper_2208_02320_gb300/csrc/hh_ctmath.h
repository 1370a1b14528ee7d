// Compile-time trigonometry for the FFT twiddle constants.
//
// cos and sin of 2 pi t / n for integers t, n, evaluated by the compiler
// (constexpr): the angle pi a / b is reduced to [0, pi/4] with the symmetries
// of the circle in exact integer arithmetic,
//     theta -> 2 pi - theta,  theta -> pi - theta,  theta -> pi/2 - theta,
// and the Taylor series of sin and cos about 0 are then summed to 12 terms
// (the first neglected term is below 1e-27 on [0, pi/4]). Plain C++17, so the
// same header compiles with a host compiler for testing.
#pragma once

#if defined(__CUDACC__)
#define HH_CT_FN __host__ __device__ constexpr
#else
#define HH_CT_FN constexpr
#endif

namespace hh {

constexpr double kCtPi = 3.141592653589793238462643383279502884;

HH_CT_FN double ct_sin_taylor(double x) {
  double x2 = x * x, term = x, sum = x;
  for (int k = 1; k <= 12; ++k) {
    term *= -x2 / double((2 * k) * (2 * k + 1));
    sum += term;
  }
  return sum;
}

HH_CT_FN double ct_cos_taylor(double x) {
  double x2 = x * x, term = 1.0, sum = 1.0;
  for (int k = 1; k <= 12; ++k) {
    term *= -x2 / double((2 * k - 1) * (2 * k));
    sum += term;
  }
  return sum;
}

// cos(2 pi t / n) (want_sin = false) or sin(2 pi t / n) (want_sin = true), n >= 1.
HH_CT_FN double ct_trig(long long t, long long n, bool want_sin) {
  long long b = n;
  long long a = ((2 * t) % (2 * n) + 2 * n) % (2 * n);  // angle = pi a / b, a in [0, 2b)
  double sc = 1.0, ss = 1.0;
  if (a > b) {  // theta in (pi, 2 pi): theta -> 2 pi - theta
    a = 2 * b - a;
    ss = -ss;
  }
  if (2 * a > b) {  // theta in (pi/2, pi]: theta -> pi - theta
    a = b - a;
    sc = -sc;
  }
  bool swap = false;
  if (4 * a > b) {  // theta in (pi/4, pi/2]: theta -> pi/2 - theta, cos <-> sin
    a = b - 2 * a;
    b = 2 * b;
    swap = true;
  }
  const double x = kCtPi * double(a) / double(b);
  const double c = ct_cos_taylor(x), s = ct_sin_taylor(x);
  return want_sin ? ss * (swap ? c : s) : sc * (swap ? s : c);
}

}  // namespace hh
