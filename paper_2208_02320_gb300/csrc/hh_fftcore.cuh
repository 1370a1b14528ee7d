// Complex values, register DFTs of radix 2..5 and the line addressing shared
// by the staged and the two-pass shared-memory transforms.
#pragma once

#include <cuda_runtime.h>

namespace hh {

template <typename T>
struct alignas(2 * sizeof(T)) C2 {
  T x, y;
};

template <typename T>
__host__ __device__ __forceinline__ C2<T> mk(T a, T b) {
  C2<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename T>
__device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ C2<T> csub(C2<T> a, C2<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T>
__device__ __forceinline__ C2<T> cmulc(C2<T> a, C2<T> b) {
  return mk<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// multiply by -i (forward) or +i (inverse)
template <typename T, bool INV>
__device__ __forceinline__ C2<T> rot(C2<T> a) {
  return INV ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}

// ---------------------------------------------------------------------------
// Small DFTs of size R on registers (forward: exp(-2 pi i rq / R)).
// ---------------------------------------------------------------------------
template <typename T, int R, bool INV>
__device__ __forceinline__ void small_dft(C2<T>* a, const C2<T>* tw, int N) {
  if constexpr (R == 2) {
    C2<T> t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
  } else if constexpr (R == 3) {
    const T h = T(0.86602540378443864676);  // sqrt(3)/2
    C2<T> s = cadd(a[1], a[2]);
    C2<T> d = csub(a[1], a[2]);
    C2<T> m = mk<T>(a[0].x - T(0.5) * s.x, a[0].y - T(0.5) * s.y);
    a[0] = cadd(a[0], s);
    // -i h d (forward) / +i h d (inverse)
    C2<T> t = rot<T, INV>(mk<T>(h * d.x, h * d.y));
    a[1] = cadd(m, t);
    a[2] = csub(m, t);
  } else if constexpr (R == 4) {
    C2<T> s02 = cadd(a[0], a[2]);
    C2<T> d02 = csub(a[0], a[2]);
    C2<T> s13 = cadd(a[1], a[3]);
    C2<T> d13 = rot<T, INV>(csub(a[1], a[3]));
    a[0] = cadd(s02, s13);
    a[2] = csub(s02, s13);
    a[1] = cadd(d02, d13);
    a[3] = csub(d02, d13);
  } else {
    C2<T> y[R];
    const int st = N / R;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      C2<T> acc = a[0];
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C2<T> w = tw[((r * q) % R) * st];
        if (INV) w.y = -w.y;
        acc = cadd(acc, cmul(a[r], w));
      }
      y[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < R; ++q) a[q] = y[q];
  }
}

// Lines addressed as off(l) = (l / lpg) * gstride + (l % lpg) * lstride, element
// k of a line at off(l) + k * es.
struct Lines {
  int n;       // number of lines
  int lpg;     // lines per group
  int gstride;
  int lstride;
  int es;
  bool fast;   // adjacent threads take adjacent lines (column access)
};

}  // namespace hh
