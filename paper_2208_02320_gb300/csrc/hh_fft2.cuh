// Two-pass (four-step) transforms of lines held in shared memory.
//
// A line of length N = N1 * N2, element n = t1 + N1 m (t1 < N1, m < N2),
// has the DFT
//     X[k2 + N2 k1] = sum_t1 W_N1^(t1 k1) * W_N^(t1 k2) * sum_m x[t1 + N1 m] W_N2^(m k2),
// so one pass does, for every (line, t1), the N2-point inner DFT and the
// twiddle W_N^(t1 k2) and stores the result at k2 N1 + t1; a second pass
// does, for every (line, k2), the N1-point outer DFT and stores X in natural
// order. Every DFT runs on registers with its cosines and sines folded in by
// the compiler (hh_ctmath.h); the only table read is the twiddle W_N^(t1 k2)
// (t1 k2 < N, no reduction needed). Each pass reads all of a round's elements
// before any is written (a barrier between, and a round never splits a line),
// so the transform is in place. Inverse transforms (INV) conjugate every
// factor.
#pragma once

#include <type_traits>

#include "hh_ctmath.h"
#include "hh_fftcore.cuh"

namespace hh {

// Lengths with a two-pass plan: X(N, N1, N2). Every 23-smooth N <= 128 that
// splits into N1 <= 23 (or N1 = N for a prime N <= 23) and N2 <= 16, choosing
// the most balanced split. Other lengths use the staged transform.
#define HH_FFT2_TABLE(X)                                                                                    \
  X(2, 2, 1) X(3, 3, 1) X(4, 2, 2) X(5, 5, 1) X(6, 3, 2) X(7, 7, 1) X(8, 4, 2) X(9, 3, 3) X(10, 5, 2)       \
  X(11, 11, 1) X(12, 4, 3) X(13, 13, 1) X(14, 7, 2) X(15, 5, 3) X(16, 4, 4) X(17, 17, 1) X(18, 6, 3)         \
  X(19, 19, 1) X(20, 5, 4) X(21, 7, 3) X(22, 11, 2) X(23, 23, 1) X(24, 6, 4) X(25, 5, 5) X(26, 13, 2)        \
  X(27, 9, 3) X(28, 7, 4) X(30, 6, 5) X(32, 8, 4) X(33, 11, 3) X(34, 17, 2) X(35, 7, 5) X(36, 6, 6)          \
  X(38, 19, 2) X(39, 13, 3) X(40, 8, 5) X(42, 7, 6) X(44, 11, 4) X(45, 9, 5) X(46, 23, 2) X(48, 8, 6)        \
  X(49, 7, 7) X(50, 10, 5) X(51, 17, 3) X(52, 13, 4) X(54, 9, 6) X(55, 11, 5) X(56, 8, 7) X(57, 19, 3)       \
  X(60, 10, 6) X(63, 9, 7) X(64, 8, 8) X(65, 13, 5) X(66, 11, 6) X(68, 17, 4) X(69, 23, 3) X(70, 10, 7)      \
  X(72, 9, 8) X(75, 15, 5) X(76, 19, 4) X(77, 11, 7) X(78, 13, 6) X(80, 10, 8) X(81, 9, 9) X(84, 12, 7)      \
  X(85, 17, 5) X(88, 11, 8) X(90, 10, 9) X(91, 13, 7) X(92, 23, 4) X(95, 19, 5) X(96, 12, 8) X(98, 14, 7)    \
  X(99, 11, 9) X(100, 10, 10) X(102, 17, 6) X(104, 13, 8) X(105, 15, 7) X(108, 12, 9) X(110, 11, 10)         \
  X(112, 14, 8) X(114, 19, 6) X(115, 23, 5) X(117, 13, 9) X(119, 17, 7) X(120, 12, 10) X(121, 11, 11)        \
  X(126, 14, 9) X(128, 16, 8)

// N1 of the two-pass plan of length n, or 0 if n has none.
__host__ __device__ inline int fft2_split(int n) {
  switch (n) {
#define HH_F2_CASE(N, A, B) \
  case N:                   \
    return A;
    HH_FFT2_TABLE(HH_F2_CASE)
#undef HH_F2_CASE
    default:
      return 0;
  }
}

// Compile-time loop: f(std::integral_constant<int, i>) for i = B .. E-1.
template <int B, int E, typename F>
__device__ __forceinline__ void sfor(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    sfor<B + 1, E>(f);
  }
}

// In-place R-point DFT of a[0..R) on registers (forward exp(-2 pi i rq / R)).
template <typename T, int R, bool INV>
__device__ __forceinline__ void dft_reg(C2<T>* a) {
  if constexpr (R == 1) {
  } else if constexpr (R <= 4) {
    small_dft<T, R, INV>(a, nullptr, R);
  } else if constexpr (R % 2 == 0) {
    // one radix-2 step on top of two R/2-point DFTs
    constexpr int H = R / 2;
    C2<T> e[H], o[H];
    sfor<0, H>([&](auto ii) {
      constexpr int i = decltype(ii)::value;
      e[i] = a[2 * i];
      o[i] = a[2 * i + 1];
    });
    dft_reg<T, H, INV>(e);
    dft_reg<T, H, INV>(o);
    sfor<0, H>([&](auto kk) {
      constexpr int k = decltype(kk)::value;
      C2<T> t = o[k];
      if constexpr (k > 0) {
        constexpr T wc = T(ct_trig(k, R, false));
        constexpr T ws = T(INV ? ct_trig(k, R, true) : -ct_trig(k, R, true));
        t = mk<T>(o[k].x * wc - o[k].y * ws, o[k].x * ws + o[k].y * wc);
      }
      a[k] = cadd(e[k], t);
      a[k + H] = csub(e[k], t);
    });
  } else {
    // odd R: the outputs q and R - q share the sums s_r = a_r + a_(R-r) and
    // differences d_r = a_r - a_(R-r):
    //   X[q], X[R-q] = A_q +- B_q,  A_q = a_0 + sum_r s_r cos(2 pi r q / R),
    //   B_q = -i sum_r d_r sin(2 pi r q / R)   (forward; +i for the inverse)
    constexpr int H = (R - 1) / 2;
    C2<T> s[H], d[H];
    sfor<1, H + 1>([&](auto rr) {
      constexpr int r = decltype(rr)::value;
      s[r - 1] = cadd(a[r], a[R - r]);
      d[r - 1] = csub(a[r], a[R - r]);
    });
    const C2<T> a0 = a[0];
    C2<T> tot = a0;
    sfor<0, H>([&](auto rr) { tot = cadd(tot, s[decltype(rr)::value]); });
    sfor<1, H + 1>([&](auto qq) {
      constexpr int q = decltype(qq)::value;
      C2<T> A = a0, B = mk<T>(T(0), T(0));
      sfor<1, H + 1>([&](auto rr) {
        constexpr int r = decltype(rr)::value;
        constexpr T c = T(ct_trig((r * q) % R, R, false));
        constexpr T sn = T(ct_trig((r * q) % R, R, true));
        A.x += s[r - 1].x * c;
        A.y += s[r - 1].y * c;
        B.x += d[r - 1].y * sn;
        B.y -= d[r - 1].x * sn;
      });
      if (INV) B = mk<T>(-B.x, -B.y);
      a[q] = cadd(A, B);
      a[R - q] = csub(A, B);
    });
    a[0] = tot;
  }
}

// Element k of line l: base + off(l) + k * es, off(l) = (l / lpg) gstride + (l % lpg) lstride.
__device__ __forceinline__ int line_off(const Lines& L, int l) {
  const int g = l / L.lpg;
  return g * L.gstride + (l - g * L.lpg) * L.lstride;
}

// Two-pass in-place transform of L.n lines of length N1 * N2 (all threads of
// the block take part; ends with __syncthreads()). Adjacent threads take
// adjacent lines, which keeps shared-memory accesses conflict-free when lines
// are adjacent (lstride 1) or rows have an odd pitch. tw: W_N[t], t < N.
// Lines per round are whole, so a block needs at least max(N1, N2) / 2
// threads (every supported length is far below that bound for 256 threads).
template <typename T, int N1, int N2, bool INV>
__device__ __noinline__ void fft2_lines(C2<T>* base, const Lines L, const C2<T>* tw) {
  const int nthr = blockDim.x;
  if constexpr (N2 > 1) {
    constexpr int P = N2 <= 2 ? 4 : (N2 <= 4 ? 2 : 1);  // (line, t1) pairs per thread per round
    const int lpr = (P * nthr) / N1;    // whole lines per round
    for (int l0 = 0; l0 < L.n; l0 += lpr) {
      const int nl = min(lpr, L.n - l0);
      const int tot = nl * N1;
      C2<T> v[P][N2];
      C2<T>* xs[P];
#pragma unroll
      for (int i = 0; i < P; ++i) {
        const int idx = threadIdx.x + i * nthr;
        xs[i] = nullptr;
        if (idx < tot) {
          const int t1 = idx / nl;
          const int line = l0 + (idx - t1 * nl);
          C2<T>* x = base + line_off(L, line) + t1 * L.es;
          xs[i] = x;
          sfor<0, N2>([&](auto mm) {
            constexpr int m = decltype(mm)::value;
            v[i][m] = x[m * N1 * L.es];
          });
          dft_reg<T, N2, INV>(v[i]);
          sfor<1, N2>([&](auto kk) {
            constexpr int k2 = decltype(kk)::value;
            const C2<T> w = tw[t1 * k2];
            v[i][k2] = INV ? cmulc(v[i][k2], w) : cmul(v[i][k2], w);
          });
        }
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < P; ++i) {
        if (xs[i]) {
          C2<T>* x = xs[i];
          sfor<0, N2>([&](auto kk) {
            constexpr int k2 = decltype(kk)::value;
            x[k2 * N1 * L.es] = v[i][k2];
          });
        }
      }
      __syncthreads();
    }
  }
  {
    constexpr int P = N1 <= 2 ? 4 : (N1 <= 4 ? 2 : 1);  // (line, k2) pairs per thread per round
    const int lpr = (P * nthr) / N2;
    for (int l0 = 0; l0 < L.n; l0 += lpr) {
      const int nl = min(lpr, L.n - l0);
      const int tot = nl * N2;
      C2<T> v[P][N1];
      C2<T>* xs[P];
#pragma unroll
      for (int i = 0; i < P; ++i) {
        const int idx = threadIdx.x + i * nthr;
        xs[i] = nullptr;
        if (idx < tot) {
          const int k2 = idx / nl;
          const int line = l0 + (idx - k2 * nl);
          const int es = L.es;
          C2<T>* x = base + line_off(L, line);
          xs[i] = x + k2 * es;  // output k2 + N2 k1 sits at xs + N2 k1 es
          const C2<T>* y = x + k2 * N1 * es;
          sfor<0, N1>([&](auto tt) {
            constexpr int t1 = decltype(tt)::value;
            v[i][t1] = y[t1 * es];
          });
          dft_reg<T, N1, INV>(v[i]);
        }
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < P; ++i) {
        if (xs[i]) {
          C2<T>* x = xs[i];
          sfor<0, N1>([&](auto kk) {
            constexpr int k1 = decltype(kk)::value;
            x[k1 * N2 * L.es] = v[i][k1];
          });
        }
      }
      __syncthreads();
    }
  }
}

// Two-pass transform of length n if it has a plan; false otherwise (nothing
// done). One definition per (precision, direction), each instantiating the
// whole table, lives in its own relocatable object (hh_fft2_inst.cu, built
// four times) so the large instantiation set compiles in parallel.
__device__ bool fft2_f32_fwd(C2<float>* base, const Lines L, int n, const C2<float>* tw);
__device__ bool fft2_f32_inv(C2<float>* base, const Lines L, int n, const C2<float>* tw);
__device__ bool fft2_f64_fwd(C2<double>* base, const Lines L, int n, const C2<double>* tw);
__device__ bool fft2_f64_inv(C2<double>* base, const Lines L, int n, const C2<double>* tw);

template <typename T, bool INV>
__device__ __forceinline__ bool fft2_dispatch(C2<T>* base, const Lines L, int n, const C2<T>* tw) {
  if constexpr (sizeof(T) == 4)
    return INV ? fft2_f32_inv(base, L, n, tw) : fft2_f32_fwd(base, L, n, tw);
  else
    return INV ? fft2_f64_inv(base, L, n, tw) : fft2_f64_fwd(base, L, n, tw);
}

}  // namespace hh
