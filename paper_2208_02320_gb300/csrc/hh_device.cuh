// Device-side types and kernels of the FFT Galerkin elasticity solver.
//
// The discrete problem (Appendix A): find the compatible strain fluctuation
// eps* with G*(C:eps*) = -G*(C:E), solved by conjugate gradients. G is the
// orthogonal projection of a symmetric tensor field onto compatible strains,
// applied mode by mode in Fourier space:
//     (P tau)_ij = n_i v_j + v_i n_j - n_i n_j (n . v),  v = tau n,  n = xi/|xi|,
// with P = 0 at xi = 0. One operator application q = P(C:p) is split into
//   plane pass  : per z-plane, the constitutive law sigma = C(x):p fused into
//                 the x (real-to-complex) and y transforms, in shared memory;
//   column pass : per ky, the z transform, the projection, the inverse z
//                 transform, in shared memory;
//   inverse pass: per z-plane, inverse y and complex-to-real x transforms and
//                 the FP64 partial of <p, q>.
// Transforms are in-place mixed-radix Cooley-Tukey: decimation in frequency
// (natural order in, digit-reversed order out) forward, decimation in time
// (digit-reversed in, natural out) inverse, so no reordering pass is needed.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hh_fftcore.cuh"

namespace hh {

constexpr int kMaxStages = 16;
constexpr int kMaxRadix = 31;

// One transform length. Twiddles W_n[t] = exp(-2 pi i t / n) live in a shared
// table of doubles at tw_off; pos_of_freq (natural frequency -> storage
// position after the forward transform) and sfreq (storage position -> signed
// frequency in (-n/2, n/2]) live in an int table. Lengths with a two-pass plan
// (hh_fft2.cuh) keep natural order, so both tables are the identity map and
// the signed frequency; other lengths use the staged transform below.
struct AxisPlan {
  int n;
  int nst;
  int rad[kMaxStages];
  int tw_off;
  int pf_off;
  int sf_off;
  int split;  // N1 of the two-pass plan (natural order in and out), 0: staged
};

// One (subimage, load case) solve.
struct Prob {
  int nx, ny, nz, nxh;
  int c0x, c0y, c0z, cnx, cny, cnz;  // core region inside the buffered box
  int px, py, pz;                    // plan index per axis
  int lc;                            // load case 0..5
  int box;                           // subimage index in the request
  int plane0;                        // first (problem, z) item of this problem
  int col0;                          // first column item of this problem
  int part0;                         // first partial-sum row of its field-pass items
  int npi;                           // field-pass items: nz, or nz * row chunks when streaming
  int rows;                          // rows per row-streaming item; 0: whole planes
  int cw;                            // spectrum columns (ky, kx) per column-pass item
  int fused;                         // 1: solved whole by the fused cluster kernel (hh_fused.cuh)
  int ct_plane;                      // plane passes: edge of the square plane's compiled body, 0: generic
  int ct_col;                        // column pass: nz * 64 + cw of the compiled body, 0: generic
  long long med_off;                 // iso: byte offset of labels; aniso: element offset of C21
  long long fld_off;                 // element offset of r, p, q (6 V each)
  long long spc_off;                 // complex offset of the spectrum (6 nz ny nxh)
};

// FP64 conjugate-gradient scalars of one problem.
struct PState {
  double rho, rho0, rho_prev, alpha, beta;
  double xbar[6];  // sum over the core of eps* (final pass)
  double sbar[6];  // sum over the core of C:(E + eps*) (final pass)
  double resid;    // final ||b - A x|| / ||b|| from the true residual
  double rt_best;  // smallest true <r, r> seen at a checkpoint
  int iters, active, status, trueflag, homog, restarts, stall;
  int pending;     // r <- r - alpha q, x <- x + alpha p not yet applied
};

enum : int { MED_ISO = 0, MED_ANISO = 1 };
enum : int { MODE_RHS = 0, MODE_ITER = 1, MODE_APPLY = 2, MODE_TRUE = 3, MODE_BASIC = 4 };
enum : int { ST_OK = 0, ST_NOT_CONVERGED = 1, ST_NONFINITE = 2 };

constexpr int kAvgParts = 12;  // per plane item: core sums of eps* (6) and C:(E + eps*) (6)
// Resident 256-thread blocks per SM the plane and column passes are compiled
// for (4: a register budget of 64 per thread; 3: 80).
#ifndef HH_FIELD_BLOCKS_PER_SM
#define HH_FIELD_BLOCKS_PER_SM 4
#endif
constexpr int kFieldBlocksPerSM = HH_FIELD_BLOCKS_PER_SM;

template <typename T>
struct KParams {
  const Prob* prob;
  PState* st;
  const int2* items;  // (problem, z or ky index)
  int nitems;
  int medium;         // MED_ISO / MED_ANISO
  int nyq_mode;       // 0 component rule, 1 mode rule
  int em;             // MODE_BASIC runs the accelerated (Eyre-Milton) scheme
  int nphase;
  const AxisPlan* plans;
  const double* tw;   // interleaved (re, im) twiddles
  const int* itab;
  const uint8_t* labels;
  const T* lammu;     // per phase (lambda, mu)
  const T* c21;       // aniso stiffness, component-major
  T* r;
  T* p;
  T* q;
  T* x;
  C2<T>* spec;
  double* part;       // per-item partial sums
  double tol;
  double rhs_floor;
  int max_iter;
  int fixed_iters;
  int nprob;
  int ycw;           // kx columns per y-column item (row-streaming problems)
  // basic scheme: Green operator of the isotropic reference medium,
  // Gamma0 = g0a (n (x) v + v (x) n) - g0b (n . v) n (x) n, v = tau n
  T g0a, g0b;
  double* cpart;     // per column item: sum h |P tau|^2_F, then Re tau^(0) (6)
};


template <typename T, int R, bool INV>
__device__ void fft_stage(C2<T>* base, const Lines& L, int N, int span, const C2<T>* tw) {
  const int sub = span / R;
  const int tstep = N / span;
  const int nb = N / R;
  const int total = L.n * nb;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    int line, b;
    if (L.fast) {
      line = idx % L.n;
      b = idx / L.n;
    } else {
      line = idx / nb;
      b = idx - line * nb;
    }
    const int blk = b / sub;
    const int j = b - blk * sub;
    C2<T>* x = base + (line / L.lpg) * L.gstride + (line % L.lpg) * L.lstride + (blk * span + j) * L.es;
    const int step = sub * L.es;
    C2<T> a[R];
#pragma unroll
    for (int r = 0; r < R; ++r) a[r] = x[r * step];
    if (!INV) {
      small_dft<T, R, false>(a, tw, N);
#pragma unroll
      for (int q = 1; q < R; ++q) a[q] = cmul(a[q], tw[q * j * tstep]);
    } else {
#pragma unroll
      for (int q = 1; q < R; ++q) a[q] = cmulc(a[q], tw[q * j * tstep]);
      small_dft<T, R, true>(a, tw, N);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) x[r * step] = a[r];
  }
}

// Stage of a prime radix R >= 7 (rare lengths): runtime R, direct O(R^2) DFT.
template <typename T, bool INV>
__device__ __noinline__ void fft_stage_generic(C2<T>* base, const Lines& L, int N, int span, int R, const C2<T>* tw) {
  const int sub = span / R;
  const int tstep = N / span;
  const int nb = N / R;
  const int total = L.n * nb;
  const int st = N / R;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    int line, b;
    if (L.fast) {
      line = idx % L.n;
      b = idx / L.n;
    } else {
      line = idx / nb;
      b = idx - line * nb;
    }
    const int blk = b / sub;
    const int j = b - blk * sub;
    C2<T>* x = base + (line / L.lpg) * L.gstride + (line % L.lpg) * L.lstride + (blk * span + j) * L.es;
    const int step = sub * L.es;
    C2<T> a[kMaxRadix];
    C2<T> y[kMaxRadix];
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
      a[r] = x[r * step];
      if (INV && r > 0) a[r] = cmulc(a[r], tw[r * j * tstep]);
    }
#pragma unroll 1
    for (int q = 0; q < R; ++q) {
      C2<T> acc = a[0];
      int m = 0;
#pragma unroll 1
      for (int r = 1; r < R; ++r) {
        m += q;
        if (m >= R) m -= R;
        C2<T> w = tw[m * st];
        if (INV) w.y = -w.y;
        acc = cadd(acc, cmul(a[r], w));
      }
      y[q] = (!INV && q > 0) ? cmul(acc, tw[q * j * tstep]) : acc;
    }
#pragma unroll 1
    for (int r = 0; r < R; ++r) x[r * step] = y[r];
  }
}

}  // namespace hh

#include "hh_fft2.cuh"

namespace hh {

// In-place transform of a set of lines in shared memory (all threads of the
// block take part; ends with __syncthreads()): the two-pass plan when the
// length has one, else the staged transform (digit-reversed order between
// forward and inverse).
template <typename T, bool INV>
__device__ __noinline__ void fft_lines_staged(C2<T>* base, const Lines L, const AxisPlan& pl, const C2<T>* tw) {
  const int N = pl.n;
  int spans[kMaxStages];
  int s = N;
  for (int i = 0; i < pl.nst; ++i) {
    spans[i] = s;
    s /= pl.rad[i];
  }
  for (int k = 0; k < pl.nst; ++k) {
    const int i = INV ? pl.nst - 1 - k : k;
    const int span = spans[i];
    switch (pl.rad[i]) {
      case 2: fft_stage<T, 2, INV>(base, L, N, span, tw); break;
      case 3: fft_stage<T, 3, INV>(base, L, N, span, tw); break;
      case 4: fft_stage<T, 4, INV>(base, L, N, span, tw); break;
      case 5: fft_stage<T, 5, INV>(base, L, N, span, tw); break;
      default: fft_stage_generic<T, INV>(base, L, N, span, pl.rad[i], tw); break;
    }
    __syncthreads();
  }
}

// The transform of a set of lines: the two-pass plan (one call into the
// transform unit) when the length has one, else the staged transform.
template <typename T, bool INV>
__device__ __forceinline__ void fft_lines(C2<T>* base, const Lines L, const AxisPlan& pl, const C2<T>* tw) {
  if (pl.split && fft2_dispatch<T, INV>(base, L, pl.n, tw)) return;
  fft_lines_staged<T, INV>(base, L, pl, tw);
}

// ---------------------------------------------------------------------------
// Block reduction of K doubles (fixed order: warp shuffle tree, then warp 0).
// Result valid in thread 0. Uses `red` (>= 32 * K doubles of shared memory).
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void block_reduce(double (&v)[K], double* red) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    v[k] = x;
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) red[warp * K + k] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double x = lane < nw ? red[lane * K + k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      v[k] = x;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ double frob_w(int c) { return c < 3 ? 1.0 : 2.0; }

// Per-thread accumulator of a sum of products with FP64-level accuracy. In
// FP32 it keeps an unevaluated sum hi + lo of two floats: each product a b is
// split exactly into p + e (p = fl(a b), e = fma(a, b, -p)), p is added to hi
// with Knuth's two-sum (hi + p = s + t exactly) and the error terms t + e go
// to lo. The FP64 pipe of this GPU runs at a small fraction of the FP32 rate,
// so per-element FP64 arithmetic is avoided; the thread's total is converted
// to FP64 once, for the block reduction. The _rn intrinsics keep the compiler
// from contracting the two-sum into fused multiply-adds. (Summing a voxel's
// six weighted products in plain FP32 before the compensated add was tried:
// at contrast 4.4e5 it moved where FP32 solves stall at their precision floor
// by up to 1 % of the stiffness, so every product is added exactly.)
template <typename T>
struct DotAcc {
  double v = 0.0;
  __device__ __forceinline__ void add(T a, T b) { v = fma(double(a), double(b), v); }
  __device__ __forceinline__ double value() const { return v; }
};
template <>
struct DotAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(t, e));
  }
  __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
};

// Weighted Frobenius product term of stored component c (weights 1, 1, 1, 2, 2, 2).
template <typename T>
__device__ __forceinline__ T frob_t(int c, T b) { return c < 3 ? b : T(2) * b; }

// ---------------------------------------------------------------------------
// Constitutive law (Section 4): isotropic sigma = lam tr(eps) I + 2 mu eps, or
// anisotropic Voigt sigma = C gamma with engineering shear gamma.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void stress_iso(const T (&e)[6], T lam, T mu, T (&s)[6]) {
  const T tr = e[0] + e[1] + e[2];
#pragma unroll
  for (int c = 0; c < 6; ++c) s[c] = T(2) * mu * e[c];
  s[0] += lam * tr;
  s[1] += lam * tr;
  s[2] += lam * tr;
}

template <typename T>
__device__ __forceinline__ void stress_aniso(const T (&e)[6], const T* c21, long long V, long long v, T (&s)[6]) {
  const T g[6] = {e[0], e[1], e[2], T(2) * e[3], T(2) * e[4], T(2) * e[5]};
  T C[21];
#pragma unroll
  for (int k = 0; k < 21; ++k) C[k] = c21[k * V + v];
  // upper-triangle index of (i, j), i <= j: i*6 - i*(i-1)/2 + (j - i)
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const int a = i < j ? i : j;
      const int b = i < j ? j : i;
      acc += C[a * 6 - a * (a - 1) / 2 + (b - a)] * g[j];
    }
    s[i] = acc;
  }
}

// a (n_i v_j + v_i n_j) - b n_i n_j (n . v), v = t n, of one mode (6 complex
// tensor components, in place); zero where the wave vector vanishes.
template <typename T>
__device__ __forceinline__ void green_mode(C2<T> (&t)[6], T x0, T x1, T x2, T a, T b) {
  const T nn = x0 * x0 + x1 * x1 + x2 * x2;
  if (!(nn > T(0))) {
#pragma unroll
    for (int c = 0; c < 6; ++c) t[c] = mk<T>(T(0), T(0));
    return;
  }
  const T inv = T(1) / sqrt(nn);
  const T n[3] = {x0 * inv, x1 * inv, x2 * inv};
  // tensor: 0=11 1=22 2=33 3=23 4=13 5=12; (i, j) of each stored component
  const int ci[6] = {0, 1, 2, 1, 0, 0}, cj[6] = {0, 1, 2, 2, 2, 1};
  C2<T> v[3];
  v[0] = mk<T>(t[0].x * n[0] + t[5].x * n[1] + t[4].x * n[2], t[0].y * n[0] + t[5].y * n[1] + t[4].y * n[2]);
  v[1] = mk<T>(t[5].x * n[0] + t[1].x * n[1] + t[3].x * n[2], t[5].y * n[0] + t[1].y * n[1] + t[3].y * n[2]);
  v[2] = mk<T>(t[4].x * n[0] + t[3].x * n[1] + t[2].x * n[2], t[4].y * n[0] + t[3].y * n[1] + t[2].y * n[2]);
  const C2<T> sv = mk<T>(n[0] * v[0].x + n[1] * v[1].x + n[2] * v[2].x, n[0] * v[0].y + n[1] * v[1].y + n[2] * v[2].y);
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const T ni = n[ci[c]], nj = n[cj[c]];
    const C2<T> vi = v[ci[c]], vj = v[cj[c]];
    t[c] = mk<T>(a * (ni * vj.x + vi.x * nj) - b * ni * nj * sv.x, a * (ni * vj.y + vi.y * nj) - b * ni * nj * sv.y);
  }
}

// Projection of one mode (6 complex tensor components, in place).
template <typename T>
__device__ __forceinline__ void project_mode(C2<T> (&t)[6], T x0, T x1, T x2) {
  const T nn = x0 * x0 + x1 * x1 + x2 * x2;
  if (!(nn > T(0))) {
#pragma unroll
    for (int c = 0; c < 6; ++c) t[c] = mk<T>(T(0), T(0));
    return;
  }
  const T inv = T(1) / sqrt(nn);
  const T n0 = x0 * inv, n1 = x1 * inv, n2 = x2 * inv;
  // tensor: 0=11 1=22 2=33 3=23 4=13 5=12
  C2<T> v0, v1, v2;
  v0.x = t[0].x * n0 + t[5].x * n1 + t[4].x * n2;
  v0.y = t[0].y * n0 + t[5].y * n1 + t[4].y * n2;
  v1.x = t[5].x * n0 + t[1].x * n1 + t[3].x * n2;
  v1.y = t[5].y * n0 + t[1].y * n1 + t[3].y * n2;
  v2.x = t[4].x * n0 + t[3].x * n1 + t[2].x * n2;
  v2.y = t[4].y * n0 + t[3].y * n1 + t[2].y * n2;
  C2<T> s;
  s.x = n0 * v0.x + n1 * v1.x + n2 * v2.x;
  s.y = n0 * v0.y + n1 * v1.y + n2 * v2.y;
  // P_ij = n_i v_j + v_i n_j - n_i n_j s
  t[0] = mk<T>(T(2) * n0 * v0.x - n0 * n0 * s.x, T(2) * n0 * v0.y - n0 * n0 * s.y);
  t[1] = mk<T>(T(2) * n1 * v1.x - n1 * n1 * s.x, T(2) * n1 * v1.y - n1 * n1 * s.y);
  t[2] = mk<T>(T(2) * n2 * v2.x - n2 * n2 * s.x, T(2) * n2 * v2.y - n2 * n2 * s.y);
  t[3] = mk<T>(n1 * v2.x + v1.x * n2 - n1 * n2 * s.x, n1 * v2.y + v1.y * n2 - n1 * n2 * s.y);
  t[4] = mk<T>(n0 * v2.x + v0.x * n2 - n0 * n2 * s.x, n0 * v2.y + v0.y * n2 - n0 * n2 * s.y);
  t[5] = mk<T>(n0 * v1.x + v0.x * n1 - n0 * n1 * s.x, n0 * v1.y + v0.y * n1 - n0 * n1 * s.y);
}

// Copy an axis' twiddles (double -> T) into shared memory.
template <typename T>
__device__ __forceinline__ void load_tw(C2<T>* dst, const double* tw, const AxisPlan& pl) {
  for (int t = threadIdx.x; t < pl.n; t += blockDim.x)
    dst[t] = mk<T>(T(tw[2 * (pl.tw_off + t)]), T(tw[2 * (pl.tw_off + t) + 1]));
}

__device__ __forceinline__ int odd_pitch(int n) { return n | 1; }

// Shared-memory layout of the plane passes (must match plane_smem_bytes on the
// host). The whole plane lives in S as three blocks of ny "pair rows", one
// block per component pair (2 c2, 2 c2 + 1), with an odd pitch RP >= nx + 2.
// In real space a pair row holds the packed complex row s_(2c2) + i s_(2c2+1)
// (nx entries); after the x transform and the unpack it holds the two half
// spectra [A_0 .. A_(nxh-1) | B_0 .. B_(nxh-1)], and the y transforms run
// down its columns.
template <typename T>
struct PlaneSmem {
  C2<T>* S;     // 3 * ny * RP
  C2<T>* twx;   // nx
  C2<T>* twy;   // ny
  int* pfx;     // nx
  T* lm;        // 2 * nphase
  double* red;  // 32 * 4
};

__device__ __forceinline__ int pair_pitch(int nx) { return (nx + 2) | 1; }

template <typename T>
__device__ __forceinline__ PlaneSmem<T> plane_layout(char* base, int nx, int ny, int nphase) {
  PlaneSmem<T> s;
  size_t o = 0;
  s.red = reinterpret_cast<double*>(base + o);
  o += 32 * 4 * sizeof(double);
  s.S = reinterpret_cast<C2<T>*>(base + o);
  o += sizeof(C2<T>) * 3 * ny * pair_pitch(nx);
  s.twx = reinterpret_cast<C2<T>*>(base + o);
  o += sizeof(C2<T>) * nx;
  s.twy = reinterpret_cast<C2<T>*>(base + o);
  o += sizeof(C2<T>) * ny;
  s.pfx = reinterpret_cast<int*>(base + o);
  o += sizeof(int) * ((nx + 3) & ~3);
  s.lm = reinterpret_cast<T*>(base + o);
  return s;
}

// Row-major walk e = hi * W + lo (0 <= lo < W) of one thread's indices
// e0, e0 + S, e0 + 2 S, ...: after the first position, each step adds the
// quotient and remainder of S / W with one carry, no division.
struct Walk2 {
  int hi, lo;
  int dhi, dlo, W;
  __device__ __forceinline__ Walk2(int e0, int S, int W_) : W(W_) {
    hi = e0 / W_;
    lo = e0 - hi * W_;
    dhi = S / W_;
    dlo = S - dhi * W_;
  }
  __device__ __forceinline__ void next() {
    lo += dlo;
    hi += dhi;
    if (lo >= W) {
      lo -= W;
      ++hi;
    }
  }
};

// Row-major walk e = (a * B + b) * W + lo (0 <= b < B, 0 <= lo < W) with a
// fixed stride S, without division after the first position: the row
// a * B + b advances by S / W or S / W + 1 (when lo carries), and each of the
// two increments is split into its quotient and remainder by B once.
struct Walk3 {
  int a, b, lo;
  int W, B, dlo, da0, db0, da1, db1;
  __device__ __forceinline__ Walk3(int e0, int S, int W_, int B_) : W(W_), B(B_) {
    const int row = e0 / W_;
    lo = e0 - row * W_;
    a = row / B_;
    b = row - a * B_;
    const int dhi = S / W_;
    dlo = S - dhi * W_;
    da0 = dhi / B_;
    db0 = dhi - da0 * B_;
    da1 = (dhi + 1) / B_;
    db1 = (dhi + 1) - da1 * B_;
  }
  __device__ __forceinline__ void next() {
    lo += dlo;
    int da = da0, db = db0;
    if (lo >= W) {
      lo -= W;
      da = da1;
      db = db1;
    }
    b += db;
    a += da;
    if (b >= B) {
      b -= B;
      ++a;
    }
  }
};

// x-line and y-line views of the pair-row plane.
__device__ __forceinline__ Lines plane_rows(int ny, int RP) { return Lines{3 * ny, 1 << 30, 0, RP, 1, false}; }
__device__ __forceinline__ Lines plane_cols(int ny, int nxh, int RP) {
  return Lines{6 * nxh, 2 * nxh, ny * RP, 1, RP, true};
}
// Position in S of spectrum component c at (ky position, kx).
__device__ __forceinline__ int plane_spec_at(int c, int ky, int kx, int ny, int nxh, int RP) {
  return ((c >> 1) * ny + ky) * RP + (c & 1) * nxh + kx;
}

constexpr int kPackPerThread = 4;

// Global-to-shared element copies are issued as cp.async (sm_80 and later):
// every copy of a thread is in flight at once and none is staged through
// registers; the caller waits with copy_async_wait() before its barrier.
__device__ __forceinline__ void copy_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Split every transformed packed row Z = A + iB (A, B spectra of real rows)
// into [A | B] in place, in rounds of whole rows (reads, barrier, writes).
template <typename T>
__device__ __forceinline__ void unpack_rows(C2<T>* S, int nrows, int RP, int nx, int nxh, const int* pfx) {
  const int rpr = max(1, (kPackPerThread * (int)blockDim.x) / nxh);
  for (int r0 = 0; r0 < nrows; r0 += rpr) {
    const int tot = min(rpr, nrows - r0) * nxh;
    C2<T> A[kPackPerThread], B[kPackPerThread];
    int o[kPackPerThread];
#pragma unroll
    for (int i = 0; i < kPackPerThread; ++i) {
      const int e = threadIdx.x + i * blockDim.x;
      o[i] = -1;
      if (e < tot) {
        const int rr = e / nxh;
        const int k = e - rr * nxh;
        const C2<T>* R = S + (r0 + rr) * RP;
        const C2<T> a = R[pfx[k]];
        const C2<T> b = R[pfx[k == 0 ? 0 : nx - k]];
        A[i] = mk<T>(T(0.5) * (a.x + b.x), T(0.5) * (a.y - b.y));
        B[i] = mk<T>(T(0.5) * (a.y + b.y), T(-0.5) * (a.x - b.x));
        o[i] = (r0 + rr) * RP + k;
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kPackPerThread; ++i)
      if (o[i] >= 0) {
        S[o[i]] = A[i];
        S[o[i] + nxh] = B[i];
      }
    __syncthreads();
  }
}

// Inverse of unpack_rows: [A | B] -> A + iB over the full row with the
// Hermitian extension, at the transform's input positions pfx[k].
template <typename T>
__device__ __forceinline__ void pack_rows(C2<T>* S, int nrows, int RP, int nx, int nxh, const int* pfx) {
  const int rpr = max(1, (kPackPerThread * (int)blockDim.x) / nx);
  for (int r0 = 0; r0 < nrows; r0 += rpr) {
    const int tot = min(rpr, nrows - r0) * nx;
    C2<T> Z[kPackPerThread];
    int o[kPackPerThread];
#pragma unroll
    for (int i = 0; i < kPackPerThread; ++i) {
      const int e = threadIdx.x + i * blockDim.x;
      o[i] = -1;
      if (e < tot) {
        const int rr = e / nx;
        const int k = e - rr * nx;
        const C2<T>* R = S + (r0 + rr) * RP;
        C2<T> A, B;
        if (k < nxh) {
          A = R[k];
          B = R[nxh + k];
        } else {
          A = R[nx - k];
          B = R[nxh + nx - k];
          A.y = -A.y;
          B.y = -B.y;
        }
        Z[i] = mk<T>(A.x - B.y, A.y + B.x);
        o[i] = (r0 + rr) * RP + pfx[k];
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kPackPerThread; ++i)
      if (o[i] >= 0) S[o[i]] = Z[i];
    __syncthreads();
  }
}

template <typename T>
__device__ __forceinline__ void plane_tables(const KParams<T>& P, const PlaneSmem<T>& sm, const AxisPlan& ax,
                                             const AxisPlan& ay, int nx, bool with_y = true) {
  load_tw<T>(sm.twx, P.tw, ax);
  if (with_y) load_tw<T>(sm.twy, P.tw, ay);
  for (int t = threadIdx.x; t < nx; t += blockDim.x) sm.pfx[t] = P.itab[ax.pf_off + t];
  if (P.medium == MED_ISO)
    for (int t = threadIdx.x; t < 2 * P.nphase; t += blockDim.x) sm.lm[t] = P.lammu[t];
}

// Plane pass (forward): constitutive law fused into the x and y transforms.
//   MODE_RHS  : tau = C : E (E = unit load of the problem); partial <tau, tau>_F
//   MODE_ITER : the deferred CG update of the previous iteration (when
//               pending) r <- r - alpha q, x <- x + alpha p, then
//               p <- r + beta p (all stored), tau = C : p; partial <r, r>_F
//   MODE_TRUE : tau = C : (E + x)  (true residual r = -G*tau follows)
//   MODE_APPLY: tau = C : p (p read only)
//   MODE_BASIC: the pending fixed-point update x <- x - q, then
//               tau = C : (E + x)  (basic scheme; x holds eps - E)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ bool skip_problem(const PState* st, int pr, int mode) {
  if (mode == MODE_ITER || mode == MODE_BASIC) return !st[pr].active;
  if (mode == MODE_TRUE) return !st[pr].trueflag;
  return false;
}

// Per-item CG scalars of the forward pass.
template <typename T, int MODE>
struct FwdScal {
  T alpha = T(0), beta = T(0);
  bool pend = false;
  __device__ __forceinline__ explicit FwdScal(const PState& s) {
    if (MODE == MODE_ITER || MODE == MODE_BASIC) {
      alpha = T(s.alpha);
      beta = T(s.beta);
      pend = s.pending != 0;
    }
  }
};

// One voxel of the forward pass: the mode's strain (with the vector updates
// it stores), its stress s, and the mode's partial sum.
template <typename T, int MODE>
__device__ __forceinline__ void fwd_voxel(const KParams<T>& P, const Prob& d, long long V, long long vo,
                                          const FwdScal<T, MODE>& k, const T* lm, T (&s)[6], DotAcc<T>& acc) {
  T* __restrict__ rr = P.r + d.fld_off + vo;
  T* __restrict__ pp = P.p + d.fld_off + vo;
  T* __restrict__ xx = P.x + d.fld_off + vo;
  const T* __restrict__ qq = P.q + d.fld_off + vo;
  const T Ed = d.lc < 3 ? T(1) : T(0.5);
  // every load of the voxel is issued before any store, so the loads of all
  // six components are in flight together
  int lab = 0;
  if (P.medium == MED_ISO) lab = P.labels[d.med_off + vo];
  T e[6];
  if (MODE == MODE_RHS) {
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = T(0);
    e[d.lc] = Ed;
  } else if (MODE == MODE_ITER) {
    T rv[6], pv[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      rv[c] = rr[c * V];
      pv[c] = pp[c * V];
    }
    if (k.pend) {
      T qv[6], xv[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        qv[c] = qq[c * V];
        xv[c] = xx[c * V];
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        rv[c] -= k.alpha * qv[c];
        rr[c * V] = rv[c];
        xx[c * V] = xv[c] + k.alpha * pv[c];
      }
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const T pn = rv[c] + k.beta * pv[c];
      pp[c * V] = pn;
      e[c] = pn;
      acc.add(rv[c], frob_t(c, rv[c]));
    }
  } else if (MODE == MODE_TRUE) {
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = xx[c * V];
    e[d.lc] += Ed;
  } else if (MODE == MODE_BASIC) {
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = xx[c * V];
    if (k.pend) {
      T qv[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) qv[c] = qq[c * V];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        e[c] -= qv[c];
        xx[c * V] = e[c];
      }
    }
    e[d.lc] += Ed;
  } else {
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = pp[c * V];
  }
  if (P.medium == MED_ISO) {
    stress_iso<T>(e, lm[2 * lab], lm[2 * lab + 1], s);
  } else {
    stress_aniso<T>(e, P.c21 + d.med_off, V, vo, s);
  }
  if (MODE == MODE_RHS) {
#pragma unroll
    for (int c = 0; c < 6; ++c) acc.add(s[c], frob_t(c, s[c]));
  }
}

// Partial-sum slot the forward pass of a mode writes (-1: none).
template <int MODE>
__device__ __forceinline__ int fwd_slot() {
  return MODE == MODE_RHS ? 0 : (MODE == MODE_ITER ? 13 : -1);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256, kFieldBlocksPerSM) k_plane_fwd(KParams<T> P) {
  extern __shared__ __align__(16) char smem[];
  int tab_px = -1, tab_py = -1;  // plans whose tables are in shared memory
  for (int it = blockIdx.x; it < P.nitems; it += gridDim.x) {
    const int2 w = P.items[it];
    if (skip_problem<T>(P.st, w.x, MODE)) continue;
    const Prob d = P.prob[w.x];
    const int z = w.y;
    const int nx = d.nx, ny = d.ny, nxh = d.nxh;
    const int RP = pair_pitch(nx);
    const long long V = (long long)nx * ny * d.nz;
    PlaneSmem<T> sm = plane_layout<T>(smem, nx, ny, P.nphase);
    const AxisPlan& ax = P.plans[d.px];  // by reference: no per-thread copy
    const AxisPlan& ay = P.plans[d.py];  // by reference: no per-thread copy
    if (d.px != tab_px || d.py != tab_py) {  // same plans: same layout, tables still in place
      plane_tables<T>(P, sm, ax, ay, nx);
      tab_px = d.px;
      tab_py = d.py;
    }
    const FwdScal<T, MODE> k(P.st[w.x]);
    __syncthreads();

    DotAcc<T> dot;
    const long long zoff = (long long)z * ny * nx;
    // voxel phase: stress of the whole plane into the pair rows
    Walk2 wv(threadIdx.x, blockDim.x, nx);
    for (int v = threadIdx.x; v < ny * nx; v += blockDim.x, wv.next()) {
      const int y = wv.hi;
      const int x = wv.lo;
      T s[6];
      fwd_voxel<T, MODE>(P, d, V, zoff + v, k, sm.lm, s, dot);
#pragma unroll
      for (int c2 = 0; c2 < 3; ++c2) sm.S[(c2 * ny + y) * RP + x] = mk<T>(s[2 * c2], s[2 * c2 + 1]);
    }
    __syncthreads();
    fft_lines<T, false>(sm.S, plane_rows(ny, RP), ax, sm.twx);
    unpack_rows<T>(sm.S, 3 * ny, RP, nx, nxh, sm.pfx);
    fft_lines<T, false>(sm.S, plane_cols(ny, nxh, RP), ay, sm.twy);
    // store the plane of the spectrum: spec[c][z][kyp][kx]
    C2<T>* sp = P.spec + d.spc_off;
    const int pl = ny * nxh;
    {
      // e = (c * ny + ky) * nxh + kx
      Walk3 wk(threadIdx.x, blockDim.x, nxh, ny);
      for (int e = threadIdx.x; e < 6 * pl; e += blockDim.x, wk.next())
        sp[((long long)wk.a * d.nz + z) * pl + wk.b * nxh + wk.lo] =
            sm.S[plane_spec_at(wk.a, wk.b, wk.lo, ny, nxh, RP)];
    }
    if (fwd_slot<MODE>() >= 0) {
      double acc[1] = {dot.value()};
      block_reduce<1>(acc, sm.red);
      if (threadIdx.x == 0) P.part[(long long)(d.part0 + z) * 16 + fwd_slot<MODE>()] = acc[0];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Row-streaming forward pass, for planes too large for one block: rows
// y0 .. y0 + nr of plane z (item w.y = z | y0 << 16), the constitutive law
// fused into the x transform; the half-spectrum rows go to spec in natural y
// order and k_ycols does the y transform.
// ---------------------------------------------------------------------------
template <typename T, int MODE>
__global__ void __launch_bounds__(256, kFieldBlocksPerSM) k_rows_fwd(KParams<T> P) {
  extern __shared__ __align__(16) char smem[];
  for (int it = blockIdx.x; it < P.nitems; it += gridDim.x) {
    const int2 w = P.items[it];
    if (skip_problem<T>(P.st, w.x, MODE)) continue;
    const Prob d = P.prob[w.x];
    const int z = w.y & 0xffff, y0 = w.y >> 16;
    const int nx = d.nx, ny = d.ny, nxh = d.nxh, R = d.rows;
    const int nr = min(R, ny - y0);
    const int RP = pair_pitch(nx);
    const long long V = (long long)nx * ny * d.nz;
    PlaneSmem<T> sm = plane_layout<T>(smem, nx, R, P.nphase);
    const AxisPlan& ax = P.plans[d.px];  // by reference: no per-thread copy
    plane_tables<T>(P, sm, ax, ax, nx, false);
    const FwdScal<T, MODE> k(P.st[w.x]);
    __syncthreads();

    DotAcc<T> dot;
    const long long off0 = ((long long)z * ny + y0) * nx;
    for (int v = threadIdx.x; v < nr * nx; v += blockDim.x) {
      const int yy = v / nx;
      const int x = v - yy * nx;
      T s[6];
      fwd_voxel<T, MODE>(P, d, V, off0 + v, k, sm.lm, s, dot);
#pragma unroll
      for (int c2 = 0; c2 < 3; ++c2) sm.S[(c2 * R + yy) * RP + x] = mk<T>(s[2 * c2], s[2 * c2 + 1]);
    }
    __syncthreads();
    fft_lines<T, false>(sm.S, Lines{3 * nr, nr, R * RP, RP, 1, false}, ax, sm.twx);
    unpack_rows<T>(sm.S, 3 * R, RP, nx, nxh, sm.pfx);
    C2<T>* sp = P.spec + d.spc_off;
    const int rl = nr * nxh;
    for (int e = threadIdx.x; e < 6 * rl; e += blockDim.x) {
      const int c = e / rl;
      const int rem = e - c * rl;
      const int yy = rem / nxh;
      sp[(((long long)c * d.nz + z) * ny + y0) * nxh + rem] = sm.S[plane_spec_at(c, yy, rem - yy * nxh, R, nxh, RP)];
    }
    if (fwd_slot<MODE>() >= 0) {
      double acc[1] = {dot.value()};
      block_reduce<1>(acc, sm.red);
      const int nch = (ny + R - 1) / R;
      if (threadIdx.x == 0) P.part[(long long)(d.part0 + z * nch + y0 / R) * 16 + fwd_slot<MODE>()] = acc[0];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// y transforms of row-streaming problems: W = ycw kx columns of plane z
// (item w.y = z | kx0 << 16), forward or inverse, in place in spec.
// ---------------------------------------------------------------------------
template <typename T, bool INV>
__global__ void __launch_bounds__(256, kFieldBlocksPerSM) k_ycols(KParams<T> P, int skip_mode) {
  extern __shared__ __align__(16) char smem[];
  for (int it = blockIdx.x; it < P.nitems; it += gridDim.x) {
    const int2 w = P.items[it];
    if (skip_problem<T>(P.st, w.x, skip_mode)) continue;
    const Prob d = P.prob[w.x];
    const int z = w.y & 0xffff, kx0 = w.y >> 16;
    const int ny = d.ny, nxh = d.nxh;
    const int W = min(P.ycw, nxh - kx0);
    C2<T>* tile = reinterpret_cast<C2<T>*>(smem);
    C2<T>* twy = tile + 6 * ny * P.ycw;
    const AxisPlan& ay = P.plans[d.py];  // by reference: no per-thread copy
    load_tw<T>(twy, P.tw, ay);
    C2<T>* sp = P.spec + d.spc_off + (long long)z * ny * nxh + kx0;
    const long long cstride = (long long)d.nz * ny * nxh;
    for (int e = threadIdx.x; e < 6 * ny * W; e += blockDim.x) {
      const int kx = e % W;
      const int cy = e / W;  // c * ny + y
      const int c = cy / ny;
      tile[e] = sp[c * cstride + (long long)(cy - c * ny) * nxh + kx];
    }
    __syncthreads();
    fft_lines<T, INV>(tile, Lines{6 * W, W, ny * W, 1, W, true}, ay, twy);
    for (int e = threadIdx.x; e < 6 * ny * W; e += blockDim.x) {
      const int kx = e % W;
      const int cy = e / W;
      const int c = cy / ny;
      sp[c * cstride + (long long)(cy - c * ny) * nxh + kx] = tile[e];
    }
    __syncthreads();
  }
}

// Shared-memory layout of the column pass (must match column_smem_bytes on
// the host): W-column tile of the six components, z twiddles, the signed
// z and y frequencies, and the block-reduction buffer.
template <typename T>
struct ColumnSmem {
  C2<T>* tile;  // 6 * nz * cw
  C2<T>* twz;   // nz
  T* fz;        // nz: wave-vector component m_z / nz of each storage position
  int* sfz;     // nz
  int* sfy;     // ny
  double* red;  // 32 * 7
};

template <typename T>
__device__ __forceinline__ ColumnSmem<T> column_layout(char* base, int cw, int nz, int ny) {
  ColumnSmem<T> s;
  size_t o = 0;
  s.tile = reinterpret_cast<C2<T>*>(base + o);
  o += sizeof(C2<T>) * 6 * (size_t)nz * cw;
  s.twz = reinterpret_cast<C2<T>*>(base + o);
  o += sizeof(C2<T>) * nz;
  s.fz = reinterpret_cast<T*>(base + o);
  o += sizeof(T) * nz;
  s.sfz = reinterpret_cast<int*>(base + o);
  o += sizeof(int) * nz;
  s.sfy = reinterpret_cast<int*>(base + o);
  o += sizeof(int) * ny;
  o = (o + 7) & ~size_t(7);
  s.red = reinterpret_cast<double*>(base + o);
  return s;
}

// ---------------------------------------------------------------------------
// Column pass: z transform, projection, inverse z transform for cw
// consecutive spectrum columns j = ky position * nxh + kx of one problem.
// `skip_mode` selects which problems take part (as in the plane passes).
// ---------------------------------------------------------------------------
//   BASIC: the basic scheme's step instead of the
//   projection: the mode becomes Gamma0 tau, and the item leaves the partial
//   sum of h |P tau|^2_F (h = 2 for the kx that stand for a conjugate pair)
//   and, from the zero mode, Re tau^(0) for the equilibrium residual.
template <typename T, bool BASIC>
__global__ void __launch_bounds__(256, kFieldBlocksPerSM) k_column(KParams<T> P, int skip_mode) {
  extern __shared__ __align__(16) char smem[];
  int tab_pz = -1, tab_py = -1, tab_cw = -1;  // layout whose tables are in shared memory
  for (int it = blockIdx.x; it < P.nitems; it += gridDim.x) {
    const int2 w = P.items[it];
    if (skip_problem<T>(P.st, w.x, skip_mode)) continue;
    const Prob d = P.prob[w.x];
    const int j0 = w.y;  // first spectrum column: j = ky position * nxh + kx
    const int nx = d.nx, ny = d.ny, nz = d.nz, nxh = d.nxh;
    const int pl = ny * nxh;
    const int W = min(d.cw, pl - j0);  // columns of this item, contiguous in every (c, z) plane
    ColumnSmem<T> sm = column_layout<T>(smem, d.cw, nz, ny);
    const AxisPlan& az = P.plans[d.pz];  // by reference: no per-thread copy
    const AxisPlan& ay = P.plans[d.py];  // by reference: no per-thread copy
    if (d.pz != tab_pz || d.py != tab_py || d.cw != tab_cw) {  // same plans and width: same layout
      load_tw<T>(sm.twz, P.tw, az);
      for (int t = threadIdx.x; t < nz; t += blockDim.x) {
        const int mz = P.itab[az.sf_off + t];
        sm.sfz[t] = mz;
        sm.fz[t] = T(mz) / T(nz);
      }
      for (int t = threadIdx.x; t < ny; t += blockDim.x) sm.sfy[t] = P.itab[ay.sf_off + t];
      tab_pz = d.pz;
      tab_py = d.py;
      tab_cw = d.cw;
    }
    C2<T>* sp = P.spec + d.spc_off + j0;
    {
      // tile[e] = sp[cz * pl + jl], e = cz * W + jl (cz = c * nz + z)
      Walk2 wk(threadIdx.x, blockDim.x, W);
      for (int e = threadIdx.x; e < 6 * nz * W; e += blockDim.x, wk.next()) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(sm.tile + e);
        const C2<T>* g = sp + (long long)wk.hi * pl + wk.lo;
        if constexpr (sizeof(C2<T>) == 8)
          asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(g) : "memory");
        else
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(g) : "memory");
      }
    }
    copy_async_wait();
    __syncthreads();
    const Lines Lz{6 * W, W, nz * W, 1, W, true};
    fft_lines<T, false>(sm.tile, Lz, az, sm.twz);
    // projection (or the basic scheme's Green operator) of every mode
    double acc[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    // (kzp, jl) of mode e = kzp * W + jl by a division-free walk; the column's
    // (ky, kx) wave-vector components change only with jl
    Walk2 wm(threadIdx.x, blockDim.x, W);
    int jl_c = -1, kx = 0, my = 0;
    T x0c = T(0), x1c = T(0);
    for (int e = threadIdx.x; e < nz * W; e += blockDim.x, wm.next()) {
      const int jl = wm.lo;
      const int kzp = wm.hi;
      if (jl != jl_c) {
        jl_c = jl;
        const int j = j0 + jl;
        const int kyp = j / nxh;
        kx = j - kyp * nxh;
        my = sm.sfy[kyp];
        x0c = T(kx) / T(nx);
        x1c = T(my) / T(ny);
      }
      const int mz = sm.sfz[kzp];
      const bool nyq_x = (nx % 2 == 0) && (2 * kx == nx);
      const bool nyq_y = (ny % 2 == 0) && (2 * my == ny);
      const bool nyq_z = (nz % 2 == 0) && (2 * mz == nz);
      T x0 = x0c, x1 = x1c, x2 = sm.fz[kzp];
      if (P.nyq_mode == 0) {
        if (nyq_x) x0 = T(0);
        if (nyq_y) x1 = T(0);
        if (nyq_z) x2 = T(0);
      } else if (nyq_x || nyq_y || nyq_z) {
        x0 = x1 = x2 = T(0);
      }
      C2<T> t[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) t[c] = sm.tile[(c * nz + kzp) * W + jl];
      if (BASIC) {
        C2<T> pt[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) pt[c] = t[c];
        project_mode<T>(pt, x0, x1, x2);
        const double h = (kx == 0 || 2 * kx == nx) ? 1.0 : 2.0;
#pragma unroll
        for (int c = 0; c < 6; ++c)
          acc[0] += h * frob_w(c) * (double(pt[c].x) * double(pt[c].x) + double(pt[c].y) * double(pt[c].y));
        if (kx == 0 && my == 0 && mz == 0) {
#pragma unroll
          for (int c = 0; c < 6; ++c) acc[1 + c] += double(t[c].x);
        }
        green_mode<T>(t, x0, x1, x2, P.g0a, P.g0b);
      } else {
        project_mode<T>(t, x0, x1, x2);
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) sm.tile[(c * nz + kzp) * W + jl] = t[c];
    }
    if (BASIC) {
      block_reduce<7>(acc, sm.red);
      if (threadIdx.x == 0) {
        double* cp = P.cpart + (long long)(d.col0 + j0 / d.cw) * 8;
#pragma unroll
        for (int k = 0; k < 7; ++k) cp[k] = acc[k];
      }
    }
    __syncthreads();
    fft_lines<T, true>(sm.tile, Lz, az, sm.twz);
    {
      Walk2 wk(threadIdx.x, blockDim.x, W);
      for (int e = threadIdx.x; e < 6 * nz * W; e += blockDim.x, wk.next())
        sp[(long long)wk.hi * pl + wk.lo] = sm.tile[e];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Plane pass (inverse): inverse y and complex-to-real x transforms.
//   MODE_RHS  : r = p = -q, x = 0, partial <r, r>_F
//   MODE_ITER : store q; partials <p, q>_F, <r, q>_F, <q, q>_F (the next
//               <r, r> follows from them without another pass)
//   MODE_TRUE : r = -q (true residual), partial <r, r>_F
//   MODE_APPLY, MODE_BASIC: store q
// ---------------------------------------------------------------------------
// One voxel of the inverse pass: q = (transformed value) / V and the mode's
// stores and partial sums (acc: MODE_ITER <p,q>, <r,q>, <q,q>; RHS/TRUE <r,r>).
template <typename T, int MODE>
__device__ __forceinline__ void inv_voxel(const KParams<T>& P, const Prob& d, long long V, long long vo,
                                          const T (&qv)[6], const T* lm, DotAcc<T> (&acc)[3]) {
  T* __restrict__ rr = P.r + d.fld_off + vo;
  T* __restrict__ pp = P.p + d.fld_off + vo;
  T* __restrict__ qq = P.q + d.fld_off + vo;
  T* __restrict__ xx = P.x + d.fld_off + vo;
  if (MODE == MODE_RHS || MODE == MODE_TRUE) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const T rv = -qv[c];
      rr[c * V] = rv;
      if (MODE == MODE_RHS) {
        pp[c * V] = rv;
        xx[c * V] = T(0);
      }
      acc[0].add(rv, frob_t(c, rv));
    }
  } else if (MODE == MODE_ITER) {
    T pv[6], rv[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      pv[c] = pp[c * V];
      rv[c] = rr[c * V];
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      qq[c * V] = qv[c];
      const T wq = frob_t(c, qv[c]);
      acc[0].add(pv[c], wq);
      acc[1].add(rv[c], wq);
      acc[2].add(qv[c], wq);
    }
  } else if (MODE == MODE_BASIC && P.em) {
    // accelerated scheme: the Lippmann-Schwinger residual B = E - eps -
    // Gamma0 * tau = -(x + q) (x holds eps - E, q = Gamma0 * tau) and the
    // update x <- x + 2 (C + C0)^-1 C0 : B, whose spherical and deviatoric
    // factors per phase the launch passes in lm; partial ||B||^2_F
    const int lab = P.labels[d.med_off + vo];
    T xv[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) xv[c] = xx[c * V];
    const T fs = lm[2 * lab], fd = lm[2 * lab + 1];
    T bv[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) bv[c] = -(xv[c] + qv[c]);
    const T sph = (bv[0] + bv[1] + bv[2]) * T(1.0 / 3.0);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      xx[c * V] = xv[c] + fd * bv[c] + (c < 3 ? (fs - fd) * sph : T(0));
      acc[0].add(bv[c], frob_t(c, bv[c]));
    }
  } else {
#pragma unroll
    for (int c = 0; c < 6; ++c) qq[c * V] = qv[c];
  }
}

// Partial sums of the inverse pass of one item into row `row` of P.part.
template <typename T, int MODE>
__device__ __forceinline__ void inv_partials(const KParams<T>& P, long long row, const DotAcc<T> (&dot)[3],
                                             double* red) {
  double acc[3] = {dot[0].value(), dot[1].value(), dot[2].value()};
  if (MODE == MODE_ITER) {
    block_reduce<3>(acc, red);
    if (threadIdx.x == 0) {
      double* pt = P.part + row * 16;
      pt[12] = acc[0];
      pt[14] = acc[1];
      pt[15] = acc[2];
    }
  } else if ((MODE != MODE_APPLY && MODE != MODE_BASIC) || (MODE == MODE_BASIC && P.em)) {
    double a1[1] = {acc[0]};
    block_reduce<1>(a1, red);
    if (threadIdx.x == 0) P.part[row * 16 + 12] = a1[0];
  }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256, kFieldBlocksPerSM) k_plane_inv(KParams<T> P) {
  extern __shared__ __align__(16) char smem[];
  int tab_px = -1, tab_py = -1;  // plans whose tables are in shared memory
  for (int it = blockIdx.x; it < P.nitems; it += gridDim.x) {
    const int2 w = P.items[it];
    if (skip_problem<T>(P.st, w.x, MODE)) continue;
    const Prob d = P.prob[w.x];
    const int z = w.y;
    const int nx = d.nx, ny = d.ny, nxh = d.nxh;
    const int RP = pair_pitch(nx);
    const long long V = (long long)nx * ny * d.nz;
    PlaneSmem<T> sm = plane_layout<T>(smem, nx, ny, P.nphase);
    const AxisPlan& ax = P.plans[d.px];  // by reference: no per-thread copy
    const AxisPlan& ay = P.plans[d.py];  // by reference: no per-thread copy
    if (d.px != tab_px || d.py != tab_py) {
      plane_tables<T>(P, sm, ax, ay, nx);
      tab_px = d.px;
      tab_py = d.py;
    }
    const C2<T>* sp = P.spec + d.spc_off;
    const int pl = ny * nxh;
    const long long zpl = (long long)z * pl, cpl = (long long)d.nz * pl;
    {
      // e = (c * ny + ky) * nxh + kx
      Walk3 wk(threadIdx.x, blockDim.x, nxh, ny);
      for (int e = threadIdx.x; e < 6 * pl; e += blockDim.x, wk.next()) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(sm.S + plane_spec_at(wk.a, wk.b, wk.lo, ny, nxh, RP));
        const C2<T>* g = sp + wk.a * cpl + zpl + wk.b * nxh + wk.lo;
        if constexpr (sizeof(C2<T>) == 8)
          asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(g) : "memory");
        else
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(g) : "memory");
      }
    }
    copy_async_wait();
    __syncthreads();
    fft_lines<T, true>(sm.S, plane_cols(ny, nxh, RP), ay, sm.twy);
    pack_rows<T>(sm.S, 3 * ny, RP, nx, nxh, sm.pfx);
    fft_lines<T, true>(sm.S, plane_rows(ny, RP), ax, sm.twx);

    DotAcc<T> acc[3];
    const T invV = T(1) / T(V);
    const long long zoff = (long long)z * ny * nx;
    Walk2 wv(threadIdx.x, blockDim.x, nx);
    for (int v = threadIdx.x; v < ny * nx; v += blockDim.x, wv.next()) {
      const int y = wv.hi;
      const int x = wv.lo;
      T qv[6];
#pragma unroll
      for (int c2 = 0; c2 < 3; ++c2) {
        const C2<T> zz = sm.S[(c2 * ny + y) * RP + x];
        qv[2 * c2] = zz.x * invV;
        qv[2 * c2 + 1] = zz.y * invV;
      }
      inv_voxel<T, MODE>(P, d, V, zoff + v, qv, sm.lm, acc);
    }
    inv_partials<T, MODE>(P, d.part0 + z, acc, sm.red);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Row-streaming inverse pass: rows y0 .. y0 + nr of plane z after the
// inverse y transform (k_ycols), complex-to-real x transform, voxel phase.
// ---------------------------------------------------------------------------
template <typename T, int MODE>
__global__ void __launch_bounds__(256, kFieldBlocksPerSM) k_rows_inv(KParams<T> P) {
  extern __shared__ __align__(16) char smem[];
  for (int it = blockIdx.x; it < P.nitems; it += gridDim.x) {
    const int2 w = P.items[it];
    if (skip_problem<T>(P.st, w.x, MODE)) continue;
    const Prob d = P.prob[w.x];
    const int z = w.y & 0xffff, y0 = w.y >> 16;
    const int nx = d.nx, ny = d.ny, nxh = d.nxh, R = d.rows;
    const int nr = min(R, ny - y0);
    const int RP = pair_pitch(nx);
    const long long V = (long long)nx * ny * d.nz;
    PlaneSmem<T> sm = plane_layout<T>(smem, nx, R, P.nphase);
    const AxisPlan& ax = P.plans[d.px];  // by reference: no per-thread copy
    plane_tables<T>(P, sm, ax, ax, nx, false);
    const C2<T>* sp = P.spec + d.spc_off;
    const int rl = nr * nxh;
    for (int e = threadIdx.x; e < 6 * rl; e += blockDim.x) {
      const int c = e / rl;
      const int rem = e - c * rl;
      const int yy = rem / nxh;
      sm.S[plane_spec_at(c, yy, rem - yy * nxh, R, nxh, RP)] = sp[(((long long)c * d.nz + z) * ny + y0) * nxh + rem];
    }
    __syncthreads();
    pack_rows<T>(sm.S, 3 * R, RP, nx, nxh, sm.pfx);
    fft_lines<T, true>(sm.S, Lines{3 * nr, nr, R * RP, RP, 1, false}, ax, sm.twx);

    DotAcc<T> acc[3];
    const T invV = T(1) / T(V);
    const long long off0 = ((long long)z * ny + y0) * nx;
    for (int v = threadIdx.x; v < nr * nx; v += blockDim.x) {
      const int yy = v / nx;
      const int x = v - yy * nx;
      T qv[6];
#pragma unroll
      for (int c2 = 0; c2 < 3; ++c2) {
        const C2<T> zz = sm.S[(c2 * R + yy) * RP + x];
        qv[2 * c2] = zz.x * invV;
        qv[2 * c2 + 1] = zz.y * invV;
      }
      inv_voxel<T, MODE>(P, d, V, off0 + v, qv, sm.lm, acc);
    }
    const int nch = (ny + R - 1) / R;
    inv_partials<T, MODE>(P, d.part0 + z * nch + y0 / R, acc, sm.red);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Deferred CG update of the problems that have one pending (before the true
// residual, the averages, or a restart): r <- r - alpha q, x <- x + alpha p.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_flush(KParams<T> P) {
  for (int it = blockIdx.x; it < P.nitems; it += gridDim.x) {
    const int2 w = P.items[it];
    if (!P.st[w.x].pending) continue;
    const Prob d = P.prob[w.x];
    const int z = w.y;
    const long long V = (long long)d.nx * d.ny * d.nz;
    const int pl = d.nx * d.ny;
    const T alpha = T(P.st[w.x].alpha);
    const long long o0 = d.fld_off + (long long)z * pl;
    T* rr = P.r + o0;
    T* xx = P.x + o0;
    const T* qq = P.q + o0;
    const T* pp = P.p + o0;
    for (int c = 0; c < 6; ++c)
      for (int e = threadIdx.x; e < pl; e += blockDim.x) {
        const long long o = c * V + e;
        rr[o] = rr[o] - alpha * qq[o];
        xx[o] = xx[o] + alpha * pp[o];
      }
  }
}

// ---------------------------------------------------------------------------
// Core sums of eps* and of C:(E + eps*) on one plane (final averages).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_avg(KParams<T> P) {
  __shared__ double red[32 * kAvgParts];
  __shared__ T lm[512];
  if (P.medium == MED_ISO)
    for (int t = threadIdx.x; t < 2 * P.nphase; t += blockDim.x) lm[t] = P.lammu[t];
  __syncthreads();
  for (int it = blockIdx.x; it < P.nitems; it += gridDim.x) {
    const int2 w = P.items[it];
    const Prob d = P.prob[w.x];
    const int z = w.y;
    const long long V = (long long)d.nx * d.ny * d.nz;
    double acc[kAvgParts];
#pragma unroll
    for (int k = 0; k < kAvgParts; ++k) acc[k] = 0.0;
    if (z >= d.c0z && z < d.c0z + d.cnz) {
      const T* xx = P.x + d.fld_off;
      const T Ed = d.lc < 3 ? T(1) : T(0.5);
      const int cells = d.cny * d.cnx;
      for (int v = threadIdx.x; v < cells; v += blockDim.x) {
        const int y = d.c0y + v / d.cnx;
        const int x = d.c0x + v % d.cnx;
        const long long vo = ((long long)z * d.ny + y) * d.nx + x;
        T e[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          e[c] = xx[c * V + vo];
          acc[c] += double(e[c]);
        }
        e[d.lc] += Ed;
        T s[6];
        if (P.medium == MED_ISO) {
          const int lab = P.labels[d.med_off + vo];
          stress_iso<T>(e, lm[2 * lab], lm[2 * lab + 1], s);
        } else {
          stress_aniso<T>(e, P.c21 + d.med_off, V, vo, s);
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[6 + c] += double(s[c]);
      }
    }
    block_reduce<kAvgParts>(acc, red);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < kAvgParts; ++k) P.part[(long long)(d.plane0 + z) * 16 + k] = acc[k];
    }
  }
}

// The scalar kernels below are plain (non-template) kernels: defined only in
// the unit that launches them (units that include this header for the
// compiled-shape kernels alone define HH_FIELD_TEMPLATES_ONLY).
#ifndef HH_FIELD_TEMPLATES_ONLY
// ---------------------------------------------------------------------------
// FP64 scalar steps of conjugate gradients, one thread per problem. Partials
// of a problem's plane items are summed in item order (deterministic).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double sum_parts(const double* part, const Prob& d, int slot) {
  double a = 0.0;
  for (int i = 0; i < d.npi; ++i) a += part[(long long)(d.part0 + i) * 16 + slot];
  return a;
}

__global__ void k_scal_init(const Prob* prob, PState* st, const double* part, int nprob, double floor2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nprob || prob[i].fused) return;
  const Prob d = prob[i];
  PState s;
  const double tt = sum_parts(part, d, 0);
  const double rho = sum_parts(part, d, 12);
  s.rho = rho;
  s.rho0 = rho;
  s.rho_prev = rho;
  s.alpha = 0.0;
  s.beta = 0.0;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    s.xbar[c] = 0.0;
    s.sbar[c] = 0.0;
  }
  s.iters = 0;
  s.status = ST_OK;
  s.resid = 0.0;
  s.active = 1;
  s.trueflag = 0;
  s.homog = 0;
  s.restarts = 0;
  s.stall = 0;
  s.pending = 0;
  s.rt_best = rho;
  if (!isfinite(rho) || !isfinite(tt)) {
    s.active = 0;
    s.status = ST_NONFINITE;
  } else if (rho <= floor2 * tt) {
    s.active = 0;  // right-hand side zero to working precision: eps* = 0
    s.homog = 1;
  }
  st[i] = s;
}

// One CG step after the inverse plane pass of iteration k. The plane passes
// left <r_k, r_k> (slot 13, from the r that the forward pass formed), <p, q>,
// <r, q> and <q, q> (slots 12, 14, 15). Then
//   alpha = <r, r> / <p, q>,
//   <r', r'> = <r, r> - 2 alpha <r, q> + alpha^2 <q, q>   (r' = r - alpha q),
//   beta = <r', r'> / <r, r>,
// and the vector updates r', x + alpha p are deferred to the next forward
// plane pass (pending = 1). <r, r> comes from the stored r every iteration,
// so the expansion does not accumulate rounding across iterations.
__global__ void k_scal_step(const Prob* prob, PState* st, const double* part, int nprob, double tol,
                            int max_iter, int fixed_iters) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nprob || !st[i].active) return;
  const Prob d = prob[i];
  PState& s = st[i];
  s.pending = 0;  // the forward pass of this iteration applied the previous update
  const double rr = sum_parts(part, d, 13);
  const double pq = sum_parts(part, d, 12);
  const double rq = sum_parts(part, d, 14);
  const double qq = sum_parts(part, d, 15);
  if (!isfinite(rr) || !isfinite(pq) || !isfinite(rq) || !isfinite(qq)) {
    s.active = 0;
    s.status = ST_NONFINITE;
    return;
  }
  if (!(pq > 0.0)) {
    // <p, A p> lost positivity to rounding: the recursion has stalled; the
    // true-residual check decides convergence.
    s.active = 0;
    return;
  }
  const double alpha = rr / pq;
  double rn = rr - 2.0 * alpha * rq + alpha * alpha * qq;
  if (rn < 0.0) rn = 0.0;
  s.alpha = alpha;
  s.pending = 1;
  s.iters += 1;
  const bool conv = fixed_iters > 0 ? (s.iters >= fixed_iters) : (sqrt(rn) <= tol * sqrt(s.rho0));
  s.rho_prev = rr;
  s.rho = rn;
  if (conv || rn == 0.0 || s.iters >= max_iter) {
    s.active = 0;
    if (!conv && rn != 0.0) s.status = ST_NOT_CONVERGED;
    return;
  }
  s.beta = rn / rr;
}

// Basic scheme: fresh state, x = eps - E = 0 (set by the host).
__global__ void k_scal_basic_init(PState* st, int nprob) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nprob) return;
  PState s;
  memset(&s, 0, sizeof(s));
  s.rho0 = 1.0;
  s.active = 1;
  st[i] = s;
}

// Basic scheme, after the column pass of iteration k: the equilibrium
// residual ||G*sigma|| / ||<sigma>|| (Frobenius norms over the box; by
// Parseval sum h |P sigma^|^2 / sum_c w_c (Re sigma^_c(0))^2) of the current
// strain decides; otherwise the update x <- x - Gamma0 * sigma that the
// inverse pass stored in q is applied by the next forward pass.
//
// Accelerated scheme (em = 1): the inverse pass of iteration k has applied
// its update and left the partials of ||B^k||^2_F (slot 12); the residual
// ||B^k|| / ||E|| (||E||^2 = V w_lc E_lc^2 for the unit load) decides
// whether that iteration was the last. Nothing is left pending.
__global__ void k_scal_basic(const Prob* prob, PState* st, const double* cpart, const double* part, int nprob,
                             double tol, int max_iter, int fixed_iters, int em) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nprob || !st[i].active) return;
  const Prob d = prob[i];
  PState& s = st[i];
  s.pending = 0;
  if (em) {
    const double Ed = d.lc < 3 ? 1.0 : 0.5;
    const double nE2 = (double)d.nx * d.ny * d.nz * frob_w(d.lc) * Ed * Ed;
    const double res = sqrt(sum_parts(part, d, 12) / nE2);
    if (!isfinite(res)) {
      s.active = 0;
      s.status = ST_NONFINITE;
      return;
    }
    s.resid = res;
    s.iters += 1;
    const bool stop = fixed_iters > 0 ? (s.iters >= fixed_iters) : (res <= tol);
    if (stop || s.iters >= max_iter) {
      s.active = 0;
      if (!stop) s.status = ST_NOT_CONVERGED;
    }
    return;
  }
  const int n = (d.ny * d.nxh + d.cw - 1) / d.cw;
  double eq = 0.0, m[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int j = 0; j < n; ++j) {
    const double* cp = cpart + (long long)(d.col0 + j) * 8;
    eq += cp[0];
#pragma unroll
    for (int c = 0; c < 6; ++c) m[c] += cp[1 + c];
  }
  double den = 0.0;
#pragma unroll
  for (int c = 0; c < 6; ++c) den += frob_w(c) * m[c] * m[c];
  const double res = den > 0.0 ? sqrt(eq / den) : 0.0;
  if (!isfinite(res)) {
    s.active = 0;
    s.status = ST_NONFINITE;
    return;
  }
  s.resid = res;
  const bool stop = fixed_iters > 0 ? (s.iters >= fixed_iters) : (res <= tol);
  if (stop || s.iters >= max_iter) {
    s.active = 0;
    if (!stop) s.status = ST_NOT_CONVERGED;
    return;
  }
  s.iters += 1;
  s.pending = 1;
}

// After k_flush: no update is pending any more.
__global__ void k_scal_clear(PState* st, int nprob) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nprob) st[i].pending = 0;
}

// which = 0: flag the active problems (residual replacement);
// which = 1: flag every problem that iterated and is finite (final check).
__global__ void k_mark_true(const Prob* prob, PState* st, int nprob, int which) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nprob || prob[i].fused) return;
  PState& s = st[i];
  s.trueflag = which == 0 ? s.active : ((!s.homog && s.status != ST_NONFINITE) ? 1 : 0);
}

// Residual replacement: r was overwritten by the true residual; restart the
// beta recursion from it (p keeps its direction). Checkpoint safeguards for
// the precision floor: stop when the true residual has grown tenfold (in
// norm) over the best seen, or has not improved for 8 checkpoints.
__global__ void k_scal_replace(const Prob* prob, PState* st, const double* part, int nprob, double tol,
                               int fixed_iters) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nprob || !st[i].trueflag) return;
  PState& s = st[i];
  s.trueflag = 0;
  const double rr = sum_parts(part, prob[i], 12);
  if (!isfinite(rr)) {
    s.active = 0;
    s.status = ST_NONFINITE;
    return;
  }
  s.beta = (s.rho_prev > 0.0) ? rr / s.rho_prev : 0.0;
  s.rho = rr;
  if (fixed_iters > 0) return;
  if (sqrt(rr) <= tol * sqrt(s.rho0)) {
    s.active = 0;
    return;
  }
  if (rr > 100.0 * s.rt_best) {
    s.active = 0;
    s.status = ST_NOT_CONVERGED;
    return;
  }
  if (rr < s.rt_best) {
    s.rt_best = rr;
    s.stall = 0;
  } else if (++s.stall >= 8) {
    s.active = 0;
    s.status = ST_NOT_CONVERGED;
  }
}

// Final check on the true residual; problems above `slack * tol` restart
// (at most max_restarts times) with r = b - A x and p = r, unless the
// checkpoint safeguards already stopped them.
__global__ void k_scal_true_final(const Prob* prob, PState* st, const double* part, int nprob, double tol,
                                  double slack, int max_restarts, int max_iter, int fixed_iters) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nprob || !st[i].trueflag) return;
  PState& s = st[i];
  s.trueflag = 0;
  const double rr = sum_parts(part, prob[i], 12);
  if (!isfinite(rr)) {
    s.status = ST_NONFINITE;
    return;
  }
  s.resid = (s.rho0 > 0.0) ? sqrt(rr / s.rho0) : 0.0;
  if (fixed_iters > 0) return;
  if (s.resid > slack * tol) {
    const bool improving = rr < s.rt_best;
    if (rr < s.rt_best) s.rt_best = rr;
    if (s.status == ST_OK && s.iters < max_iter && s.restarts < max_restarts && improving) {
      s.active = 1;
      s.restarts += 1;
      s.stall = 0;
      s.rho = rr;
      s.rho_prev = rr;
      s.beta = 0.0;  // p <- r on the next plane pass
    } else {
      s.status = ST_NOT_CONVERGED;
    }
  }
}

__global__ void k_scal_avg(const Prob* prob, PState* st, const double* part, int nprob) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nprob || prob[i].fused) return;
  const Prob d = prob[i];
  PState& s = st[i];
  // k_avg leaves one row of partials per (problem, z) item
  for (int c = 0; c < 6; ++c) {
    double a = 0.0, b = 0.0;
    for (int z = 0; z < d.nz; ++z) {
      a += part[(long long)(d.plane0 + z) * 16 + c];
      b += part[(long long)(d.plane0 + z) * 16 + 6 + c];
    }
    s.xbar[c] = a;
    s.sbar[c] = b;
  }
}

// Number of active problems and, over them, the real-field voxels and the
// half-spectrum elements (6 nz ny nxh) one iteration touches.
__global__ void k_count_active(const PState* st, const Prob* prob, int nprob, int* out_n,
                               unsigned long long* out_vs) {
  __shared__ int cnt;
  __shared__ unsigned long long sv, ss;
  if (threadIdx.x == 0) {
    cnt = 0;
    sv = 0;
    ss = 0;
  }
  __syncthreads();
  int c = 0;
  unsigned long long v = 0, sp = 0;
  for (int i = threadIdx.x; i < nprob; i += blockDim.x)
    if (st[i].active) {
      const Prob& d = prob[i];
      ++c;
      v += (unsigned long long)d.nx * d.ny * d.nz;
      sp += 6ull * d.nz * d.ny * d.nxh;
    }
  atomicAdd(&cnt, c);
  atomicAdd(&sv, v);
  atomicAdd(&ss, sp);
  __syncthreads();
  if (threadIdx.x == 0) {
    *out_n = cnt;
    out_vs[0] = sv;
    out_vs[1] = ss;
  }
}

#endif  // HH_FIELD_TEMPLATES_ONLY

}  // namespace hh

#include "hh_plane_ct.cuh"
