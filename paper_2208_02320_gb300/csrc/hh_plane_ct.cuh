// Field-pass bodies compiled for one shape each: the plane passes of xy
// planes whose edges are even in 16..48 and differ by 0, 8 or 16, and the
// column pass of z lines of even length 16..48 - the buffered boxes of cores
// with edges 16, 24 or 32 and one buffer width b = 0..8 (edge = core + 2 b),
// which carry the work of uneven partitions on an 8-voxel coarse unit.
//
// The arithmetic is the generic passes' (the same two-pass transforms of
// hh_fft2.cuh with the same splits, twiddles and operation order, the same
// voxel functions, the same shared-memory layout), so a problem may take
// either path; what changes is the bookkeeping:
//   * every length, stride, pitch and trip count is a compile-time constant,
//     so index division becomes multiply-shift and loops unroll;
//   * the transforms are inlined (no call into the separately compiled
//     transform table, no callee-saved register traffic);
//   * the first pass of a two-pass transform reads and writes the same
//     positions in every thread ({t1 + N1 j : j < N2}), so it needs no barrier
//     of its own; the second pass stages all lines of a round before its
//     barrier and writes them after it;
//   * the inverse x transform reads the packed row Z = A + iB straight from
//     the two half spectra [A | B] (Hermitian extension), without a separate
//     packing step;
//   * they run as kernels of their own (k_plane_fwd_ct, k_plane_inv_ct,
//     k_column_ct) with one block per item, on launch classes that hold only
//     problems with a compiled shape (the CG iterations in FP32; the other
//     modes take the generic kernels on the same items).
// Blocks have kNT = 256 threads (the launch shape of the field kernels).
#pragma once

namespace hh {
namespace ct {

constexpr int kNT = 256;

__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int cdiv(int a, int b) { return (a + b - 1) / b; }

// N1 of the two-pass plan of length n (the table of hh_fft2.cuh), 0 if none.
__host__ __device__ constexpr int split_of(int n) {
#define HH_CT_SPLIT(N, A, B) \
  if (n == N) return A;
  HH_FFT2_TABLE(HH_CT_SPLIT)
#undef HH_CT_SPLIT
  return 0;
}

// Complex values a thread stages at once in one pass (registers), and the
// voxels of a thread whose global loads are issued together in the voxel
// phases.
#ifndef HH_CT_STAGE
#define HH_CT_STAGE 4
#endif
#ifndef HH_CT_VOXELS
#define HH_CT_VOXELS 1
#endif
constexpr int kStage = HH_CT_STAGE;
constexpr int kVoxels = HH_CT_VOXELS;

}  // namespace ct

// Resident 256-thread blocks per SM the compiled-shape kernels are built for:
// the inverse plane and column passes at 5 (48 registers per thread; 40 warps
// per SM to hide their load latency, measured faster than 4 blocks with 64
// registers), the forward plane pass at 4 (64 registers: its voxel phase
// holds four fields per voxel).
#ifndef HH_CT_BLOCKS_PER_SM
#define HH_CT_BLOCKS_PER_SM 5
#endif
#ifndef HH_CT_FWD_BLOCKS_PER_SM
#define HH_CT_FWD_BLOCKS_PER_SM 4
#endif
constexpr int kCtBlocksPerSM = HH_CT_BLOCKS_PER_SM;
constexpr int kCtFwdBlocksPerSM = HH_CT_FWD_BLOCKS_PER_SM;

namespace ct {

// NL lines; line l starts at (l / LPG) GS + (l % LPG) LS, element k of it
// sits ES further on per k.
template <int NL_, int LPG_, int GS_, int LS_, int ES_>
struct Geo {
  static constexpr int NL = NL_, LPG = LPG_, GS = GS_, LS = LS_, ES = ES_;
  static __device__ __forceinline__ int off(unsigned l) {
    if constexpr (LPG >= NL)
      return (int)(l * LS);
    else
      return (int)((l / LPG) * GS + (l % LPG) * LS);
  }
};

// The thread index, read so that the compiler cannot treat it as invariant:
// the indices a body derives from it are recomputed where they are used
// instead of being hoisted out of the round and chunk loops and held in
// registers (or spilled) for the whole body. (With a persistent item loop
// around the bodies such hoisting cost 2-4 KB of spill code per kernel.)
__device__ __forceinline__ unsigned tid_item() {
  unsigned t;
  asm volatile("mov.u32 %0, %%tid.x;" : "=r"(t));
  return t;
}

template <typename T>
__device__ __forceinline__ void cp_async_elem(C2<T>* dst_smem, const C2<T>* src) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(dst_smem);
  if constexpr (sizeof(C2<T>) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}

// First pass of the two-pass transform, for every (line, t1): the N2-point
// DFT of x[t1 + N1 m], the twiddle W_N^(t1 k2), stored at k2 N1 + t1. A
// thread writes only the positions it read, so no barrier is needed inside;
// adjacent threads take adjacent lines. (Loops with compile-time trip counts
// are unrolled, so the staged arrays stay in registers.)
template <typename T, int N1, int N2, bool INV, class G>
__device__ __forceinline__ void pass1_local(C2<T>* S, const C2<T>* tw) {
  constexpr int TOT = G::NL * N1;
  constexpr int IT = cdiv(TOT, kNT);
  constexpr int B = cmax(1, kStage / N2);
  const unsigned tid = tid_item();
  // one chunk of B pairs per trip (the code of one chunk, not of all)
#pragma unroll 1
  for (int i0 = 0; i0 < IT; i0 += B) {
    C2<T> v[B][N2];
    int o[B], t1s[B];
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const int i = i0 + j;
      const unsigned p = tid + i * kNT;
      o[j] = -1;
      if (i < IT && ((i + 1) * kNT <= TOT || p < TOT)) {
        const unsigned line = p % G::NL, t1 = p / G::NL;
        o[j] = G::off(line) + (int)t1 * G::ES;
        t1s[j] = (int)t1;
#pragma unroll
        for (int m = 0; m < N2; ++m) v[j][m] = S[o[j] + m * N1 * G::ES];
      }
    }
#pragma unroll
    for (int j = 0; j < B; ++j) {
      if (o[j] >= 0) {
        dft_reg<T, N2, INV>(v[j]);
#pragma unroll
        for (int k2 = 1; k2 < N2; ++k2) {
          const C2<T> w = tw[t1s[j] * k2];
          v[j][k2] = INV ? cmulc(v[j][k2], w) : cmul(v[j][k2], w);
        }
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) S[o[j] + k2 * N1 * G::ES] = v[j][k2];
      }
    }
  }
}

enum : int { KIND_P2 = 0, KIND_P1_PACKED = 1 };

// A pass that moves values between positions of a line, in rounds of whole
// lines: every pair of a round is read and transformed, then (after a
// barrier) written; different rounds touch different lines. Ends with a
// barrier.
//   KIND_P2       : second pass, pair (line, k2): the N1-point DFT of the
//                   first pass's results at k2 N1 + t1, stored at k2 + N2 k1
//                   (natural order).
//   KIND_P1_PACKED: first pass of an inverse row transform whose row holds the
//                   half spectra [A | B] (A at 0..NXH-1, B at NXH..2 NXH-1) of
//                   two real rows: element n of the packed row is
//                   Z[n] = A[n] + i B[n], with A[n] = conj(A[N - n]) (same for
//                   B) for n >= NXH.
template <typename T, int N1, int N2, bool INV, class G, int KIND, int NXH = 0>
__device__ __forceinline__ void pass_rounds(C2<T>* S, const C2<T>* tw) {
  constexpr int N = N1 * N2;
  constexpr int J = KIND == KIND_P2 ? N2 : N1;     // pairs per line
  constexpr int R = KIND == KIND_P2 ? N1 : N2;     // values per pair
  constexpr int STEP = KIND == KIND_P2 ? N2 : N1;  // output stride in a line
  constexpr int PMAX = cmax(1, kStage / R);
  constexpr int LPR0 = cmax(1, PMAX * kNT / J);
  constexpr int NR = cdiv(G::NL, LPR0);
  constexpr int LPR = cdiv(G::NL, NR);
  constexpr int IT = cdiv(LPR * J, kNT);
  constexpr int TOT = LPR * J;  // pairs of a round (the last may have fewer lines)
  static_assert(KIND == KIND_P2 || G::ES == 1, "packed rows are contiguous");
  const unsigned tid = tid_item();
  // every round runs the same code (LPR lines, the last round's missing lines
  // skipped), so the loop is not unrolled and its constants stay constants
#pragma unroll 1
  for (int r = 0; r < NR; ++r) {
    const unsigned L0 = r * LPR;
    C2<T> v[IT][R];
    int o[IT];
#pragma unroll
    for (int i = 0; i < IT; ++i) {
      const unsigned p = tid + i * kNT;
      const unsigned line = L0 + p % LPR, jj = p / LPR;
      o[i] = -1;
      if (((i + 1) * kNT <= TOT || p < (unsigned)TOT) && (NR * LPR == G::NL || line < (unsigned)G::NL)) {
        const int lo = G::off(line);
        if constexpr (KIND == KIND_P2) {
#pragma unroll
          for (int t1 = 0; t1 < N1; ++t1) v[i][t1] = S[lo + ((int)jj * N1 + t1) * G::ES];
          dft_reg<T, N1, INV>(v[i]);
          o[i] = lo + (int)jj * G::ES;
        } else {
#pragma unroll
          for (int m = 0; m < N2; ++m) {
            const int n = (int)jj + N1 * m;
            const bool low = n < NXH;
            const int ia = low ? n : N - n;
            C2<T> A = S[lo + ia], B = S[lo + NXH + ia];
            if (!low) {
              A.y = -A.y;
              B.y = -B.y;
            }
            v[i][m] = mk<T>(A.x - B.y, A.y + B.x);
          }
          dft_reg<T, N2, INV>(v[i]);
#pragma unroll
          for (int k2 = 1; k2 < N2; ++k2) {
            const C2<T> w = tw[(int)jj * k2];
            v[i][k2] = INV ? cmulc(v[i][k2], w) : cmul(v[i][k2], w);
          }
          o[i] = lo + (int)jj;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IT; ++i)
      if (o[i] >= 0) {
#pragma unroll
        for (int k = 0; k < R; ++k) S[o[i] + k * STEP * G::ES] = v[i][k];
      }
  }
  __syncthreads();
}

// Whole transform of natural-order lines (caller has synchronized the block
// since the lines were written; ends with a barrier).
template <typename T, int N, bool INV, class G>
__device__ __forceinline__ void fft_ct(C2<T>* S, const C2<T>* tw) {
  constexpr int N1 = split_of(N), N2 = N / N1;
  static_assert(N1 > 0, "length without a two-pass plan");
  if constexpr (N2 > 1) {
    pass1_local<T, N1, N2, INV, G>(S, tw);
    __syncthreads();
  }
  pass_rounds<T, N1, N2, INV, G, KIND_P2>(S, tw);
}

// Inverse transform of rows held as half spectra [A | B]: the results are the
// packed real rows a + i b at natural positions 0..N-1.
template <typename T, int N, class G>
__device__ __forceinline__ void fft_inv_packed_ct(C2<T>* S, const C2<T>* tw) {
  constexpr int N1 = split_of(N), N2 = N / N1;
  static_assert(N1 > 0 && N2 > 1, "packed rows need a two-pass length");
  pass_rounds<T, N1, N2, true, G, KIND_P1_PACKED, N / 2 + 1>(S, tw);
  pass_rounds<T, N1, N2, true, G, KIND_P2>(S, tw);
}

// Split each transformed packed row Z = A + iB into [A | B] in place (the
// generic passes' unpack_rows for natural order), in rounds of whole rows.
template <typename T, int NX, int NROWS, int RP>
__device__ __forceinline__ void unpack_ct(C2<T>* S) {
  constexpr int NXH = NX / 2 + 1;
  constexpr int EMAX = cmax(1, kStage / 2);
  constexpr int RPR0 = cmax(1, EMAX * kNT / NXH);
  constexpr int NR = cdiv(NROWS, RPR0);
  constexpr int RPR = cdiv(NROWS, NR);
  constexpr int IT = cdiv(RPR * NXH, kNT);
  constexpr int TOT = RPR * NXH;
  const unsigned tid = tid_item();
#pragma unroll 1
  for (int r = 0; r < NR; ++r) {
    const unsigned R0 = r * RPR;
    C2<T> A[IT], B[IT];
    int o[IT];
#pragma unroll
    for (int i = 0; i < IT; ++i) {
      const unsigned e = tid + i * kNT;
      const unsigned row = R0 + e / NXH, k = e % NXH;
      o[i] = -1;
      if (((i + 1) * kNT <= TOT || e < (unsigned)TOT) && (NR * RPR == NROWS || row < (unsigned)NROWS)) {
        const int base = (int)row * RP;
        const C2<T> a = S[base + (int)k];
        const C2<T> b = S[base + (k == 0 ? 0 : NX - (int)k)];
        A[i] = mk<T>(T(0.5) * (a.x + b.x), T(0.5) * (a.y - b.y));
        B[i] = mk<T>(T(0.5) * (a.y + b.y), T(-0.5) * (a.x - b.x));
        o[i] = base + (int)k;
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IT; ++i)
      if (o[i] >= 0) {
        S[o[i]] = A[i];
        S[o[i] + NXH] = B[i];
      }
  }
  __syncthreads();
}

// Forward plane pass of plane z of problem d with an NX x NY plane (the body
// of k_plane_fwd after its tables and scalars are in place).
template <typename T, int MODE, int NX, int NY>
__device__ __forceinline__ void plane_fwd(const KParams<T>& P, const Prob& d, int z, const PlaneSmem<T>& sm,
                                          const FwdScal<T, MODE>& k) {
  constexpr int NXH = NX / 2 + 1, RP = (NX + 2) | 1, PL = NY * NXH, NV = NX * NY;
  const unsigned tid = tid_item();
  const long long V = (long long)NV * d.nz;
  const long long zoff = (long long)z * NV;
  DotAcc<T> dot;
  constexpr int ITV = cdiv(NV, kNT);
#pragma unroll 1
  for (int i0 = 0; i0 < ITV; i0 += kVoxels)
#pragma unroll
  for (int i = i0; i < i0 + kVoxels; ++i) {
    const unsigned v = tid + i * kNT;
    if (i < ITV && ((i + 1) * kNT <= NV || v < NV)) {
      const int y = (int)(v / NX), x = (int)(v % NX);
      T s[6];
      fwd_voxel<T, MODE>(P, d, V, zoff + v, k, sm.lm, s, dot);
#pragma unroll
      for (int c2 = 0; c2 < 3; ++c2) sm.S[(c2 * NY + y) * RP + x] = mk<T>(s[2 * c2], s[2 * c2 + 1]);
    }
  }
  __syncthreads();
  fft_ct<T, NX, false, Geo<3 * NY, (1 << 30), 0, RP, 1>>(sm.S, sm.twx);
  unpack_ct<T, NX, 3 * NY, RP>(sm.S);
  fft_ct<T, NY, false, Geo<6 * NXH, 2 * NXH, NY * RP, 1, RP>>(sm.S, sm.twy);
  // spectrum of the plane: spec[c][z][ky][kx]
  C2<T>* sp = P.spec + d.spc_off + (long long)z * PL;
  const long long cpl = (long long)d.nz * PL;
  constexpr int ITS = cdiv(PL, kNT);
#pragma unroll 1
  for (int i = 0; i < ITS; ++i) {
    const unsigned e = tid + i * kNT;
    if ((i + 1) * kNT <= PL || e < PL) {
      const int ky = (int)(e / NXH), kx = (int)(e % NXH);
#pragma unroll
      for (int c = 0; c < 6; ++c) sp[c * cpl + e] = sm.S[((c >> 1) * NY + ky) * RP + (c & 1) * NXH + kx];
    }
  }
  if (fwd_slot<MODE>() >= 0) {
    double acc[1] = {dot.value()};
    block_reduce<1>(acc, sm.red);
    if (threadIdx.x == 0) P.part[(long long)(d.part0 + z) * 16 + fwd_slot<MODE>()] = acc[0];
  }
  __syncthreads();
}

// Inverse plane pass of plane z of problem d with an NX x NY plane.
template <typename T, int MODE, int NX, int NY>
__device__ __forceinline__ void plane_inv(const KParams<T>& P, const Prob& d, int z, const PlaneSmem<T>& sm) {
  constexpr int NXH = NX / 2 + 1, RP = (NX + 2) | 1, PL = NY * NXH, NV = NX * NY;
  const unsigned tid = tid_item();
  const long long cpl = (long long)d.nz * PL;
  {
    const C2<T>* sp = P.spec + d.spc_off + (long long)z * PL;
    constexpr int ITS = cdiv(PL, kNT);
#pragma unroll 1
    for (int i = 0; i < ITS; ++i) {
      const unsigned e = tid + i * kNT;
      if ((i + 1) * kNT <= PL || e < PL) {
        const int ky = (int)(e / NXH), kx = (int)(e % NXH);
#pragma unroll
        for (int c = 0; c < 6; ++c)
          cp_async_elem<T>(sm.S + ((c >> 1) * NY + ky) * RP + (c & 1) * NXH + kx, sp + c * cpl + e);
      }
    }
  }
  copy_async_wait();
  __syncthreads();
  fft_ct<T, NY, true, Geo<6 * NXH, 2 * NXH, NY * RP, 1, RP>>(sm.S, sm.twy);
  fft_inv_packed_ct<T, NX, Geo<3 * NY, (1 << 30), 0, RP, 1>>(sm.S, sm.twx);
  DotAcc<T> acc[3];
  const long long V = (long long)NV * d.nz;
  const T invV = T(1) / T(V);
  const long long zoff = (long long)z * NV;
  constexpr int ITV = cdiv(NV, kNT);
#pragma unroll 1
  for (int i0 = 0; i0 < ITV; i0 += kVoxels)
#pragma unroll
  for (int i = i0; i < i0 + kVoxels; ++i) {
    const unsigned v = tid + i * kNT;
    if (i < ITV && ((i + 1) * kNT <= NV || v < NV)) {
      const int y = (int)(v / NX), x = (int)(v % NX);
      T qv[6];
#pragma unroll
      for (int c2 = 0; c2 < 3; ++c2) {
        const C2<T> zz = sm.S[(c2 * NY + y) * RP + x];
        qv[2 * c2] = zz.x * invV;
        qv[2 * c2 + 1] = zz.y * invV;
      }
      inv_voxel<T, MODE>(P, d, V, zoff + v, qv, sm.lm, acc);
    }
  }
  inv_partials<T, MODE>(P, d.part0 + z, acc, sm.red);
  __syncthreads();
}

// Column pass of CW consecutive spectrum columns starting at j0 of problem d
// with z length NZ (the body of k_column for the projection): columns past
// the end of the plane are transformed but neither read nor written.
template <typename T, int NZ, int CW>
__device__ __forceinline__ void column(const KParams<T>& P, const Prob& d, int j0, const ColumnSmem<T>& sm) {
  static_assert(kNT % CW == 0, "a thread keeps one column");
  const int nx = d.nx, ny = d.ny, nxh = d.nxh;
  const int pl = ny * nxh;
  const int W = min(CW, pl - j0);
  const unsigned tid = tid_item();
  C2<T>* sp = P.spec + d.spc_off + j0;
  constexpr int TOT = 6 * NZ * CW;
  constexpr int ITL = cdiv(TOT, kNT);
  const int jl = (int)(tid % CW);  // the one column of every element this thread moves
  const unsigned cz0 = tid / CW;
  constexpr int DCZ = kNT / CW;
  if (jl < W) {
#pragma unroll 4
    for (int i = 0; i < ITL; ++i) {
      const unsigned cz = cz0 + i * DCZ;
      if ((i + 1) * kNT <= TOT || cz < 6 * NZ) cp_async_elem<T>(sm.tile + cz * CW + jl, sp + (long long)cz * pl + jl);
    }
  }
  copy_async_wait();
  __syncthreads();
  using GZ = Geo<6 * CW, CW, NZ * CW, 1, CW>;
  fft_ct<T, NZ, false, GZ>(sm.tile, sm.twz);
  {
    // modes e = kzp * CW + jl: this thread's column is jl for every e
    const int j = j0 + jl;
    const int kyp = j / nxh;
    const int kx = j - kyp * nxh;
    const int my = sm.sfy[min(kyp, ny - 1)];
    const bool nyq_x = (nx % 2 == 0) && (2 * kx == nx);
    const bool nyq_y = (ny % 2 == 0) && (2 * my == ny);
    const T x0c = (P.nyq_mode == 0 && nyq_x) ? T(0) : T(kx) / T(nx);
    const T x1c = (P.nyq_mode == 0 && nyq_y) ? T(0) : T(my) / T(ny);
    constexpr int NM = NZ * CW;
    constexpr int ITM = cdiv(NM, kNT);
#pragma unroll 1
    for (int i = 0; i < ITM; ++i) {
      const unsigned kzp = cz0 + i * DCZ;
      if ((i + 1) * kNT <= NM || kzp < NZ) {
        const int mz = sm.sfz[kzp];
        const bool nyq_z = (NZ % 2 == 0) && (2 * mz == NZ);
        T x0 = x0c, x1 = x1c, x2 = sm.fz[kzp];
        if (P.nyq_mode == 0) {
          if (nyq_z) x2 = T(0);
        } else if (nyq_x || nyq_y || nyq_z) {
          x0 = x1 = x2 = T(0);
        }
        C2<T> t[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) t[c] = sm.tile[(c * NZ + kzp) * CW + jl];
        project_mode<T>(t, x0, x1, x2);
#pragma unroll
        for (int c = 0; c < 6; ++c) sm.tile[(c * NZ + kzp) * CW + jl] = t[c];
      }
    }
  }
  __syncthreads();
  fft_ct<T, NZ, true, GZ>(sm.tile, sm.twz);
  if (jl < W) {
#pragma unroll 4
    for (int i = 0; i < ITL; ++i) {
      const unsigned cz = cz0 + i * DCZ;
      if ((i + 1) * kNT <= TOT || cz < 6 * NZ) sp[(long long)cz * pl + jl] = sm.tile[cz * CW + jl];
    }
  }
  __syncthreads();
}

}  // namespace ct

// Shape codes of the compiled bodies: nx * 64 + ny of the xy plane for the
// plane passes, nz * 64 + cw (z length and column width) for the column pass;
// 0 = none. The plane shapes are the buffered boxes of cores whose edges
// are 16, 24 or 32 (multiples of the coarse unit 8) with one buffer width:
// both edges even in 16..48, differing by 0, 8 or 16. They are compiled in
// four groups by nx, one kernel per group and pass, each built on its own.
__host__ __device__ constexpr int ct_plane_group(int nx, int ny) {
  const int d = nx > ny ? nx - ny : ny - nx;
  if (nx % 2 || ny % 2 || nx < 16 || ny < 16 || nx > 48 || ny > 48 || (d != 0 && d != 8 && d != 16)) return -1;
  return nx <= 22 ? 0 : (nx <= 30 ? 1 : (nx <= 38 ? 2 : 3));
}
constexpr int kCtPlaneGroups = 4;
__host__ __device__ constexpr bool ct_col_length(int n) { return n >= 16 && n <= 48 && n % 2 == 0; }

#define HH_CT_PLANES_0(X) X(16, 16) X(16, 24) X(16, 32) X(18, 18) X(18, 26) X(18, 34) X(20, 20) X(20, 28) \
  X(20, 36) X(22, 22) X(22, 30) X(22, 38)
#define HH_CT_PLANES_1(X) X(24, 16) X(24, 24) X(24, 32) X(24, 40) X(26, 18) X(26, 26) X(26, 34) X(26, 42) \
  X(28, 20) X(28, 28) X(28, 36) X(28, 44) X(30, 22) X(30, 30) X(30, 38) X(30, 46)
#define HH_CT_PLANES_2(X) X(32, 16) X(32, 24) X(32, 32) X(32, 40) X(32, 48) X(34, 18) X(34, 26) X(34, 34) \
  X(34, 42) X(36, 20) X(36, 28) X(36, 36) X(36, 44) X(38, 22) X(38, 30) X(38, 38) X(38, 46)
#define HH_CT_PLANES_3(X) X(40, 24) X(40, 32) X(40, 40) X(40, 48) X(42, 26) X(42, 34) X(42, 42) X(44, 28) \
  X(44, 36) X(44, 44) X(46, 30) X(46, 38) X(46, 46) X(48, 32) X(48, 40) X(48, 48)
#define HH_CT_COL_LENGTHS(X) X(16) X(18) X(20) X(22) X(24) X(26) X(28) X(30) X(32) X(34) X(36) X(38) X(40) \
  X(42) X(44) X(46) X(48)

// Kernels of the compiled bodies: one block per item of a launch class whose
// problems all carry a shape code of one group (the host keeps them apart
// from the generic passes' classes). No persistent loop: inside one, the
// compiler keeps the bodies' thread-dependent indices live across items,
// which costs more in registers and spills than reloading the few tables per
// block saves. The shared-memory layout is taken per shape, so its offsets
// are constants too.
namespace ct {
template <typename T, int NX, int NY>
__device__ __forceinline__ void fwd_item(const KParams<T>& P, int2 w, char* smem) {
  const Prob& d = P.prob[w.x];
  PlaneSmem<T> sm = plane_layout<T>(smem, NX, NY, P.nphase);
  plane_tables<T>(P, sm, P.plans[d.px], P.plans[d.py], NX);
  const FwdScal<T, MODE_ITER> k(P.st[w.x]);
  __syncthreads();
  plane_fwd<T, MODE_ITER, NX, NY>(P, d, w.y, sm, k);
}
template <typename T, int NX, int NY>
__device__ __forceinline__ void inv_item(const KParams<T>& P, int2 w, char* smem) {
  const Prob& d = P.prob[w.x];
  PlaneSmem<T> sm = plane_layout<T>(smem, NX, NY, P.nphase);
  plane_tables<T>(P, sm, P.plans[d.px], P.plans[d.py], NX);
  plane_inv<T, MODE_ITER, NX, NY>(P, d, w.y, sm);
}

#define HH_CT_FWD_CASE(NX, NY)                  \
  case NX * 64 + NY:                            \
    fwd_item<T, NX, NY>(P, w, smem);            \
    break;
#define HH_CT_INV_CASE(NX, NY)                  \
  case NX * 64 + NY:                            \
    inv_item<T, NX, NY>(P, w, smem);            \
    break;
template <typename T, int G, bool FWD>
__device__ __forceinline__ void plane_item(const KParams<T>& P, int2 w, char* smem) {
  const int code = P.prob[w.x].ct_plane;
  if constexpr (FWD) {
    if constexpr (G == 0) {
      switch (code) { HH_CT_PLANES_0(HH_CT_FWD_CASE) default: break; }
    } else if constexpr (G == 1) {
      switch (code) { HH_CT_PLANES_1(HH_CT_FWD_CASE) default: break; }
    } else if constexpr (G == 2) {
      switch (code) { HH_CT_PLANES_2(HH_CT_FWD_CASE) default: break; }
    } else {
      switch (code) { HH_CT_PLANES_3(HH_CT_FWD_CASE) default: break; }
    }
  } else {
    if constexpr (G == 0) {
      switch (code) { HH_CT_PLANES_0(HH_CT_INV_CASE) default: break; }
    } else if constexpr (G == 1) {
      switch (code) { HH_CT_PLANES_1(HH_CT_INV_CASE) default: break; }
    } else if constexpr (G == 2) {
      switch (code) { HH_CT_PLANES_2(HH_CT_INV_CASE) default: break; }
    } else {
      switch (code) { HH_CT_PLANES_3(HH_CT_INV_CASE) default: break; }
    }
  }
}
#undef HH_CT_FWD_CASE
#undef HH_CT_INV_CASE
}  // namespace ct

template <typename T, int G>
__global__ void __launch_bounds__(256, kCtFwdBlocksPerSM) k_plane_fwd_ct(KParams<T> P) {
  if constexpr (sizeof(T) == 4) {
    extern __shared__ __align__(16) char smem[];
    if ((int)blockIdx.x >= P.nitems) return;
    const int2 w = P.items[blockIdx.x];
    if (skip_problem<T>(P.st, w.x, MODE_ITER)) return;
    ct::plane_item<T, G, true>(P, w, smem);
  }
}

template <typename T, int G>
__global__ void __launch_bounds__(256, kCtBlocksPerSM) k_plane_inv_ct(KParams<T> P) {
  if constexpr (sizeof(T) == 4) {
    extern __shared__ __align__(16) char smem[];
    if ((int)blockIdx.x >= P.nitems) return;
    const int2 w = P.items[blockIdx.x];
    if (skip_problem<T>(P.st, w.x, MODE_ITER)) return;
    ct::plane_item<T, G, false>(P, w, smem);
  }
}

// Column widths of the compiled column pass.
__host__ __device__ constexpr bool ct_width(int cw) { return cw == 16 || cw == 32; }

// Column pass (projection) of the problems with a compiled z length; every
// mode but the basic scheme's (`skip_mode` as in k_column). One block per item.
namespace ct {
template <typename T, int NZ, int CW>
__device__ __forceinline__ void column_item(const KParams<T>& P, int2 w, char* smem) {
  const Prob& d = P.prob[w.x];
  const int ny = d.ny;
  ColumnSmem<T> sm = column_layout<T>(smem, CW, NZ, ny);
  const AxisPlan& az = P.plans[d.pz];
  const AxisPlan& ay = P.plans[d.py];
  load_tw<T>(sm.twz, P.tw, az);
  for (int t = threadIdx.x; t < NZ; t += kNT) {
    const int mz = P.itab[az.sf_off + t];
    sm.sfz[t] = mz;
    sm.fz[t] = T(mz) / T(NZ);
  }
  for (int t = threadIdx.x; t < ny; t += kNT) sm.sfy[t] = P.itab[ay.sf_off + t];
  column<T, NZ, CW>(P, d, w.y, sm);
}
}  // namespace ct

template <typename T>
__global__ void __launch_bounds__(256, kCtBlocksPerSM) k_column_ct(KParams<T> P, int skip_mode) {
  if constexpr (sizeof(T) == 4) {
    extern __shared__ __align__(16) char smem[];
    if ((int)blockIdx.x >= P.nitems) return;
    const int2 w = P.items[blockIdx.x];
    if (skip_problem<T>(P.st, w.x, skip_mode)) return;
    switch (P.prob[w.x].ct_col) {
#define HH_CT_COL(N)                          \
  case N * 64 + 16:                           \
    ct::column_item<T, N, 16>(P, w, smem);    \
    break;                                    \
  case N * 64 + 32:                           \
    ct::column_item<T, N, 32>(P, w, smem);    \
    break;
      HH_CT_COL_LENGTHS(HH_CT_COL)
#undef HH_CT_COL
      default:
        break;
    }
  }
}

}  // namespace hh
