// Fused on-chip subimage solver: the whole conjugate-gradient solve of one
// (subimage, load case) problem (Appendix A: G*(C:eps*) = -G*(C:E)) runs in
// one thread-block cluster, without returning to the host between
// iterations.
//
// Layout. The C blocks of a cluster split the buffered box Omega_B into
// slabs of consecutive z planes. A block keeps its slab of the six-component
// half spectrum in shared memory, as the plane passes do, one "pair row"
// block of ny rows per component pair and plane: the constitutive law and
// the x (real-to-complex) and y transforms run on the block's own planes;
// the z transform, the projection and the inverse z transform run on spectrum
// columns (ky, kx) that every block gathers from the whole cluster through
// distributed shared memory and scatters back; the inverse y and x transforms
// again run on the block's own planes. The spectrum never leaves the chip.
// After the inverse transforms the slab holds q = A p in real space, which
// stays there for the deferred update r <- r - alpha q, x <- x + alpha p of
// the next forward phase: per iteration only r, p, x (read and written once)
// and the labels go through global memory, plus p and r read again for
// <p, q> and <r, q>.
//
// Scalars. Every block reduces its partial sums (fixed-order warp and block
// trees, as the multi-pass solver does), the cluster's C partials are summed
// in block-rank order by every block, and every block applies the same FP64
// conjugate-gradient step to its own copy of the problem state, so all
// blocks take the same control decisions (same iteration count, same
// residual checks) and arrive at the same cluster barriers. The stopping
// rule, the residual replacement every `chunk` iterations, the stall and
// growth safeguards and the final true-residual check with bounded restarts
// are those of the multi-pass solver, step for step.
//
// Work. A persistent grid of clusters takes problems from a device counter
// (one atomic per problem, no waiting) in the order the host sorted them.
#pragma once

#include <cooperative_groups.h>

#include "hh_device.cuh"

namespace hh {

namespace cgr = cooperative_groups;

constexpr int kFusedThreads = 256;
constexpr int kFusedRed = 12;  // largest block reduction (the core averages)

template <typename T>
struct FusedParams {
  const Prob* prob;
  PState* st;
  const int* order;  // problem indices in the order clusters take them
  int nwork;
  int* queue;        // next entry of `order` (zeroed before the launch)
  const AxisPlan* plans;
  const double* tw;
  const int* itab;
  const uint8_t* labels;
  const T* lammu;
  int nphase;
  int nyq_mode;
  T* r;
  T* p;
  T* x;
  double tol, floor2;
  int max_iter, fixed_iters, chunk, replace, max_restarts;
  long long max_chunks;
};

// Spectrum columns per z-phase round: about 256 z lines of work per round.
__host__ __device__ inline int fused_cols(int nz) { return nz >= 128 ? 2 : (256 / nz < 2 ? 2 : (256 / nz > 16 ? 16 : 256 / nz)); }

// Shared-memory layout of a block for one problem (the same in every block
// of the cluster, so that a remote block's slab sits at the same offset).
// fused_smem_bytes() on the host must match.
template <typename T>
struct FusedSmem {
  double* red;     // 32 * kFusedRed: block reduction
  double* cred;    // 2 * 16: this block's partials for the cluster, two rounds alternating
  PState* ps;      // the problem's CG state (an identical copy in every block)
  int* next;       // the problem index rank 0 took from the queue
  T* lm;           // 2 * nphase
  C2<T>* twx;      // nx
  C2<T>* twy;      // ny
  C2<T>* twz;      // nz
  int* pfx;        // nx
  int* sfy;        // ny
  int* sfz;        // nz
  C2<T>* slab;     // zper * 3 * ny * RP
  C2<T>* zt;       // W * 6 * nz
};

__host__ __device__ inline size_t fused_align(size_t v) { return (v + 15) & ~size_t(15); }
constexpr size_t kFusedFixed = 32 * kFusedRed * 8 + 2 * 16 * 8 + 256 + 16;
static_assert(sizeof(PState) <= 256, "the problem state must fit its shared-memory slot");

template <typename T>
__host__ __device__ inline size_t fused_smem_bytes(int nx, int ny, int nz, int zper, int nphase) {
  const size_t RP = (size_t)((nx + 2) | 1);
  const int W = fused_cols(nz);
  size_t o = kFusedFixed;
  o = fused_align(o + sizeof(T) * 2 * (size_t)nphase);
  o = fused_align(o + sizeof(C2<T>) * (size_t)(nx + ny + nz));
  o = fused_align(o + sizeof(int) * (size_t)(nx + ny + nz));
  o = fused_align(o + sizeof(C2<T>) * (size_t)zper * 3 * ny * RP);
  o = fused_align(o + sizeof(C2<T>) * (size_t)W * 6 * nz);
  return o;
}

template <typename T>
__device__ __forceinline__ FusedSmem<T> fused_layout(char* base, int nx, int ny, int nz, int zper, int nphase) {
  FusedSmem<T> s;
  const size_t RP = (size_t)((nx + 2) | 1);
  s.red = reinterpret_cast<double*>(base);
  s.cred = s.red + 32 * kFusedRed;
  s.ps = reinterpret_cast<PState*>(s.cred + 2 * 16);
  s.next = reinterpret_cast<int*>(base + 32 * kFusedRed * 8 + 2 * 16 * 8 + 256);
  size_t o = kFusedFixed;
  s.lm = reinterpret_cast<T*>(base + o);
  o = fused_align(o + sizeof(T) * 2 * (size_t)nphase);
  s.twx = reinterpret_cast<C2<T>*>(base + o);
  s.twy = s.twx + nx;
  s.twz = s.twy + ny;
  o = fused_align(o + sizeof(C2<T>) * (size_t)(nx + ny + nz));
  s.pfx = reinterpret_cast<int*>(base + o);
  s.sfy = s.pfx + nx;
  s.sfz = s.sfy + ny;
  o = fused_align(o + sizeof(int) * (size_t)(nx + ny + nz));
  s.slab = reinterpret_cast<C2<T>*>(base + o);
  o = fused_align(o + sizeof(C2<T>) * (size_t)zper * 3 * ny * RP);
  s.zt = reinterpret_cast<C2<T>*>(base + o);
  return s;
}

// Geometry of the problem a cluster works on, the same in all its blocks.
struct FusedGeo {
  int nx, ny, nz, nxh, RP, zper;
  int z0, zc;     // this block's planes [z0, z0 + zc)
  long long V;    // voxels of Omega_B
  int pl;         // nx * ny
};

// ---------------------------------------------------------------------------
// CG scalar steps (the multi-pass solver's k_scal_* kernels, on one state).
// ---------------------------------------------------------------------------
__device__ inline void fused_scal_init(PState& s, double tt, double rho, double floor2) {
  s.rho = rho;
  s.rho0 = rho;
  s.rho_prev = rho;
  s.alpha = 0.0;
  s.beta = 0.0;
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
    s.active = 0;
    s.homog = 1;
  }
}

__device__ inline void fused_scal_step(PState& s, double rr, double pq, double rq, double qq, double tol,
                                       int max_iter, int fixed_iters) {
  s.pending = 0;
  if (!isfinite(rr) || !isfinite(pq) || !isfinite(rq) || !isfinite(qq)) {
    s.active = 0;
    s.status = ST_NONFINITE;
    return;
  }
  if (!(pq > 0.0)) {
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

__device__ inline void fused_scal_replace(PState& s, double rr, double tol, int fixed_iters) {
  s.trueflag = 0;
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

__device__ inline void fused_scal_true_final(PState& s, double rr, double tol, double slack, int max_restarts,
                                             int max_iter, int fixed_iters) {
  s.trueflag = 0;
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
      s.beta = 0.0;
    } else {
      s.status = ST_NOT_CONVERGED;
    }
  }
}

// ---------------------------------------------------------------------------
// Phases of one operator application.
// ---------------------------------------------------------------------------

// Sum of K partials over the cluster: block tree, then the C block totals in
// rank order (every block reads all C slots, so every block gets the same
// doubles). The result is valid in thread 0. `round` alternates the slot
// buffer: between two uses of one buffer there is always the other round's
// cluster barrier, after which every block has read the older values.
template <int K>
__device__ __forceinline__ void fused_cluster_sum(double (&v)[K], double* red, double* cred, int& round,
                                                  cgr::cluster_group& cl) {
  block_reduce<K>(v, red);
  double* slot = cred + 16 * round;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) slot[k] = v[k];
  }
  cl.sync();
  if (threadIdx.x == 0) {
    const int C = (int)cl.num_blocks();
    double tot[K];
#pragma unroll
    for (int k = 0; k < K; ++k) tot[k] = 0.0;
    for (int rk = 0; rk < C; ++rk) {
      const double* rs = cl.map_shared_rank(slot, rk);
#pragma unroll
      for (int k = 0; k < K; ++k) tot[k] += rs[k];
    }
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = tot[k];
  }
  round ^= 1;
}

// Forward transforms of the block's planes (x real-to-complex with the pair
// packing, unpack, y), then the z phase over the cluster, with the
// projection (Appendix A) of every mode.
template <typename T>
__device__ __noinline__ void fused_spectral(const FusedParams<T>& P, const FusedGeo& g, const FusedSmem<T>& sm,
                               const AxisPlan& ax, const AxisPlan& ay, const AxisPlan& az, C2<T>* const* rb,
                               cgr::cluster_group& cl) {
  const int ny = g.ny, nz = g.nz, nxh = g.nxh, RP = g.RP;
  if (g.zc > 0) {
    fft_lines<T, false>(sm.slab, Lines{3 * ny * g.zc, 1 << 30, 0, RP, 1, false}, ax, sm.twx);
    unpack_rows<T>(sm.slab, 3 * ny * g.zc, RP, g.nx, nxh, sm.pfx);
    fft_lines<T, false>(sm.slab, Lines{6 * nxh * g.zc, 2 * nxh, ny * RP, 1, RP, true}, ay, sm.twy);
  }
  cl.sync();  // every block's planes are transformed in x and y
  // z phase: this block's share of the ny * nxh spectrum columns
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const long long J = (long long)ny * nxh;
  const int jb = (int)(J * rank / C), je = (int)(J * (rank + 1) / C);
  const int zper = g.zper;
  const int W = fused_cols(nz);
  for (int j0 = jb; j0 < je; j0 += W) {
    const int Wc = min(W, je - j0);
    const int tot = 6 * nz * Wc;
    // gather: zt[(c * nz + z) * Wc + jl] = component c of column j0 + jl at plane z
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
      const int jl = e % Wc;
      const int cz = e / Wc;
      const int c = cz / nz;
      const int z = cz - c * nz;
      const int j = j0 + jl;
      const int ky = j / nxh;
      const int kx = j - ky * nxh;
      const int ow = z / zper;
      const int zl = z - ow * zper;
      sm.zt[e] = rb[ow][((zl * 3 + (c >> 1)) * ny + ky) * RP + (c & 1) * nxh + kx];
    }
    __syncthreads();
    const Lines Lz{6 * Wc, Wc, nz * Wc, 1, Wc, true};
    fft_lines<T, false>(sm.zt, Lz, az, sm.twz);
    for (int e = threadIdx.x; e < nz * Wc; e += blockDim.x) {
      const int jl = e % Wc;
      const int kzp = e / Wc;
      const int j = j0 + jl;
      const int kyp = j / nxh;
      const int kx = j - kyp * nxh;
      const int my = sm.sfy[kyp];
      const int mz = sm.sfz[kzp];
      const bool nyq_x = (g.nx % 2 == 0) && (2 * kx == g.nx);
      const bool nyq_y = (ny % 2 == 0) && (2 * my == ny);
      const bool nyq_z = (nz % 2 == 0) && (2 * mz == nz);
      T x0 = T(kx) / T(g.nx), x1 = T(my) / T(ny), x2 = T(mz) / T(nz);
      if (P.nyq_mode == 0) {
        if (nyq_x) x0 = T(0);
        if (nyq_y) x1 = T(0);
        if (nyq_z) x2 = T(0);
      } else if (nyq_x || nyq_y || nyq_z) {
        x0 = x1 = x2 = T(0);
      }
      C2<T> t[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) t[c] = sm.zt[(c * nz + kzp) * Wc + jl];
      project_mode<T>(t, x0, x1, x2);
#pragma unroll
      for (int c = 0; c < 6; ++c) sm.zt[(c * nz + kzp) * Wc + jl] = t[c];
    }
    __syncthreads();
    fft_lines<T, true>(sm.zt, Lz, az, sm.twz);
    // scatter back to the owners' slabs
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
      const int jl = e % Wc;
      const int cz = e / Wc;
      const int c = cz / nz;
      const int z = cz - c * nz;
      const int j = j0 + jl;
      const int ky = j / nxh;
      const int kx = j - ky * nxh;
      const int ow = z / zper;
      const int zl = z - ow * zper;
      rb[ow][((zl * 3 + (c >> 1)) * ny + ky) * RP + (c & 1) * nxh + kx] = sm.zt[e];
    }
    __syncthreads();
  }
  cl.sync();  // every column is back in its owner's slab
  if (g.zc > 0) {
    fft_lines<T, true>(sm.slab, Lines{6 * nxh * g.zc, 2 * nxh, ny * RP, 1, RP, true}, ay, sm.twy);
    pack_rows<T>(sm.slab, 3 * ny * g.zc, RP, g.nx, nxh, sm.pfx);
    fft_lines<T, true>(sm.slab, Lines{3 * ny * g.zc, 1 << 30, 0, RP, 1, false}, ax, sm.twx);
  }
}

// Voxel v of the block's planes: its offset in Omega_B and the slab position
// of its first component pair (pairs c2 = 1, 2 follow at c2 * ny * RP).
__device__ __forceinline__ void fused_voxel_at(const FusedGeo& g, int v, long long& vo, int& so) {
  const int zl = v / g.pl;
  const int rem = v - zl * g.pl;
  const int y = rem / g.nx;
  const int x = rem - y * g.nx;
  vo = (long long)(g.z0 + zl) * g.pl + rem;
  so = (zl * 3 * g.ny + y) * g.RP + x;
}

// One operator application q = G*(C:e) in mode MODE with the voxel work of
// the forward and inverse phases; returns the cluster sums in sums[] (valid
// in thread 0):
//   MODE_RHS : e = E;            sums = {<tau, tau>, <r, r>}; r = p = -q, x = 0
//   MODE_ITER: pending update, p <- r + beta p, e = p;
//              sums = {<r, r>, <p, q>, <r, q>, <q, q>}; q kept in the slab
//   MODE_TRUE: e = E + x;        sums = {<r, r>}; r = -q
template <typename T, int MODE>
__device__ __noinline__ void fused_apply(const FusedParams<T>& P, const Prob& d, const FusedGeo& g, const FusedSmem<T>& sm,
                            const AxisPlan& ax, const AxisPlan& ay, const AxisPlan& az, C2<T>* const* rb,
                            int& round, cgr::cluster_group& cl, double (&sums)[4]) {
  const long long V = g.V;
  const int sstr = g.ny * g.RP;  // slab stride between component pairs
  T* __restrict__ R = P.r + d.fld_off;
  T* __restrict__ Pp = P.p + d.fld_off;
  T* __restrict__ X = P.x + d.fld_off;
  const uint8_t* __restrict__ lab = P.labels + d.med_off;
  const T Ed = d.lc < 3 ? T(1) : T(0.5);
  const T alpha = T(sm.ps->alpha), beta = T(sm.ps->beta);
  const bool pend = sm.ps->pending != 0;
  DotAcc<T> a0;
  const int nv = g.zc * g.pl;
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    long long vo;
    int so;
    fused_voxel_at(g, v, vo, so);
    const int lb = lab[vo];
    T e[6];
    if (MODE == MODE_RHS) {
#pragma unroll
      for (int c = 0; c < 6; ++c) e[c] = T(0);
      e[d.lc] = Ed;
    } else if (MODE == MODE_ITER) {
      T rv[6], pv[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        rv[c] = R[c * V + vo];
        pv[c] = Pp[c * V + vo];
      }
      if (pend) {
        T xv[6], qv[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) xv[c] = X[c * V + vo];
#pragma unroll
        for (int c2 = 0; c2 < 3; ++c2) {
          const C2<T> qq = sm.slab[so + c2 * sstr];
          qv[2 * c2] = qq.x;
          qv[2 * c2 + 1] = qq.y;
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          rv[c] -= alpha * qv[c];
          R[c * V + vo] = rv[c];
          X[c * V + vo] = xv[c] + alpha * pv[c];
        }
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const T pn = rv[c] + beta * pv[c];
        Pp[c * V + vo] = pn;
        e[c] = pn;
        a0.add(rv[c], frob_t(c, rv[c]));
      }
    } else {  // MODE_TRUE
#pragma unroll
      for (int c = 0; c < 6; ++c) e[c] = X[c * V + vo];
      e[d.lc] += Ed;
    }
    T s[6];
    stress_iso<T>(e, sm.lm[2 * lb], sm.lm[2 * lb + 1], s);
    if (MODE == MODE_RHS) {
#pragma unroll
      for (int c = 0; c < 6; ++c) a0.add(s[c], frob_t(c, s[c]));
    }
#pragma unroll
    for (int c2 = 0; c2 < 3; ++c2) sm.slab[so + c2 * sstr] = mk<T>(s[2 * c2], s[2 * c2 + 1]);
  }
  __syncthreads();
  fused_spectral<T>(P, g, sm, ax, ay, az, rb, cl);
  // inverse voxel phase
  DotAcc<T> a1, a2, a3;
  const T invV = T(1) / T(V);
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    long long vo;
    int so;
    fused_voxel_at(g, v, vo, so);
    T qv[6];
#pragma unroll
    for (int c2 = 0; c2 < 3; ++c2) {
      const C2<T> zz = sm.slab[so + c2 * sstr];
      qv[2 * c2] = zz.x * invV;
      qv[2 * c2 + 1] = zz.y * invV;
    }
    if (MODE == MODE_ITER) {
      T pv[6], rv[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        pv[c] = Pp[c * V + vo];
        rv[c] = R[c * V + vo];
      }
#pragma unroll
      for (int c2 = 0; c2 < 3; ++c2) sm.slab[so + c2 * sstr] = mk<T>(qv[2 * c2], qv[2 * c2 + 1]);
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const T wq = frob_t(c, qv[c]);
        a1.add(pv[c], wq);
        a2.add(rv[c], wq);
        a3.add(qv[c], wq);
      }
    } else {
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const T rv = -qv[c];
        R[c * V + vo] = rv;
        if (MODE == MODE_RHS) {
          Pp[c * V + vo] = rv;
          X[c * V + vo] = T(0);
        }
        a1.add(rv, frob_t(c, rv));
      }
    }
  }
  if (MODE == MODE_ITER) {
    double v4[4] = {a0.value(), a1.value(), a2.value(), a3.value()};
    fused_cluster_sum<4>(v4, sm.red, sm.cred, round, cl);
#pragma unroll
    for (int k = 0; k < 4; ++k) sums[k] = v4[k];
  } else {
    double v2[2] = {a0.value(), a1.value()};
    fused_cluster_sum<2>(v2, sm.red, sm.cred, round, cl);
    sums[0] = v2[0];
    sums[1] = v2[1];
  }
}

// The deferred update r <- r - alpha q, x <- x + alpha p (q from the slab).
template <typename T>
__device__ __noinline__ void fused_flush(const FusedParams<T>& P, const Prob& d, const FusedGeo& g, const FusedSmem<T>& sm) {
  const long long V = g.V;
  const int sstr = g.ny * g.RP;
  T* __restrict__ R = P.r + d.fld_off;
  const T* __restrict__ Pp = P.p + d.fld_off;
  T* __restrict__ X = P.x + d.fld_off;
  const T alpha = T(sm.ps->alpha);
  const int nv = g.zc * g.pl;
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    long long vo;
    int so;
    fused_voxel_at(g, v, vo, so);
#pragma unroll
    for (int c2 = 0; c2 < 3; ++c2) {
      const C2<T> qq = sm.slab[so + c2 * sstr];
      const int c = 2 * c2;
      R[c * V + vo] = R[c * V + vo] - alpha * qq.x;
      R[(c + 1) * V + vo] = R[(c + 1) * V + vo] - alpha * qq.y;
      X[c * V + vo] = X[c * V + vo] + alpha * Pp[c * V + vo];
      X[(c + 1) * V + vo] = X[(c + 1) * V + vo] + alpha * Pp[(c + 1) * V + vo];
    }
  }
}

// Core sums of eps* and of C:(E + eps*) (Section 4 averages over Omega_R).
template <typename T>
__device__ __noinline__ void fused_averages(const FusedParams<T>& P, const Prob& d, const FusedGeo& g, const FusedSmem<T>& sm,
                               int& round, cgr::cluster_group& cl, double (&out)[kFusedRed]) {
  const long long V = g.V;
  const T* __restrict__ X = P.x + d.fld_off;
  const uint8_t* __restrict__ lab = P.labels + d.med_off;
  const T Ed = d.lc < 3 ? T(1) : T(0.5);
  double acc[kFusedRed];
#pragma unroll
  for (int k = 0; k < kFusedRed; ++k) acc[k] = 0.0;
  const int nv = g.zc * g.pl;
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    const int zl = v / g.pl;
    const int rem = v - zl * g.pl;
    const int y = rem / g.nx;
    const int x = rem - y * g.nx;
    const int z = g.z0 + zl;
    if (z < d.c0z || z >= d.c0z + d.cnz || y < d.c0y || y >= d.c0y + d.cny || x < d.c0x || x >= d.c0x + d.cnx)
      continue;
    const long long vo = (long long)z * g.pl + rem;
    T e[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      e[c] = X[c * V + vo];
      acc[c] += double(e[c]);
    }
    e[d.lc] += Ed;
    T s[6];
    const int lb = lab[vo];
    stress_iso<T>(e, sm.lm[2 * lb], sm.lm[2 * lb + 1], s);
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[6 + c] += double(s[c]);
  }
  fused_cluster_sum<kFusedRed>(acc, sm.red, sm.cred, round, cl);
#pragma unroll
  for (int k = 0; k < kFusedRed; ++k) out[k] = acc[k];
}

// ---------------------------------------------------------------------------
// The persistent kernel.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kFusedThreads, 4) k_fused(FusedParams<T> P) {
  extern __shared__ __align__(16) char smem[];
  cgr::cluster_group cl = cgr::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  __shared__ C2<T>* rb[16];  // slab base of every block of the cluster
  int* next = reinterpret_cast<int*>(smem + 32 * kFusedRed * 8 + 2 * 16 * 8 + 256);
  int round = 0;
  while (true) {
    if (rank == 0 && threadIdx.x == 0) *next = atomicAdd(P.queue, 1);
    cl.sync();
    const int w = *cl.map_shared_rank(next, 0);
    cl.sync();  // rank 0 writes `next` again only after every block has read it
    if (w >= P.nwork) break;
    const int pr = P.order[w];
    const Prob d = P.prob[pr];
    FusedGeo g;
    g.nx = d.nx;
    g.ny = d.ny;
    g.nz = d.nz;
    g.nxh = d.nxh;
    g.RP = pair_pitch(d.nx);
    g.zper = (d.nz + C - 1) / C;
    g.z0 = min(rank * g.zper, d.nz);
    g.zc = min(d.nz, g.z0 + g.zper) - g.z0;
    g.V = (long long)d.nx * d.ny * d.nz;
    g.pl = d.nx * d.ny;
    const FusedSmem<T> sm = fused_layout<T>(smem, d.nx, d.ny, d.nz, g.zper, P.nphase);
    const AxisPlan& ax = P.plans[d.px];
    const AxisPlan& ay = P.plans[d.py];
    const AxisPlan& az = P.plans[d.pz];
    load_tw<T>(sm.twx, P.tw, ax);
    load_tw<T>(sm.twy, P.tw, ay);
    load_tw<T>(sm.twz, P.tw, az);
    for (int t = threadIdx.x; t < d.nx; t += blockDim.x) sm.pfx[t] = P.itab[ax.pf_off + t];
    for (int t = threadIdx.x; t < d.ny; t += blockDim.x) sm.sfy[t] = P.itab[ay.sf_off + t];
    for (int t = threadIdx.x; t < d.nz; t += blockDim.x) sm.sfz[t] = P.itab[az.sf_off + t];
    for (int t = threadIdx.x; t < 2 * P.nphase; t += blockDim.x) sm.lm[t] = P.lammu[t];
    if (threadIdx.x < C) rb[threadIdx.x] = cl.map_shared_rank(sm.slab, (int)threadIdx.x);
    __syncthreads();

    double sums[4];
    PState& s = *sm.ps;
    // ---- right-hand side b = -G*(C:E), r = p = b, x = 0
    fused_apply<T, MODE_RHS>(P, d, g, sm, ax, ay, az, rb, round, cl, sums);
    if (threadIdx.x == 0) fused_scal_init(s, sums[0], sums[1], P.floor2);
    __syncthreads();
    int final_rounds = 0;
    long long chunks = 0;
    while (true) {
      if (!s.active) {
        // every iteration of this problem has stopped: check the true residual
        if (final_rounds > P.max_restarts) break;
        if (s.pending) {
          fused_flush<T>(P, d, g, sm);
          __syncthreads();
          if (threadIdx.x == 0) s.pending = 0;
          __syncthreads();
        }
        const bool check = !s.homog && s.status != ST_NONFINITE;
        if (check) {
          fused_apply<T, MODE_TRUE>(P, d, g, sm, ax, ay, az, rb, round, cl, sums);
          if (threadIdx.x == 0)
            fused_scal_true_final(s, sums[1], P.tol, 2.0, P.max_restarts, P.max_iter, P.fixed_iters);
          __syncthreads();
        }
        ++final_rounds;
        if (!s.active) break;
      }
      if (chunks >= P.max_chunks) break;
      for (int m = 0; m < P.chunk && s.active; ++m) {
        fused_apply<T, MODE_ITER>(P, d, g, sm, ax, ay, az, rb, round, cl, sums);
        if (threadIdx.x == 0) fused_scal_step(s, sums[0], sums[1], sums[2], sums[3], P.tol, P.max_iter, P.fixed_iters);
        __syncthreads();
      }
      if (P.replace) {
        if (s.pending) {
          fused_flush<T>(P, d, g, sm);
          __syncthreads();
          if (threadIdx.x == 0) s.pending = 0;
          __syncthreads();
        }
        if (s.active) {
          fused_apply<T, MODE_TRUE>(P, d, g, sm, ax, ay, az, rb, round, cl, sums);
          if (threadIdx.x == 0) fused_scal_replace(s, sums[1], P.tol, P.fixed_iters);
          __syncthreads();
        }
      }
      ++chunks;
    }
    if (s.pending) {
      fused_flush<T>(P, d, g, sm);
      __syncthreads();
      if (threadIdx.x == 0) s.pending = 0;
    }
    __syncthreads();
    double avg[kFusedRed];
    fused_averages<T>(P, d, g, sm, round, cl, avg);
    if (threadIdx.x == 0 && rank == 0) {
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        s.xbar[c] = avg[c];
        s.sbar[c] = avg[6 + c];
      }
      s.trueflag = 0;
      P.st[pr] = s;
    }
    // the next problem may have another layout: no block may still be reading
    // this one's slab or partial slots
    cl.sync();
  }
}

}  // namespace hh
