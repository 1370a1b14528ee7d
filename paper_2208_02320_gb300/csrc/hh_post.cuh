// Device kernels around the solver: subimage extraction (Section 4, Fig. 4),
// effective stiffness C_R = Sigma Eps^-1 (Section 4), assembly of the
// intermediate anisotropic image (Section 3), isotropic projections of a
// stiffness, arithmetic means, and the power-law fit in 1/n (Section 5).
// All stiffness algebra is FP64.
#pragma once

#include "hh_device.cuh"

namespace hh {

struct BoxReq {
  int ox, oy, oz, cnx, cny, cnz, b, pad;
  long long lab_off;  // offset of the buffered label box in the label workspace
};

struct BoxRes {
  double C[36];     // raw Sigma Eps^-1
  double Sig[36];   // columns = load cases (stress Voigt)
  double Eps[36];   // columns = load cases (engineering strain Voigt)
  double Csym[36];
  double Cspd[36];  // sym(C_R) raised to the stiffness floor (level-2 voxel)
  double K, G, KR, GR;
  double resid[6];
  int iters[6];
  int status;
  int clipped;
};

// Extraction of the buffered boxes with periodic wrap; one block per (box, z).
// Labels >= nphase set *bad.
__global__ void k_gather(const uint8_t* img, int Nx, int Ny, int Nz, const BoxReq* boxes, const int2* items,
                         int nitems, uint8_t* out, int nphase, int* bad) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int2 w = items[it];
    const BoxReq B = boxes[w.x];
    const int bx = B.cnx + 2 * B.b, by = B.cny + 2 * B.b, bz = B.cnz + 2 * B.b;
    const int k = w.y;
    int sz = (B.oz - B.b + k) % Nz;
    if (sz < 0) sz += Nz;
    uint8_t* dst = out + B.lab_off + (long long)k * by * bx;
    for (int e = threadIdx.x; e < by * bx; e += blockDim.x) {
      const int j = e / bx;
      const int i = e - j * bx;
      int sy = (B.oy - B.b + j) % Ny;
      if (sy < 0) sy += Ny;
      int sx = (B.ox - B.b + i) % Nx;
      if (sx < 0) sx += Nx;
      const uint8_t v = img[((long long)sz * Ny + sy) * Nx + sx];
      dst[e] = v;
      if (v >= nphase) atomicOr(bad, 1);
    }
    (void)bz;
  }
}

// Sets *bad when any of the n labels is >= nphase (the phase table of the
// plane passes has nphase entries).
__global__ void k_check_labels(const uint8_t* lab, long long n, int nphase, int* bad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (lab[i] >= nphase) atomicOr(bad, 1);
}

// Gauss-Jordan inverse with partial pivoting of a 6x6 row-major matrix.
__device__ inline bool inv6(const double* A, double* X) {
  double M[6][12];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      M[i][j] = A[i * 6 + j];
      M[i][6 + j] = (i == j) ? 1.0 : 0.0;
    }
  for (int c = 0; c < 6; ++c) {
    int piv = c;
    double best = fabs(M[c][c]);
    for (int r = c + 1; r < 6; ++r)
      if (fabs(M[r][c]) > best) {
        best = fabs(M[r][c]);
        piv = r;
      }
    if (!(best > 0.0)) return false;
    if (piv != c)
      for (int j = 0; j < 12; ++j) {
        double t = M[c][j];
        M[c][j] = M[piv][j];
        M[piv][j] = t;
      }
    const double d = 1.0 / M[c][c];
    for (int j = 0; j < 12; ++j) M[c][j] *= d;
    for (int r = 0; r < 6; ++r)
      if (r != c) {
        const double f = M[r][c];
        if (f != 0.0)
          for (int j = 0; j < 12; ++j) M[r][j] -= f * M[c][j];
      }
  }
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) X[i * 6 + j] = M[i][6 + j];
  return true;
}

// Cyclic Jacobi eigen-decomposition of a symmetric 6x6 matrix (row-major
// A[36], overwritten): A = V diag(w) V^T. Each rotation zeroes the (p, q)
// pair and updates the symmetric pairs of rows/columns p and q explicitly.
__device__ inline void jacobi6(double* A, double* V, double* w) {
  for (int i = 0; i < 36; ++i) V[i] = (i % 7 == 0) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int p = 0; p < 6; ++p) {
      diag += A[p * 6 + p] * A[p * 6 + p];
      for (int q = p + 1; q < 6; ++q) off += A[p * 6 + q] * A[p * 6 + q];
    }
    if (off <= 1e-32 * diag) break;
    for (int p = 0; p < 5; ++p)
      for (int q = p + 1; q < 6; ++q) {
        const double apq = A[p * 6 + q];
        if (apq == 0.0) continue;
        const double app = A[p * 6 + p], aqq = A[q * 6 + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0);
        const double sn = t * c;
        A[p * 6 + p] = app - t * apq;
        A[q * 6 + q] = aqq + t * apq;
        A[p * 6 + q] = 0.0;
        A[q * 6 + p] = 0.0;
        for (int r = 0; r < 6; ++r) {
          if (r == p || r == q) continue;
          const double arp = A[r * 6 + p], arq = A[r * 6 + q];
          const double nrp = c * arp - sn * arq, nrq = sn * arp + c * arq;
          A[r * 6 + p] = nrp;
          A[p * 6 + r] = nrp;
          A[r * 6 + q] = nrq;
          A[q * 6 + r] = nrq;
        }
        for (int r = 0; r < 6; ++r) {
          const double vrp = V[r * 6 + p], vrq = V[r * 6 + q];
          V[r * 6 + p] = c * vrp - sn * vrq;
          V[r * 6 + q] = sn * vrp + c * vrq;
        }
      }
  }
  for (int i = 0; i < 6; ++i) w[i] = A[i * 7];
}

// sym(C) with every tensor eigenvalue (Mandel form D C D, D = diag(1,1,1,
// sqrt2,sqrt2,sqrt2)) below `floor` raised to `floor`; returns whether it
// changed anything. Used for the level-2 voxels of buffered subimages.
__device__ inline bool clip_spd6(const double* Cs, double floor, double* out) {
  const double D[6] = {1.0, 1.0, 1.0, 1.4142135623730951, 1.4142135623730951, 1.4142135623730951};
  double A[36], V[36], w[6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) A[i * 6 + j] = D[i] * Cs[i * 6 + j] * D[j];
  jacobi6(A, V, w);
  double wmin = w[0];
  for (int i = 1; i < 6; ++i) wmin = fmin(wmin, w[i]);
  if (!(floor > 0.0) || wmin >= floor * (1.0 - 1e-12)) {
    for (int i = 0; i < 36; ++i) out[i] = Cs[i];
    return false;
  }
  for (int i = 0; i < 6; ++i) w[i] = fmax(w[i], floor);
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 6; ++k) acc += V[i * 6 + k] * w[k] * V[j * 6 + k];
      out[i * 6 + j] = acc / (D[i] * D[j]);
    }
  return true;
}

// Isotropic Voigt and Reuss projections of a 6x6 stiffness.
__device__ inline void moduli(const double* C, double* K, double* G, double* KR, double* GR) {
  const double a = C[0] + C[7] + C[14];
  const double b = C[1] + C[2] + C[8];
  const double c = C[21] + C[28] + C[35];
  *K = (a + 2.0 * b) / 9.0;
  *G = (a - b + 3.0 * c) / 15.0;
  double S[36];
  if (inv6(C, S)) {
    const double sa = S[0] + S[7] + S[14];
    const double sb = S[1] + S[2] + S[8];
    const double sc = S[21] + S[28] + S[35];
    *KR = 1.0 / (sa + 2.0 * sb);
    *GR = 15.0 / (4.0 * sa - 4.0 * sb + 3.0 * sc);
  } else {
    *KR = nan("");
    *GR = nan("");
  }
}

// Sigma, Eps and C_R of each box from the CG scalars of its six load cases
// (problems 6 b .. 6 b + 5 of the wave). Core averages:
//   <sigma>_R = sum_R C:(E + eps*) / |R|,  <eps>_R = E + sum_R eps* / |R|.
__global__ void k_finalize(const Prob* prob, const PState* st, int nbox, BoxRes* out, int box_base, double floor) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  BoxRes R;
  int status = ST_OK;
  const Prob d0 = prob[6 * b];
  const double Vc = double(d0.cnx) * d0.cny * d0.cnz;
  for (int a = 0; a < 6; ++a) {
    const PState s = st[6 * b + a];
    for (int i = 0; i < 6; ++i) {
      R.Sig[i * 6 + a] = s.sbar[i] / Vc;
      const double Ei = (i == a) ? (a < 3 ? 1.0 : 0.5) : 0.0;
      R.Eps[i * 6 + a] = (i < 3 ? 1.0 : 2.0) * (Ei + s.xbar[i] / Vc);
    }
    R.iters[a] = s.iters;
    R.resid[a] = s.resid;
    if (s.status == ST_NONFINITE) status = ST_NONFINITE;
    else if (s.status == ST_NOT_CONVERGED && status == ST_OK) status = ST_NOT_CONVERGED;
  }
  double Ei[36];
  if (!inv6(R.Eps, Ei)) status = ST_NONFINITE;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 6; ++k) acc += R.Sig[i * 6 + k] * Ei[k * 6 + j];
      R.C[i * 6 + j] = acc;
    }
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) R.Csym[i * 6 + j] = 0.5 * (R.C[i * 6 + j] + R.C[j * 6 + i]);
  moduli(R.Csym, &R.K, &R.G, &R.KR, &R.GR);
  R.clipped = clip_spd6(R.Csym, floor, R.Cspd) ? 1 : 0;
  R.status = status;
  out[box_base + b] = R;
}

// Level-1 results of the subimages whose surrogate prediction was accepted:
// C = sym(C) = the predicted stiffness (21 upper-triangle values, FP64), its
// moduli, and the same projection onto the stiffness floor as FFT results.
__global__ void k_accept_pred(const double* c21, const int* idx, int n, BoxRes* res, double floor) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  BoxRes R;
  memset(&R, 0, sizeof(R));
  for (int a = 0, t = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b, ++t) {
      R.C[a * 6 + b] = R.C[b * 6 + a] = c21[(long long)i * 21 + t];
      R.Csym[a * 6 + b] = R.Csym[b * 6 + a] = c21[(long long)i * 21 + t];
    }
  moduli(R.Csym, &R.K, &R.G, &R.KR, &R.GR);
  R.clipped = clip_spd6(R.Csym, floor, R.Cspd) ? 1 : 0;
  res[idx[i]] = R;
}

// res[pos[i]] = src[i] (FFT results of the remaining subimages into place).
__global__ void k_scatter_res(const BoxRes* src, const int* pos, int n, BoxRes* res) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) res[pos[i]] = src[i];
}

// Assembly (Section 3): each box fills its block of unit-size coarse cells
// with the 21 upper-triangle entries of sym(C_R) (component-major, FP64).
__global__ void k_assemble(const BoxReq* boxes, const BoxRes* res, int nbox, int unit, int rx, int ry, int rz, int Cx,
                           int Cy, int Cz, double* c21) {
  const int b = blockIdx.x;
  if (b >= nbox) return;
  const BoxReq B = boxes[b];
  const long long V = (long long)Cx * Cy * Cz;
  const int x0 = B.ox / unit - rx, y0 = B.oy / unit - ry, z0 = B.oz / unit - rz;
  const int ex = B.cnx / unit, ey = B.cny / unit, ez = B.cnz / unit;
  const int cells = ex * ey * ez;
  for (int e = threadIdx.x; e < cells * 21; e += blockDim.x) {
    const int k = e / cells;
    const int cidx = e - k * cells;
    const int i = cidx % ex;
    const int j = (cidx / ex) % ey;
    const int l = cidx / (ex * ey);
    int a = 0, t = k;
    while (t >= 6 - a) {
      t -= 6 - a;
      ++a;
    }
    const int bcol = a + t;
    const long long v = ((long long)(z0 + l) * Cy + (y0 + j)) * Cx + (x0 + i);
    c21[k * V + v] = res[b].Cspd[a * 6 + bcol];
  }
}

// FP64 -> T copy of a C21 field with a Cholesky check of every voxel's 6x6.
template <typename T>
__global__ void k_c21_prepare(const double* src, T* dst, long long V, int* bad) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    double A[6][6];
    int k = 0;
    for (int i = 0; i < 6; ++i)
      for (int j = i; j < 6; ++j) {
        const double x = src[k * V + v];
        A[i][j] = x;
        A[j][i] = x;
        dst[k * V + v] = T(x);
        ++k;
      }
    // Cholesky: positive pivots <=> symmetric positive definite
    bool ok = true;
    for (int j = 0; j < 6 && ok; ++j) {
      double s = A[j][j];
      for (int m = 0; m < j; ++m) s -= A[j][m] * A[j][m];
      if (!(s > 0.0) || !isfinite(s)) {
        ok = false;
        break;
      }
      const double ljj = sqrt(s);
      A[j][j] = ljj;
      for (int i = j + 1; i < 6; ++i) {
        double t = A[i][j];
        for (int m = 0; m < j; ++m) t -= A[i][m] * A[j][m];
        A[i][j] = t / ljj;
      }
    }
    if (!ok) atomicOr(bad, 1);
  }
}

// Extraction of buffered boxes from a stiffness field (21 upper-triangle
// components, component-major over the whole Nx x Ny x Nz field, FP64) with
// periodic wrap, into each box's own component-major block (element offset
// boxes[b].lab_off) in the solver's precision, with the positive-definite
// check of every voxel. One block per (box, z) item.
template <typename T>
__global__ void k_gather_c21(const double* src, int Nx, int Ny, int Nz, const BoxReq* boxes, const int2* items,
                             int nitems, T* dst, int* bad) {
  const long long Vs = (long long)Nx * Ny * Nz;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int2 w = items[it];
    const BoxReq B = boxes[w.x];
    const int ex = B.cnx + 2 * B.b, ey = B.cny + 2 * B.b, ez = B.cnz + 2 * B.b;
    const long long Vb = (long long)ex * ey * ez;
    const int z = w.y;
    const int sz = ((B.oz - B.b + z) % Nz + Nz) % Nz;
    for (int v = threadIdx.x; v < ex * ey; v += blockDim.x) {
      const int y = v / ex, x = v - (v / ex) * ex;
      const int sy = ((B.oy - B.b + y) % Ny + Ny) % Ny;
      const int sx = ((B.ox - B.b + x) % Nx + Nx) % Nx;
      const long long s = ((long long)sz * Ny + sy) * Nx + sx;
      const long long d = B.lab_off + (long long)z * ex * ey + v;
      double A[6][6];
      int k = 0;
      for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j) {
          const double val = src[k * Vs + s];
          A[i][j] = val;
          A[j][i] = val;
          dst[d + k * Vb] = T(val);
          ++k;
        }
      bool ok = true;
      for (int j = 0; j < 6 && ok; ++j) {
        double t = A[j][j];
        for (int m = 0; m < j; ++m) t -= A[j][m] * A[j][m];
        if (!(t > 0.0) || !isfinite(t)) {
          ok = false;
          break;
        }
        const double ljj = sqrt(t);
        A[j][j] = ljj;
        for (int i = j + 1; i < 6; ++i) {
          double q = A[i][j];
          for (int m = 0; m < j; ++m) q -= A[i][m] * A[j][m];
          A[i][j] = q / ljj;
        }
      }
      if (!ok) atomicOr(bad, 1);
    }
  }
}

// Two-point pair counts of the material indicator M = [label != pore] along
// one axis (0 = x, 1 = y, 2 = z): counts[l] += sum of M(v) M(v + l e_axis)
// over the pairs inside the image, l = 0..lmax. One thread per line along
// the axis (adjacent threads take adjacent lines); per-block shared counts,
// then one 64-bit atomic per l and block (integer sums: exact).
__global__ void k_corr_counts(const uint8_t* lab, int Nx, int Ny, int Nz, int axis, int pore, int lmax,
                              unsigned long long* counts) {
  extern __shared__ unsigned long long cnt[];
  for (int t = threadIdx.x; t <= lmax; t += blockDim.x) cnt[t] = 0ull;
  __syncthreads();
  const long long nline = axis == 0 ? (long long)Ny * Nz : (axis == 1 ? (long long)Nx * Nz : (long long)Nx * Ny);
  const int n = axis == 0 ? Nx : (axis == 1 ? Ny : Nz);
  const long long stride = axis == 0 ? 1 : (axis == 1 ? Nx : (long long)Nx * Ny);
  for (long long line = blockIdx.x * (long long)blockDim.x + threadIdx.x; line < nline;
       line += (long long)gridDim.x * blockDim.x) {
    long long base;
    if (axis == 0) {
      base = line * Nx;  // line = z * Ny + y
    } else if (axis == 1) {
      const long long z = line / Nx, x = line - z * Nx;
      base = z * Nx * Ny + x;
    } else {
      base = line;  // line = y * Nx + x
    }
    const uint8_t* p = lab + base;
    for (int l = 0; l <= lmax && l < n; ++l) {
      unsigned int c = 0;
      for (int i = 0; i + l < n; ++i) c += (p[i * stride] != pore) & (p[(i + l) * stride] != pore);
      if (c) atomicAdd(&cnt[l], (unsigned long long)c);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t <= lmax; t += blockDim.x)
    if (cnt[t]) atomicAdd(&counts[t], cnt[t]);
}

// Core-volume-weighted means of subimage K and G (one block, fixed order).
__global__ void k_am(const BoxRes* res, const BoxReq* boxes, int nbox, double* out3) {
  __shared__ double red[32 * 4];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nbox; b += blockDim.x) {
    const double w = double(boxes[b].cnx) * boxes[b].cny * boxes[b].cnz;
    v[0] += w * res[b].K;
    v[1] += w * res[b].G;
    v[2] += w;
    v[3] += res[b].clipped;
  }
  block_reduce<4>(v, red);
  if (threadIdx.x == 0) {
    out3[0] = v[0] / v[2];
    out3[1] = v[1] / v[2];
    out3[2] = v[2];
    out3[3] = v[3];
  }
}

// Least squares of M = M_inf + C x, x = 1/n (Section 5, Eq. fit_power_law).
__global__ void k_fit_inverse_n(const int* ns, const double* M, int count, double* out2) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double xm = 0.0, ym = 0.0;
  for (int i = 0; i < count; ++i) {
    xm += 1.0 / double(ns[i]);
    ym += M[i];
  }
  xm /= count;
  ym /= count;
  double Sxx = 0.0, Sxy = 0.0;  // centred sums (two-pass)
  for (int i = 0; i < count; ++i) {
    const double dx = 1.0 / double(ns[i]) - xm;
    Sxx += dx * dx;
    Sxy += dx * (M[i] - ym);
  }
  const double C = Sxy / Sxx;
  out2[0] = ym - C * xm;
  out2[1] = C;
}

}  // namespace hh
