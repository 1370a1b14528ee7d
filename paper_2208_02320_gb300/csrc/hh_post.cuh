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
  double K, G, KR, GR;
  double resid[6];
  int iters[6];
  int status;
  int pad;
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
__global__ void k_finalize(const Prob* prob, const PState* st, int nbox, BoxRes* out, int box_base) {
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
  R.status = status;
  R.pad = 0;
  out[box_base + b] = R;
}

// Assembly (Section 3): each box fills its block of unit-size coarse cells
// with the 21 upper-triangle entries of sym(C_R) (component-major, FP64).
__global__ void k_assemble(const BoxReq* boxes, const BoxRes* res, int nbox, int unit, int Cx, int Cy, int Cz,
                           double* c21) {
  const int b = blockIdx.x;
  if (b >= nbox) return;
  const BoxReq B = boxes[b];
  const long long V = (long long)Cx * Cy * Cz;
  const int x0 = B.ox / unit, y0 = B.oy / unit, z0 = B.oz / unit;
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
    c21[k * V + v] = res[b].Csym[a * 6 + bcol];
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

// Core-volume-weighted means of subimage K and G (one block, fixed order).
__global__ void k_am(const BoxRes* res, const BoxReq* boxes, int nbox, double* out3) {
  __shared__ double red[32 * 3];
  double v[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nbox; b += blockDim.x) {
    const double w = double(boxes[b].cnx) * boxes[b].cny * boxes[b].cnz;
    v[0] += w * res[b].K;
    v[1] += w * res[b].G;
    v[2] += w;
  }
  block_reduce<3>(v, red);
  if (threadIdx.x == 0) {
    out3[0] = v[0] / v[2];
    out3[1] = v[1] / v[2];
    out3[2] = v[2];
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
