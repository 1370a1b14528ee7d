// Subimage surrogate network (not in the paper): a small 3D CNN that maps a
// buffered subimage's phase labels to the 21 upper-triangle components of its
// core's effective Voigt stiffness, trained on GPU with the library's own
// kernels, and the gate that decides whether the ensemble's prediction stands
// in for an FFT solve.
//
//   input   one-hot of the labels 0, 1, 2 and the core mask (4 channels; the
//           box Omega_B has any shape, the core Omega_R is 1, the buffer 0)
//   conv1   4 -> 16, 3x3x3, stride 1, zero padding 1, bias, ReLU
//   conv2  16 -> 32, stride 2, ReLU
//   conv3  32 -> 64, stride 2, ReLU
//   conv4  64 -> 64, stride 1, ReLU
//   pool    mean over the voxels -> 64;  fc1 64 -> 128, ReLU;  fc2 128 -> 21
//
// Activations are channels-last BF16 ([sample][z][y][x][c]); weights are FP32
// master copies with BF16 copies for the convolutions; every sum accumulates in
// FP32. conv1 reads the labels directly (a one-hot input turns its contraction
// into a lookup of the weight row of each neighbour's label, plus the mask
// row where the neighbour lies in the core). conv2..conv4, their data
// gradients and their weight gradients are implicit GEMMs on the fifth-
// generation tensor cores (tcgen05.mma kind::f16, BF16 operands staged in
// shared memory, FP32 accumulator in tensor memory) with the operands
// gathered from the channels-last activations in 16-byte runs of channels
// (no im2col buffer). Subimages of one shape form a batch; a call with
// several shapes runs one batch sequence per shape.
//
// Parameter layout (flat FP32): per conv layer W[tap][ci][co] with
// tap = (kz * 3 + ky) * 3 + kx, then bias[co]; per fully connected layer
// W[in][out], then bias[out]; layers in order.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hh.h"
#include "hh_internal.h"

namespace hh {
namespace cnn {

using bf16 = __nv_bfloat16;

struct ConvSpec {
  int ci, co, stride;
};
constexpr ConvSpec kConv[4] = {{4, 16, 1}, {16, 32, 2}, {32, 64, 2}, {64, 64, 1}};
constexpr int kIn = 4;  // input channels: labels 0, 1, 2 one-hot and the core mask

// Box of a batch (all samples share it) and the core of each sample inside it.
struct Box3 {
  int x, y, z;
};
struct Core {
  int ox, oy, oz, nx, ny, nz;
  __device__ __forceinline__ bool in(int x, int y, int z) const {
    return x >= ox && x < ox + nx && y >= oy && y < oy + ny && z >= oz && z < oz + nz;
  }
};
constexpr int kFc[2][2] = {{64, 128}, {128, 21}};
constexpr int kOut = 21;
constexpr int kPoolC = 64;
constexpr int kHid = 128;

struct Offsets {
  long long w[6], b[6], total;
};
inline Offsets offsets() {
  Offsets o;
  long long p = 0;
  for (int i = 0; i < 4; ++i) {
    o.w[i] = p;
    p += 27LL * kConv[i].ci * kConv[i].co;
    o.b[i] = p;
    p += kConv[i].co;
  }
  for (int i = 0; i < 2; ++i) {
    o.w[4 + i] = p;
    p += (long long)kFc[i][0] * kFc[i][1];
    o.b[4 + i] = p;
    p += kFc[i][1];
  }
  o.total = p;
  return o;
}

__host__ __device__ inline int out_size(int n, int s) { return (n + 2 - 3) / s + 1; }

// ---------------------------------------------------------------------------
// conv1 on the labels and the core mask:
// y[m][co] = relu(b[co] + sum_tap (W1[tap][label(m + tap - 1)][co] + [m + tap - 1 in core] W1[tap][3][co])).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_conv1_fwd(const uint8_t* lab, const Core* core, int B, Box3 D,
                                                   const float* W1, const float* b1, bf16* Y) {
  __shared__ float w[27 * kIn * 16 + 16];
  for (int t = threadIdx.x; t < 27 * kIn * 16; t += blockDim.x) w[t] = W1[t];
  for (int t = threadIdx.x; t < 16; t += blockDim.x) w[27 * kIn * 16 + t] = b1[t];
  __syncthreads();
  const long long V = (long long)D.x * D.y * D.z;
  const long long M = (long long)B * V;
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < M; m += (long long)gridDim.x * blockDim.x) {
    const long long n = m / V;
    const int v = (int)(m - n * V);
    const int z = v / (D.x * D.y), y = (v / D.x) % D.y, x = v % D.x;
    const Core cr = core[n];
    float acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = w[27 * kIn * 16 + c];
    for (int kz = 0; kz < 3; ++kz) {
      const int iz = z + kz - 1;
      if (iz < 0 || iz >= D.z) continue;
      for (int ky = 0; ky < 3; ++ky) {
        const int iy = y + ky - 1;
        if (iy < 0 || iy >= D.y) continue;
        for (int kx = 0; kx < 3; ++kx) {
          const int ix = x + kx - 1;
          if (ix < 0 || ix >= D.x) continue;
          const float* wt = w + ((kz * 3 + ky) * 3 + kx) * kIn * 16;
          const int l = lab[n * V + ((long long)iz * D.y + iy) * D.x + ix];
          if (l < 3) {
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[c] += wt[l * 16 + c];
          }
          if (cr.in(ix, iy, iz)) {
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[c] += wt[3 * 16 + c];
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 16; ++c) Y[m * 16 + c] = __float2bfloat16(fmaxf(acc[c], 0.f));
  }
}

// conv1 weight gradient: dW1[tap][l][co] += sum over voxels m whose neighbour at
// tap has label l of dZ1[m][co], and dW1[tap][3][co] over those whose neighbour
// lies in the core (shared-memory partial sums, then global atomics).
__global__ void __launch_bounds__(256) k_conv1_wgrad(const uint8_t* lab, const Core* core, int B, Box3 D,
                                                     const bf16* dZ, float* dW1) {
  __shared__ float acc[27 * kIn * 16];
  for (int t = threadIdx.x; t < 27 * kIn * 16; t += blockDim.x) acc[t] = 0.f;
  __syncthreads();
  const long long V = (long long)D.x * D.y * D.z;
  const long long M = (long long)B * V;
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < M; m += (long long)gridDim.x * blockDim.x) {
    const long long n = m / V;
    const int v = (int)(m - n * V);
    const int z = v / (D.x * D.y), y = (v / D.x) % D.y, x = v % D.x;
    float g[16];
    bool any = false;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      g[c] = __bfloat162float(dZ[m * 16 + c]);
      any |= g[c] != 0.f;
    }
    if (!any) continue;
    const Core cr = core[n];
    for (int tap = 0; tap < 27; ++tap) {
      const int iz = z + tap / 9 - 1, iy = y + (tap / 3) % 3 - 1, ix = x + tap % 3 - 1;
      if (iz < 0 || iz >= D.z || iy < 0 || iy >= D.y || ix < 0 || ix >= D.x) continue;
      const int l = lab[n * V + ((long long)iz * D.y + iy) * D.x + ix];
      if (l < 3) {
#pragma unroll
        for (int c = 0; c < 16; ++c)
          if (g[c] != 0.f) atomicAdd(&acc[(tap * kIn + l) * 16 + c], g[c]);
      }
      if (cr.in(ix, iy, iz)) {
#pragma unroll
        for (int c = 0; c < 16; ++c)
          if (g[c] != 0.f) atomicAdd(&acc[(tap * kIn + 3) * 16 + c], g[c]);
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 27 * kIn * 16; t += blockDim.x)
    if (acc[t] != 0.f) atomicAdd(&dW1[t], acc[t]);
}

// Bias gradient: db[c] += sum over rows of dZ[m][c] (C channels).
__global__ void __launch_bounds__(256) k_bias_grad(const bf16* dZ, long long M, int C, float* db) {
  __shared__ float acc[64];
  for (int t = threadIdx.x; t < C; t += blockDim.x) acc[t] = 0.f;
  __syncthreads();
  const int c = threadIdx.x % C;
  const int rows_per = blockDim.x / C;
  float a = 0.f;
  if ((int)threadIdx.x < rows_per * C)
    for (long long m = blockIdx.x * (long long)rows_per + threadIdx.x / C; m < M; m += (long long)gridDim.x * rows_per)
      a += __bfloat162float(dZ[m * C + c]);
  atomicAdd(&acc[c], a);
  __syncthreads();
  for (int t = threadIdx.x; t < C; t += blockDim.x) atomicAdd(&db[t], acc[t]);
}

// Geometry of one convolution layer: input box Di, output box Do (per axis).
struct Geo {
  Box3 Di, Do;
  int ci, co, s;
};

// ---------------------------------------------------------------------------
// Implicit GEMM on the fifth-generation tensor cores (tcgen05, sm_100 family):
// D[M][N] = sum_k A(m, k) B(n, k), M tile 128, N <= 64 (a multiple of 16),
// K in chunks of 64. Four warps stage each chunk's A (128 x 64) and B (N x 64)
// BF16 tiles into shared memory in the no-swizzle K-major layout of the
// matrix descriptors (8-row x 16-byte core matrices; core (i, j) of rows
// 8i..8i+7 and K elements 8j..8j+7 at byte ((8 i) + j) * 128, so the K step
// between core matrices is 128 bytes and the row-group step 1024 bytes); one
// thread issues the chunk's four 128 x N x 16 MMAs with the FP32 accumulator
// in tensor memory and commits them to the chunk buffer's mbarrier. Two
// chunk buffers: the staging of chunk i + 1 overlaps the MMAs of chunk i.
// The epilogue reads the accumulator back (tcgen05.ld, one row per thread)
// and hands each row to Op::store_row. Every mbarrier wait is bounded (about
// a second of the global timer); a wait that runs out sets *err, and the
// kernel still waits (bounded) for its MMAs before freeing tensor memory.
// blockIdx.y splits K (Op::store_row then accumulates with atomics).
// ---------------------------------------------------------------------------
namespace tc {

constexpr int kChunkK = 64;
constexpr int kABytes = 128 * kChunkK * 2;  // 16 KB
constexpr int kBBytes = 64 * kChunkK * 2;   // 8 KB (N <= 64)
constexpr int kStageBytes = kABytes + kBBytes;
constexpr int kSmemBytes = 2 * kStageBytes + 1024;  // two stages, 1 KB alignment slack
constexpr int kTmemCols = 64;

// Byte offset of the 16-byte segment (row r, K elements 8 k8 .. 8 k8 + 7).
__device__ __forceinline__ uint32_t kmaj(int r, int k8) {
  return (uint32_t)(((((r >> 3) << 3) + k8) << 7) + ((r & 7) << 4));
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);  // start address / 16
  d |= (uint64_t)(128 >> 4) << 16;                  // leading (K) byte offset / 16
  d |= (uint64_t)(1024 >> 4) << 32;                 // stride (row-group) byte offset / 16
  d |= (uint64_t)1 << 46;                           // descriptor version 1; no swizzle, base offset 0
  return d;
}

// kind::f16 instruction descriptor: BF16 A and B, FP32 D, both K-major.
__host__ __device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void cp16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void st_u16(uint32_t addr, unsigned short v) {
  asm volatile("st.shared.u16 [%0], %1;\n" ::"r"(addr), "h"(v) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = gtimer();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (gtimer() - t0 > 1000000000ull) return false;
  }
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

template <class Op>
__global__ void __launch_bounds__(128) k_gemm(Op op, long long M, int N, long long K, long long kper, int* err) {
  extern __shared__ __align__(1024) uint8_t dsm[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tmem_slot;
  const uint32_t base = ((uint32_t)__cvta_generic_to_shared(dsm) + 1023u) & ~1023u;
  const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(&bars[0]);
  const uint32_t bar1 = (uint32_t)__cvta_generic_to_shared(&bars[1]);
  const int warp = threadIdx.x >> 5;
  const long long m0 = (long long)blockIdx.x * 128;
  const long long kb = (long long)blockIdx.y * kper;
  const long long ke = min(K, kb + kper);
  const int nch = ke > kb ? (int)((ke - kb + kChunkK - 1) / kChunkK) : 0;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t id = idesc_bf16(128, N);
  bool ok = true;
  for (int i = 0; i < nch; ++i) {
    const int b = i & 1;
    const uint32_t bar = b ? bar1 : bar0;
    if (i >= 2 && ok) ok = mbar_wait(bar, (uint32_t)((i - 2) >> 1) & 1u);  // this buffer's MMAs are done
    const uint32_t sA = base + (uint32_t)b * kStageBytes, sB = sA + kABytes;
    op.stage(m0, kb + (long long)i * kChunkK, ke, M, N, sA, sB);
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && ok) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
      for (int s = 0; s < kChunkK / 16; ++s)
        mma(tmem, sdesc(sA + 256u * s), sdesc(sB + 256u * s), id, (i > 0 || s > 0) ? 1u : 0u);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                   : "memory");
    }
  }
  if (nch > 0 && ok) ok = mbar_wait((nch - 1) & 1 ? bar1 : bar0, (uint32_t)((nch - 1) >> 1) & 1u);
  ok = __syncthreads_and(ok) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (ok && nch > 0) {
    const long long m = m0 + threadIdx.x;
    float v[64];
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    for (int j = 0; j < N; j += 16) ld16(lane_addr + (uint32_t)j, v + j);
    if (m < M) op.store_row(m, v, N);
  }
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    // bounded wait for the MMAs this block issued before tensor memory is freed
    if (nch > 0) (void)mbar_wait((nch - 1) & 1 ? bar1 : bar0, (uint32_t)((nch - 1) >> 1) & 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// Output voxel m's input voxel at tap (or -1 in the zero padding).
__device__ __forceinline__ long long in_voxel(const Geo& g, long long m, int tap) {
  const long long V = (long long)g.Do.x * g.Do.y * g.Do.z;
  const long long n = m / V;
  const int v = (int)(m - n * V);
  const int iz = (v / (g.Do.x * g.Do.y)) * g.s + tap / 9 - 1;
  const int iy = ((v / g.Do.x) % g.Do.y) * g.s + (tap / 3) % 3 - 1;
  const int ix = (v % g.Do.x) * g.s + tap % 3 - 1;
  if (iz < 0 || iz >= g.Di.z || iy < 0 || iy >= g.Di.y || ix < 0 || ix >= g.Di.x) return -1;
  return ((n * g.Di.z + iz) * g.Di.y + iy) * g.Di.x + ix;
}

// Input voxel m's output voxel reached through tap (or -1): the output
// voxel o with o * s + tap offset - 1 = in(m) on every axis.
__device__ __forceinline__ long long out_voxel(const Geo& g, long long m, int tap) {
  const long long V = (long long)g.Di.x * g.Di.y * g.Di.z;
  const long long n = m / V;
  const int v = (int)(m - n * V);
  int q[3] = {v / (g.Di.x * g.Di.y) + 1 - tap / 9, (v / g.Di.x) % g.Di.y + 1 - (tap / 3) % 3, v % g.Di.x + 1 - tap % 3};
  const int lim[3] = {g.Do.z, g.Do.y, g.Do.x};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (q[d] < 0 || q[d] % g.s) return -1;
    q[d] /= g.s;
    if (q[d] >= lim[d]) return -1;
  }
  return ((n * g.Do.z + q[0]) * g.Do.y + q[1]) * g.Do.x + q[2];
}

// Forward: Y[m][o] = relu(b[o] + sum_{tap, c} X[in(m, tap)][c] W[tap][c][o]);
// A rows = output voxels (16-byte runs of 8 input channels), B rows = o from
// Wt[tap][o][c] (the weights transposed so that c is contiguous).
struct Fwd {
  const bf16* X;
  const bf16* Wt;
  const float* bias;
  bf16* Y;
  Geo g;
  __device__ __forceinline__ void stage(long long m0, long long k0, long long ke, long long M, int N, uint32_t sA,
                                        uint32_t sB) const {
    for (int e = threadIdx.x; e < 128 * 8; e += 128) {
      const int r = e >> 3, k8 = e & 7;
      const long long m = m0 + r, k = k0 + 8 * k8;
      const bf16* src = X;
      int bytes = 0;
      if (m < M && k < ke) {
        const int tap = (int)(k / g.ci), c = (int)(k - (long long)tap * g.ci);
        const long long iv = in_voxel(g, m, tap);
        if (iv >= 0) {
          src = X + iv * g.ci + c;
          bytes = 16;
        }
      }
      cp16(sA + kmaj(r, k8), src, bytes);
    }
    for (int e = threadIdx.x; e < N * 8; e += 128) {
      const int n = e >> 3, k8 = e & 7;
      const long long k = k0 + 8 * k8;
      const bf16* src = Wt;
      int bytes = 0;
      if (k < ke) {
        const int tap = (int)(k / g.ci), c = (int)(k - (long long)tap * g.ci);
        src = Wt + ((long long)tap * g.co + n) * g.ci + c;
        bytes = 16;
      }
      cp16(sB + kmaj(n, k8), src, bytes);
    }
  }
  __device__ __forceinline__ void store_row(long long m, const float* v, int N) const {
    bf16* y = Y + m * g.co;
    for (int n = 0; n < N; n += 2)
      *reinterpret_cast<__nv_bfloat162*>(y + n) =
          __floats2bfloat162_rn(fmaxf(v[n] + bias[n], 0.f), fmaxf(v[n + 1] + bias[n + 1], 0.f));
  }
};

// Data gradient masked by the ReLU of the layer's input:
// dZin[m][c] = [X[m][c] > 0] sum_{tap, o} dZ[out(m, tap)][o] W[tap][c][o];
// A rows = input voxels (runs of 8 output channels of dZ), B rows = c
// (runs of 8 o of W[tap][c][.], contiguous in the parameter layout).
struct Dgrad {
  const bf16* dZ;
  const bf16* W;
  const bf16* X;
  bf16* dZin;
  Geo g;
  __device__ __forceinline__ void stage(long long m0, long long k0, long long ke, long long M, int N, uint32_t sA,
                                        uint32_t sB) const {
    for (int e = threadIdx.x; e < 128 * 8; e += 128) {
      const int r = e >> 3, k8 = e & 7;
      const long long m = m0 + r, k = k0 + 8 * k8;
      const bf16* src = dZ;
      int bytes = 0;
      if (m < M && k < ke) {
        const int tap = (int)(k / g.co), o = (int)(k - (long long)tap * g.co);
        const long long ov = out_voxel(g, m, tap);
        if (ov >= 0) {
          src = dZ + ov * g.co + o;
          bytes = 16;
        }
      }
      cp16(sA + kmaj(r, k8), src, bytes);
    }
    for (int e = threadIdx.x; e < N * 8; e += 128) {
      const int n = e >> 3, k8 = e & 7;
      const long long k = k0 + 8 * k8;
      const bf16* src = W;
      int bytes = 0;
      if (k < ke) {
        const int tap = (int)(k / g.co), o = (int)(k - (long long)tap * g.co);
        src = W + ((long long)tap * g.ci + n) * g.co + o;
        bytes = 16;
      }
      cp16(sB + kmaj(n, k8), src, bytes);
    }
  }
  __device__ __forceinline__ void store_row(long long m, const float* v, int N) const {
    const bf16* x = X + m * g.ci;
    bf16* d = dZin + m * g.ci;
    for (int n = 0; n < N; ++n) d[n] = __float2bfloat16(__bfloat162float(x[n]) > 0.f ? v[n] : 0.f);
  }
};

// Weight gradient: dW[tap][c][o] += sum_m X[in(m, tap)][c] dZ[m][o]; rows
// r = tap * ci + c, K = output voxels m. Both operands run along the
// channels in memory, so each 16-byte load (8 channels of one voxel) is
// written to shared memory transposed, one BF16 element per K position.
struct Wgrad {
  const bf16* X;
  const bf16* dZ;
  float* dW;
  Geo g;
  __device__ __forceinline__ void stage(long long r0, long long k0, long long ke, long long M, int N, uint32_t sA,
                                        uint32_t sB) const {
    for (int e = threadIdx.x; e < 16 * kChunkK; e += 128) {
      const int r8 = e / kChunkK, kl = e - r8 * kChunkK;  // rows 8 r8 .. 8 r8 + 7 at K position kl
      const long long r = r0 + 8 * r8, m = k0 + kl;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (r < M && m < ke) {
        const int tap = (int)(r / g.ci), c = (int)(r - (long long)tap * g.ci);
        const long long iv = in_voxel(g, m, tap);
        if (iv >= 0) val = *reinterpret_cast<const uint4*>(X + iv * g.ci + c);
      }
      const unsigned short* h = reinterpret_cast<const unsigned short*>(&val);
#pragma unroll
      for (int j = 0; j < 8; ++j) st_u16(sA + kmaj(8 * r8 + j, kl >> 3) + ((kl & 7) << 1), h[j]);
    }
    for (int e = threadIdx.x; e < (N / 8) * kChunkK; e += 128) {
      const int n8 = e / kChunkK, kl = e - n8 * kChunkK;
      const long long m = k0 + kl;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (m < ke) val = *reinterpret_cast<const uint4*>(dZ + m * g.co + 8 * n8);
      const unsigned short* h = reinterpret_cast<const unsigned short*>(&val);
#pragma unroll
      for (int j = 0; j < 8; ++j) st_u16(sB + kmaj(8 * n8 + j, kl >> 3) + ((kl & 7) << 1), h[j]);
    }
  }
  __device__ __forceinline__ void store_row(long long r, const float* v, int N) const {
    float* d = dW + r * g.co;
    for (int n = 0; n < N; ++n)
      if (v[n] != 0.f) atomicAdd(d + n, v[n]);
  }
};

}  // namespace tc

// Wt[tap][o][c] = W[tap][c][o] (BF16), the forward pass's B operand layout.
__global__ void k_transpose_w(const bf16* W, bf16* Wt, int ci, int co) {
  const int n = 27 * ci * co;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int tap = i / (ci * co), rem = i - tap * ci * co, c = rem / co, o = rem - c * co;
    Wt[((long long)tap * co + o) * ci + c] = W[i];
  }
}

// ---------------------------------------------------------------------------
// Head: mean pool, fc1 + ReLU, fc2 (one block per sample, FP32).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_head_fwd(const bf16* Y4, int V4, const float* W5, const float* b5,
                                                  const float* W6, const float* b6, float* h0, float* h1,
                                                  float* out) {
  __shared__ float s0[kPoolC], s1[kHid], part[128];
  const int n = blockIdx.x;
  const bf16* y = Y4 + (long long)n * V4 * kPoolC;
  // pool: thread t sums channel t % 64 over voxels of parity t / 64
  {
    const int c = threadIdx.x % kPoolC, h = threadIdx.x / kPoolC;
    float a = 0.f;
    for (int v = h; v < V4; v += 2) a += __bfloat162float(y[(long long)v * kPoolC + c]);
    part[threadIdx.x] = a;
  }
  __syncthreads();
  if (threadIdx.x < kPoolC) s0[threadIdx.x] = (part[threadIdx.x] + part[threadIdx.x + kPoolC]) / float(V4);
  __syncthreads();
  if (threadIdx.x < kHid) {
    float a = b5[threadIdx.x];
    for (int i = 0; i < kPoolC; ++i) a += s0[i] * W5[i * kHid + threadIdx.x];
    s1[threadIdx.x] = fmaxf(a, 0.f);
  }
  __syncthreads();
  if (threadIdx.x < kOut) {
    float a = b6[threadIdx.x];
    for (int i = 0; i < kHid; ++i) a += s1[i] * W6[i * kOut + threadIdx.x];
    out[n * kOut + threadIdx.x] = a;
  }
  if (threadIdx.x < kPoolC) h0[n * kPoolC + threadIdx.x] = s0[threadIdx.x];
  if (threadIdx.x < kHid) h1[n * kHid + threadIdx.x] = s1[threadIdx.x];
}

// Loss gradient and head backward: dout = 2 (out - t) / (B * 21); fc2 and fc1
// weight and bias gradients (atomics over the batch); dZ4 = dpool masked by
// conv4's ReLU. loss_part[n] = |out - t|^2.
__global__ void __launch_bounds__(128) k_head_bwd(const bf16* Y4, int V4, int B, const float* W5, const float* W6,
                                                  const float* h0, const float* h1, const float* out,
                                                  const float* tgt, float* dW5, float* db5, float* dW6, float* db6,
                                                  bf16* dZ4, double* loss_part) {
  __shared__ float dout[kOut], dh1[kHid], dh0[kPoolC];
  const int n = blockIdx.x;
  if (threadIdx.x < kOut) {
    const float r = out[n * kOut + threadIdx.x] - tgt[n * kOut + threadIdx.x];
    dout[threadIdx.x] = 2.f * r / float(B * kOut);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double l = 0.0;
    for (int i = 0; i < kOut; ++i) {
      const double r = (double)out[n * kOut + i] - (double)tgt[n * kOut + i];
      l += r * r;
    }
    loss_part[n] = l;
  }
  for (int e = threadIdx.x; e < kHid * kOut; e += blockDim.x) {
    const int i = e / kOut, j = e % kOut;
    atomicAdd(&dW6[e], h1[n * kHid + i] * dout[j]);
  }
  if (threadIdx.x < kOut) atomicAdd(&db6[threadIdx.x], dout[threadIdx.x]);
  if (threadIdx.x < kHid) {
    float a = 0.f;
    for (int j = 0; j < kOut; ++j) a += W6[threadIdx.x * kOut + j] * dout[j];
    dh1[threadIdx.x] = h1[n * kHid + threadIdx.x] > 0.f ? a : 0.f;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kPoolC * kHid; e += blockDim.x) {
    const int i = e / kHid, j = e % kHid;
    atomicAdd(&dW5[e], h0[n * kPoolC + i] * dh1[j]);
  }
  if (threadIdx.x < kHid) atomicAdd(&db5[threadIdx.x], dh1[threadIdx.x]);
  if (threadIdx.x < kPoolC) {
    float a = 0.f;
    for (int j = 0; j < kHid; ++j) a += W5[threadIdx.x * kHid + j] * dh1[j];
    dh0[threadIdx.x] = a / float(V4);
  }
  __syncthreads();
  const bf16* y = Y4 + (long long)n * V4 * kPoolC;
  bf16* dz = dZ4 + (long long)n * V4 * kPoolC;
  for (int e = threadIdx.x; e < V4 * kPoolC; e += blockDim.x)
    dz[e] = __float2bfloat16(__bfloat162float(y[e]) > 0.f ? dh0[e % kPoolC] : 0.f);
}

// Adam (Kingma and Ba) with bias correction; refreshes the BF16 weight copy.
__global__ void k_adam(float* theta, const float* grad, float* m, float* v, long long n, float lr, float c1, float c2,
                       bf16* theta16) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float th = theta[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    theta[i] = th;
    theta16[i] = __float2bfloat16(th);
  }
}

__global__ void k_to_bf16(const float* a, bf16* b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16(a[i]);
}

// Scale the network outputs (normalised stiffness) to GPa.
__global__ void k_scale(const float* a, float s, float* b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = a[i] * s;
}

// ---------------------------------------------------------------------------
// Gate: one block per subimage. Phase fractions of the core -> Reuss and
// Voigt bounds of K and G; each member's Voigt-projected K, G must lie
// inside; the relative
// spread (max - min) / mean of K and of G must be <= spread; the mean
// stiffness must be positive definite (Cholesky, FP64).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void kg_of(const double* c21, double& K, double& G) {
  // upper-triangle index of (i, j), i <= j
  auto at = [&](int i, int j) { return c21[i * 6 - i * (i - 1) / 2 + (j - i)]; };
  K = (at(0, 0) + at(1, 1) + at(2, 2) + 2.0 * (at(0, 1) + at(0, 2) + at(1, 2))) / 9.0;
  G = (at(0, 0) + at(1, 1) + at(2, 2) - (at(0, 1) + at(0, 2) + at(1, 2)) + 3.0 * (at(3, 3) + at(4, 4) + at(5, 5))) /
      15.0;
}

__global__ void __launch_bounds__(256) k_gate(const uint8_t* lab, Box3 D, const Core* core, const double* ph,
                                              int nphase, const float* members, int E, double spread, int* accept,
                                              double* c21_out) {
  __shared__ unsigned int cnt[256];
  const int n = blockIdx.x;
  const long long V = (long long)D.x * D.y * D.z;
  const Core cr = core[n];
  const long long Vc = (long long)cr.nx * cr.ny * cr.nz;
  for (int t = threadIdx.x; t < 256; t += blockDim.x) cnt[t] = 0;
  __syncthreads();
  for (long long v = threadIdx.x; v < Vc; v += blockDim.x) {
    const int x = (int)(v % cr.nx), y = (int)((v / cr.nx) % cr.ny), z = (int)(v / ((long long)cr.nx * cr.ny));
    atomicAdd(&cnt[lab[n * V + ((long long)(cr.oz + z) * D.y + (cr.oy + y)) * D.x + (cr.ox + x)]], 1u);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double sKf = 0, sKr = 0, sGf = 0, sGr = 0;
  bool badlab = false;
  for (int p = 0; p < 256; ++p) {
    if (!cnt[p]) continue;
    if (p >= nphase) {
      badlab = true;
      break;
    }
    const double f = double(cnt[p]) / double(Vc);
    sKf += f * ph[2 * p];
    sKr += f / ph[2 * p];
    sGf += f * ph[2 * p + 1];
    sGr += f / ph[2 * p + 1];
  }
  const double KV = sKf, KR = 1.0 / sKr, GV = sGf, GR = 1.0 / sGr;
  double mean[21];
  for (int i = 0; i < 21; ++i) mean[i] = 0.0;
  double Kmin = 1e300, Kmax = -1e300, Gmin = 1e300, Gmax = -1e300, Ks = 0, Gs = 0;
  bool ok = !badlab;
  for (int e = 0; e < E; ++e) {
    double c[21];
    for (int i = 0; i < 21; ++i) {
      c[i] = members[((long long)n * E + e) * 21 + i];
      mean[i] += c[i] / E;
    }
    double K, G;
    kg_of(c, K, G);
    ok = ok && K >= KR && K <= KV && G >= GR && G <= GV;
    Kmin = fmin(Kmin, K);
    Kmax = fmax(Kmax, K);
    Gmin = fmin(Gmin, G);
    Gmax = fmax(Gmax, G);
    Ks += K / E;
    Gs += G / E;
  }
  ok = ok && (Kmax - Kmin) <= spread * Ks && (Gmax - Gmin) <= spread * Gs;
  // Cholesky of the mean (Voigt form; same definiteness as the Mandel form)
  double A[6][6];
  for (int i = 0, t = 0; i < 6; ++i)
    for (int j = i; j < 6; ++j, ++t) A[i][j] = A[j][i] = mean[t];
  for (int j = 0; j < 6 && ok; ++j) {
    double d = A[j][j];
    for (int k = 0; k < j; ++k) d -= A[j][k] * A[j][k];
    if (!(d > 0.0)) {
      ok = false;
      break;
    }
    d = sqrt(d);
    A[j][j] = d;
    for (int i = j + 1; i < 6; ++i) {
      double s = A[i][j];
      for (int k = 0; k < j; ++k) s -= A[i][k] * A[j][k];
      A[i][j] = s / d;
    }
  }
  accept[n] = ok ? 1 : 0;
  for (int i = 0; i < 21; ++i) c21_out[(long long)n * 21 + i] = mean[i];
}

// ---------------------------------------------------------------------------
// Host side: device workspace of one batch and the passes over it.
// ---------------------------------------------------------------------------
#define CNN_CK(x)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (x);                                                                  \
    if (e_ != cudaSuccess) {                                                               \
      err = std::string(#x) + ": " + cudaGetErrorString(e_);                               \
      return HH_ERR_CUDA;                                                                  \
    }                                                                                      \
  } while (0)

struct Net {
  cudaStream_t st = nullptr;
  int B = 0;
  Box3 dims[5];  // box before conv1 .. after conv4
  Offsets off;
  std::string err;
  std::vector<void*> allocs;
  float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  bf16* theta16 = nullptr;
  bf16* theta16t = nullptr;  // conv weights as Wt[tap][co][ci] (the forward pass's B operand)
  int* terr = nullptr;       // set by a tensor-core GEMM whose bounded wait ran out
  uint8_t* lab = nullptr;
  Core* core = nullptr;
  bf16* act[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // act[i]: output of conv i (1-based)
  bf16* dact[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // gradient at conv i's output (pre-ReLU)
  float *h0 = nullptr, *h1 = nullptr, *out = nullptr, *tgt = nullptr;
  double* loss_part = nullptr;
  long long launches = 0;

  ~Net() {
    for (void* p : allocs) cudaFree(p);
  }
  template <typename T>
  hh_status alloc(T** p, long long n) {
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<long long>(n, 1) * sizeof(T)) != cudaSuccess) {
      (void)cudaGetLastError();
      err = "device allocation failed";
      return HH_ERR_OOM;
    }
    allocs.push_back(q);
    *p = reinterpret_cast<T*>(q);
    return HH_OK;
  }

  static long long vox(const Box3& b) { return (long long)b.x * b.y * b.z; }

  // workspace for batches of up to `batch` samples of box `box`; with `shared`
  // the parameters, their gradient and Adam's moments are those of `shared`
  hh_status init(cudaStream_t s, int batch, Box3 box, bool train, const Net* shared = nullptr) {
    st = s;
    B = batch;
    off = offsets();
    dims[0] = box;
    for (int i = 0; i < 4; ++i)
      dims[i + 1] = Box3{out_size(dims[i].x, kConv[i].stride), out_size(dims[i].y, kConv[i].stride),
                         out_size(dims[i].z, kConv[i].stride)};
    hh_status r;
    if (shared) {
      theta = shared->theta;
      theta16 = shared->theta16;
      theta16t = shared->theta16t;
      terr = shared->terr;
      grad = shared->grad;
      m = shared->m;
      v = shared->v;
    } else if ((r = alloc(&theta, off.total)) || (r = alloc(&theta16, off.total)) ||
               (r = alloc(&theta16t, off.total)) || (r = alloc(&terr, 1))) {
      return r;
    } else if (cudaMemsetAsync(terr, 0, sizeof(int), st) != cudaSuccess) {
      err = "device memset failed";
      return HH_ERR_CUDA;
    }
    if ((r = alloc(&lab, B * vox(box))) ||
        (r = alloc(&core, B)) || (r = alloc(&h0, (long long)B * kPoolC)) || (r = alloc(&h1, (long long)B * kHid)) ||
        (r = alloc(&out, (long long)B * kOut)) || (r = alloc(&tgt, (long long)B * kOut)) ||
        (r = alloc(&loss_part, B)))
      return r;
    for (int i = 1; i <= 4; ++i) {
      const long long n = (long long)B * vox(dims[i]) * kConv[i - 1].co;
      if ((r = alloc(&act[i], n))) return r;
      if (train && (r = alloc(&dact[i], n))) return r;
    }
    if (train && !shared &&
        ((r = alloc(&grad, off.total)) || (r = alloc(&m, off.total)) || (r = alloc(&v, off.total))))
      return r;
    return HH_OK;
  }

  hh_status set_params(const float* host) {
    CNN_CK(cudaMemcpyAsync(theta, host, off.total * sizeof(float), cudaMemcpyHostToDevice, st));
    ++launches;
    k_to_bf16<<<256, 256, 0, st>>>(theta, theta16, off.total);
    CNN_CK(cudaGetLastError());
    return HH_OK;
  }

  // tensor-core implicit GEMM: M rows in tiles of 128, N (16, 32 or 64)
  // columns, K split over `splits` blocks in whole chunks of 64
  template <class Op>
  hh_status gemm(const Op& op, long long M, int N, long long K, int splits = 1) {
    if (N < 16 || N > 64 || N % 16) {
      err = "surrogate: GEMM width outside 16..64";
      return HH_ERR_UNSUPPORTED;
    }
    const long long kper = ((K + splits - 1) / splits + tc::kChunkK - 1) / tc::kChunkK * tc::kChunkK;
    const int sp = (int)((K + kper - 1) / kper);
    CNN_CK(cudaFuncSetAttribute(tc::k_gemm<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes));
    dim3 grid((unsigned)((M + 127) / 128), (unsigned)sp);
    ++launches;
    tc::k_gemm<Op><<<grid, 128, tc::kSmemBytes, st>>>(op, M, N, K, kper, terr);
    CNN_CK(cudaGetLastError());
    return HH_OK;
  }

  // after a synchronization: HH_ERR_DEVICE_TIMEOUT if a GEMM's wait ran out
  hh_status timeout_check() {
    int e = 0;
    CNN_CK(cudaMemcpyAsync(&e, terr, sizeof(int), cudaMemcpyDeviceToHost, st));
    CNN_CK(cudaStreamSynchronize(st));
    if (e) {
      err = "surrogate: a tensor-core GEMM's mbarrier wait ran out";
      return HH_ERR_DEVICE_TIMEOUT;
    }
    return HH_OK;
  }

  Geo geo(int i) const { return Geo{dims[i], dims[i + 1], kConv[i].ci, kConv[i].co, kConv[i].stride}; }

  // forward of nb <= B samples already in lab and core
  hh_status forward(int nb) {
    const long long V1 = vox(dims[1]);
    ++launches;
    k_conv1_fwd<<<(unsigned)std::min<long long>(4096, (nb * V1 + 255) / 256), 256, 0, st>>>(
        lab, core, nb, dims[0], theta + off.w[0], theta + off.b[0], act[1]);
    CNN_CK(cudaGetLastError());
    for (int i = 1; i < 4; ++i) {
      ++launches;
      k_transpose_w<<<64, 256, 0, st>>>(theta16 + off.w[i], theta16t + off.w[i], kConv[i].ci, kConv[i].co);
      CNN_CK(cudaGetLastError());
    }
    for (int i = 1; i < 4; ++i) {
      const Geo g = geo(i);
      const long long M = nb * vox(g.Do);
      tc::Fwd op{act[i], theta16t + off.w[i], theta + off.b[i], act[i + 1], g};
      hh_status r = gemm(op, M, g.co, 27LL * g.ci);
      if (r) return r;
    }
    const int V4 = (int)vox(dims[4]);
    ++launches;
    k_head_fwd<<<nb, 128, 0, st>>>(act[4], V4, theta + off.w[4], theta + off.b[4], theta + off.w[5],
                                   theta + off.b[5], h0, h1, out);
    CNN_CK(cudaGetLastError());
    return HH_OK;
  }

  // gradients of the loss of nb samples (of a mean over `total` samples) added
  // to grad (zeroed by the caller); needs tgt
  hh_status backward(int nb, int total) {
    const int V4 = (int)vox(dims[4]);
    ++launches;
    k_head_bwd<<<nb, 128, 0, st>>>(act[4], V4, total, theta + off.w[4], theta + off.w[5], h0, h1, out, tgt,
                                   grad + off.w[4], grad + off.b[4], grad + off.w[5], grad + off.b[5], dact[4],
                                   loss_part);
    CNN_CK(cudaGetLastError());
    for (int i = 3; i >= 1; --i) {
      const Geo g = geo(i);
      const long long Mo = nb * vox(g.Do);
      const long long Mi = nb * vox(g.Di);
      // weight and bias gradients of conv i+1 (0-based i)
      const int splits = (int)std::min<long long>(64, std::max<long long>(1, Mo / 4096));
      tc::Wgrad ow{act[i], dact[i + 1], grad + off.w[i], g};
      hh_status r = gemm(ow, 27LL * g.ci, g.co, Mo, splits);
      if (r) return r;
      ++launches;
      k_bias_grad<<<(unsigned)std::min<long long>(1024, (Mo + 63) / 64), 256, 0, st>>>(dact[i + 1], Mo, g.co,
                                                                                      grad + off.b[i]);
      CNN_CK(cudaGetLastError());
      // gradient at the layer's input, masked by the previous ReLU
      tc::Dgrad od{dact[i + 1], theta16 + off.w[i], act[i], dact[i], g};
      if ((r = gemm(od, Mi, g.ci, 27LL * g.co))) return r;
    }
    const long long V1 = vox(dims[1]);
    ++launches;
    k_conv1_wgrad<<<(unsigned)std::min<long long>(2048, (nb * V1 + 255) / 256), 256, 0, st>>>(
        lab, core, nb, dims[0], dact[1], grad + off.w[0]);
    CNN_CK(cudaGetLastError());
    ++launches;
    k_bias_grad<<<(unsigned)std::min<long long>(1024, (nb * V1 + 63) / 64), 256, 0, st>>>(dact[1], nb * V1, 16,
                                                                                         grad + off.b[0]);
    CNN_CK(cudaGetLastError());
    return HH_OK;
  }
};

// One subimage of a call: its box, its core inside the box and the offset of
// its labels in the concatenated input. Subimages of one box shape are
// batched together (`groups`, in the order the shapes first appear).
struct Sub {
  Box3 box;
  Core core;
  long long off;
};

static bool same_box(const Box3& a, const Box3& b) { return a.x == b.x && a.y == b.y && a.z == b.z; }

hh_status parse_subs(hh_ctx* h, int count, const int32_t* boxes, std::vector<Sub>& subs,
                     std::vector<std::vector<int>>& groups) {
  if (count < 1 || !boxes) return ctx_fail(h, HH_ERR_ARG, "surrogate: count >= 1 and a box table");
  subs.resize(count);
  groups.clear();
  long long off = 0;
  for (int i = 0; i < count; ++i) {
    const int32_t* r = boxes + 9 * (long long)i;
    Sub& u = subs[i];
    u.box = Box3{r[0], r[1], r[2]};
    u.core = Core{r[3], r[4], r[5], r[6], r[7], r[8]};
    const bool ok = u.box.x >= 8 && u.box.x <= 256 && u.box.y >= 8 && u.box.y <= 256 && u.box.z >= 8 &&
                    u.box.z <= 256 && u.core.nx >= 1 && u.core.ny >= 1 && u.core.nz >= 1 && u.core.ox >= 0 &&
                    u.core.oy >= 0 && u.core.oz >= 0 && u.core.ox + u.core.nx <= u.box.x &&
                    u.core.oy + u.core.ny <= u.box.y && u.core.oz + u.core.nz <= u.box.z;
    if (!ok)
      return ctx_fail(h, HH_ERR_ARG,
                      ("surrogate: subimage " + std::to_string(i) +
                       ": box edges 8..256 and a core of at least one voxel inside the box").c_str());
    u.off = off;
    off += Net::vox(u.box);
    int g = 0;
    while (g < (int)groups.size() && !same_box(subs[groups[g][0]].box, u.box)) ++g;
    if (g == (int)groups.size()) groups.emplace_back();
    groups[g].push_back(i);
  }
  return HH_OK;
}

// Stages samples ids[0..n) of a group (labels and cores) into the workspace.
static hh_status stage(Net& net, const uint8_t* labels, const std::vector<Sub>& subs, const int* ids, int n,
                       std::vector<uint8_t>& lab_h, std::vector<Core>& core_h) {
  const long long V = Net::vox(subs[ids[0]].box);
  lab_h.resize((size_t)n * V);
  core_h.resize(n);
  for (int j = 0; j < n; ++j) {
    std::memcpy(lab_h.data() + (size_t)j * V, labels + subs[ids[j]].off, (size_t)V);
    core_h[j] = subs[ids[j]].core;
  }
  if (cudaMemcpyAsync(net.lab, lab_h.data(), (size_t)n * V, cudaMemcpyHostToDevice, net.st) != cudaSuccess ||
      cudaMemcpyAsync(net.core, core_h.data(), n * sizeof(Core), cudaMemcpyHostToDevice, net.st) != cudaSuccess ||
      cudaStreamSynchronize(net.st) != cudaSuccess) {
    net.err = "surrogate: staging copy failed";
    return HH_ERR_CUDA;
  }
  return HH_OK;
}

}  // namespace cnn
}  // namespace hh

using namespace hh;
using namespace hh::cnn;

extern "C" int64_t hh_cnn_num_params(void) { return offsets().total; }

extern "C" hh_status hh_cnn_init_params(uint64_t seed, float* params) {
  if (!params) return ctx_fail(nullptr, HH_ERR_ARG, "hh_cnn_init_params: NULL params");
  const Offsets o = offsets();
  for (long long i = 0; i < o.total; ++i) params[i] = 0.f;
  // the i-th SplitMix64 output (Steele, Lea and Flood 2014) of `seed` as a
  // double in [0, 1) from its top 53 bits
  auto draw = [&](long long i) {
    uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-53;
  };
  for (int l = 0; l < 6; ++l) {
    const long long fan_in = l < 4 ? 27LL * kConv[l].ci : kFc[l - 4][0];
    const long long n = l < 4 ? 27LL * kConv[l].ci * kConv[l].co : (long long)kFc[l - 4][0] * kFc[l - 4][1];
    const double bound = std::sqrt(6.0 / double(fan_in));
    for (long long i = o.w[l]; i < o.w[l] + n; ++i) params[i] = float((2.0 * draw(i) - 1.0) * bound);
  }
  return HH_OK;
}

extern "C" hh_status hh_cnn_forward(hh_ctx* h, const uint8_t* labels, int count, const int32_t* boxes,
                                   const float* params, float* out) {
  if (!h || !labels || !params || !out) return ctx_fail(h, HH_ERR_ARG, "hh_cnn_forward: NULL argument");
  std::vector<Sub> subs;
  std::vector<std::vector<int>> groups;
  hh_status s = parse_subs(h, count, boxes, subs, groups);
  if (s) return s;
  if ((s = ctx_enter(h))) return s;
  std::vector<uint8_t> lab_h;
  std::vector<Core> core_h;
  std::vector<float> o((size_t)64 * kOut);
  for (const std::vector<int>& g : groups) {
    const int B = std::min((int)g.size(), 64);
    Net net;
    if ((s = net.init(ctx_stream(h), B, subs[g[0]].box, false)) || (s = net.set_params(params)))
      return ctx_fail(h, s, net.err.c_str());
    for (int b0 = 0; b0 < (int)g.size(); b0 += B) {
      const int nb = std::min(B, (int)g.size() - b0);
      if ((s = stage(net, labels, subs, g.data() + b0, nb, lab_h, core_h)) || (s = net.forward(nb)))
        return ctx_fail(h, s, net.err.c_str());
      if (cudaMemcpyAsync(o.data(), net.out, (size_t)nb * kOut * sizeof(float), cudaMemcpyDeviceToHost, net.st) !=
              cudaSuccess ||
          cudaStreamSynchronize(net.st) != cudaSuccess)
        return ctx_fail(h, HH_ERR_CUDA, "surrogate forward failed");
      if ((s = net.timeout_check())) return ctx_fail(h, s, net.err.c_str());
      for (int j = 0; j < nb; ++j) std::memcpy(out + (size_t)g[b0 + j] * kOut, o.data() + (size_t)j * kOut, kOut * 4);
    }
  }
  return HH_OK;
}

extern "C" hh_status hh_cnn_loss_grad(hh_ctx* h, const uint8_t* labels, int count, const int32_t* boxes,
                                     const float* params, const float* targets, double* loss, float* grad) {
  if (!h || !labels || !params || !targets || !loss || !grad)
    return ctx_fail(h, HH_ERR_ARG, "hh_cnn_loss_grad: NULL argument");
  std::vector<Sub> subs;
  std::vector<std::vector<int>> groups;
  hh_status s = parse_subs(h, count, boxes, subs, groups);
  if (s) return s;
  if ((s = ctx_enter(h))) return s;
  Net par;  // the parameters and their gradient, shared by the shape groups
  if ((s = par.init(ctx_stream(h), 1, Box3{8, 8, 8}, true)) || (s = par.set_params(params)))
    return ctx_fail(h, s, par.err.c_str());
  if (cudaMemsetAsync(par.grad, 0, par.off.total * sizeof(float), par.st) != cudaSuccess)
    return ctx_fail(h, HH_ERR_CUDA, "surrogate gradients: memset failed");
  std::vector<uint8_t> lab_h;
  std::vector<Core> core_h;
  double l = 0.0;
  for (const std::vector<int>& g : groups) {
    const int n = (int)g.size();
    Net net;
    if ((s = net.init(par.st, n, subs[g[0]].box, true, &par)) || (s = stage(net, labels, subs, g.data(), n, lab_h, core_h)))
      return ctx_fail(h, s, net.err.c_str());
    std::vector<float> t((size_t)n * kOut);
    for (int j = 0; j < n; ++j) std::memcpy(t.data() + (size_t)j * kOut, targets + (size_t)g[j] * kOut, kOut * 4);
    std::vector<double> lp(n);
    if (cudaMemcpyAsync(net.tgt, t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice, net.st) != cudaSuccess)
      return ctx_fail(h, HH_ERR_CUDA, "surrogate gradients: copy failed");
    if ((s = net.forward(n)) || (s = net.backward(n, count))) return ctx_fail(h, s, net.err.c_str());
    if (cudaMemcpyAsync(lp.data(), net.loss_part, n * sizeof(double), cudaMemcpyDeviceToHost, net.st) != cudaSuccess ||
        cudaStreamSynchronize(net.st) != cudaSuccess)
      return ctx_fail(h, HH_ERR_CUDA, "surrogate gradients failed");
    for (double x : lp) l += x;
  }
  if (cudaMemcpyAsync(grad, par.grad, par.off.total * sizeof(float), cudaMemcpyDeviceToHost, par.st) != cudaSuccess ||
      cudaStreamSynchronize(par.st) != cudaSuccess)
    return ctx_fail(h, HH_ERR_CUDA, "surrogate gradients failed");
  if ((s = par.timeout_check())) return ctx_fail(h, s, par.err.c_str());
  *loss = l / (double(count) * kOut);
  return HH_OK;
}

// Host shuffle: SplitMix64 stream (Steele, Lea and Flood 2014) driving a
// Fisher-Yates permutation.
static uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

extern "C" hh_status hh_surrogate_train(hh_ctx* h, const uint8_t* labels, int count, const int32_t* boxes,
                                       const float* targets, const float* init, int epochs, int batch, double lr,
                                       uint64_t seed, float* params_out, double* loss_history) {
  if (!h || !labels || !targets || !init || !params_out || epochs < 1 || batch < 1 || !(lr > 0.0))
    return ctx_fail(h, HH_ERR_ARG, "hh_surrogate_train: NULL argument, epochs < 1, batch < 1 or lr <= 0");
  std::vector<Sub> subs;
  std::vector<std::vector<int>> groups;
  hh_status s = parse_subs(h, count, boxes, subs, groups);
  if (s) return s;
  if ((s = ctx_enter(h))) return s;
  const cudaStream_t st = ctx_stream(h);
  Net par;  // parameters, gradient and Adam's moments, shared by the shape groups
  if ((s = par.init(st, 1, Box3{8, 8, 8}, true)) || (s = par.set_params(init))) return ctx_fail(h, s, par.err.c_str());
  if (cudaMemsetAsync(par.m, 0, par.off.total * sizeof(float), st) != cudaSuccess ||
      cudaMemsetAsync(par.v, 0, par.off.total * sizeof(float), st) != cudaSuccess)
    return ctx_fail(h, HH_ERR_CUDA, "surrogate training: setup failed");
  // per shape group: a workspace for its minibatches (min(batch, group size)
  // subimages, whole batches only) and the group's labels, cores and targets
  const int G = (int)groups.size();
  std::vector<Net> nets(G);
  std::vector<uint8_t*> all_lab(G);
  std::vector<Core*> all_core(G);
  std::vector<float*> all_tgt(G);
  std::vector<int> Bg(G), nbat(G);
  long long per_epoch = 0;
  std::vector<uint8_t> lab_h;
  std::vector<Core> core_h;
  for (int g = 0; g < G; ++g) {
    const std::vector<int>& ids = groups[g];
    const int n = (int)ids.size();
    const long long V = Net::vox(subs[ids[0]].box);
    Bg[g] = std::min(batch, n);
    nbat[g] = n / Bg[g];
    per_epoch += nbat[g];
    Net& net = nets[g];
    if ((s = net.init(st, Bg[g], subs[ids[0]].box, true, &par)) || (s = net.alloc(&all_lab[g], n * V)) ||
        (s = net.alloc(&all_core[g], n)) || (s = net.alloc(&all_tgt[g], (long long)n * kOut)))
      return ctx_fail(h, s, net.err.c_str());
    lab_h.resize((size_t)n * V);
    core_h.resize(n);
    std::vector<float> t((size_t)n * kOut);
    for (int j = 0; j < n; ++j) {
      std::memcpy(lab_h.data() + (size_t)j * V, labels + subs[ids[j]].off, (size_t)V);
      core_h[j] = subs[ids[j]].core;
      std::memcpy(t.data() + (size_t)j * kOut, targets + (size_t)ids[j] * kOut, kOut * 4);
    }
    if (cudaMemcpyAsync(all_lab[g], lab_h.data(), lab_h.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(all_core[g], core_h.data(), n * sizeof(Core), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(all_tgt[g], t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return ctx_fail(h, HH_ERR_CUDA, "surrogate training: setup failed");
  }
  std::vector<std::vector<int>> perm(G);
  for (int g = 0; g < G; ++g) {
    perm[g].resize(groups[g].size());
    for (size_t i = 0; i < perm[g].size(); ++i) perm[g][i] = (int)i;
  }
  uint64_t rs = seed;
  std::vector<double> lp(batch);
  long long step = 0;
  const long long total_steps = (long long)epochs * per_epoch;
  for (int ep = 0; ep < epochs; ++ep) {
    // a seeded permutation of every group, and a seeded order of the
    // epoch's minibatches over the groups
    for (int g = 0; g < G; ++g)
      for (int i = (int)perm[g].size() - 1; i > 0; --i)
        std::swap(perm[g][i], perm[g][(int)(splitmix64(rs) % (uint64_t)(i + 1))]);
    std::vector<std::pair<int, int>> order;
    for (int g = 0; g < G; ++g)
      for (int b = 0; b < nbat[g]; ++b) order.emplace_back(g, b);
    for (int i = (int)order.size() - 1; i > 0; --i)
      std::swap(order[i], order[(int)(splitmix64(rs) % (uint64_t)(i + 1))]);
    double ep_loss = 0.0;
    long long ep_n = 0;
    for (const std::pair<int, int>& gb : order) {
      const int g = gb.first, B = Bg[g];
      Net& net = nets[g];
      const long long V = Net::vox(net.dims[0]);
      for (int j = 0; j < B; ++j) {
        const int k = perm[g][gb.second * B + j];
        if (cudaMemcpyAsync(net.lab + j * V, all_lab[g] + k * V, V, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(net.core + j, all_core[g] + k, sizeof(Core), cudaMemcpyDeviceToDevice, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(net.tgt + j * kOut, all_tgt[g] + (long long)k * kOut, kOut * sizeof(float),
                            cudaMemcpyDeviceToDevice, st) != cudaSuccess)
          return ctx_fail(h, HH_ERR_CUDA, "surrogate training: batch copy failed");
      }
      if (cudaMemsetAsync(par.grad, 0, par.off.total * sizeof(float), st) != cudaSuccess)
        return ctx_fail(h, HH_ERR_CUDA, "surrogate training: memset failed");
      if ((s = net.forward(B)) || (s = net.backward(B, B))) return ctx_fail(h, s, net.err.c_str());
      // cosine decay of the step size over the whole run
      const double lr_t = 0.5 * lr * (1.0 + cos(3.14159265358979323846 * double(step) / double(total_steps)));
      ++step;
      const float c1 = 1.f - powf(0.9f, (float)step), c2 = 1.f - powf(0.999f, (float)step);
      k_adam<<<256, 256, 0, st>>>(par.theta, par.grad, par.m, par.v, par.off.total, (float)lr_t, c1, c2,
                                  par.theta16);
      ++net.launches;
      if (cudaGetLastError() != cudaSuccess) return ctx_fail(h, HH_ERR_CUDA, "surrogate training: adam failed");
      if (loss_history) {
        if (cudaMemcpyAsync(lp.data(), net.loss_part, B * sizeof(double), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
          return ctx_fail(h, HH_ERR_CUDA, "surrogate training failed");
        for (int j = 0; j < B; ++j) ep_loss += lp[j];
        ep_n += B;
      }
    }
    if (loss_history) loss_history[ep] = ep_n ? ep_loss / (double(ep_n) * kOut) : 0.0;
  }
  if (cudaMemcpyAsync(params_out, par.theta, par.off.total * sizeof(float), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ctx_fail(h, HH_ERR_CUDA, "surrogate training failed");
  if ((s = par.timeout_check())) return ctx_fail(h, s, par.err.c_str());
  return HH_OK;
}

extern "C" hh_status hh_surrogate_predict(hh_ctx* h, const uint8_t* labels, int count, const int32_t* boxes,
                                         const float* params, int ensemble, double scale, float* out) {
  if (!h || !labels || !params || !out || ensemble < 1 || !(scale > 0.0))
    return ctx_fail(h, HH_ERR_ARG, "hh_surrogate_predict: NULL argument, ensemble < 1 or scale <= 0");
  if (count < 1) return ctx_fail(h, HH_ERR_ARG, "hh_surrogate_predict: count >= 1");
  const long long np = offsets().total;
  std::vector<float> tmp((size_t)count * kOut);
  for (int e = 0; e < ensemble; ++e) {
    hh_status s = hh_cnn_forward(h, labels, count, boxes, params + e * np, tmp.data());
    if (s) return s;
    for (int i = 0; i < count; ++i)
      for (int j = 0; j < kOut; ++j) out[((long long)i * ensemble + e) * kOut + j] = float(tmp[(size_t)i * kOut + j] * scale);
  }
  return HH_OK;
}

extern "C" hh_status hh_surrogate_gate(hh_ctx* h, const uint8_t* labels, int count, const int32_t* boxes,
                                      const hh_phase* phases, int nphase, const float* members, int ensemble,
                                      double spread, int* accept, double* c21) {
  if (!h || !labels || !phases || nphase < 1 || nphase > 256 || !members || ensemble < 1 || !accept || !c21 ||
      !(spread >= 0.0))
    return ctx_fail(h, HH_ERR_ARG, "hh_surrogate_gate: NULL argument or bad phase count, ensemble or spread");
  std::vector<Sub> subs;
  std::vector<std::vector<int>> groups;
  hh_status s = parse_subs(h, count, boxes, subs, groups);
  if (s) return s;
  for (int i = 0; i < nphase; ++i)
    if (!(phases[i].K > 0.0) || !(phases[i].G > 0.0)) return ctx_fail(h, HH_ERR_ARG, "surrogate gate: phase moduli");
  if ((s = ctx_enter(h))) return s;
  const cudaStream_t st = ctx_stream(h);
  std::vector<double> ph(2 * nphase);
  for (int i = 0; i < nphase; ++i) {
    ph[2 * i] = phases[i].K;
    ph[2 * i + 1] = phases[i].G;
  }
  for (const std::vector<int>& g : groups) {
    const int n = (int)g.size();
    Net net;  // only its label and core buffers (and the allocation list) are used
    net.st = st;
    double *d_ph = nullptr, *d_c = nullptr;
    float* d_mem = nullptr;
    int* d_acc = nullptr;
    const Box3 box = subs[g[0]].box;
    if ((s = net.alloc(&net.lab, n * Net::vox(box))) || (s = net.alloc(&net.core, n)) ||
        (s = net.alloc(&d_ph, 2 * nphase)) || (s = net.alloc(&d_mem, (long long)n * ensemble * kOut)) ||
        (s = net.alloc(&d_acc, n)) || (s = net.alloc(&d_c, (long long)n * kOut)))
      return ctx_fail(h, s, "surrogate gate: device allocation failed");
    std::vector<uint8_t> lab_h;
    std::vector<Core> core_h;
    if ((s = stage(net, labels, subs, g.data(), n, lab_h, core_h))) return ctx_fail(h, s, net.err.c_str());
    std::vector<float> mem((size_t)n * ensemble * kOut);
    for (int j = 0; j < n; ++j)
      std::memcpy(mem.data() + (size_t)j * ensemble * kOut, members + (size_t)g[j] * ensemble * kOut,
                  (size_t)ensemble * kOut * sizeof(float));
    std::vector<int> acc(n);
    std::vector<double> c(n * (size_t)kOut);
    if (cudaMemcpyAsync(d_ph, ph.data(), ph.size() * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_mem, mem.data(), mem.size() * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return ctx_fail(h, HH_ERR_CUDA, "surrogate gate: copy failed");
    k_gate<<<n, 256, 0, st>>>(net.lab, box, net.core, d_ph, nphase, d_mem, ensemble, spread, d_acc, d_c);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(acc.data(), d_acc, n * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(c.data(), d_c, c.size() * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return ctx_fail(h, HH_ERR_CUDA, "surrogate gate failed");
    for (int j = 0; j < n; ++j) {
      accept[g[j]] = acc[j];
      std::memcpy(c21 + (size_t)g[j] * kOut, c.data() + (size_t)j * kOut, kOut * sizeof(double));
    }
  }
  return HH_OK;
}

// ---------------------------------------------------------------------------
// Ensemble files (host only). Fields are written byte by byte in
// little-endian order, so the file is the same on every host.
// ---------------------------------------------------------------------------
namespace {

constexpr char kSurrMagic[8] = {'H', 'H', 'S', 'U', 'R', 'R', '0', '1'};
constexpr size_t kSurrHeader = 8 + 4 + 4 + 8 + 8 + 8;

// FNV-1a, 64-bit (Fowler, Noll and Vo): offset basis 0xcbf29ce484222325,
// prime 0x100000001b3.
uint64_t fnv1a64(const unsigned char* p, size_t n) {
  uint64_t h = 0xcbf29ce484222325ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 0x100000001b3ull;
  }
  return h;
}

void put_le(unsigned char* dst, uint64_t v, int bytes) {
  for (int i = 0; i < bytes; ++i) dst[i] = (unsigned char)(v >> (8 * i));
}

uint64_t get_le(const unsigned char* src, int bytes) {
  uint64_t v = 0;
  for (int i = 0; i < bytes; ++i) v |= (uint64_t)src[i] << (8 * i);
  return v;
}

// The parameters as little-endian bytes (FP32 bit patterns).
std::vector<unsigned char> params_bytes(const float* params, size_t n) {
  std::vector<unsigned char> b(4 * n);
  for (size_t i = 0; i < n; ++i) {
    uint32_t u;
    std::memcpy(&u, params + i, 4);
    put_le(b.data() + 4 * i, u, 4);
  }
  return b;
}

}  // namespace

extern "C" hh_status hh_surrogate_save(const char* path, const float* params, int ensemble, double scale) {
  if (!path || !params || ensemble < 1 || !(scale > 0.0) || !std::isfinite(scale))
    return ctx_fail(nullptr, HH_ERR_ARG, "hh_surrogate_save: NULL path or params, ensemble < 1 or bad scale");
  const int64_t np = hh_cnn_num_params();
  const std::vector<unsigned char> body = params_bytes(params, (size_t)ensemble * (size_t)np);
  unsigned char head[kSurrHeader];
  std::memcpy(head, kSurrMagic, 8);
  put_le(head + 8, (uint32_t)ensemble, 4);
  put_le(head + 12, 0, 4);
  put_le(head + 16, (uint64_t)np, 8);
  uint64_t sb;
  std::memcpy(&sb, &scale, 8);
  put_le(head + 24, sb, 8);
  put_le(head + 32, fnv1a64(body.data(), body.size()), 8);
  FILE* f = std::fopen(path, "wb");
  if (!f) return ctx_fail(nullptr, HH_ERR_ARG, (std::string("hh_surrogate_save: cannot open ") + path).c_str());
  const bool ok = std::fwrite(head, 1, kSurrHeader, f) == kSurrHeader &&
                  std::fwrite(body.data(), 1, body.size(), f) == body.size();
  if (std::fclose(f) != 0 || !ok)
    return ctx_fail(nullptr, HH_ERR_ARG, (std::string("hh_surrogate_save: cannot write ") + path).c_str());
  return HH_OK;
}

extern "C" hh_status hh_surrogate_load(const char* path, float* params, int64_t capacity, int* ensemble,
                                       double* scale) {
  if (!path || !ensemble || !scale)
    return ctx_fail(nullptr, HH_ERR_ARG, "hh_surrogate_load: NULL path, ensemble or scale");
  FILE* f = std::fopen(path, "rb");
  if (!f) return ctx_fail(nullptr, HH_ERR_ARG, (std::string("hh_surrogate_load: cannot open ") + path).c_str());
  unsigned char head[kSurrHeader];
  const bool got_head = std::fread(head, 1, kSurrHeader, f) == kSurrHeader;
  const int64_t np = hh_cnn_num_params();
  const int ens = got_head ? (int)(uint32_t)get_le(head + 8, 4) : 0;
  if (!got_head || std::memcmp(head, kSurrMagic, 8) != 0 || (int64_t)get_le(head + 16, 8) != np || ens < 1) {
    std::fclose(f);
    return ctx_fail(nullptr, HH_ERR_ARG, "hh_surrogate_load: not an ensemble file of this network");
  }
  double sc;
  const uint64_t sb = get_le(head + 24, 8);
  std::memcpy(&sc, &sb, 8);
  const size_t n = (size_t)ens * (size_t)np;
  std::vector<unsigned char> body(4 * n);
  const bool got_body = std::fread(body.data(), 1, body.size(), f) == body.size();
  unsigned char extra;
  const bool at_end = std::fread(&extra, 1, 1, f) == 0;
  std::fclose(f);
  if (!got_body || !at_end)
    return ctx_fail(nullptr, HH_ERR_ARG, "hh_surrogate_load: file length does not match its header");
  if (fnv1a64(body.data(), body.size()) != get_le(head + 32, 8))
    return ctx_fail(nullptr, HH_ERR_ARG, "hh_surrogate_load: parameter hash does not match");
  if (!(sc > 0.0) || !std::isfinite(sc)) return ctx_fail(nullptr, HH_ERR_ARG, "hh_surrogate_load: bad scale");
  *ensemble = ens;
  *scale = sc;
  if (!params) return HH_OK;
  if (capacity < (int64_t)n) return ctx_fail(nullptr, HH_ERR_ARG, "hh_surrogate_load: capacity too small");
  for (size_t i = 0; i < n; ++i) {
    const uint32_t u = (uint32_t)get_le(body.data() + 4 * i, 4);
    std::memcpy(params + i, &u, 4);
  }
  return HH_OK;
}
