// Host side of libhh: FFT planning, context and workspace, the batched
// wave driver of the conjugate-gradient solves (CUDA-graph-captured iteration
// chunks), and the C ABI declared in include/hh.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "hh.h"
#include "hh_device.cuh"
#include "hh_fused.cuh"
#include "hh_post.cuh"
#include "hh_internal.h"

namespace hh {

// The compiled-shape kernels are instantiated in hh_ct_inst.cu.
#define HH_CT_EXTERN(G)                                                       \
  extern template __global__ void k_plane_fwd_ct<float, G>(KParams<float>);   \
  extern template __global__ void k_plane_fwd_ct<double, G>(KParams<double>); \
  extern template __global__ void k_plane_inv_ct<float, G>(KParams<float>);   \
  extern template __global__ void k_plane_inv_ct<double, G>(KParams<double>);
HH_CT_EXTERN(0)
HH_CT_EXTERN(1)
HH_CT_EXTERN(2)
HH_CT_EXTERN(3)
#undef HH_CT_EXTERN
extern template __global__ void k_column_ct<float>(KParams<float>, int);
extern template __global__ void k_column_ct<double>(KParams<double>, int);

// ---------------------------------------------------------------------------
// FFT planning: radices, twiddles, digit-reversal tables.
// ---------------------------------------------------------------------------
// Radices of n (4s, then 2, then odd primes up to 31) into rad[kMaxStages].
static bool factorize(int n, int* rad, int* nst) {
  int k = 0;
  auto push = [&](int r) {
    if (k >= kMaxStages) return false;
    rad[k++] = r;
    return true;
  };
  while (n % 4 == 0) {
    if (!push(4)) return false;
    n /= 4;
  }
  while (n % 2 == 0) {
    if (!push(2)) return false;
    n /= 2;
  }
  const int primes[] = {3, 5, 7, 11, 13, 17, 19, 23, 29, 31};
  for (int p : primes)
    while (n % p == 0) {
      if (!push(p)) return false;
      n /= p;
    }
  *nst = k;
  return n == 1;
}

// Fill the plan of length n and its tables without allocating: tw receives
// 2n doubles (W_n[t] = exp(-2 pi i t / n)), pf and sf n ints each
// (natural frequency -> storage position, storage position -> signed frequency).
static bool plan_fill(int n, AxisPlan* p, double* tw, int* pf, int* sf) {
  std::memset(p, 0, sizeof(*p));
  if (n < 1 || !factorize(n, p->rad, &p->nst)) return false;
  p->n = n;
  p->split = fft2_split(n);
  const long double two_pi = 6.283185307179586476925286766559005768L;
  for (int t = 0; t < n; ++t) {
    const long double a = two_pi * (long double)t / (long double)n;
    tw[2 * t] = (double)cosl(a);
    tw[2 * t + 1] = (double)-sinl(a);
  }
  if (p->split) {
    // two-pass plan: natural order in and out
    for (int k = 0; k < n; ++k) {
      pf[k] = k;
      sf[k] = (2 * k <= n) ? k : k - n;
    }
    return true;
  }
  for (int k = 0; k < n; ++k) {
    int rem = k, span = n, pos = 0;
    for (int s = 0; s < p->nst; ++s) {
      const int R = p->rad[s];
      const int q = rem % R;
      rem /= R;
      span /= R;
      pos += q * span;
    }
    pf[k] = pos;
  }
  for (int k = 0; k < n; ++k) sf[pf[k]] = (2 * k <= n) ? k : k - n;
  return true;
}

struct Tables {
  std::vector<AxisPlan> plans;
  std::vector<double> tw;
  std::vector<int> itab;
  std::map<int, int> index;
};

// Returns the plan index for length n, or -1 if n is not supported.
static int plan_for(Tables& T, int n) {
  auto it = T.index.find(n);
  if (it != T.index.end()) return it->second;
  if (n < 1) return -1;
  AxisPlan p;
  std::vector<double> tw(2 * (size_t)n);
  std::vector<int> pf(n), sf(n);
  if (!plan_fill(n, &p, tw.data(), pf.data(), sf.data())) return -1;
  p.tw_off = (int)(T.tw.size() / 2);
  T.tw.insert(T.tw.end(), tw.begin(), tw.end());
  p.pf_off = (int)T.itab.size();
  T.itab.insert(T.itab.end(), pf.begin(), pf.end());
  p.sf_off = (int)T.itab.size();
  T.itab.insert(T.itab.end(), sf.begin(), sf.end());
  const int idx = (int)T.plans.size();
  T.plans.push_back(p);
  T.index[n] = idx;
  return idx;
}

// ---------------------------------------------------------------------------
// Context and workspace.
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
};

// Streams a pass's launch classes are spread over: the classes of one pass
// touch disjoint problems, so they run side by side (branches of the chunk's
// graph when it is captured) and fill one another's tails. 1: one stream.
#ifndef HH_PASS_STREAMS
#define HH_PASS_STREAMS 4
#endif
constexpr int kPassStreams = HH_PASS_STREAMS;

struct Ctx {
  int dev = 0;
  int nsm = 0;
  size_t smem_optin = 0;
  cudaStream_t st = nullptr;   // internal stream (captures graphs)
  cudaStream_t user = nullptr; // caller's stream, or nullptr
  Tables tab;
  size_t tab_uploaded = 0;
  DevBuf d_plans, d_tw, d_itab;
  std::map<std::string, DevBuf> bufs;
  int* h_int = nullptr;        // pinned scratch
  double* h_dbl = nullptr;
  std::string err;
  long long launches = 0;      // kernels launched on this context
  cudaEvent_t ev_call0 = nullptr, ev_call1 = nullptr;
  cudaStream_t side[kPassStreams] = {};           // the pass streams (fork from st, join back)
  cudaEvent_t ev_fork = nullptr, ev_join[kPassStreams] = {};
  struct KStat {
    long long launches = 0, sampled = 0;
    double ms = 0.0, bytes = 0.0;
  };
  std::map<std::string, KStat> prof;
  std::map<long long, int> col_tune;  // autotuned column-pass width per (precision, shape)
  size_t mem_limit = 0;               // cap on the workspace buffers (0: none)
  std::map<long long, int> fused_occ; // resident clusters per (precision, cluster size, shared memory)
};

#define HH_CK(call)                                                         \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) {                                                \
      c.err = std::string(#call) + " (line " + std::to_string(__LINE__) +   \
              "): " + cudaGetErrorString(e_);                                \
      return e_ == cudaErrorMemoryAllocation ? HH_ERR_OOM : HH_ERR_CUDA;    \
    }                                                                       \
  } while (0)

static hh_status ensure(Ctx& c, const char* name, size_t bytes, void** out) {
  DevBuf& b = c.bufs[name];
  if (b.n < bytes || !b.p) {
    size_t want = std::max<size_t>(bytes, 256);
    if (c.mem_limit) {
      size_t held = 0;
      for (auto& kv : c.bufs) held += kv.second.n;
      if (held - b.n + want > c.mem_limit) {
        c.err = std::string("workspace '") + name + "' of " + std::to_string(want) + " bytes would exceed the " +
                "context's device memory limit of " + std::to_string(c.mem_limit) + " bytes";
        return HH_ERR_OOM;
      }
    }
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
    HH_CK(cudaMalloc(&b.p, want));
    b.n = want;
  }
  *out = b.p;
  return HH_OK;
}

static hh_status upload_tables(Ctx& c) {
  const size_t sig = c.tab.plans.size();
  if (sig == c.tab_uploaded) return HH_OK;
  auto up = [&](DevBuf& b, const void* src, size_t bytes) -> hh_status {
    if (b.n < bytes) {
      if (b.p) cudaFree(b.p);
      b.p = nullptr;
      HH_CK(cudaMalloc(&b.p, std::max<size_t>(bytes, 256)));
      b.n = std::max<size_t>(bytes, 256);
    }
    HH_CK(cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, c.st));
    return HH_OK;
  };
  hh_status s;
  if ((s = up(c.d_plans, c.tab.plans.data(), c.tab.plans.size() * sizeof(AxisPlan))) != HH_OK) return s;
  if ((s = up(c.d_tw, c.tab.tw.data(), c.tab.tw.size() * sizeof(double))) != HH_OK) return s;
  if ((s = up(c.d_itab, c.tab.itab.data(), c.tab.itab.size() * sizeof(int))) != HH_OK) return s;
  HH_CK(cudaStreamSynchronize(c.st));
  c.tab_uploaded = sig;
  return HH_OK;
}

template <typename T>
static size_t plane_smem_bytes(int nx, int ny, int nphase) {
  size_t o = 32 * 4 * sizeof(double);
  o += sizeof(C2<T>) * 3 * (size_t)ny * (size_t)((nx + 2) | 1);
  o += sizeof(C2<T>) * (size_t)nx;
  o += sizeof(C2<T>) * (size_t)ny;
  o += sizeof(int) * (size_t)((nx + 3) & ~3);
  o += sizeof(T) * 2 * (size_t)std::max(nphase, 1);
  return (o + 15) & ~size_t(15);
}

template <typename T>
static size_t column_smem_bytes(int cw, int nz, int ny) {
  size_t o = sizeof(C2<T>) * (6 * (size_t)nz * cw + nz) + sizeof(T) * (size_t)nz + sizeof(int) * ((size_t)nz + ny);
  o = (o + 7) & ~size_t(7);
  o += 32 * 7 * sizeof(double);  // block reduction of the basic scheme's residual partials
  return (o + 15) & ~size_t(15);
}
constexpr size_t kColumnSmem = 48 * 1024;  // per-block target of the column pass

// Spectrum columns per column-pass item: the widest power of two up to 32
// (FP32) or 16 (FP64) whose tile fits the column target, else what fits at all.
template <typename T>
static int column_width(int nz, int ny, size_t optin) {
  int cw = sizeof(T) == 4 ? 32 : 16;
  while (cw > 1 && column_smem_bytes<T>(cw, nz, ny) > kColumnSmem) cw /= 2;
  while (cw > 1 && column_smem_bytes<T>(cw, nz, ny) > optin) cw /= 2;
  return cw;
}

// Row-streaming passes: R rows of a plane per block; y columns: W kx columns.
template <typename T>
static size_t rows_smem_bytes(int nx, int R, int nphase) {
  return plane_smem_bytes<T>(nx, R, nphase);
}
template <typename T>
static size_t ycol_smem_bytes(int ny, int W) {
  return (sizeof(C2<T>) * (6 * (size_t)ny * W + ny) + 15) & ~size_t(15);
}
constexpr size_t kStreamSmem = 48 * 1024;  // per-block target of the streaming passes

// Launch classes: shared-memory footprints are rounded up to these sizes and
// every class gets its own launch, so small subimages are not held to the
// occupancy of the largest one.
// The field kernels run at most kFieldBlocksPerSM blocks per SM (register
// bound), so footprints are grouped by the blocks per SM their shared memory
// allows (228 KB per SM, 1 KB reserved per block): one launch per tier, with
// the tier's largest footprint.
static size_t smem_bucket(size_t bytes) {
  const size_t per_sm = 228 * 1024, reserve = 1024;
  for (int nb = kFieldBlocksPerSM; nb > 1; --nb)
    if (bytes <= per_sm / nb - reserve) return per_sm / nb - reserve;
  return bytes;
}

// ---------------------------------------------------------------------------
// The batched solver.
// ---------------------------------------------------------------------------
struct Medium {
  int kind = MED_ISO;
  // iso: device image and phase table
  const uint8_t* d_img = nullptr;
  int Nx = 0, Ny = 0, Nz = 0;
  std::vector<double> lam, mu;
  // aniso: device FP64 C21 field of the single whole-grid box
  const double* d_c21 = nullptr;
  // smallest tensor eigenvalue min(3K, 2G) of the phases (level-2 voxel floor)
  double floor = 0.0;
};

struct Stats {
  int iters_max = 0;
  double resid_max = 0.0;
  long long voxel_iters = 0;
  int worst = ST_OK;
  int fused_boxes = 0;  // subimages solved by the fused cluster kernel
};

template <typename T>
static int grid_for(Ctx& c, const void* kern, int threads, size_t smem, int nitems) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem) != cudaSuccess || nb < 1) nb = 1;
  long long g = (long long)nb * c.nsm;
  if (g > nitems) g = nitems;
  return (int)std::max<long long>(g, 1);
}

// Autotuner: the spectrum columns per column-pass block for one subimage
// shape, chosen by timing the column pass on a scratch batch of that shape
// (8 problems, zero spectrum) for the widths that fit, once per context. The
// width changes no arithmetic (every z line is transformed and projected the
// same way), only the speed.
// With `ct` (a z length that has compiled column bodies) the candidates are
// the compiled widths, timed through those bodies.
template <typename T>
static int tuned_column_width(Ctx& c, int nx, int ny, int nz, int nyq_mode, bool enabled, bool ct = false) {
  int rule = column_width<T>(nz, ny, c.smem_optin);
  if (ct) rule = rule >= 32 ? 32 : 16;
  if (!enabled) return rule;
  const long long key = ((long long)ct << 56) | ((long long)sizeof(T) << 48) | ((long long)nz << 32) |
                        ((long long)ny << 16) | nx;
  auto it = c.col_tune.find(key);
  if (it != c.col_tune.end()) return it->second;
  const int nxh = nx / 2 + 1, np = 8;
  const long long pl = (long long)ny * nxh;
  C2<T>* d_spec = nullptr;
  Prob* d_prob = nullptr;
  int2* d_items = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int best = rule;
  float best_ms = 1e30f;
  bool ok = ensure(c, "tune_spec", np * 6 * nz * pl * sizeof(C2<T>), (void**)&d_spec) == HH_OK &&
            ensure(c, "tune_prob", np * sizeof(Prob), (void**)&d_prob) == HH_OK &&
            ensure(c, "tune_items", np * pl * sizeof(int2), (void**)&d_items) == HH_OK &&
            cudaMemsetAsync(d_spec, 0, np * 6 * nz * pl * sizeof(C2<T>), c.st) == cudaSuccess &&
            cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  auto* kc = ct ? k_column_ct<T> : k_column<T, false>;
  ok = ok && cudaFuncSetAttribute((const void*)kc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)c.smem_optin) == cudaSuccess;
  const std::vector<int> cands = ct ? std::vector<int>{16, 32} : std::vector<int>{rule / 2, rule, rule * 2};
  for (int cw : cands) {
    if (!ok || cw < 1 || column_smem_bytes<T>(cw, nz, ny) > c.smem_optin) continue;
    std::vector<Prob> probs(np);
    std::vector<int2> items;
    for (int i = 0; i < np; ++i) {
      Prob& d = probs[i];
      std::memset(&d, 0, sizeof(d));
      d.nx = nx;
      d.ny = ny;
      d.nz = nz;
      d.nxh = nxh;
      d.px = c.tab.index[nx];
      d.py = c.tab.index[ny];
      d.pz = c.tab.index[nz];
      d.cw = cw;
      d.ct_col = ct ? nz * 64 + cw : 0;
      d.spc_off = (long long)i * 6 * nz * pl;
      for (int j0 = 0; j0 < pl; j0 += cw) items.push_back(make_int2(i, j0));
    }
    if (cudaMemcpyAsync(d_prob, probs.data(), np * sizeof(Prob), cudaMemcpyHostToDevice, c.st) != cudaSuccess ||
        cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, c.st) !=
            cudaSuccess) {
      ok = false;
      break;
    }
    KParams<T> kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.prob = d_prob;
    kp.items = d_items;
    kp.nitems = (int)items.size();
    kp.nyq_mode = nyq_mode;
    kp.plans = (const AxisPlan*)c.d_plans.p;
    kp.tw = (const double*)c.d_tw.p;
    kp.itab = (const int*)c.d_itab.p;
    kp.spec = d_spec;
    const size_t smem = column_smem_bytes<T>(cw, nz, ny);
    // (the compiled-shape kernel takes one block per item)
    const int grid = ct ? kp.nitems : grid_for<T>(c, (const void*)kc, 256, smem, kp.nitems);
    kc<<<grid, 256, smem, c.st>>>(kp, MODE_APPLY);
    cudaEventRecord(e0, c.st);
    for (int r = 0; r < 3; ++r) kc<<<grid, 256, smem, c.st>>>(kp, MODE_APPLY);
    cudaEventRecord(e1, c.st);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      ok = false;
      break;
    }
    c.launches += 4;
    if (ms < best_ms) {
      best_ms = ms;
      best = cw;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (!ok) {
    (void)cudaGetLastError();
    return rule;
  }
  c.col_tune[key] = best;
  return best;
}

// Cluster shape of the fused solver for one subimage: blocks per cluster (C)
// and shared memory per block, or C = 0 when the subimage takes the
// multi-pass solver. The slab of the half spectrum is split over C blocks of
// consecutive z planes; the shape with the most blocks per SM (four, three or
// two, by shared memory) is taken, with the fewest blocks per cluster among
// those, else the fewest blocks that fit the per-block limit at all.
struct FusedPlan {
  int C = 0;
  size_t smem = 0;
};
constexpr int kFusedMaxCluster = 8;  // the portable cluster size

// Launch configuration of the fused kernel: C blocks per cluster, `smem`
// bytes of dynamic shared memory per block, `grid` blocks.
template <typename T>
static cudaLaunchConfig_t fused_config(Ctx& c, int C, size_t smem, int grid, cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(kFusedThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c.st;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

// Clusters of C blocks with `smem` bytes each that the device holds at once
// (0: the shape cannot be launched); cached per context.
template <typename T>
static int fused_resident_clusters(Ctx& c, int C, size_t smem) {
  const long long key = ((long long)sizeof(T) << 40) | ((long long)C << 32) | (long long)smem;
  auto it = c.fused_occ.find(key);
  if (it != c.fused_occ.end()) return it->second;
  const void* kern = (const void*)k_fused<T>;
  int n = 0;
  cudaFuncAttributes fa;
  // the dynamic limit leaves room for the kernel's static shared memory
  if (cudaFuncGetAttributes(&fa, kern) == cudaSuccess && smem + fa.sharedSizeBytes <= c.smem_optin &&
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(c.smem_optin - fa.sharedSizeBytes)) == cudaSuccess) {
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = fused_config<T>(c, C, smem, C, at);
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) n = 0;
  }
  (void)cudaGetLastError();
  c.fused_occ[key] = n;
  return n;
}

template <typename T>
static FusedPlan fused_plan(Ctx& c, int nx, int ny, int nz, int nphase) {
  const size_t per_sm = 228 * 1024, reserve = 1024;
  for (int nb : {4, 3, 2, 1}) {
    const size_t lim = nb > 1 ? per_sm / nb - reserve : c.smem_optin;
    for (int C = 1; C <= kFusedMaxCluster && C <= nz; C *= 2) {
      const size_t bytes = fused_smem_bytes<T>(nx, ny, nz, (nz + C - 1) / C, nphase);
      // (the kernel's static shared memory, 16 pointers, comes on top)
      if (bytes <= lim && bytes + 256 <= c.smem_optin && fused_resident_clusters<T>(c, C, smem_bucket(bytes)) > 0)
        return FusedPlan{C, bytes};
    }
  }
  return FusedPlan();
}

// One persistent cluster launch per group of fused problems (same blocks per
// cluster and shared-memory tier). Clusters take the group's problems from a
// device counter, largest subimage first; each solves its problem to the end
// and writes its CG state (iterations, status, residual, core sums).
template <typename T>
static hh_status run_fused(Ctx& c, const std::map<std::pair<int, size_t>, std::vector<int>>& groups,
                           const std::vector<Prob>& probs, const FusedParams<T>& base, int nphase) {
  std::vector<int> order;
  std::vector<int> start;
  for (auto& kv : groups) {
    start.push_back((int)order.size());
    std::vector<int> g = kv.second;
    std::stable_sort(g.begin(), g.end(), [&](int a, int b) {
      const Prob& pa = probs[a];
      const Prob& pb = probs[b];
      return (long long)pa.nx * pa.ny * pa.nz > (long long)pb.nx * pb.ny * pb.nz;
    });
    order.insert(order.end(), g.begin(), g.end());
  }
  int *d_order, *d_queue;
  hh_status s;
  if ((s = ensure(c, "fused_order", order.size() * sizeof(int), (void**)&d_order)) != HH_OK) return s;
  if ((s = ensure(c, "fused_queue", groups.size() * sizeof(int), (void**)&d_queue)) != HH_OK) return s;
  HH_CK(cudaMemcpyAsync(d_order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice, c.st));
  HH_CK(cudaMemsetAsync(d_queue, 0, groups.size() * sizeof(int), c.st));
  int gi = 0;
  for (auto& kv : groups) {
    const int C = kv.first.first;
    size_t smem = 0;
    for (int pr : kv.second) {
      const Prob& d = probs[pr];
      smem = std::max(smem, fused_smem_bytes<T>(d.nx, d.ny, d.nz, (d.nz + C - 1) / C, nphase));
    }
    smem = smem_bucket(smem);
    const int n = (int)kv.second.size();
    const int ncl = std::min(fused_resident_clusters<T>(c, C, smem), n);
    if (ncl < 1) {
      c.err = "fused solver: no cluster of " + std::to_string(C) + " blocks fits";
      return HH_ERR_UNSUPPORTED;
    }
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = fused_config<T>(c, C, smem, ncl * C, at);
    FusedParams<T> fp = base;
    fp.order = d_order + start[gi];
    fp.nwork = n;
    fp.queue = d_queue + gi;
    ++c.launches;
    HH_CK(cudaLaunchKernelEx(&cfg, k_fused<T>, fp));
    ++gi;
  }
  return HH_OK;
}

// Solve the six load cases of every box; per-box results land in d_res[box].
template <typename T>
static hh_status solve_boxes(Ctx& c, const hh_options& o, const Medium& med, const std::vector<BoxReq>& boxes_in,
                             BoxRes* d_res, Stats& stats) {
  const int nbox = (int)boxes_in.size();
  if (nbox == 0) return HH_OK;
  const int threads = 256;
  // plans for every axis length in the request
  std::vector<int> bdim(3 * nbox);
  for (int b = 0; b < nbox; ++b) {
    const BoxReq& B = boxes_in[b];
    const int n3[3] = {B.cnx + 2 * B.b, B.cny + 2 * B.b, B.cnz + 2 * B.b};
    for (int a = 0; a < 3; ++a) {
      const int pi = plan_for(c.tab, n3[a]);
      if (pi < 0) {
        c.err = "unsupported FFT length " + std::to_string(n3[a]);
        return HH_ERR_UNSUPPORTED;
      }
      bdim[3 * b + a] = n3[a];
    }
  }
  hh_status s = upload_tables(c);
  if (s != HH_OK) return s;
  const int nphase = (int)med.lam.size();

  // per-box workspace bytes
  auto box_bytes = [&](int b) -> size_t {
    const size_t nx = bdim[3 * b], ny = bdim[3 * b + 1], nz = bdim[3 * b + 2];
    const size_t V = nx * ny * nz, nxh = nx / 2 + 1;
    size_t m = (med.kind == MED_ISO) ? V : 21 * V * sizeof(T);
    m += 6 * (24 * V * sizeof(T) + 12 * nz * ny * nxh * sizeof(T) + nz * 16 * sizeof(double) + 64 * sizeof(int2));
    m += 6 * (sizeof(Prob) + sizeof(PState)) + sizeof(BoxReq) + 4096;
    return m;
  };
  size_t budget = (size_t)o.workspace_bytes;
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    HH_CK(cudaMemGetInfo(&fr, &tot));
    size_t have = 0;
    for (auto& kv : c.bufs) have += kv.second.n;
    budget = (size_t)((fr + have) * 0.75);
  }
  if (c.mem_limit) budget = std::min(budget, c.mem_limit / 4 * 3);

  // shared memory: a whole plane per plane-pass block when it fits the plane
  // limit, else R rows per block and W kx columns per y-column block (row
  // streaming); column_width() spectrum columns per column-pass block
  const size_t plane_lim = o.plane_smem_limit > 0 ? std::min<size_t>(o.plane_smem_limit, c.smem_optin) : c.smem_optin;
  int ycw = 16;
  const size_t stream_target = std::min(kStreamSmem, plane_lim);
  for (int b = 0; b < nbox; ++b) {
    const int nx = bdim[3 * b], ny = bdim[3 * b + 1], nz = bdim[3 * b + 2];
    if (plane_smem_bytes<T>(nx, ny, nphase) > plane_lim) {
      while (ycw > 1 && ycol_smem_bytes<T>(ny, ycw) > std::max(stream_target, ycol_smem_bytes<T>(ny, 1))) ycw /= 2;
      if (rows_smem_bytes<T>(nx, 1, nphase) > c.smem_optin || ycol_smem_bytes<T>(ny, 1) > c.smem_optin) {
        c.err = "row or y column too long for shared memory";
        return HH_ERR_UNSUPPORTED;
      }
    }
    if (column_smem_bytes<T>(1, nz, ny) > c.smem_optin) {
      c.err = "z column too long for shared memory";
      return HH_ERR_UNSUPPORTED;
    }
  }
  // rows per streaming item: as many as fit the streaming target
  auto stream_rows = [&](int nx, int ny) {
    int R = 1;
    while (R < ny && rows_smem_bytes<T>(nx, R + 1, nphase) <= std::max(stream_target, rows_smem_bytes<T>(nx, 1, nphase)))
      ++R;
    return R;
  };
  auto* kf_rhs = k_plane_fwd<T, MODE_RHS>;
  auto* kf_it = k_plane_fwd<T, MODE_ITER>;
  auto* kf_tr = k_plane_fwd<T, MODE_TRUE>;
  auto* ki_rhs = k_plane_inv<T, MODE_RHS>;
  auto* ki_it = k_plane_inv<T, MODE_ITER>;
  auto* ki_tr = k_plane_inv<T, MODE_TRUE>;
  auto* kc = k_column<T, false>;
  auto* kcb = k_column<T, true>;
  auto* ku = k_flush<T>;
  auto* ka = k_avg<T>;
  auto* kf_b = k_plane_fwd<T, MODE_BASIC>;
  auto* ki_b = k_plane_inv<T, MODE_BASIC>;
  using KFn = void (*)(KParams<T>);
  // forward / inverse kernels per mode: whole planes and row streaming
  auto kfwd = [&](int mode, bool rows) -> KFn {
    switch (mode) {
      case MODE_RHS: return rows ? k_rows_fwd<T, MODE_RHS> : kf_rhs;
      case MODE_ITER: return rows ? k_rows_fwd<T, MODE_ITER> : kf_it;
      case MODE_TRUE: return rows ? k_rows_fwd<T, MODE_TRUE> : kf_tr;
      default: return rows ? k_rows_fwd<T, MODE_BASIC> : kf_b;
    }
  };
  auto kinv = [&](int mode, bool rows) -> KFn {
    switch (mode) {
      case MODE_RHS: return rows ? k_rows_inv<T, MODE_RHS> : ki_rhs;
      case MODE_ITER: return rows ? k_rows_inv<T, MODE_ITER> : ki_it;
      case MODE_TRUE: return rows ? k_rows_inv<T, MODE_TRUE> : ki_tr;
      default: return rows ? k_rows_inv<T, MODE_BASIC> : ki_b;
    }
  };
  auto* kyf = k_ycols<T, false>;
  auto* kyi = k_ycols<T, true>;
  KFn kfct[kCtPlaneGroups] = {k_plane_fwd_ct<T, 0>, k_plane_fwd_ct<T, 1>, k_plane_fwd_ct<T, 2>, k_plane_fwd_ct<T, 3>};
  KFn kict[kCtPlaneGroups] = {k_plane_inv_ct<T, 0>, k_plane_inv_ct<T, 1>, k_plane_inv_ct<T, 2>, k_plane_inv_ct<T, 3>};
  auto* kcct = k_column_ct<T>;
  for (int m : {MODE_RHS, MODE_ITER, MODE_TRUE, MODE_BASIC})
    for (bool rows : {false, true})
      for (KFn f : {kfwd(m, rows), kinv(m, rows)})
        HH_CK(cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem_optin));
  for (const void* f : {(const void*)kc, (const void*)kcb, (const void*)kyf, (const void*)kyi, (const void*)kcct})
    HH_CK(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem_optin));
  for (int g = 0; g < kCtPlaneGroups; ++g)
    for (KFn f : {kfct[g], kict[g]})
      HH_CK(cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem_optin));
  const bool replace = o.replace == 1 || (o.replace == -1 && sizeof(T) == 4);

  // lambda/mu table
  std::vector<T> lm(2 * std::max(nphase, 1));
  for (int i = 0; i < nphase; ++i) {
    lm[2 * i] = T(med.lam[i]);
    lm[2 * i + 1] = T(med.mu[i]);
  }
  T* d_lm = nullptr;
  if ((s = ensure(c, "lammu", lm.size() * sizeof(T), (void**)&d_lm)) != HH_OK) return s;
  HH_CK(cudaMemcpyAsync(d_lm, lm.data(), lm.size() * sizeof(T), cudaMemcpyHostToDevice, c.st));

  // basic and accelerated schemes: isotropic reference medium, given, or
  // for the basic scheme the means of the extreme phase values of lambda and
  // mu, for the accelerated scheme the geometric means of the extreme phase
  // values of K and mu
  const bool em = o.scheme == HH_EYRE_MILTON;
  const bool basic = o.scheme == HH_BASIC || em;
  if (em && med.kind != MED_ISO) {
    c.err = "the accelerated scheme takes isotropic phases only";
    return HH_ERR_UNSUPPORTED;
  }
  double lam0 = o.ref_lambda, mu0 = o.ref_mu;
  if (basic && !(mu0 > 0.0 && lam0 + 2.0 * mu0 / 3.0 > 0.0)) {
    if (med.kind != MED_ISO || nphase < 1) {
      c.err = "the basic scheme on an anisotropic medium needs ref_lambda and ref_mu";
      return HH_ERR_UNSUPPORTED;
    }
    if (em) {
      double kmin = 1e300, kmax = 0.0, mmin = 1e300, mmax = 0.0;
      for (int i = 0; i < nphase; ++i) {
        const double K = med.lam[i] + 2.0 * med.mu[i] / 3.0;
        kmin = std::min(kmin, K);
        kmax = std::max(kmax, K);
        mmin = std::min(mmin, med.mu[i]);
        mmax = std::max(mmax, med.mu[i]);
      }
      mu0 = std::sqrt(mmin * mmax);
      lam0 = std::sqrt(kmin * kmax) - 2.0 * mu0 / 3.0;
    } else {
      lam0 = 0.5 * (*std::min_element(med.lam.begin(), med.lam.end()) +
                    *std::max_element(med.lam.begin(), med.lam.end()));
      mu0 = 0.5 * (*std::min_element(med.mu.begin(), med.mu.end()) + *std::max_element(med.mu.begin(), med.mu.end()));
    }
  }
  // accelerated scheme: per phase the polarization moduli (lambda - lam0,
  // mu - mu0) for the forward pass and the factors of 2 (C + C0)^-1 C0
  // (spherical 2 K0 / (K + K0), deviatoric 2 mu0 / (mu + mu0)) for the
  // inverse pass
  T* d_lm_tau = nullptr;
  T* d_lm_em = nullptr;
  if (em) {
    const double K0 = lam0 + 2.0 * mu0 / 3.0;
    std::vector<T> lt(2 * std::max(nphase, 1)), le(2 * std::max(nphase, 1));
    for (int i = 0; i < nphase; ++i) {
      const double K = med.lam[i] + 2.0 * med.mu[i] / 3.0;
      lt[2 * i] = T(med.lam[i] - lam0);
      lt[2 * i + 1] = T(med.mu[i] - mu0);
      le[2 * i] = T(2.0 * K0 / (K + K0));
      le[2 * i + 1] = T(2.0 * mu0 / (med.mu[i] + mu0));
    }
    if ((s = ensure(c, "lm_tau", lt.size() * sizeof(T), (void**)&d_lm_tau)) != HH_OK) return s;
    if ((s = ensure(c, "lm_em", le.size() * sizeof(T), (void**)&d_lm_em)) != HH_OK) return s;
    HH_CK(cudaMemcpyAsync(d_lm_tau, lt.data(), lt.size() * sizeof(T), cudaMemcpyHostToDevice, c.st));
    HH_CK(cudaMemcpyAsync(d_lm_em, le.data(), le.size() * sizeof(T), cudaMemcpyHostToDevice, c.st));
  }
  const double floor2 = (sizeof(T) == 4) ? 1e-12 : 1e-28;
  int b0 = 0;
  while (b0 < nbox) {
    // ---- choose the wave [b0, b1)
    int b1 = b0;
    size_t used = 0;
    while (b1 < nbox && (b1 == b0 || (used + box_bytes(b1) <= budget && (o.wave_boxes <= 0 || b1 - b0 < o.wave_boxes))))
      used += box_bytes(b1++);
    const int nb = b1 - b0;
    const int np = 6 * nb;
    std::vector<Prob> probs(np);
    std::vector<BoxReq> wboxes(boxes_in.begin() + b0, boxes_in.begin() + b1);
    std::vector<int2> pitems, citems, gitems;
    // launch classes by shared-memory size: whole planes, streaming rows,
    // streaming y columns, z columns
    std::map<size_t, std::vector<int2>> pclass, rclass, yclass, cclass;
    // largest footprint in each class: the launch asks for no more, so small
    // planes leave the SM's remaining shared memory to L1
    std::map<size_t, size_t> pneed, rneed, yneed, cneed;
    auto need = [](std::map<size_t, size_t>& m, size_t key, size_t bytes) {
      size_t& v = m[key];
      v = std::max(v, (bytes + 1023) & ~size_t(1023));
      return key;
    };
    long long lab_off = 0, fld_off = 0, spc_off = 0, c21_off = 0, ccount = 0, prow = 0;
    // fused solves: problems per (blocks per cluster, shared memory per block)
    std::map<std::pair<int, size_t>, std::vector<int>> fgroups;
    int n_multipass = 0;
    for (int b = 0; b < nb; ++b) {
      const BoxReq& B = wboxes[b];
      const int nx = bdim[3 * (b0 + b)], ny = bdim[3 * (b0 + b) + 1], nz = bdim[3 * (b0 + b) + 2];
      const long long V = (long long)nx * ny * nz;
      const int nxh = nx / 2 + 1;
      wboxes[b].lab_off = (med.kind == MED_ISO) ? lab_off : c21_off;  // labels: bytes; stiffness: elements
      for (int k = 0; k < nz; ++k) gitems.push_back(make_int2(b, k));
      const FusedPlan fp = (o.fused && med.kind == MED_ISO && !basic) ? fused_plan<T>(c, nx, ny, nz, nphase)
                                                                       : FusedPlan();
      if (fp.C > 0) {
        // solved whole by the fused kernel: no multi-pass items, partials or spectrum
        std::vector<int>& grp = fgroups[std::make_pair(fp.C, smem_bucket(fp.smem))];
        for (int a = 0; a < 6; ++a) {
          Prob& d = probs[6 * b + a];
          std::memset(&d, 0, sizeof(d));
          d.nx = nx;
          d.ny = ny;
          d.nz = nz;
          d.nxh = nxh;
          d.c0x = B.b;
          d.c0y = B.b;
          d.c0z = B.b;
          d.cnx = B.cnx;
          d.cny = B.cny;
          d.cnz = B.cnz;
          d.px = c.tab.index[nx];
          d.py = c.tab.index[ny];
          d.pz = c.tab.index[nz];
          d.lc = a;
          d.box = b0 + b;
          d.cw = 1;
          d.fused = 1;
          d.med_off = lab_off;
          d.fld_off = fld_off;
          grp.push_back(6 * b + a);
          fld_off += 6 * V;
        }
        lab_off += V;
        c21_off += 21 * V;
        continue;
      }
      n_multipass += 6;
      for (int a = 0; a < 6; ++a) {
        Prob& d = probs[6 * b + a];
        std::memset(&d, 0, sizeof(d));
        d.nx = nx;
        d.ny = ny;
        d.nz = nz;
        d.nxh = nxh;
        d.c0x = B.b;
        d.c0y = B.b;
        d.c0z = B.b;
        d.cnx = B.cnx;
        d.cny = B.cny;
        d.cnz = B.cnz;
        d.px = c.tab.index[nx];
        d.py = c.tab.index[ny];
        d.pz = c.tab.index[nz];
        d.lc = a;
        d.box = b0 + b;
        d.plane0 = (int)pitems.size();
        const bool ct_on = o.shape_kernels != 0 && sizeof(T) == 4;
        d.cw = tuned_column_width<T>(c, nx, ny, nz, o.nyquist, o.autotune != 0, ct_on && ct_col_length(nz));
        d.ct_col = (ct_on && ct_col_length(nz) && ct_width(d.cw)) ? nz * 64 + d.cw : 0;
        d.col0 = (int)ccount;
        ccount += ((long long)ny * nxh + d.cw - 1) / d.cw;
        d.med_off = (med.kind == MED_ISO) ? lab_off : c21_off;
        d.fld_off = fld_off;
        d.spc_off = spc_off;
        const int pr = 6 * b + a;
        for (int k = 0; k < nz; ++k) pitems.push_back(make_int2(pr, k));
        d.part0 = (int)prow;
        if (plane_smem_bytes<T>(nx, ny, nphase) <= plane_lim) {
          d.rows = 0;
          d.npi = nz;
          const int g = ct_on ? ct_plane_group(nx, ny) : -1;
          d.ct_plane = g >= 0 ? nx * 64 + ny : 0;
          const size_t pb = plane_smem_bytes<T>(nx, ny, nphase);
          // compiled-shape problems get launch classes of their own, one per group
          std::vector<int2>& pc = pclass[need(pneed, (smem_bucket(pb) << 3) | (g >= 0 ? 1 + g : 0), pb)];
          for (int k = 0; k < nz; ++k) pc.push_back(make_int2(pr, k));
        } else {
          const int R = stream_rows(nx, ny);
          const int nch = (ny + R - 1) / R;
          d.rows = R;
          d.npi = nz * nch;
          const size_t rb = rows_smem_bytes<T>(nx, R, nphase), yb = ycol_smem_bytes<T>(ny, ycw);
          std::vector<int2>& rc = rclass[need(rneed, smem_bucket(rb) << 3, rb)];
          std::vector<int2>& yc = yclass[need(yneed, smem_bucket(yb) << 3, yb)];
          for (int k = 0; k < nz; ++k) {
            for (int j = 0; j < nch; ++j) rc.push_back(make_int2(pr, k | ((j * R) << 16)));
            for (int x0 = 0; x0 < nxh; x0 += ycw) yc.push_back(make_int2(pr, k | (x0 << 16)));
          }
        }
        prow += d.npi;
        const size_t cb = column_smem_bytes<T>(d.cw, nz, ny);
        const size_t ckey = need(cneed, (smem_bucket(cb) << 3) | (d.ct_col ? 1 : 0), cb);
        std::vector<int2>& cc = cclass[ckey];
        for (int j0 = 0; j0 < ny * nxh; j0 += d.cw) cc.push_back(make_int2(6 * b + a, j0));
        fld_off += 6 * V;
        spc_off += 6LL * nz * ny * nxh;
      }
      lab_off += V;
      c21_off += 21 * V;
    }
    // class item lists, concatenated: plane classes first, then column classes
    struct Cls {
      size_t smem;
      long long off;
      int n;
      int grid_f, grid_i;
      bool rows;
      int ct;   // 1 + group when every problem has a compiled shape (k_plane_*_ct, k_column_ct), else 0
      int grid_fc, grid_ic;
    };
    std::vector<Cls> pcl, ycl, ccl;
    citems.clear();
    std::vector<int2> clsitems;
    // within a launch, the largest problems first (shortest tail)
    auto by_size = [&](const int2& a, const int2& b) {
      const Prob& pa = probs[a.x];
      const Prob& pb = probs[b.x];
      return (long long)pa.nx * pa.ny * pa.nz > (long long)pb.nx * pb.ny * pb.nz;
    };
    auto add_classes = [&](std::map<size_t, std::vector<int2>>& m, std::map<size_t, size_t>& nd, std::vector<Cls>& out,
                           bool rows) {
      for (auto& kv : m) {
        std::stable_sort(kv.second.begin(), kv.second.end(), by_size);
        out.push_back({nd[kv.first], (long long)clsitems.size(), (int)kv.second.size(), 0, 0, rows,
                       (int)(kv.first & 7), 0, 0});
        clsitems.insert(clsitems.end(), kv.second.begin(), kv.second.end());
      }
    };
    add_classes(pclass, pneed, pcl, false);
    add_classes(rclass, rneed, pcl, true);
    add_classes(yclass, yneed, ycl, false);
    add_classes(cclass, cneed, ccl, false);
    citems = clsitems;
    // ---- device buffers
    Prob* d_prob;
    PState* d_st;
    int2 *d_pit, *d_cit, *d_git;
    BoxReq* d_boxes;
    T *d_r, *d_p, *d_q, *d_x, *d_c21 = nullptr;
    C2<T>* d_spec;
    double* d_part;
    uint8_t* d_lab = nullptr;
    int* d_flag;
    if ((s = ensure(c, "prob", np * sizeof(Prob), (void**)&d_prob)) != HH_OK) return s;
    if ((s = ensure(c, "state", np * sizeof(PState), (void**)&d_st)) != HH_OK) return s;
    if ((s = ensure(c, "pitems", pitems.size() * sizeof(int2), (void**)&d_pit)) != HH_OK) return s;
    if ((s = ensure(c, "citems", citems.size() * sizeof(int2), (void**)&d_cit)) != HH_OK) return s;
    if ((s = ensure(c, "gitems", gitems.size() * sizeof(int2), (void**)&d_git)) != HH_OK) return s;
    if ((s = ensure(c, "boxes", nb * sizeof(BoxReq), (void**)&d_boxes)) != HH_OK) return s;
    if ((s = ensure(c, "r", fld_off * sizeof(T), (void**)&d_r)) != HH_OK) return s;
    if ((s = ensure(c, "p", fld_off * sizeof(T), (void**)&d_p)) != HH_OK) return s;
    if ((s = ensure(c, "q", fld_off * sizeof(T), (void**)&d_q)) != HH_OK) return s;
    if ((s = ensure(c, "x", fld_off * sizeof(T), (void**)&d_x)) != HH_OK) return s;
    if ((s = ensure(c, "spec", spc_off * sizeof(C2<T>), (void**)&d_spec)) != HH_OK) return s;
    if ((s = ensure(c, "part", std::max<size_t>(pitems.size(), prow) * 16 * sizeof(double), (void**)&d_part)) !=
        HH_OK)
      return s;
    double* d_cpart = nullptr;
    if (basic && (s = ensure(c, "cpart", std::max<long long>(ccount, 1) * 8 * sizeof(double), (void**)&d_cpart)) != HH_OK)
      return s;
    if ((s = ensure(c, "flag", 64, (void**)&d_flag)) != HH_OK) return s;
    HH_CK(cudaMemcpyAsync(d_prob, probs.data(), np * sizeof(Prob), cudaMemcpyHostToDevice, c.st));
    HH_CK(cudaMemcpyAsync(d_pit, pitems.data(), pitems.size() * sizeof(int2), cudaMemcpyHostToDevice, c.st));
    HH_CK(cudaMemcpyAsync(d_cit, citems.data(), citems.size() * sizeof(int2), cudaMemcpyHostToDevice, c.st));
    HH_CK(cudaMemcpyAsync(d_git, gitems.data(), gitems.size() * sizeof(int2), cudaMemcpyHostToDevice, c.st));
    HH_CK(cudaMemcpyAsync(d_boxes, wboxes.data(), nb * sizeof(BoxReq), cudaMemcpyHostToDevice, c.st));
    HH_CK(cudaMemsetAsync(d_flag, 0, 64, c.st));
    if (med.kind == MED_ISO) {
      if ((s = ensure(c, "labels", lab_off, (void**)&d_lab)) != HH_OK) return s;
      ++c.launches;
      k_gather<<<grid_for<T>(c, (const void*)k_gather, 256, 0, (int)gitems.size()), 256, 0, c.st>>>(
          med.d_img, med.Nx, med.Ny, med.Nz, d_boxes, d_git, (int)gitems.size(), d_lab, nphase, d_flag);
      HH_CK(cudaGetLastError());
    } else {
      if ((s = ensure(c, "c21T", c21_off * sizeof(T), (void**)&d_c21)) != HH_OK) return s;
      ++c.launches;
      k_gather_c21<T><<<grid_for<T>(c, (const void*)k_gather_c21<T>, 256, 0, (int)gitems.size()), 256, 0, c.st>>>(
          med.d_c21, med.Nx, med.Ny, med.Nz, d_boxes, d_git, (int)gitems.size(), d_c21, d_flag);
      HH_CK(cudaGetLastError());
    }
    HH_CK(cudaMemcpyAsync(c.h_int, d_flag, sizeof(int), cudaMemcpyDeviceToHost, c.st));
    HH_CK(cudaStreamSynchronize(c.st));
    if (c.h_int[0]) {
      if (med.kind == MED_ISO) {
        c.err = "label >= nphase in image";
        return HH_ERR_ARG;
      }
      c.err = "stiffness not symmetric positive definite";
      return HH_ERR_BAD_STIFFNESS;
    }

    KParams<T> kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.prob = d_prob;
    kp.st = d_st;
    kp.medium = med.kind;
    kp.nyq_mode = o.nyquist;
    kp.ycw = ycw;
    kp.nphase = std::max(nphase, 1);
    kp.plans = (const AxisPlan*)c.d_plans.p;
    kp.tw = (const double*)c.d_tw.p;
    kp.itab = (const int*)c.d_itab.p;
    kp.labels = d_lab;
    kp.lammu = d_lm;
    kp.c21 = d_c21;
    kp.r = d_r;
    kp.p = d_p;
    kp.q = d_q;
    kp.x = d_x;
    kp.spec = d_spec;
    kp.part = d_part;
    kp.tol = o.tol;
    kp.max_iter = o.max_iter;
    kp.fixed_iters = o.fixed_iters;
    kp.g0a = T(1.0 / (2.0 * mu0));
    kp.g0b = T((lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0)));
    kp.cpart = d_cpart;
    kp.nprob = np;
    KParams<T> kpp = kp;
    kpp.items = d_pit;
    kpp.nitems = (int)pitems.size();
    for (Cls& k : pcl) {
      k.grid_f = grid_for<T>(c, (const void*)kfwd(MODE_ITER, k.rows), threads, k.smem, k.n);
      k.grid_i = grid_for<T>(c, (const void*)kinv(MODE_ITER, k.rows), threads, k.smem, k.n);
      if (k.ct) k.grid_fc = k.grid_ic = k.n;  // one block per item
    }
    for (Cls& k : ycl) k.grid_f = k.grid_i = grid_for<T>(c, (const void*)kyf, threads, k.smem, k.n);
    for (Cls& k : ccl) {
      k.grid_f = grid_for<T>(c, (const void*)kc, threads, k.smem, k.n);
      if (k.ct) k.grid_fc = k.n;
    }
    auto cls_params = [&](const Cls& k) {
      KParams<T> q = kp;
      q.items = d_cit + k.off;
      q.nitems = k.n;
      return q;
    };
    // one launch per class for the plane and column passes, the classes of
    // one group spread over the pass streams (fork from c.st, join back)
    int nfork = 0;  // pass streams forked in the current group
    auto gstream = [&](int i, int n) -> cudaStream_t {
      if (kPassStreams <= 1 || n <= 1) return c.st;
      const int j = i % kPassStreams;
      if (j >= nfork) {
        if (nfork == 0) (void)cudaEventRecord(c.ev_fork, c.st);
        (void)cudaStreamWaitEvent(c.side[j], c.ev_fork, 0);
        nfork = j + 1;
      }
      return c.side[j];
    };
    auto gjoin = [&]() {
      for (int j = 0; j < nfork; ++j) {
        (void)cudaEventRecord(c.ev_join[j], c.side[j]);
        (void)cudaStreamWaitEvent(c.st, c.ev_join[j], 0);
      }
      nfork = 0;
    };
    // forward pass of a mode: whole planes and streaming rows, then the
    // streaming problems' y transforms; the inverse pass in reverse order
    auto fwd_pass = [&](int mode) {
      const int n = (int)pcl.size();
      for (int i = 0; i < n; ++i) {
        const Cls& k = pcl[i];
        ++c.launches;
        cudaStream_t s = gstream(i, n);
        if (k.ct && mode == MODE_ITER)
          kfct[k.ct - 1]<<<k.grid_fc, threads, k.smem, s>>>(cls_params(k));
        else
          kfwd(mode, k.rows)<<<k.grid_f, threads, k.smem, s>>>(cls_params(k));
      }
      gjoin();
      const int ny_ = (int)ycl.size();
      for (int i = 0; i < ny_; ++i) {
        ++c.launches;
        kyf<<<ycl[i].grid_f, threads, ycl[i].smem, gstream(i, ny_)>>>(cls_params(ycl[i]), mode);
      }
      gjoin();
    };
    auto inv_pass = [&](int mode) {
      const int ny_ = (int)ycl.size();
      for (int i = 0; i < ny_; ++i) {
        ++c.launches;
        kyi<<<ycl[i].grid_i, threads, ycl[i].smem, gstream(i, ny_)>>>(cls_params(ycl[i]), mode);
      }
      gjoin();
      const int n = (int)pcl.size();
      for (int i = 0; i < n; ++i) {
        const Cls& k = pcl[i];
        ++c.launches;
        cudaStream_t s = gstream(i, n);
        if (k.ct && mode == MODE_ITER)
          kict[k.ct - 1]<<<k.grid_ic, threads, k.smem, s>>>(cls_params(k));
        else
          kinv(mode, k.rows)<<<k.grid_i, threads, k.smem, s>>>(cls_params(k));
      }
      gjoin();
    };
    auto column_pass = [&](int mode) {
      const int n = (int)ccl.size();
      for (int i = 0; i < n; ++i) {
        const Cls& k = ccl[i];
        ++c.launches;
        cudaStream_t s = gstream(i, n);
        if (k.ct && mode != MODE_BASIC)
          kcct<<<k.grid_fc, threads, k.smem, s>>>(cls_params(k), mode);
        else
          (mode == MODE_BASIC ? kcb : kc)<<<k.grid_f, threads, k.smem, s>>>(cls_params(k), mode);
      }
      gjoin();
    };
    const int gu = grid_for<T>(c, (const void*)ku, threads, 0, kpp.nitems);
    const int gs = (np + 127) / 128;

    hh_status rs = HH_OK;
    const int chunk = std::max(1, o.check_every);
    const long long max_chunks =
        ((long long)(o.fixed_iters > 0 ? o.fixed_iters : o.max_iter) / chunk + 2) * (o.max_restarts + 2);
    // ---- fused solves first: they leave their problems' states final
    //      (inactive, nothing pending), which the multi-pass kernels skip
    cudaEvent_t fev[2] = {nullptr, nullptr};
    if (!fgroups.empty()) {
      FusedParams<T> fp;
      std::memset(&fp, 0, sizeof(fp));
      fp.prob = d_prob;
      fp.st = d_st;
      fp.plans = (const AxisPlan*)c.d_plans.p;
      fp.tw = (const double*)c.d_tw.p;
      fp.itab = (const int*)c.d_itab.p;
      fp.labels = d_lab;
      fp.lammu = d_lm;
      fp.nphase = std::max(nphase, 1);
      fp.nyq_mode = o.nyquist;
      fp.r = d_r;
      fp.p = d_p;
      fp.x = d_x;
      fp.tol = o.tol;
      fp.floor2 = floor2;
      fp.max_iter = o.max_iter;
      fp.fixed_iters = o.fixed_iters;
      fp.chunk = chunk;
      fp.replace = replace ? 1 : 0;
      fp.max_restarts = o.max_restarts;
      fp.max_chunks = max_chunks;
      if (o.profile) {
        for (auto& e : fev) HH_CK(cudaEventCreate(&e));
        HH_CK(cudaEventRecord(fev[0], c.st));
      }
      if ((s = run_fused<T>(c, fgroups, probs, fp, std::max(nphase, 1))) != HH_OK) return s;
      if (o.profile) HH_CK(cudaEventRecord(fev[1], c.st));
    }
    if (n_multipass == 0) {
      // every problem of the wave was solved by the fused kernel
    } else if (basic) {
      // ---- basic scheme (Moulinec-Suquet fixed point): x = eps - E = 0, then
      //      per iteration sigma = C:(E + x), residual, x <- x - Gamma0 * sigma.
      //      Accelerated scheme: tau = (C - C0):(E + x) forward, the inverse
      //      pass applies x <- x + 2 (C + C0)^-1 C0 : B with B = -(x + Gamma0 * tau)
      HH_CK(cudaMemsetAsync(d_x, 0, fld_off * sizeof(T), c.st));
      ++c.launches;
      k_scal_basic_init<<<gs, 128, 0, c.st>>>(d_st, np);
      HH_CK(cudaGetLastError());
      kp.em = em ? 1 : 0;
      auto basic_chunk = [&]() {
        for (int m = 0; m < chunk; ++m) {
          if (em) kp.lammu = d_lm_tau;
          fwd_pass(MODE_BASIC);
          column_pass(MODE_BASIC);
          if (em) kp.lammu = d_lm_em;
          inv_pass(MODE_BASIC);
          kp.lammu = d_lm;
          ++c.launches;
          k_scal_basic<<<gs, 128, 0, c.st>>>(d_prob, d_st, d_cpart, d_part, np, o.tol, o.max_iter, o.fixed_iters,
                                             em ? 1 : 0);
        }
      };
      cudaGraphExec_t bexec = nullptr;
      long long bk = 0;
      if (o.use_graphs) {
        cudaGraph_t g = nullptr;
        HH_CK(cudaStreamBeginCapture(c.st, cudaStreamCaptureModeThreadLocal));
        const long long l0 = c.launches;
        basic_chunk();
        bk = c.launches - l0;
        c.launches = l0;
        cudaError_t ce = cudaStreamEndCapture(c.st, &g);
        if (ce == cudaSuccess) {
          ce = cudaGraphInstantiate(&bexec, g, 0);
          cudaGraphDestroy(g);
        }
        if (ce != cudaSuccess) {
          c.err = std::string("graph: ") + cudaGetErrorString(ce);
          return HH_ERR_CUDA;
        }
      }
      for (long long chunks = 0;; ++chunks) {
        ++c.launches;
        k_count_active<<<1, 256, 0, c.st>>>(d_st, d_prob, np, d_flag,
                                            reinterpret_cast<unsigned long long*>(d_flag + 4));
        cudaMemcpyAsync(c.h_int, d_flag, sizeof(int), cudaMemcpyDeviceToHost, c.st);
        cudaError_t e = cudaStreamSynchronize(c.st);
        if (e != cudaSuccess) {
          c.err = std::string("solve: ") + cudaGetErrorString(e);
          rs = HH_ERR_CUDA;
          break;
        }
        if (c.h_int[0] == 0 || chunks >= max_chunks) break;
        if (bexec) {
          e = cudaGraphLaunch(bexec, c.st);
          c.launches += bk;
        } else {
          basic_chunk();
          e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
          c.err = std::string("launch: ") + cudaGetErrorString(e);
          rs = HH_ERR_CUDA;
          break;
        }
      }
      if (bexec) cudaGraphExecDestroy(bexec);
    } else {
      // ---- right-hand side b = -G*(C:E), r = p = b, x = 0
      fwd_pass(MODE_RHS);
      column_pass(MODE_RHS);
      inv_pass(MODE_RHS);
      ++c.launches;
      k_scal_init<<<gs, 128, 0, c.st>>>(d_prob, d_st, d_part, np, floor2);
      HH_CK(cudaGetLastError());

      // profiling: events around the field kernels of the first iteration of every chunk
      const bool prof = o.profile != 0;
      cudaEvent_t pev[4] = {nullptr, nullptr, nullptr, nullptr};
      if (prof)
        for (auto& e : pev) HH_CK(cudaEventCreate(&e));
      // external record nodes, so that the events are timed inside graph replays
      auto rec = [&](int m, int k) {
        if (prof && m == 0) {
          if (cudaEventRecordWithFlags(pev[k], c.st, cudaEventRecordExternal) != cudaSuccess) (void)cudaGetLastError();
        }
      };
      // apply the deferred CG updates of every problem that has one
      auto flush = [&]() {
        ++c.launches;
        ku<<<gu, threads, 0, c.st>>>(kpp);
        ++c.launches;
        k_scal_clear<<<gs, 128, 0, c.st>>>(d_st, np);
      };
      // true residual r = -G*(C:(E + x)) of the flagged problems
      auto true_pass = [&]() {
        fwd_pass(MODE_TRUE);
        column_pass(MODE_TRUE);
        inv_pass(MODE_TRUE);
      };
      // ---- iterations, in chunks captured as CUDA graphs; residual
      //      replacement at the end of every chunk (when enabled)
      auto launch_chunk = [&]() {
        for (int m = 0; m < chunk; ++m) {
          rec(m, 0);
          fwd_pass(MODE_ITER);
          rec(m, 1);
          column_pass(MODE_ITER);
          rec(m, 2);
          inv_pass(MODE_ITER);
          rec(m, 3);
          ++c.launches;
          k_scal_step<<<gs, 128, 0, c.st>>>(d_prob, d_st, d_part, np, o.tol, o.max_iter, o.fixed_iters);
        }
        if (replace) {
          flush();
          ++c.launches;
          k_mark_true<<<gs, 128, 0, c.st>>>(d_prob, d_st, np, 0);
          true_pass();
          ++c.launches;
          k_scal_replace<<<gs, 128, 0, c.st>>>(d_prob, d_st, d_part, np, o.tol, o.fixed_iters);
        }
      };
      cudaGraphExec_t exec = nullptr;
      long long chunk_kernels = 0;
      if (o.use_graphs) {
        cudaGraph_t g = nullptr;
        HH_CK(cudaStreamBeginCapture(c.st, cudaStreamCaptureModeThreadLocal));
        const long long l0 = c.launches;
        launch_chunk();
        chunk_kernels = c.launches - l0;
        c.launches = l0;
        cudaError_t ce = cudaStreamEndCapture(c.st, &g);
        if (ce != cudaSuccess) {
          c.err = std::string("graph capture: ") + cudaGetErrorString(ce);
          return HH_ERR_CUDA;
        }
        ce = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) {
          c.err = std::string("graph instantiate: ") + cudaGetErrorString(ce);
          return HH_ERR_CUDA;
        }
      }
      long long chunks = 0;
      int final_rounds = 0;
      // algorithmic bytes per voxel (a) and per half-spectrum element (b) of the
      // four field kernels: every field value read or written once
      const double Tb = sizeof(T);
      const double lab_b = (med.kind == MED_ISO) ? 1.0 : 21.0 * Tb;
      // (plane_fwd: r, q, p, x read, r, x, p written, label, half spectrum
      // written; plane_inv: half spectrum read, p, r read, q written)
      const char* pnames[3] = {"plane_fwd", "column", "plane_inv"};
      const double pa[3] = {42.0 * Tb + lab_b, 0.0, 18.0 * Tb};
      const double pb[3] = {2.0 * Tb, 4.0 * Tb, 2.0 * Tb};
      unsigned long long* h_vs = reinterpret_cast<unsigned long long*>(c.h_dbl);
      double act_v = 0.0, act_s = 0.0;
      bool sampled_pending = false;
      auto count_active = [&](int* out) -> cudaError_t {
        ++c.launches;
        k_count_active<<<1, 256, 0, c.st>>>(d_st, d_prob, np, d_flag, reinterpret_cast<unsigned long long*>(d_flag + 4));
        cudaMemcpyAsync(c.h_int, d_flag, sizeof(int), cudaMemcpyDeviceToHost, c.st);
        cudaMemcpyAsync(h_vs, d_flag + 4, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c.st);
        cudaError_t e = cudaStreamSynchronize(c.st);
        *out = c.h_int[0];
        if (e == cudaSuccess && prof && sampled_pending) {
          const int pairs[3][2] = {{0, 1}, {1, 2}, {2, 3}};
          for (int k = 0; k < 3; ++k) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, pev[pairs[k][0]], pev[pairs[k][1]]) == cudaSuccess) {
              Ctx::KStat& ks = c.prof[pnames[k]];
              ks.sampled += 1;
              ks.ms += ms;
              ks.bytes += pa[k] * act_v + pb[k] * act_s;
            } else {
              (void)cudaGetLastError();  // profiling is best effort; keep the error state clean
            }
          }
          sampled_pending = false;
        }
        if (e == cudaSuccess) {
          act_v = double(h_vs[0]);
          act_s = double(h_vs[1]);
        }
        return e;
      };
      while (true) {
        int nact = 0;
        cudaError_t e = count_active(&nact);
        if (e != cudaSuccess) {
          c.err = std::string("solve: ") + cudaGetErrorString(e);
          rs = HH_ERR_CUDA;
          break;
        }
        if (nact == 0) {
          // every problem stopped on its recursive residual: check the true one
          if (final_rounds > o.max_restarts) break;
          flush();
          ++c.launches;
          k_mark_true<<<gs, 128, 0, c.st>>>(d_prob, d_st, np, 1);
          true_pass();
          ++c.launches;
          k_scal_true_final<<<gs, 128, 0, c.st>>>(d_prob, d_st, d_part, np, o.tol, 2.0, o.max_restarts, o.max_iter,
                                                   o.fixed_iters);
          ++final_rounds;
          if ((e = count_active(&nact)) != cudaSuccess) {
            c.err = std::string("solve: ") + cudaGetErrorString(e);
            rs = HH_ERR_CUDA;
            break;
          }
          if (nact == 0) break;
        }
        if (chunks >= max_chunks) break;
        if (exec) {
          e = cudaGraphLaunch(exec, c.st);
          c.launches += chunk_kernels;
        } else {
          launch_chunk();
          e = cudaGetLastError();
        }
        if (prof) {
          sampled_pending = true;
          const long long per[3] = {(long long)(pcl.size() + ycl.size()), (long long)ccl.size(),
                                    (long long)(pcl.size() + ycl.size())};
          for (int k = 0; k < 3; ++k) c.prof[pnames[k]].launches += chunk * per[k];
        }
        if (e != cudaSuccess) {
          c.err = std::string("launch: ") + cudaGetErrorString(e);
          rs = HH_ERR_CUDA;
          break;
        }
        ++chunks;
      }
      if (exec) cudaGraphExecDestroy(exec);
      for (auto& e : pev)
        if (e) cudaEventDestroy(e);
    }
    if (rs != HH_OK) return rs;

    // ---- core averages from x (the fused kernel formed its own)
    if (n_multipass > 0) {
      if (!basic) {
        ++c.launches;
        ku<<<gu, threads, 0, c.st>>>(kpp);
        ++c.launches;
        k_scal_clear<<<gs, 128, 0, c.st>>>(d_st, np);
      }
      const int ga = grid_for<T>(c, (const void*)ka, threads, 0, kpp.nitems);
      ++c.launches;
      ka<<<ga, threads, 0, c.st>>>(kpp);
      ++c.launches;
      k_scal_avg<<<gs, 128, 0, c.st>>>(d_prob, d_st, d_part, np);
      HH_CK(cudaGetLastError());
    }

    // ---- per-box results
    ++c.launches;
    k_finalize<<<(nb + 63) / 64, 64, 0, c.st>>>(d_prob, d_st, nb, d_res, b0, med.floor);
    HH_CK(cudaGetLastError());
    // statistics
    std::vector<PState> hst(np);
    HH_CK(cudaMemcpyAsync(hst.data(), d_st, np * sizeof(PState), cudaMemcpyDeviceToHost, c.st));
    HH_CK(cudaStreamSynchronize(c.st));
    double fused_units = 0.0;
    for (int i = 0; i < np; ++i) {
      const Prob& d = probs[i];
      stats.iters_max = std::max(stats.iters_max, hst[i].iters);
      stats.resid_max = std::max(stats.resid_max, hst[i].resid);
      stats.voxel_iters += (long long)d.nx * d.ny * d.nz * hst[i].iters;
      if (d.fused) fused_units += double(d.nx) * d.ny * d.nz * hst[i].iters;
      if (d.fused && d.lc == 0) ++stats.fused_boxes;
      if (hst[i].status == ST_NONFINITE) stats.worst = ST_NONFINITE;
      else if (hst[i].status == ST_NOT_CONVERGED && stats.worst == ST_OK) stats.worst = ST_NOT_CONVERGED;
    }
    if (fev[0]) {
      // the fused launches of the wave: algorithmic bytes per voxel-iteration
      // = r, p, x read, r, x, p written, the label, and p, r read again
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, fev[0], fev[1]) == cudaSuccess) {
        Ctx::KStat& ks = c.prof["fused"];
        ks.launches += (long long)fgroups.size();
        ks.sampled += 1;
        ks.ms += ms;
        ks.bytes += fused_units * (48.0 * sizeof(T) + 1.0);
        Ctx::KStat& ku = c.prof["fused_units"];
        ku.sampled += 1;
        ku.bytes += fused_units;
      }
      (void)cudaGetLastError();
      for (auto& e : fev) cudaEventDestroy(e);
    }
    b0 = b1;
  }
  return HH_OK;
}

// q = G*(C:p) for one field (parity of the operator).
template <typename T>
static hh_status apply_operator(Ctx& c, const hh_options& o, const Medium& med, int nx, int ny, int nz,
                                const double* h_p, double* h_q) {
  const int px = plan_for(c.tab, nx), py = plan_for(c.tab, ny), pz = plan_for(c.tab, nz);
  if (px < 0 || py < 0 || pz < 0) {
    c.err = "unsupported FFT length";
    return HH_ERR_UNSUPPORTED;
  }
  hh_status s = upload_tables(c);
  if (s != HH_OK) return s;
  const int nphase = (int)med.lam.size();
  const long long V = (long long)nx * ny * nz;
  const int nxh = nx / 2 + 1;
  const size_t psm = plane_smem_bytes<T>(nx, ny, nphase);
  const int colw = column_width<T>(nz, ny, c.smem_optin);
  const size_t csm = column_smem_bytes<T>(colw, nz, ny);
  if (psm > c.smem_optin || csm > c.smem_optin) {
    c.err = "plane too large for shared memory";
    return HH_ERR_UNSUPPORTED;
  }
  Prob d;
  std::memset(&d, 0, sizeof(d));
  d.nx = nx;
  d.ny = ny;
  d.nz = nz;
  d.nxh = nxh;
  d.cnx = nx;
  d.cny = ny;
  d.cnz = nz;
  d.px = px;
  d.py = py;
  d.pz = pz;
  d.cw = colw;
  d.npi = nz;
  std::vector<int2> pit, cit;
  for (int k = 0; k < nz; ++k) pit.push_back(make_int2(0, k));
  for (int j0 = 0; j0 < ny * nxh; j0 += colw) cit.push_back(make_int2(0, j0));
  Prob* d_prob;
  int2 *d_pit, *d_cit;
  T *d_p, *d_q, *d_c21 = nullptr, *d_lm;
  C2<T>* d_spec;
  uint8_t* d_lab = nullptr;
  int* d_flag;
  if ((s = ensure(c, "prob", sizeof(Prob), (void**)&d_prob)) != HH_OK) return s;
  if ((s = ensure(c, "pitems", pit.size() * sizeof(int2), (void**)&d_pit)) != HH_OK) return s;
  if ((s = ensure(c, "citems", cit.size() * sizeof(int2), (void**)&d_cit)) != HH_OK) return s;
  if ((s = ensure(c, "p", 6 * V * sizeof(T), (void**)&d_p)) != HH_OK) return s;
  if ((s = ensure(c, "q", 6 * V * sizeof(T), (void**)&d_q)) != HH_OK) return s;
  if ((s = ensure(c, "spec", 6LL * nz * ny * nxh * sizeof(C2<T>), (void**)&d_spec)) != HH_OK) return s;
  if ((s = ensure(c, "lammu", 2 * std::max(nphase, 1) * sizeof(T), (void**)&d_lm)) != HH_OK) return s;
  if ((s = ensure(c, "flag", 64, (void**)&d_flag)) != HH_OK) return s;
  std::vector<T> hp(6 * V);
  for (long long i = 0; i < 6 * V; ++i) hp[i] = T(h_p[i]);
  HH_CK(cudaMemcpyAsync(d_prob, &d, sizeof(Prob), cudaMemcpyHostToDevice, c.st));
  HH_CK(cudaMemcpyAsync(d_pit, pit.data(), pit.size() * sizeof(int2), cudaMemcpyHostToDevice, c.st));
  HH_CK(cudaMemcpyAsync(d_cit, cit.data(), cit.size() * sizeof(int2), cudaMemcpyHostToDevice, c.st));
  HH_CK(cudaMemcpyAsync(d_p, hp.data(), 6 * V * sizeof(T), cudaMemcpyHostToDevice, c.st));
  HH_CK(cudaMemsetAsync(d_flag, 0, 64, c.st));
  std::vector<T> lm(2 * std::max(nphase, 1));
  for (int i = 0; i < nphase; ++i) {
    lm[2 * i] = T(med.lam[i]);
    lm[2 * i + 1] = T(med.mu[i]);
  }
  HH_CK(cudaMemcpyAsync(d_lm, lm.data(), lm.size() * sizeof(T), cudaMemcpyHostToDevice, c.st));
  if (med.kind == MED_ISO) {
    if ((s = ensure(c, "labels", V, (void**)&d_lab)) != HH_OK) return s;
    HH_CK(cudaMemcpyAsync(d_lab, med.d_img, V, cudaMemcpyDeviceToDevice, c.st));
  } else {
    if ((s = ensure(c, "c21T", 21 * V * sizeof(T), (void**)&d_c21)) != HH_OK) return s;
    ++c.launches;
    k_c21_prepare<T><<<std::max(1, std::min<int>(c.nsm * 8, (int)((V + 255) / 256))), 256, 0, c.st>>>(
        med.d_c21, d_c21, V, d_flag);
    HH_CK(cudaGetLastError());
  }
  KParams<T> kp;
  std::memset(&kp, 0, sizeof(kp));
  kp.prob = d_prob;
  kp.medium = med.kind;
  kp.nyq_mode = o.nyquist;
  kp.nphase = std::max(nphase, 1);
  kp.plans = (const AxisPlan*)c.d_plans.p;
  kp.tw = (const double*)c.d_tw.p;
  kp.itab = (const int*)c.d_itab.p;
  kp.labels = d_lab;
  kp.lammu = d_lm;
  kp.c21 = d_c21;
  kp.p = d_p;
  kp.q = d_q;
  kp.r = d_q;
  kp.x = d_q;
  kp.spec = d_spec;
  kp.nprob = 1;
  KParams<T> kpp = kp, kpc = kp;
  kpp.items = d_pit;
  kpp.nitems = nz;
  kpc.items = d_cit;
  kpc.nitems = (int)cit.size();
  auto* kf = k_plane_fwd<T, MODE_APPLY>;
  auto* ki = k_plane_inv<T, MODE_APPLY>;
  auto* kc = k_column<T, false>;
  HH_CK(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm));
  HH_CK(cudaFuncSetAttribute(ki, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm));
  HH_CK(cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm));
  ++c.launches;
  kf<<<std::min(nz, 4 * c.nsm), 256, psm, c.st>>>(kpp);
  ++c.launches;
  kc<<<std::min((int)cit.size(), 4 * c.nsm), 256, csm, c.st>>>(kpc, MODE_APPLY);
  ++c.launches;
  ki<<<std::min(nz, 4 * c.nsm), 256, psm, c.st>>>(kpp);
  HH_CK(cudaGetLastError());
  HH_CK(cudaMemcpyAsync(c.h_int, d_flag, sizeof(int), cudaMemcpyDeviceToHost, c.st));
  std::vector<T> hq(6 * V);
  HH_CK(cudaMemcpyAsync(hq.data(), d_q, 6 * V * sizeof(T), cudaMemcpyDeviceToHost, c.st));
  HH_CK(cudaStreamSynchronize(c.st));
  if (med.kind == MED_ANISO && c.h_int[0]) {
    c.err = "stiffness not symmetric positive definite";
    return HH_ERR_BAD_STIFFNESS;
  }
  for (long long i = 0; i < 6 * V; ++i) h_q[i] = double(hq[i]);
  return HH_OK;
}

}  // namespace hh

// ===========================================================================
// C ABI
// ===========================================================================
using namespace hh;

struct hh_ctx {
  Ctx c;
};

static thread_local char g_last_error[512];

static void set_last_error(const char* msg) {
  std::strncpy(g_last_error, msg, sizeof(g_last_error) - 1);
  g_last_error[sizeof(g_last_error) - 1] = 0;
}

static hh_status fail(hh_ctx* ctx, hh_status s, const std::string& msg) {
  if (ctx) ctx->c.err = msg;
  set_last_error(msg.c_str());
  return s;
}

extern "C" const char* hh_version(void) { return "libhh 0.1 (sm_103a)"; }

extern "C" const char* hh_status_string(hh_status s) {
  switch (s) {
    case HH_OK: return "ok";
    case HH_WARN_NOT_CONVERGED: return "warning: not converged within max_iter";
    case HH_WARN_TARGET_UNMET: return "warning: no candidate meets the error target";
    case HH_ERR_ARG: return "error: invalid argument";
    case HH_ERR_OOM: return "error: out of memory";
    case HH_ERR_CUDA: return "error: CUDA runtime failure";
    case HH_ERR_NONFINITE: return "error: non-finite value in the solver";
    case HH_ERR_DEVICE_TIMEOUT: return "error: bounded device wait ran out";
    case HH_ERR_BAD_STIFFNESS: return "error: stiffness not symmetric positive definite";
    case HH_ERR_UNSUPPORTED: return "error: unsupported size";
    default: return "error: unknown status";
  }
}

extern "C" const char* hh_last_error(hh_ctx* ctx) {
  return ctx ? ctx->c.err.c_str() : g_last_error;
}

extern "C" hh_status hh_options_default(hh_options* o) {
  if (!o) return HH_ERR_ARG;
  std::memset(o, 0, sizeof(*o));
  o->precision = HH_FP32;
  o->tol = 1e-6;
  o->max_iter = 20000;
  o->scheme = HH_CG;
  o->nyquist = HH_NYQ_ZERO_COMPONENT;
  o->fixed_iters = 0;
  o->use_graphs = 1;
  o->check_every = 32;
  o->replace = -1;
  o->max_restarts = 4;
  o->autotune = 1;
  o->fused = 0;
  o->shape_kernels = 1;
  return HH_OK;
}

extern "C" hh_status hh_create(hh_ctx** out, int device, void* cuda_stream) {
  if (!out) return HH_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n)
    return fail(nullptr, HH_ERR_ARG, "no such CUDA device");
  hh_ctx* h = new (std::nothrow) hh_ctx();
  if (!h) return HH_ERR_OOM;
  Ctx& c = h->c;
  c.dev = device;
  auto bad = [&](cudaError_t e) {
    set_last_error(cudaGetErrorString(e));
    delete h;
    return e == cudaErrorMemoryAllocation ? HH_ERR_OOM : HH_ERR_CUDA;
  };
  cudaError_t e;
  if ((e = cudaSetDevice(device)) != cudaSuccess) return bad(e);
  cudaDeviceProp prop;
  if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess) return bad(e);
  c.nsm = prop.multiProcessorCount;
  c.smem_optin = prop.sharedMemPerBlockOptin;
  if ((e = cudaStreamCreateWithFlags(&c.st, cudaStreamNonBlocking)) != cudaSuccess) return bad(e);
  c.user = (cudaStream_t)cuda_stream;
  if ((e = cudaMallocHost((void**)&c.h_int, 64 * sizeof(int))) != cudaSuccess) return bad(e);
  if ((e = cudaMallocHost((void**)&c.h_dbl, 64 * sizeof(double))) != cudaSuccess) return bad(e);
  if ((e = cudaEventCreate(&c.ev_call0)) != cudaSuccess) return bad(e);
  if ((e = cudaEventCreate(&c.ev_call1)) != cudaSuccess) return bad(e);
  if (kPassStreams > 1) {
    if ((e = cudaEventCreateWithFlags(&c.ev_fork, cudaEventDisableTiming)) != cudaSuccess) return bad(e);
    for (int j = 0; j < kPassStreams; ++j) {
      if ((e = cudaStreamCreateWithFlags(&c.side[j], cudaStreamNonBlocking)) != cudaSuccess) return bad(e);
      if ((e = cudaEventCreateWithFlags(&c.ev_join[j], cudaEventDisableTiming)) != cudaSuccess) return bad(e);
    }
  }
  *out = h;
  return HH_OK;
}

extern "C" void hh_destroy(hh_ctx* h) {
  if (!h) return;
  Ctx& c = h->c;
  cudaSetDevice(c.dev);
  if (c.st) cudaStreamSynchronize(c.st);
  for (auto& kv : c.bufs)
    if (kv.second.p) cudaFree(kv.second.p);
  if (c.d_plans.p) cudaFree(c.d_plans.p);
  if (c.d_tw.p) cudaFree(c.d_tw.p);
  if (c.d_itab.p) cudaFree(c.d_itab.p);
  if (c.h_int) cudaFreeHost(c.h_int);
  if (c.h_dbl) cudaFreeHost(c.h_dbl);
  if (c.ev_call0) cudaEventDestroy(c.ev_call0);
  if (c.ev_call1) cudaEventDestroy(c.ev_call1);
  if (c.ev_fork) cudaEventDestroy(c.ev_fork);
  for (int j = 0; j < kPassStreams; ++j) {
    if (c.ev_join[j]) cudaEventDestroy(c.ev_join[j]);
    if (c.side[j]) cudaStreamDestroy(c.side[j]);
  }
  if (c.st) cudaStreamDestroy(c.st);
  delete h;
}

extern "C" hh_status hh_set_memory_limit(hh_ctx* h, int64_t bytes) {
  if (!h || bytes < 0) return fail(h, HH_ERR_ARG, "NULL context or negative limit");
  Ctx& c = h->c;
  HH_CK(cudaSetDevice(c.dev));
  HH_CK(cudaStreamSynchronize(c.st));
  for (auto& kv : c.bufs)
    if (kv.second.p) cudaFree(kv.second.p);
  c.bufs.clear();
  c.mem_limit = (size_t)bytes;
  return HH_OK;
}

// Order the internal stream after the caller's stream (for device inputs),
// and start the call's device timer.
static thread_local long long g_launch0 = 0;
static hh_status enter(hh_ctx* h) {
  Ctx& c = h->c;
  HH_CK(cudaSetDevice(c.dev));
  g_launch0 = c.launches;
  if (c.user) {
    cudaEvent_t ev;
    HH_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    HH_CK(cudaEventRecord(ev, c.user));
    HH_CK(cudaStreamWaitEvent(c.st, ev, 0));
    cudaEventDestroy(ev);
  }
  HH_CK(cudaEventRecord(c.ev_call0, c.st));
  return HH_OK;
}

// Stop the device timer of a call and fill the counters of its result.
// Bridge for the surrogate unit (hh_internal.h).
namespace hh {
int ctx_device(hh_ctx* h) { return h->c.dev; }
cudaStream_t ctx_stream(hh_ctx* h) { return h->c.st; }
hh_status ctx_fail(hh_ctx* h, hh_status s, const char* msg) { return fail(h, s, msg); }
hh_status ctx_enter(hh_ctx* h) { return enter(h); }
}  // namespace hh

static hh_status finish(hh_ctx* h, hh_status s, hh_result* out) {
  Ctx& c = h->c;
  if (s < 0) return s;
  float ms = 0.f;
  if (cudaEventRecord(c.ev_call1, c.st) == cudaSuccess && cudaEventSynchronize(c.ev_call1) == cudaSuccess &&
      cudaEventElapsedTime(&ms, c.ev_call0, c.ev_call1) == cudaSuccess && out) {
    out->device_ms = ms;
  }
  if (out) out->kernel_launches = c.launches - g_launch0;
  return s;
}

static hh_status check_opts(hh_ctx* h, const hh_options* o) {
  if (!o) return fail(h, HH_ERR_ARG, "options is NULL");
  if (o->precision != HH_FP32 && o->precision != HH_FP64) return fail(h, HH_ERR_ARG, "bad precision");
  if (!(o->tol > 0.0) && o->fixed_iters <= 0) return fail(h, HH_ERR_ARG, "tol must be > 0");
  if (o->max_iter < 1 || o->fixed_iters < 0) return fail(h, HH_ERR_ARG, "bad iteration limits");
  if (o->nyquist != HH_NYQ_ZERO_COMPONENT && o->nyquist != HH_NYQ_ZERO_MODE) return fail(h, HH_ERR_ARG, "bad nyquist");
  if (o->scheme != HH_CG && o->scheme != HH_BASIC && o->scheme != HH_EYRE_MILTON) return fail(h, HH_ERR_ARG, "bad scheme");
  if (o->check_every < 0 || o->max_restarts < 0 || o->replace < -1 || o->replace > 1 || o->wave_boxes < 0 ||
      o->fused < 0 || o->fused > 1)
    return fail(h, HH_ERR_ARG, "bad check_every, replace, max_restarts, wave_boxes or fused");
  return HH_OK;
}

static hh_status check_phases(hh_ctx* h, const hh_phase* ph, int nphase, Medium& m) {
  if (!ph || nphase < 1 || nphase > 256) return fail(h, HH_ERR_ARG, "phase table");
  m.lam.resize(nphase);
  m.mu.resize(nphase);
  for (int i = 0; i < nphase; ++i) {
    if (!(ph[i].K > 0.0) || !(ph[i].G > 0.0) || !std::isfinite(ph[i].K) || !std::isfinite(ph[i].G))
      return fail(h, HH_ERR_ARG, "phase moduli must be finite and > 0");
    m.lam[i] = ph[i].K - 2.0 * ph[i].G / 3.0;
    m.mu[i] = ph[i].G;
    const double f = std::min(3.0 * ph[i].K, 2.0 * ph[i].G);
    m.floor = (i == 0) ? f : std::min(m.floor, f);
  }
  return HH_OK;
}

// Place the image on the device (copy of a host image into context memory).
static hh_status stage_image(hh_ctx* h, const uint8_t* img, long long V, int on_dev, const uint8_t** d_img) {
  Ctx& c = h->c;
  if (!img) return fail(h, HH_ERR_ARG, "image is NULL");
  if (on_dev) {
    *d_img = img;
    return HH_OK;
  }
  uint8_t* d;
  hh_status s = ensure(c, "image", (size_t)V, (void**)&d);
  if (s != HH_OK) return s;
  HH_CK(cudaMemcpyAsync(d, img, (size_t)V, cudaMemcpyHostToDevice, c.st));
  *d_img = d;
  return HH_OK;
}

static void fill_result(hh_result* out, const BoxRes& R, const Stats& st) {
  std::memcpy(out->C, R.C, sizeof(out->C));
  std::memcpy(out->C_sym, R.Csym, sizeof(out->C_sym));
  out->K = R.K;
  out->G = R.G;
  out->K_reuss = R.KR;
  out->G_reuss = R.GR;
  out->iters_max = st.iters_max;
  out->resid_max = st.resid_max;
  out->voxel_iters = st.voxel_iters;
  out->n_fused = st.fused_boxes;
  out->status = st.worst == ST_NONFINITE ? HH_ERR_NONFINITE : (st.worst == ST_NOT_CONVERGED ? HH_WARN_NOT_CONVERGED : HH_OK);
}

template <typename T>
static hh_status run_boxes(hh_ctx* h, const hh_options& o, const Medium& m, const std::vector<BoxReq>& boxes,
                           BoxRes** d_res_out, Stats& st) {
  Ctx& c = h->c;
  BoxRes* d_res;
  hh_status s = ensure(c, "boxres", boxes.size() * sizeof(BoxRes), (void**)&d_res);
  if (s != HH_OK) return s;
  s = solve_boxes<T>(c, o, m, boxes, d_res, st);
  *d_res_out = d_res;
  return s;
}

static hh_status run_boxes_p(hh_ctx* h, const hh_options& o, const Medium& m, const std::vector<BoxReq>& boxes,
                             BoxRes** d_res, Stats& st) {
  return o.precision == HH_FP64 ? run_boxes<double>(h, o, m, boxes, d_res, st)
                                : run_boxes<float>(h, o, m, boxes, d_res, st);
}

static hh_status status_of(const Stats& st) {
  return st.worst == ST_NONFINITE ? HH_ERR_NONFINITE : (st.worst == ST_NOT_CONVERGED ? HH_WARN_NOT_CONVERGED : HH_OK);
}

extern "C" hh_status hh_homogenize_direct(hh_ctx* h, const uint8_t* img, int nx, int ny, int nz, int on_dev,
                                          const hh_phase* phases, int nphase, const hh_options* opt,
                                          hh_result* out) {
  if (!h || !out) return fail(h, HH_ERR_ARG, "NULL context or output");
  hh_status s;
  if ((s = check_opts(h, opt)) != HH_OK) return s;
  if (nx < 1 || ny < 1 || nz < 1) return fail(h, HH_ERR_ARG, "dims must be >= 1");
  Medium m;
  if ((s = check_phases(h, phases, nphase, m)) != HH_OK) return s;
  if ((s = enter(h)) != HH_OK) return s;
  m.kind = MED_ISO;
  m.Nx = nx;
  m.Ny = ny;
  m.Nz = nz;
  if ((s = stage_image(h, img, (long long)nx * ny * nz, on_dev, &m.d_img)) != HH_OK) return s;
  std::vector<BoxReq> boxes(1);
  std::memset(boxes.data(), 0, sizeof(BoxReq));
  boxes[0].cnx = nx;
  boxes[0].cny = ny;
  boxes[0].cnz = nz;
  Stats st;
  BoxRes* d_res;
  if ((s = run_boxes_p(h, *opt, m, boxes, &d_res, st)) != HH_OK) return s;
  Ctx& c = h->c;
  BoxRes R;
  HH_CK(cudaMemcpyAsync(&R, d_res, sizeof(BoxRes), cudaMemcpyDeviceToHost, c.st));
  HH_CK(cudaStreamSynchronize(c.st));
  std::memset(out, 0, sizeof(*out));
  fill_result(out, R, st);
  out->n_subimages = 1;
  out->K_am = R.K;
  out->G_am = R.G;
  return finish(h, out->status, out);
}

static hh_status parse_boxes(hh_ctx* h, const int32_t* boxes, int nbox, int nx, int ny, int nz,
                             std::vector<BoxReq>& out) {
  if (!boxes || nbox < 1) return fail(h, HH_ERR_ARG, "no boxes");
  out.resize(nbox);
  for (int i = 0; i < nbox; ++i) {
    const int32_t* r = boxes + 7 * i;
    BoxReq& B = out[i];
    std::memset(&B, 0, sizeof(B));
    B.ox = r[0];
    B.oy = r[1];
    B.oz = r[2];
    B.cnx = r[3];
    B.cny = r[4];
    B.cnz = r[5];
    B.b = r[6];
    if (B.cnx < 1 || B.cny < 1 || B.cnz < 1 || B.b < 0 || B.ox < 0 || B.oy < 0 || B.oz < 0 || B.ox >= nx ||
        B.oy >= ny || B.oz >= nz || B.cnx > nx || B.cny > ny || B.cnz > nz)
      return fail(h, HH_ERR_ARG, "box " + std::to_string(i) + " out of range");
  }
  return HH_OK;
}

// level 1 + assembly + level 2 on a validated tiling partition. Subimages
// listed in acc_idx take the stiffness acc_c21 (21 values each, accepted
// surrogate predictions) instead of an FFT solve.
static hh_status hierarchical_core(hh_ctx* h, const hh_options& o, Medium& m, const std::vector<BoxReq>& boxes, int unit,
                                   const int* reg, hh_result* out, double* per_sub_C, int* per_sub_iters,
                                   const std::vector<int>* acc_idx = nullptr,
                                   const std::vector<double>* acc_c21 = nullptr) {
  Ctx& c = h->c;
  hh_status s;
  Stats st1;
  BoxRes* d_res = nullptr;
  const int nbox = (int)boxes.size();
  const int nacc = acc_idx ? (int)acc_idx->size() : 0;
  std::vector<int> rest;  // subimages that the FFT solver homogenizes
  if (nacc) {
    std::vector<char> is_acc(nbox, 0);
    for (int i : *acc_idx) is_acc[i] = 1;
    for (int i = 0; i < nbox; ++i)
      if (!is_acc[i]) rest.push_back(i);
    std::vector<BoxReq> rb;
    for (int i : rest) rb.push_back(boxes[i]);
    if (!rb.empty() && (s = run_boxes_p(h, o, m, rb, &d_res, st1)) != HH_OK) return s;
  } else if ((s = run_boxes_p(h, o, m, boxes, &d_res, st1)) != HH_OK) {
    return s;
  }
  // assembly of the intermediate image (FP64)
  const int Cx = reg[3], Cy = reg[4], Cz = reg[5];
  const long long Vc = (long long)Cx * Cy * Cz;
  double* d_c21;
  BoxReq* d_boxes;
  double* d_am;
  BoxRes* d_res1;
  // keep level-1 results: move them out of the buffer the level-2 solve reuses
  if ((s = ensure(c, "boxres1", nbox * sizeof(BoxRes), (void**)&d_res1)) != HH_OK) return s;
  if (!nacc) {
    HH_CK(cudaMemcpyAsync(d_res1, d_res, nbox * sizeof(BoxRes), cudaMemcpyDeviceToDevice, c.st));
  } else {
    int *d_pos, *d_acc;
    double* d_pc;
    if ((s = ensure(c, "surr_pos", std::max<size_t>(rest.size(), 1) * sizeof(int), (void**)&d_pos)) != HH_OK ||
        (s = ensure(c, "surr_idx", nacc * sizeof(int), (void**)&d_acc)) != HH_OK ||
        (s = ensure(c, "surr_c21", nacc * 21 * sizeof(double), (void**)&d_pc)) != HH_OK)
      return s;
    if (!rest.empty()) {
      HH_CK(cudaMemcpyAsync(d_pos, rest.data(), rest.size() * sizeof(int), cudaMemcpyHostToDevice, c.st));
      ++c.launches;
      k_scatter_res<<<((int)rest.size() + 127) / 128, 128, 0, c.st>>>(d_res, d_pos, (int)rest.size(), d_res1);
    }
    HH_CK(cudaMemcpyAsync(d_acc, acc_idx->data(), nacc * sizeof(int), cudaMemcpyHostToDevice, c.st));
    HH_CK(cudaMemcpyAsync(d_pc, acc_c21->data(), nacc * 21 * sizeof(double), cudaMemcpyHostToDevice, c.st));
    ++c.launches;
    k_accept_pred<<<(nacc + 127) / 128, 128, 0, c.st>>>(d_pc, d_acc, nacc, d_res1, m.floor);
    HH_CK(cudaGetLastError());
  }
  if ((s = ensure(c, "coarse", 21 * Vc * sizeof(double), (void**)&d_c21)) != HH_OK) return s;
  if ((s = ensure(c, "aboxes", nbox * sizeof(BoxReq), (void**)&d_boxes)) != HH_OK) return s;
  if ((s = ensure(c, "am", 4 * sizeof(double), (void**)&d_am)) != HH_OK) return s;
  HH_CK(cudaMemcpyAsync(d_boxes, boxes.data(), nbox * sizeof(BoxReq), cudaMemcpyHostToDevice, c.st));
  ++c.launches;
  k_assemble<<<nbox, 128, 0, c.st>>>(d_boxes, d_res1, nbox, unit, reg[0], reg[1], reg[2], Cx, Cy, Cz, d_c21);
  ++c.launches;
  k_am<<<1, 256, 0, c.st>>>(d_res1, d_boxes, nbox, d_am);
  HH_CK(cudaGetLastError());
  // level 2
  Medium m2;
  m2.kind = MED_ANISO;
  m2.d_c21 = d_c21;
  m2.Nx = Cx;
  m2.Ny = Cy;
  m2.Nz = Cz;
  std::vector<BoxReq> one(1);
  std::memset(one.data(), 0, sizeof(BoxReq));
  one[0].cnx = Cx;
  one[0].cny = Cy;
  one[0].cnz = Cz;
  Stats st2;
  BoxRes* d_res2;
  hh_options o2 = o;
  o2.scheme = HH_CG;  // the basic scheme is a mode of the subimage (level-1) solves
  if ((s = run_boxes_p(h, o2, m2, one, &d_res2, st2)) != HH_OK) return s;
  BoxRes R;
  double am[4];
  HH_CK(cudaMemcpyAsync(&R, d_res2, sizeof(BoxRes), cudaMemcpyDeviceToHost, c.st));
  HH_CK(cudaMemcpyAsync(am, d_am, 4 * sizeof(double), cudaMemcpyDeviceToHost, c.st));
  std::vector<BoxRes> all;
  if (per_sub_C || per_sub_iters) {
    all.resize(nbox);
    HH_CK(cudaMemcpyAsync(all.data(), d_res1, nbox * sizeof(BoxRes), cudaMemcpyDeviceToHost, c.st));
  }
  HH_CK(cudaStreamSynchronize(c.st));
  Stats tot;
  tot.iters_max = std::max(st1.iters_max, st2.iters_max);
  tot.resid_max = std::max(st1.resid_max, st2.resid_max);
  tot.voxel_iters = st1.voxel_iters + st2.voxel_iters;
  tot.worst = std::max(st1.worst, st2.worst);
  tot.fused_boxes = st1.fused_boxes;
  std::memset(out, 0, sizeof(*out));
  fill_result(out, R, tot);
  out->K_am = am[0];
  out->G_am = am[1];
  out->n_subimages = nbox;
  out->n_surrogate_accepted = nacc;
  out->n_clipped = (int)am[3];
  for (int b = 0; b < (int)all.size(); ++b) {
    if (per_sub_C) std::memcpy(per_sub_C + 36 * b, all[b].C, 36 * sizeof(double));
    if (per_sub_iters) std::memcpy(per_sub_iters + 6 * b, all[b].iters, 6 * sizeof(int));
  }
  return out->status;
}

// Largest cell edge that divides every core origin and edge (the coarse unit
// when the caller passes none).
static int derive_unit(const std::vector<BoxReq>& boxes) {
  int g = 0;
  for (const BoxReq& B : boxes)
    for (int v : {B.ox, B.oy, B.oz, B.cnx, B.cny, B.cnz}) g = std::gcd(g, v);
  return std::max(g, 1);
}

// The cores must tile their bounding box (in unit cells); reg receives the
// box origin and extent in unit cells.
static hh_status check_tiling(hh_ctx* h, const std::vector<BoxReq>& boxes, int unit, int nx, int ny, int nz, int* reg) {
  if (unit < 1) return fail(h, HH_ERR_ARG, "unit must be >= 1");
  int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {0, 0, 0};
  for (const BoxReq& B : boxes) {
    if (B.ox % unit || B.oy % unit || B.oz % unit || B.cnx % unit || B.cny % unit || B.cnz % unit ||
        B.ox + B.cnx > nx || B.oy + B.cny > ny || B.oz + B.cnz > nz)
      return fail(h, HH_ERR_ARG, "box not aligned to unit or outside the image");
    const int o3[3] = {B.ox / unit, B.oy / unit, B.oz / unit};
    const int e3[3] = {(B.ox + B.cnx) / unit, (B.oy + B.cny) / unit, (B.oz + B.cnz) / unit};
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], o3[a]);
      hi[a] = std::max(hi[a], e3[a]);
    }
  }
  const int Cx = hi[0] - lo[0], Cy = hi[1] - lo[1], Cz = hi[2] - lo[2];
  std::vector<uint8_t> cover((size_t)Cx * Cy * Cz, 0);
  for (const BoxReq& B : boxes) {
    for (int k = B.oz / unit; k < (B.oz + B.cnz) / unit; ++k)
      for (int j = B.oy / unit; j < (B.oy + B.cny) / unit; ++j)
        for (int i = B.ox / unit; i < (B.ox + B.cnx) / unit; ++i) {
          uint8_t& v = cover[((size_t)(k - lo[2]) * Cy + (j - lo[1])) * Cx + (i - lo[0])];
          if (v) return fail(h, HH_ERR_ARG, "boxes overlap");
          v = 1;
        }
  }
  for (uint8_t v : cover)
    if (!v) return fail(h, HH_ERR_ARG, "boxes do not tile a box-shaped region");
  reg[0] = lo[0];
  reg[1] = lo[1];
  reg[2] = lo[2];
  reg[3] = Cx;
  reg[4] = Cy;
  reg[5] = Cz;
  return HH_OK;
}

extern "C" hh_status hh_homogenize_partition(hh_ctx* h, const uint8_t* img, int nx, int ny, int nz, int on_dev,
                                             const hh_phase* phases, int nphase, const int32_t* boxes, int nbox,
                                             int unit, const hh_options* opt, hh_result* out, double* per_sub_C,
                                             int* per_sub_iters) {
  if (!h || !out) return fail(h, HH_ERR_ARG, "NULL context or output");
  hh_status s;
  if ((s = check_opts(h, opt)) != HH_OK) return s;
  if (nx < 1 || ny < 1 || nz < 1) return fail(h, HH_ERR_ARG, "dims must be >= 1");
  Medium m;
  if ((s = check_phases(h, phases, nphase, m)) != HH_OK) return s;
  std::vector<BoxReq> bx;
  if ((s = parse_boxes(h, boxes, nbox, nx, ny, nz, bx)) != HH_OK) return s;
  if (unit <= 0) unit = derive_unit(bx);
  int reg[6];
  if ((s = check_tiling(h, bx, unit, nx, ny, nz, reg)) != HH_OK) return s;
  if ((s = enter(h)) != HH_OK) return s;
  m.kind = MED_ISO;
  m.Nx = nx;
  m.Ny = ny;
  m.Nz = nz;
  if ((s = stage_image(h, img, (long long)nx * ny * nz, on_dev, &m.d_img)) != HH_OK) return s;
  return finish(h, hierarchical_core(h, *opt, m, bx, unit, reg, out, per_sub_C, per_sub_iters), out);
}

// The i-th draw (i from 0) of the SplitMix64 generator (Steele, Lea and
// Flood, 2014) seeded with `seed`, as a double in [0, 1) from its top 53 bits.
static double audit_draw(uint64_t seed, int i) {
  uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1.0p-53;
}

// Isotropic Voigt projection of a 6x6 Voigt stiffness: K = (C11 + C22 + C33 +
// 2 (C12 + C13 + C23)) / 9, G = (C11 + C22 + C33 - C12 - C13 - C23 + 3 (C44 +
// C55 + C66)) / 15.
static void voigt_kg(const double* C, double* K, double* G) {
  const double d = C[0] + C[7] + C[14], o = C[1] + C[2] + C[8], sh = C[21] + C[28] + C[35];
  *K = (d + 2.0 * o) / 9.0;
  *G = (d - o + 3.0 * sh) / 15.0;
}

extern "C" hh_status hh_homogenize_partition_surrogate(hh_ctx* h, const uint8_t* img, int nx, int ny, int nz,
                                                       int on_dev, const hh_phase* phases, int nphase,
                                                       const int32_t* boxes, int nbox, int unit, const float* params,
                                                       int ensemble, double scale, double spread,
                                                       double audit_fraction, uint64_t audit_seed,
                                                       const hh_options* opt, hh_result* out, double* per_sub_C,
                                                       int* accepted, double* audit_err) {
  if (!h || !out || !params || ensemble < 1 || !(scale > 0.0) || !(spread >= 0.0) ||
      !(audit_fraction >= 0.0 && audit_fraction <= 1.0))
    return fail(h, HH_ERR_ARG, "NULL context, output or parameters, or bad ensemble/scale/spread/audit fraction");
  hh_status s;
  if ((s = check_opts(h, opt)) != HH_OK) return s;
  if (nx < 1 || ny < 1 || nz < 1) return fail(h, HH_ERR_ARG, "dims must be >= 1");
  Medium m;
  if ((s = check_phases(h, phases, nphase, m)) != HH_OK) return s;
  std::vector<BoxReq> bx;
  if ((s = parse_boxes(h, boxes, nbox, nx, ny, nz, bx)) != HH_OK) return s;
  if (unit <= 0) unit = derive_unit(bx);
  int reg[6];
  if ((s = check_tiling(h, bx, unit, nx, ny, nz, reg)) != HH_OK) return s;
  // candidates: every subimage whose buffered box has edges 8..256, offered
  // to the network with its buffer and its core
  std::vector<int> cand;
  std::vector<int32_t> rows, sboxes;
  long long lab_len = 0;
  for (int i = 0; i < nbox; ++i) {
    const int ex = bx[i].cnx + 2 * bx[i].b, ey = bx[i].cny + 2 * bx[i].b, ez = bx[i].cnz + 2 * bx[i].b;
    if (ex < 8 || ey < 8 || ez < 8 || ex > 256 || ey > 256 || ez > 256) continue;
    cand.push_back(i);
    rows.insert(rows.end(), boxes + 7 * i, boxes + 7 * i + 7);
    const int32_t r[9] = {ex, ey, ez, bx[i].b, bx[i].b, bx[i].b, bx[i].cnx, bx[i].cny, bx[i].cnz};
    sboxes.insert(sboxes.end(), r, r + 9);
    lab_len += (long long)ex * ey * ez;
  }
  std::vector<int> acc_idx, aud_idx;  // accepted: ensemble stiffness used; audited: FFT solve
  std::vector<double> acc_c21, aud_c21;
  if (!cand.empty()) {
    const int nc = (int)cand.size();
    std::vector<uint8_t> lab(lab_len);
    std::vector<float> pred((size_t)nc * ensemble * 21);
    std::vector<int> ok(nc);
    std::vector<double> c21((size_t)nc * 21);
    if ((s = hh_extract_subimages(h, img, nx, ny, nz, on_dev, rows.data(), nc, lab.data(), (int64_t)lab.size())) !=
            HH_OK ||
        (s = hh_surrogate_predict(h, lab.data(), nc, sboxes.data(), params, ensemble, scale, pred.data())) != HH_OK ||
        (s = hh_surrogate_gate(h, lab.data(), nc, sboxes.data(), phases, nphase, pred.data(), ensemble, spread,
                               ok.data(), c21.data())) != HH_OK)
      return s;
    for (int j = 0; j < nc; ++j)
      if (ok[j]) {
        const int i = cand[j];
        const bool audit = audit_draw(audit_seed, i) < audit_fraction;
        (audit ? aud_idx : acc_idx).push_back(i);
        std::vector<double>& c_to = audit ? aud_c21 : acc_c21;
        c_to.insert(c_to.end(), c21.begin() + 21 * j, c21.begin() + 21 * j + 21);
      }
  }
  if (accepted) {
    std::memset(accepted, 0, nbox * sizeof(int));
    for (int i : acc_idx) accepted[i] = 1;
    for (int i : aud_idx) accepted[i] = 2;
  }
  if ((s = enter(h)) != HH_OK) return s;
  m.kind = MED_ISO;
  m.Nx = nx;
  m.Ny = ny;
  m.Nz = nz;
  if ((s = stage_image(h, img, (long long)nx * ny * nz, on_dev, &m.d_img)) != HH_OK) return s;
  // the audited subimages are solved by the FFT solver with the rejected ones
  std::vector<double> Cb;
  double* Cout = per_sub_C;
  if (!Cout && audit_err && !aud_idx.empty()) {
    Cb.resize((size_t)nbox * 36);
    Cout = Cb.data();
  }
  s = hierarchical_core(h, *opt, m, bx, unit, reg, out, Cout, nullptr, &acc_idx, &acc_c21);
  out->n_surrogate_accepted = (int)(acc_idx.size() + aud_idx.size());
  if (audit_err && s >= 0) {
    for (int i = 0; i < nbox; ++i) audit_err[i] = -1.0;
    for (size_t j = 0; j < aud_idx.size(); ++j) {
      const int i = aud_idx[j];
      double P[36], F[36];
      for (int a = 0, t = 0; a < 6; ++a)
        for (int b = a; b < 6; ++b, ++t) P[6 * a + b] = P[6 * b + a] = aud_c21[21 * j + t];
      for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) F[6 * a + b] = 0.5 * (Cout[36 * i + 6 * a + b] + Cout[36 * i + 6 * b + a]);
      double Kp, Gp, Kf, Gf;
      voigt_kg(P, &Kp, &Gp);
      voigt_kg(F, &Kf, &Gf);
      audit_err[i] = std::max(std::fabs(Kp - Kf) / Kf, std::fabs(Gp - Gf) / Gf);
    }
  }
  return finish(h, s, out);
}

// Least-squares fit of exp(-l / xi) to corr(0..L), L the first l with
// corr(l) < 0.05 (at least 1), by golden-section search on log(xi) over
// (0.01, 1e4); 200 steps.
static double fit_xi(const double* corr, int n) {
  int L = n - 1;
  for (int l = 0; l < n; ++l)
    if (corr[l] < 0.05) {
      L = l;
      break;
    }
  L = std::max(L, 1);
  auto f = [&](double lx) {
    const double xi = std::exp(lx);
    double s = 0.0;
    for (int l = 0; l <= L && l < n; ++l) {
      const double r = corr[l] - std::exp(-double(l) / xi);
      s += r * r;
    }
    return s;
  };
  double a = std::log(0.01), b = std::log(1e4);
  const double g = (std::sqrt(5.0) - 1.0) / 2.0;
  double x1 = b - g * (b - a), x2 = a + g * (b - a), f1 = f(x1), f2 = f(x2);
  for (int it = 0; it < 200; ++it) {
    if (f1 < f2) {
      b = x2;
      x2 = x1;
      f2 = f1;
      x1 = b - g * (b - a);
      f1 = f(x1);
    } else {
      a = x1;
      x1 = x2;
      f1 = f2;
      x2 = a + g * (b - a);
      f2 = f(x2);
    }
  }
  return std::exp(0.5 * (a + b));
}

extern "C" hh_status hh_correlation(hh_ctx* h, const uint8_t* img, int nx, int ny, int nz, int on_dev, int pore_label,
                                    int lmax, int64_t* counts, double* corr, double* xi, int* n_min) {
  if (!h || !counts || !corr || !xi || lmax < 1 || lmax > 4096 || pore_label < 0 || pore_label > 255)
    return fail(h, HH_ERR_ARG, "NULL output, lmax outside 1..4096 or pore label outside 0..255");
  if (nx < 2 || ny < 2 || nz < 2) return fail(h, HH_ERR_ARG, "dims must be >= 2");
  hh_status s;
  if ((s = enter(h)) != HH_OK) return s;
  Ctx& c = h->c;
  const long long V = (long long)nx * ny * nz;
  const uint8_t* d_img;
  if ((s = stage_image(h, img, V, on_dev, &d_img)) != HH_OK) return s;
  unsigned long long* d_cnt;
  if ((s = ensure(c, "corr_counts", 3 * (lmax + 1) * sizeof(unsigned long long), (void**)&d_cnt)) != HH_OK) return s;
  HH_CK(cudaMemsetAsync(d_cnt, 0, 3 * (lmax + 1) * sizeof(unsigned long long), c.st));
  const int dims[3] = {nx, ny, nz};
  for (int a = 0; a < 3; ++a) {
    const long long nline = V / dims[a];
    const int grid = (int)std::min<long long>(8LL * c.nsm, (nline + 255) / 256);
    ++c.launches;
    k_corr_counts<<<std::max(grid, 1), 256, (lmax + 1) * sizeof(unsigned long long), c.st>>>(
        d_img, nx, ny, nz, a, pore_label, lmax, d_cnt + a * (lmax + 1));
    HH_CK(cudaGetLastError());
  }
  std::vector<unsigned long long> h_cnt(3 * (lmax + 1));
  HH_CK(cudaMemcpyAsync(h_cnt.data(), d_cnt, h_cnt.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                        c.st));
  HH_CK(cudaStreamSynchronize(c.st));
  // <M> over all voxels = the l = 0 count of any axis / V
  const double m = double(h_cnt[0]) / double(V);
  for (int a = 0; a < 3; ++a) {
    const int n = dims[a];
    const long long other = V / n;
    const int nl = std::min(lmax, n - 1) + 1;
    for (int l = 0; l <= lmax; ++l) {
      counts[a * (lmax + 1) + l] = (int64_t)h_cnt[a * (lmax + 1) + l];
      corr[a * (lmax + 1) + l] = (l < n && m > 0.0 && m < 1.0)
                                     ? (double(h_cnt[a * (lmax + 1) + l]) / double((long long)(n - l) * other) - m * m) /
                                           (m - m * m)
                                     : 0.0;
    }
    xi[a] = (m > 0.0 && m < 1.0) ? fit_xi(corr + a * (lmax + 1), nl) : 0.0;
  }
  // Section 2: subimages of at least three correlation lengths
  if (n_min) n_min[0] = (int)std::ceil(3.0 * std::max(xi[0], std::max(xi[1], xi[2])));
  return HH_OK;
}

// Choice of the subimage edge n and buffer b from the error model of
// Section 5 (HH error ~ C_b / n for each buffer width, Eq. fit_power_law with
// the constants fitted per buffer as in Table fit_pad) and the cost model of
// Section 3 (Eq. 2: (N/n)^3 subimage solves, each costing (n + 2b)^a, the
// solved box being the buffered one), subject to n >= n_min (Section 2).
extern "C" hh_status hh_plan_partition(int nx, int ny, int nz, int n_min, const int* bs, const double* c_rel, int nb,
                                       double a, double eps, int* n_out, int* b_out, double* err_out,
                                       double* cost_out) {
  if (nx < 1 || ny < 1 || nz < 1 || !bs || !c_rel || nb < 1 || !(a > 0.0) || !(eps > 0.0) || !n_out || !b_out)
    return ctx_fail(nullptr, HH_ERR_ARG, "hh_plan_partition: bad dimensions, NULL array, nb < 1, a <= 0 or eps <= 0");
  for (int i = 0; i < nb; ++i)
    if (bs[i] < 0 || !(c_rel[i] >= 0.0) || !std::isfinite(c_rel[i]))
      return ctx_fail(nullptr, HH_ERR_ARG, "hh_plan_partition: a buffer < 0 or a constant that is negative or not finite");
  const int lo = std::max(n_min, 1), hi = std::min(nx, std::min(ny, nz));
  const double V = (double)nx * (double)ny * (double)nz;
  int bn = 0, bb = 0;
  double be = 0.0, bc = 0.0;
  bool bmet = false;
  for (int n = lo; n <= hi; ++n) {
    if (nx % n || ny % n || nz % n) continue;
    for (int i = 0; i < nb; ++i) {
      const int edge = n + 2 * bs[i];
      int rad[kMaxStages], nst = 0;
      if (!factorize(edge, rad, &nst)) continue;  // an FFT length the solver does not take
      const double err = c_rel[i] / n;
      const double cost = V / ((double)n * n * n) * std::pow((double)edge, a);
      const bool met = err <= eps;
      // order: candidates meeting eps first; among them (cost, error), else
      // (error, cost); then the larger n, then the smaller b
      bool better;
      if (bn == 0) {
        better = true;
      } else if (met != bmet) {
        better = met;
      } else {
        const double k1 = met ? cost : err, k1b = met ? bc : be;
        const double k2 = met ? err : cost, k2b = met ? be : bc;
        if (k1 != k1b) better = k1 < k1b;
        else if (k2 != k2b) better = k2 < k2b;
        else better = n > bn || (n == bn && bs[i] < bb);
      }
      if (better) {
        bn = n;
        bb = bs[i];
        be = err;
        bc = cost;
        bmet = met;
      }
    }
  }
  if (bn == 0)
    return ctx_fail(nullptr, HH_ERR_ARG, "hh_plan_partition: no edge n >= n_min divides the image with a supported box");
  *n_out = bn;
  *b_out = bb;
  if (err_out) *err_out = be;
  if (cost_out) *cost_out = bc;
  return bmet ? HH_OK : HH_WARN_TARGET_UNMET;
}

// Cubic cores of edge n tiling an nx x ny x nz grid (x fastest), buffer b.
static std::vector<BoxReq> uniform_boxes(int nx, int ny, int nz, int n, int b) {
  std::vector<BoxReq> out;
  for (int k = 0; k < nz / n; ++k)
    for (int j = 0; j < ny / n; ++j)
      for (int i = 0; i < nx / n; ++i) {
        BoxReq B;
        std::memset(&B, 0, sizeof(B));
        B.ox = i * n;
        B.oy = j * n;
        B.oz = k * n;
        B.cnx = B.cny = B.cnz = n;
        B.b = b;
        out.push_back(B);
      }
  return out;
}

extern "C" hh_status hh_homogenize_multilevel(hh_ctx* h, const uint8_t* img, int nx, int ny, int nz, int on_dev,
                                              const hh_phase* phases, int nphase, const int* ns, const int* bs,
                                              int nlevels, const hh_options* opt, hh_result* out) {
  if (!h || !out || !ns || !bs || nlevels < 1) return fail(h, HH_ERR_ARG, "NULL argument or nlevels < 1");
  hh_status s;
  if ((s = check_opts(h, opt)) != HH_OK) return s;
  if (nx < 1 || ny < 1 || nz < 1) return fail(h, HH_ERR_ARG, "dims must be >= 1");
  int gx = nx, gy = ny, gz = nz;
  for (int l = 0; l < nlevels; ++l) {
    const int n = ns[l];
    if (n < 1 || bs[l] < 0 || gx % n || gy % n || gz % n)
      return fail(h, HH_ERR_ARG, "level " + std::to_string(l) + ": n must divide the grid, b >= 0");
    gx /= n;
    gy /= n;
    gz /= n;
  }
  Medium m;
  if ((s = check_phases(h, phases, nphase, m)) != HH_OK) return s;
  if ((s = enter(h)) != HH_OK) return s;
  Ctx& c = h->c;
  m.kind = MED_ISO;
  m.Nx = nx;
  m.Ny = ny;
  m.Nz = nz;
  if ((s = stage_image(h, img, (long long)nx * ny * nz, on_dev, &m.d_img)) != HH_OK) return finish(h, s, out);
  Stats tot;
  int cx = nx, cy = ny, cz = nz;  // grid of the current level
  double* d_cur = nullptr;        // coarse stiffness image of the previous level
  for (int l = 0; l < nlevels; ++l) {
    const int n = ns[l];
    std::vector<BoxReq> boxes = uniform_boxes(cx, cy, cz, n, bs[l]);
    Medium ml = m;
    if (l > 0) {
      ml.kind = MED_ANISO;
      ml.d_c21 = d_cur;
      ml.Nx = cx;
      ml.Ny = cy;
      ml.Nz = cz;
    }
    Stats st;
    BoxRes* d_res;
    if ((s = run_boxes_p(h, *opt, ml, boxes, &d_res, st)) != HH_OK) return finish(h, s, out);
    tot.iters_max = std::max(tot.iters_max, st.iters_max);
    tot.resid_max = std::max(tot.resid_max, st.resid_max);
    tot.voxel_iters += st.voxel_iters;
    tot.worst = std::max(tot.worst, st.worst);
    // assembly into the next coarse image (ping-pong buffers)
    const int nbox = (int)boxes.size();
    const int Cx = cx / n, Cy = cy / n, Cz = cz / n;
    double* d_next;
    BoxReq* d_boxes;
    BoxRes* d_keep;
    if ((s = ensure(c, (l & 1) ? "ml_b" : "ml_a", 21LL * Cx * Cy * Cz * sizeof(double), (void**)&d_next)) != HH_OK ||
        (s = ensure(c, "ml_boxes", nbox * sizeof(BoxReq), (void**)&d_boxes)) != HH_OK ||
        (s = ensure(c, "ml_res", nbox * sizeof(BoxRes), (void**)&d_keep)) != HH_OK)
      return finish(h, s, out);
    HH_CK(cudaMemcpyAsync(d_keep, d_res, nbox * sizeof(BoxRes), cudaMemcpyDeviceToDevice, c.st));
    HH_CK(cudaMemcpyAsync(d_boxes, boxes.data(), nbox * sizeof(BoxReq), cudaMemcpyHostToDevice, c.st));
    ++c.launches;
    k_assemble<<<nbox, 128, 0, c.st>>>(d_boxes, d_keep, nbox, n, 0, 0, 0, Cx, Cy, Cz, d_next);
    HH_CK(cudaGetLastError());
    d_cur = d_next;
    cx = Cx;
    cy = Cy;
    cz = Cz;
  }
  // the last coarse image, solved whole (always by CG, like level 2)
  Medium mf = m;
  mf.kind = MED_ANISO;
  mf.d_c21 = d_cur;
  mf.Nx = cx;
  mf.Ny = cy;
  mf.Nz = cz;
  std::vector<BoxReq> one = uniform_boxes(cx, cy, cz, 1, 0);
  one.resize(1);
  one[0].cnx = cx;
  one[0].cny = cy;
  one[0].cnz = cz;
  hh_options of = *opt;
  of.scheme = HH_CG;
  Stats st;
  BoxRes* d_res;
  if ((s = run_boxes_p(h, of, mf, one, &d_res, st)) != HH_OK) return finish(h, s, out);
  BoxRes R;
  HH_CK(cudaMemcpyAsync(&R, d_res, sizeof(BoxRes), cudaMemcpyDeviceToHost, c.st));
  HH_CK(cudaStreamSynchronize(c.st));
  tot.iters_max = std::max(tot.iters_max, st.iters_max);
  tot.resid_max = std::max(tot.resid_max, st.resid_max);
  tot.voxel_iters += st.voxel_iters;
  tot.worst = std::max(tot.worst, st.worst);
  std::memset(out, 0, sizeof(*out));
  fill_result(out, R, tot);
  return finish(h, out->status, out);
}

extern "C" hh_status hh_homogenize_hierarchical(hh_ctx* h, const uint8_t* img, int nx, int ny, int nz, int on_dev,
                                                const hh_phase* phases, int nphase, int n, int b,
                                                const hh_options* opt, hh_result* out, double* per_sub_C,
                                                int* per_sub_iters) {
  if (n < 1 || b < 0 || nx % n || ny % n || nz % n) return fail(h, HH_ERR_ARG, "n must divide the image, b >= 0");
  std::vector<int32_t> rows;
  for (int k = 0; k < nz / n; ++k)
    for (int j = 0; j < ny / n; ++j)
      for (int i = 0; i < nx / n; ++i) {
        const int32_t r[7] = {i * n, j * n, k * n, n, n, n, b};
        rows.insert(rows.end(), r, r + 7);
      }
  return hh_homogenize_partition(h, img, nx, ny, nz, on_dev, phases, nphase, rows.data(), (int)(rows.size() / 7), n,
                                 opt, out, per_sub_C, per_sub_iters);
}

extern "C" hh_status hh_solve_subimages(hh_ctx* h, const uint8_t* img, int nx, int ny, int nz, int on_dev,
                                        const hh_phase* phases, int nphase, const int32_t* boxes, int nbox,
                                        const hh_options* opt, double* C_out, double* Sigma_out, double* Eps_out,
                                        int* iters_out, double* resid_out) {
  if (!h) return HH_ERR_ARG;
  hh_status s;
  if ((s = check_opts(h, opt)) != HH_OK) return s;
  if (nx < 1 || ny < 1 || nz < 1) return fail(h, HH_ERR_ARG, "dims must be >= 1");
  Medium m;
  if ((s = check_phases(h, phases, nphase, m)) != HH_OK) return s;
  std::vector<BoxReq> bx;
  if ((s = parse_boxes(h, boxes, nbox, nx, ny, nz, bx)) != HH_OK) return s;
  if ((s = enter(h)) != HH_OK) return s;
  m.kind = MED_ISO;
  m.Nx = nx;
  m.Ny = ny;
  m.Nz = nz;
  if ((s = stage_image(h, img, (long long)nx * ny * nz, on_dev, &m.d_img)) != HH_OK) return s;
  Stats st;
  BoxRes* d_res;
  if ((s = run_boxes_p(h, *opt, m, bx, &d_res, st)) != HH_OK) return s;
  Ctx& c = h->c;
  std::vector<BoxRes> all(nbox);
  HH_CK(cudaMemcpyAsync(all.data(), d_res, nbox * sizeof(BoxRes), cudaMemcpyDeviceToHost, c.st));
  HH_CK(cudaStreamSynchronize(c.st));
  for (int b = 0; b < nbox; ++b) {
    if (C_out) std::memcpy(C_out + 36 * b, all[b].C, 36 * sizeof(double));
    if (Sigma_out) std::memcpy(Sigma_out + 36 * b, all[b].Sig, 36 * sizeof(double));
    if (Eps_out) std::memcpy(Eps_out + 36 * b, all[b].Eps, 36 * sizeof(double));
    if (iters_out) std::memcpy(iters_out + 6 * b, all[b].iters, 6 * sizeof(int));
    if (resid_out) std::memcpy(resid_out + 6 * b, all[b].resid, 6 * sizeof(double));
  }
  return status_of(st);
}

extern "C" hh_status hh_homogenize_aniso(hh_ctx* h, const double* C21, int nx, int ny, int nz, int on_dev,
                                         const hh_options* opt, hh_result* out) {
  if (!h || !out || !C21) return fail(h, HH_ERR_ARG, "NULL argument");
  hh_status s;
  if ((s = check_opts(h, opt)) != HH_OK) return s;
  if (nx < 1 || ny < 1 || nz < 1) return fail(h, HH_ERR_ARG, "dims must be >= 1");
  if ((s = enter(h)) != HH_OK) return s;
  Ctx& c = h->c;
  const long long V = (long long)nx * ny * nz;
  const double* d_c21 = C21;
  if (!on_dev) {
    double* d;
    if ((s = ensure(c, "c21in", 21 * V * sizeof(double), (void**)&d)) != HH_OK) return s;
    HH_CK(cudaMemcpyAsync(d, C21, 21 * V * sizeof(double), cudaMemcpyHostToDevice, c.st));
    d_c21 = d;
  }
  Medium m;
  m.kind = MED_ANISO;
  m.d_c21 = d_c21;
  m.Nx = nx;
  m.Ny = ny;
  m.Nz = nz;
  std::vector<BoxReq> one(1);
  std::memset(one.data(), 0, sizeof(BoxReq));
  one[0].cnx = nx;
  one[0].cny = ny;
  one[0].cnz = nz;
  Stats st;
  BoxRes* d_res;
  if ((s = run_boxes_p(h, *opt, m, one, &d_res, st)) != HH_OK) return s;
  BoxRes R;
  HH_CK(cudaMemcpyAsync(&R, d_res, sizeof(BoxRes), cudaMemcpyDeviceToHost, c.st));
  HH_CK(cudaStreamSynchronize(c.st));
  std::memset(out, 0, sizeof(*out));
  fill_result(out, R, st);
  return finish(h, out->status, out);
}

extern "C" hh_status hh_apply_operator(hh_ctx* h, const uint8_t* labels, const hh_phase* phases, int nphase,
                                       const double* C21, int nx, int ny, int nz, const double* p, double* q,
                                       const hh_options* opt) {
  if (!h || !p || !q) return fail(h, HH_ERR_ARG, "NULL argument");
  hh_status s;
  if ((s = check_opts(h, opt)) != HH_OK) return s;
  if (nx < 1 || ny < 1 || nz < 1) return fail(h, HH_ERR_ARG, "dims must be >= 1");
  if ((s = enter(h)) != HH_OK) return s;
  Ctx& c = h->c;
  const long long V = (long long)nx * ny * nz;
  Medium m;
  if (C21) {
    m.kind = MED_ANISO;
    double* d;
    if ((s = ensure(c, "c21in", 21 * V * sizeof(double), (void**)&d)) != HH_OK) return s;
    HH_CK(cudaMemcpyAsync(d, C21, 21 * V * sizeof(double), cudaMemcpyHostToDevice, c.st));
    m.d_c21 = d;
  } else {
    if ((s = check_phases(h, phases, nphase, m)) != HH_OK) return s;
    if (!labels) return fail(h, HH_ERR_ARG, "labels is NULL");
    for (long long i = 0; i < V; ++i)
      if (labels[i] >= nphase) return fail(h, HH_ERR_ARG, "label >= nphase");
    m.kind = MED_ISO;
    if ((s = stage_image(h, labels, V, 0, &m.d_img)) != HH_OK) return s;
  }
  return opt->precision == HH_FP64 ? apply_operator<double>(c, *opt, m, nx, ny, nz, p, q)
                                   : apply_operator<float>(c, *opt, m, nx, ny, nz, p, q);
}

extern "C" hh_status hh_extract_subimages(hh_ctx* h, const uint8_t* img, int nx, int ny, int nz, int on_dev,
                                          const int32_t* boxes, int nbox, uint8_t* out, int64_t out_len) {
  if (!h || !out) return fail(h, HH_ERR_ARG, "NULL argument");
  if (nx < 1 || ny < 1 || nz < 1) return fail(h, HH_ERR_ARG, "dims must be >= 1");
  hh_status s;
  std::vector<BoxReq> bx;
  if ((s = parse_boxes(h, boxes, nbox, nx, ny, nz, bx)) != HH_OK) return s;
  long long tot = 0;
  std::vector<int2> items;
  for (int b = 0; b < nbox; ++b) {
    bx[b].lab_off = tot;
    const long long ex = bx[b].cnx + 2LL * bx[b].b, ey = bx[b].cny + 2LL * bx[b].b, ez = bx[b].cnz + 2LL * bx[b].b;
    tot += ex * ey * ez;
    for (int k = 0; k < ez; ++k) items.push_back(make_int2(b, k));
  }
  if (out_len < tot) return fail(h, HH_ERR_ARG, "output buffer too small");
  if ((s = enter(h)) != HH_OK) return s;
  Ctx& c = h->c;
  const uint8_t* d_img;
  if ((s = stage_image(h, img, (long long)nx * ny * nz, on_dev, &d_img)) != HH_OK) return s;
  uint8_t* d_out;
  BoxReq* d_b;
  int2* d_it;
  int* d_flag;
  if ((s = ensure(c, "labels", tot, (void**)&d_out)) != HH_OK) return s;
  if ((s = ensure(c, "boxes", nbox * sizeof(BoxReq), (void**)&d_b)) != HH_OK) return s;
  if ((s = ensure(c, "gitems", items.size() * sizeof(int2), (void**)&d_it)) != HH_OK) return s;
  if ((s = ensure(c, "flag", 64, (void**)&d_flag)) != HH_OK) return s;
  HH_CK(cudaMemcpyAsync(d_b, bx.data(), nbox * sizeof(BoxReq), cudaMemcpyHostToDevice, c.st));
  HH_CK(cudaMemcpyAsync(d_it, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, c.st));
  HH_CK(cudaMemsetAsync(d_flag, 0, 64, c.st));
  ++c.launches;
  k_gather<<<std::min<int>((int)items.size(), 8 * c.nsm), 256, 0, c.st>>>(d_img, nx, ny, nz, d_b, d_it,
                                                                           (int)items.size(), d_out, 256, d_flag);
  HH_CK(cudaGetLastError());
  HH_CK(cudaMemcpyAsync(out, d_out, tot, cudaMemcpyDeviceToHost, c.st));
  HH_CK(cudaStreamSynchronize(c.st));
  return HH_OK;
}

extern "C" hh_status hh_profile_read(hh_ctx* h, hh_kernel_stat* out, int cap, int* count) {
  if (!h || !count || (cap > 0 && !out)) return fail(h, HH_ERR_ARG, "bad arguments");
  Ctx& c = h->c;
  int i = 0;
  for (auto& kv : c.prof) {
    if (i < cap) {
      hh_kernel_stat& k = out[i];
      std::memset(&k, 0, sizeof(k));
      std::strncpy(k.name, kv.first.c_str(), sizeof(k.name) - 1);
      k.launches = kv.second.launches;
      k.sampled = kv.second.sampled;
      k.sampled_ms = kv.second.ms;
      k.sampled_bytes = kv.second.bytes;
    }
    ++i;
  }
  *count = i;
  return HH_OK;
}

extern "C" hh_status hh_profile_reset(hh_ctx* h) {
  if (!h) return HH_ERR_ARG;
  h->c.prof.clear();
  return HH_OK;
}

extern "C" hh_status hh_fit_inverse_n(hh_ctx* h, const int* ns, const double* M, int count, double* M_inf,
                                      double* C) {
  if (!h || !ns || !M || !M_inf || !C || count < 2) return fail(h, HH_ERR_ARG, "fit needs >= 2 points");
  bool distinct = false;
  for (int i = 0; i < count; ++i) {
    if (ns[i] < 1) return fail(h, HH_ERR_ARG, "n must be >= 1");
    if (ns[i] != ns[0]) distinct = true;
  }
  if (!distinct) return fail(h, HH_ERR_ARG, "fit needs two distinct n");
  hh_status s;
  if ((s = enter(h)) != HH_OK) return s;
  Ctx& c = h->c;
  int* d_n;
  double *d_m, *d_o;
  if ((s = ensure(c, "fit_n", count * sizeof(int), (void**)&d_n)) != HH_OK) return s;
  if ((s = ensure(c, "fit_m", count * sizeof(double), (void**)&d_m)) != HH_OK) return s;
  if ((s = ensure(c, "fit_o", 2 * sizeof(double), (void**)&d_o)) != HH_OK) return s;
  HH_CK(cudaMemcpyAsync(d_n, ns, count * sizeof(int), cudaMemcpyHostToDevice, c.st));
  HH_CK(cudaMemcpyAsync(d_m, M, count * sizeof(double), cudaMemcpyHostToDevice, c.st));
  ++c.launches;
  k_fit_inverse_n<<<1, 32, 0, c.st>>>(d_n, d_m, count, d_o);
  HH_CK(cudaGetLastError());
  HH_CK(cudaMemcpyAsync(c.h_dbl, d_o, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.st));
  HH_CK(cudaStreamSynchronize(c.st));
  *M_inf = c.h_dbl[0];
  *C = c.h_dbl[1];
  return HH_OK;
}

extern "C" hh_status hh_extrapolate(hh_ctx* h, const uint8_t* img, int nx, int ny, int nz, int on_dev,
                                    const hh_phase* phases, int nphase, const int* ns, int count, int b,
                                    const hh_options* opt, double* K_inf, double* C_K, double* G_inf, double* C_G,
                                    hh_result* per_n) {
  if (!h || !ns || count < 2 || !K_inf || !C_K || !G_inf || !C_G) return fail(h, HH_ERR_ARG, "bad arguments");
  std::vector<double> Ks(count), Gs(count);
  hh_status worst = HH_OK;
  for (int i = 0; i < count; ++i) {
    hh_result r;
    hh_status s = hh_homogenize_hierarchical(h, img, nx, ny, nz, on_dev, phases, nphase, ns[i], b, opt, &r, nullptr,
                                             nullptr);
    if (s < 0) return s;
    if (s > 0) worst = s;
    Ks[i] = r.K;
    Gs[i] = r.G;
    if (per_n) per_n[i] = r;
  }
  hh_status s = hh_fit_inverse_n(h, ns, Ks.data(), count, K_inf, C_K);
  if (s != HH_OK) return s;
  s = hh_fit_inverse_n(h, ns, Gs.data(), count, G_inf, C_G);
  if (s != HH_OK) return s;
  return worst;
}

// ===========================================================================
// Operator application without allocation
// ===========================================================================
// Some callers cannot allocate device memory: code running inside a memory
// pool or arena they do not own, allocation-free real-time loops, or hosts
// whose allocator must not be re-entered. hh_apply_operator_noalloc serves
// them. Its scratch (problem descriptor, work items, FFT tables, phase table
// and the half spectrum) lives in the file-scope device array below, which
// every GPU that loads this library holds until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(HH_NOALLOC_SCRATCH_BYTES);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array, looked up once per device (with that
// device current) by the first call made on it.
constexpr int kNoAllocMaxDevices = 64;
static void* g_noalloc_addr[kNoAllocMaxDevices];
static int g_noalloc_optin[kNoAllocMaxDevices];
static std::mutex g_noalloc_mu;

static size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

extern "C" hh_status hh_apply_operator_noalloc(const uint8_t* labels, const hh_phase* phases, int nphase, int nx,
                                               int ny, int nz, const float* p, float* q, int nyquist,
                                               void* cuda_stream) {
  if (!labels || !phases || !p || !q) {
    set_last_error("hh_apply_operator_noalloc: NULL pointer");
    return HH_ERR_ARG;
  }
  if (nx < 1 || ny < 1 || nz < 1 || nx > HH_NOALLOC_MAX_EDGE || ny > HH_NOALLOC_MAX_EDGE ||
      nz > HH_NOALLOC_MAX_EDGE) {
    set_last_error("hh_apply_operator_noalloc: each edge must be in 1..HH_NOALLOC_MAX_EDGE");
    return HH_ERR_ARG;
  }
  if (nphase < 1 || nphase > 256 || (nyquist != HH_NYQ_ZERO_COMPONENT && nyquist != HH_NYQ_ZERO_MODE)) {
    set_last_error("hh_apply_operator_noalloc: bad phase count or Nyquist rule");
    return HH_ERR_ARG;
  }
  float lm[2 * 256];
  for (int i = 0; i < nphase; ++i) {
    if (!(phases[i].K > 0.0) || !(phases[i].G > 0.0) || !std::isfinite(phases[i].K) || !std::isfinite(phases[i].G)) {
      set_last_error("hh_apply_operator_noalloc: phase moduli must be finite and > 0");
      return HH_ERR_ARG;
    }
    lm[2 * i] = float(phases[i].K - 2.0 * phases[i].G / 3.0);
    lm[2 * i + 1] = float(phases[i].G);
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
    set_last_error("hh_apply_operator_noalloc: no usable current device");
    return HH_ERR_CUDA;
  }
  auto* kf = k_plane_fwd<float, MODE_APPLY>;
  auto* ki = k_plane_inv<float, MODE_APPLY>;
  auto* kc = k_column<float, false>;
  void* base = nullptr;
  int smem_optin = 0;
  {
    // once per device, with that device current: the scratch array's device
    // address, and the kernels' shared-memory limit raised to the device's
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* a = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
      if (e != cudaSuccess || !a) {
        set_last_error("hh_apply_operator_noalloc: cudaGetSymbolAddress failed");
        return HH_ERR_CUDA;
      }
      int optin = 0;
      if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
          cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess ||
          cudaFuncSetAttribute(ki, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess ||
          cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess) {
        set_last_error("hh_apply_operator_noalloc: device query or kernel attribute failed");
        return HH_ERR_CUDA;
      }
      g_noalloc_optin[dev] = optin;
      g_noalloc_addr[dev] = a;
    }
    base = g_noalloc_addr[dev];
    smem_optin = g_noalloc_optin[dev];
  }

  // host staging of the small tables in static storage (no allocation)
  const int nxh = nx / 2 + 1;
  const int colw = column_width<float>(nz, ny, (size_t)smem_optin);
  const size_t psm = plane_smem_bytes<float>(nx, ny, nphase);
  const size_t csm = column_smem_bytes<float>(colw, nz, ny);
  if (psm > (size_t)smem_optin || csm > (size_t)smem_optin) {
    set_last_error("hh_apply_operator_noalloc: plane too large for shared memory");
    return HH_ERR_UNSUPPORTED;
  }
  const int ncol = (ny * nxh + colw - 1) / colw;
  struct Staging {
    int bad_label;  // set on the device by the label check; 0 in every staged copy
    int pad_[3];
    Prob prob;
    AxisPlan plans[3];
    double tw[2 * 3 * HH_NOALLOC_MAX_EDGE];
    int itab[2 * 3 * HH_NOALLOC_MAX_EDGE];
    float lm[2 * 256];
    int2 items[HH_NOALLOC_MAX_EDGE + HH_NOALLOC_MAX_EDGE * (HH_NOALLOC_MAX_EDGE / 2 + 1)];
  };
  static thread_local Staging h;  // static storage: no heap or stack growth per call
  h.bad_label = 0;
  std::memset(&h.prob, 0, sizeof(h.prob));
  const int dims[3] = {nx, ny, nz};
  int tw_off = 0, it_off = 0;
  for (int a = 0; a < 3; ++a) {
    AxisPlan& pl = h.plans[a];
    if (!plan_fill(dims[a], &pl, h.tw + 2 * tw_off, h.itab + it_off, h.itab + it_off + dims[a])) {
      set_last_error("hh_apply_operator_noalloc: FFT length with a prime factor above 31");
      return HH_ERR_UNSUPPORTED;
    }
    pl.tw_off = tw_off;
    pl.pf_off = it_off;
    pl.sf_off = it_off + dims[a];
    tw_off += dims[a];
    it_off += 2 * dims[a];
  }
  Prob& d = h.prob;
  d.nx = nx;
  d.ny = ny;
  d.nz = nz;
  d.nxh = nxh;
  d.cnx = nx;
  d.cny = ny;
  d.cnz = nz;
  d.px = 0;
  d.py = 1;
  d.pz = 2;
  for (int i = 0; i < 2 * nphase; ++i) h.lm[i] = lm[i];
  for (int k = 0; k < nz; ++k) h.items[k] = make_int2(0, k);
  d.cw = colw;
  d.npi = nz;
  int nc = 0;
  for (int j0 = 0; j0 < ny * nxh; j0 += colw) h.items[nz + nc++] = make_int2(0, j0);

  // scratch layout: [staging][half spectrum]
  const size_t spec_off = align256(sizeof(Staging));
  const size_t need = spec_off + sizeof(C2<float>) * 6 * (size_t)nz * ny * nxh;
  if (need > kNoAllocScratchBytes) {
    set_last_error("hh_apply_operator_noalloc: grid needs more than the HH_NOALLOC_SCRATCH_BYTES scratch");
    return HH_ERR_ARG;
  }
  unsigned char* sbase = static_cast<unsigned char*>(base);
  const Staging* dst = reinterpret_cast<const Staging*>(sbase);
  if (cudaMemcpyAsync(sbase, &h, sizeof(Staging), cudaMemcpyHostToDevice, st) != cudaSuccess) {
    set_last_error("hh_apply_operator_noalloc: staging copy failed");
    return HH_ERR_CUDA;
  }
  KParams<float> kp;
  std::memset(&kp, 0, sizeof(kp));
  kp.prob = &dst->prob;
  kp.medium = MED_ISO;
  kp.nyq_mode = nyquist;
  kp.nphase = nphase;
  kp.plans = dst->plans;
  kp.tw = dst->tw;
  kp.itab = dst->itab;
  kp.labels = labels;
  kp.lammu = dst->lm;
  kp.p = const_cast<float*>(p);
  kp.q = q;
  kp.r = q;
  kp.x = q;
  kp.spec = reinterpret_cast<C2<float>*>(sbase + spec_off);
  kp.nprob = 1;
  KParams<float> kpp = kp, kpc = kp;
  kpp.items = dst->items;
  kpp.nitems = nz;
  kpc.items = dst->items + nz;
  kpc.nitems = nc;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  nsm = std::max(nsm, 1);
  // every label must index the phase table before the plane pass reads it
  const long long V = (long long)nx * ny * nz;
  int bad = 0;
  k_check_labels<<<(int)std::min<long long>(4LL * nsm, (V + 255) / 256), 256, 0, st>>>(
      labels, V, nphase, const_cast<int*>(&dst->bad_label));
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, &dst->bad_label, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return HH_ERR_CUDA;
  }
  if (bad) {
    set_last_error("hh_apply_operator_noalloc: a label is >= nphase");
    return HH_ERR_ARG;
  }
  kf<<<std::min(nz, 4 * nsm), 256, psm, st>>>(kpp);
  kc<<<std::min(nc, 4 * nsm), 256, csm, st>>>(kpc, MODE_APPLY);
  ki<<<std::min(nz, 4 * nsm), 256, psm, st>>>(kpp);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return HH_ERR_CUDA;
  }
  return HH_OK;
}
