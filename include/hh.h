/*
 * hh.h -- C ABI of the GB300 hierarchical-homogenization library (libhh).
 *
 * Computes effective elastic stiffness of segmented 3D images by the
 * hierarchical homogenization of Ahmad, Liu, Ortiz, Mukerji and Cai (2022):
 * every subimage (core plus buffer, periodic) is homogenized by an FFT-based
 * Galerkin elasticity solver (Appendix A), the resulting anisotropic 6x6
 * stiffnesses are assembled into an intermediate image (Section 3) and that
 * image is homogenized again; K and G of the result are extrapolated in 1/n
 * (Section 5, Eq. fit_power_law).
 *
 * Conventions shared by every call
 *  - Images are uint8 labels, x fastest: index = (z * ny + y) * nx + x.
 *  - A label indexes the caller's phase table; every label must be < nphase.
 *  - Voigt order (11, 22, 33, 23, 13, 12); stress Voigt vectors hold sigma_ij,
 *    strain Voigt vectors hold engineering shear (2 eps_ij), so an isotropic
 *    phase has C44 = G. Matrices are 6x6 row-major doubles.
 *  - Ownership: the caller owns every buffer it passes; the library never
 *    keeps a caller pointer after a call returns. A context owns its device
 *    workspace, FFT tables and pinned staging memory.
 *  - `*_on_device` = 1 means the pointer is device memory readable on the
 *    context's stream; 0 means host memory.
 *  - Every call returns hh_status (0 = OK, < 0 error, > 0 warning). No call
 *    throws or aborts. On an error, outputs are left in an unspecified state.
 *  - Calls on one context are not thread-safe; use one context per thread.
 */
#ifndef HH_H
#define HH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int hh_status;
#define HH_OK 0
#define HH_WARN_NOT_CONVERGED 1   /* a load case stopped with its true residual above 2 tol:
                                     max_iter reached, or its restarts spent or no longer
                                     reducing the residual (the FP32 floor at high phase
                                     contrast); results filled, resid_max reported */
#define HH_WARN_TARGET_UNMET 2    /* hh_plan_partition: no candidate meets the error target;
                                     the candidate with the least predicted error is returned */
#define HH_ERR_ARG (-1)           /* invalid argument (dims, labels, moduli, partition, options) */
#define HH_ERR_OOM (-2)           /* device or pinned allocation failed */
#define HH_ERR_CUDA (-3)          /* a CUDA runtime call failed */
#define HH_ERR_NONFINITE (-4)     /* NaN/Inf in a CG scalar */
#define HH_ERR_DEVICE_TIMEOUT (-5)/* a bounded device-side wait ran out */
#define HH_ERR_BAD_STIFFNESS (-6) /* a stiffness that is not symmetric positive definite */
#define HH_ERR_UNSUPPORTED (-7)   /* FFT length with a prime factor above 31, or a row or z
                                     column too long for shared memory */

#define HH_FP32 0                 /* FP32 fields and FFTs, FP64 scalars and averages */
#define HH_FP64 1                 /* FP64 everywhere */
#define HH_CG 0                   /* conjugate gradients (Appendix A) */
#define HH_BASIC 1                /* basic fixed point with an isotropic reference medium
                                     (Moulinec-Suquet, cited in Appendix A) for the subimage
                                     and direct solves; the level-2 solve always uses CG */
#define HH_EYRE_MILTON 2          /* accelerated fixed point (Eyre-Milton) with an isotropic
                                     reference medium C0: tau = (C - C0) : eps,
                                     B = E - eps - Gamma0 * tau,
                                     eps <- eps + 2 (C + C0)^-1 C0 : B; stops after the
                                     iteration whose ||B|| / ||E|| <= tol (Frobenius norms);
                                     isotropic phases only; level 2 uses CG */
#define HH_NYQ_ZERO_COMPONENT 0   /* even N: Nyquist wave-vector component set to 0 */
#define HH_NYQ_ZERO_MODE 1        /* even N: projection zero on every Nyquist mode */

typedef struct hh_ctx hh_ctx;

typedef struct {
    double K; /* bulk modulus, GPa, > 0 */
    double G; /* shear modulus, GPa, > 0 */
} hh_phase;

typedef struct {
    int precision;        /* HH_FP32 (default) or HH_FP64 */
    double tol;           /* HH_CG: stop when ||r|| <= tol ||b|| (Frobenius norm);
                             HH_BASIC: stop when the equilibrium residual
                             ||G*sigma|| / ||<sigma>|| <= tol; default 1e-6 */
    int max_iter;         /* per load case, default 20000 */
    int scheme;           /* HH_CG (default), HH_BASIC or HH_EYRE_MILTON */
    int nyquist;          /* HH_NYQ_ZERO_COMPONENT (default) or HH_NYQ_ZERO_MODE */
    int fixed_iters;      /* > 0: run exactly this many iterations, ignore tol (parity runs) */
    double ref_lambda;    /* HH_BASIC / HH_EYRE_MILTON reference medium (Lame lambda, mu, GPa).
                             When ref_mu <= 0 or lambda + 2 mu / 3 <= 0: for HH_BASIC the means
                             of the smallest and largest phase lambda and mu, for
                             HH_EYRE_MILTON K0 = sqrt(K_min K_max), mu0 = sqrt(mu_min mu_max)
                             over the phases (isotropic phases only; an anisotropic medium
                             with no valid reference returns HH_ERR_UNSUPPORTED) */
    double ref_mu;
    int64_t workspace_bytes; /* device workspace budget for batched solves; 0 = 3/4 of free memory */
    int use_graphs;       /* 1 (default): capture the iteration loop in CUDA graphs */
    int check_every;      /* iterations between host convergence checks, default 32 */
    int replace;          /* residual replacement at every check: r <- -G*(C:(E + x));
                             1 on, 0 off, -1 (default) on in FP32 and off in FP64 */
    int max_restarts;     /* restarts allowed when the final true residual exceeds
                             2 tol (default 4) */
    int profile;          /* 1: time the field kernels of the first iteration of every
                             chunk with CUDA events (read with hh_profile_read) */
    int plane_smem_limit; /* largest shared-memory footprint (bytes) of a whole-plane
                             block; a subimage whose xy plane needs more takes the
                             row/column streaming passes (x rows and y columns
                             through HBM). 0 (default): the device's per-block limit */
    int autotune;         /* 1 (default): the column pass's width (spectrum columns per
                             block) is chosen per subimage shape by timing the
                             candidates once per context; 0: a fixed rule. The width
                             changes no result, only the speed */
    int wave_boxes;       /* > 0: at most this many subimages are solved together (one
                             wave of launches); 1 solves the subimages one at a time,
                             the plain unbatched solver. 0 (default): as many as the
                             workspace budget allows. Changes no result */
    int fused;            /* 1: every level-1 CG solve of isotropic phases whose half
                             spectrum fits the shared memory of a cluster of up to 8
                             thread blocks runs whole in one cluster (iterations, residual
                             checks and averages on chip; one persistent launch per
                             cluster size, fed by a device work counter); 0 (default):
                             the multi-pass solver for every subimage. Same arithmetic
                             but for the order of the partial sums */
    int shape_kernels;    /* 1 (default): FP32 CG iterations of subimages whose xy plane
                             has even edges in 16..48 differing by 0, 8 or 16 take plane
                             passes compiled for that shape, and z lengths 16..48 (even)
                             a column pass compiled for that length (column widths 16 or
                             32); 0: the generic passes for every shape. Same transforms,
                             voxel arithmetic and operation order: results agree to FP32
                             rounding */
} hh_options;

typedef struct {
    double C[36];         /* effective stiffness, raw Sigma Eps^-1 of the last solve, row-major Voigt */
    double C_sym[36];     /* (C + C^T) / 2 */
    double K, G;          /* isotropic Voigt projection of C_sym */
    double K_reuss, G_reuss; /* isotropic Reuss projection of C_sym */
    double K_am, G_am;    /* core-volume-weighted mean of subimage K, G (hierarchical calls only) */
    int iters_max;        /* most iterations of any load case of any solve */
    int n_subimages;      /* level-1 subimages solved (hierarchical calls) */
    int n_surrogate_accepted;
    int n_clipped;        /* subimages whose sym(C_R) was raised to the stiffness floor
                             min(3K, 2G) before assembly (indefinite with a buffer) */
    double resid_max;     /* largest final true residual ||b - A x|| / ||b|| */
    long long voxel_iters;/* sum over solves of (voxels x iterations), all load cases */
    long long kernel_launches; /* libhh kernels launched by this call */
    double device_ms;     /* device time of the call: CUDA events on the library's stream */
    hh_status status;
    int n_fused;          /* level-1 subimages solved by the fused cluster kernel (options.fused) */
} hh_result;

/* Per-kernel timing gathered while options.profile = 1. */
typedef struct {
    char name[32];
    long long launches;       /* launches of this kernel in profiled calls */
    long long sampled;        /* launches bracketed by CUDA events */
    double sampled_ms;        /* device time of the sampled launches */
    double sampled_bytes;     /* algorithmic DRAM bytes of the sampled launches: every field
                                 byte the kernel must read or write once */
} hh_kernel_stat;

/* Text of the last error on this context (or of the last failed hh_create
 * when ctx is NULL); never NULL. */
const char *hh_last_error(hh_ctx *ctx);

/* Library version string. */
const char *hh_version(void);

/* Human-readable text for a status code; never NULL. */
const char *hh_status_string(hh_status s);

/* Fill `o` with defaults (FP32, tol 1e-6, max_iter 20000, CG, component rule). */
hh_status hh_options_default(hh_options *o);

/* Create a context on CUDA device `device`. `cuda_stream` is a cudaStream_t to
 * run on (e.g. a PyTorch stream) or NULL for a context-owned stream. */
hh_status hh_create(hh_ctx **out, int device, void *cuda_stream);

/* Free everything the context owns. NULL is allowed. */
void hh_destroy(hh_ctx *ctx);

/* Cap, in bytes, on the device workspace the context's solver calls hold
 * (fields, spectra, work lists and per-subimage results; the FFT tables and
 * the surrogate network's buffers are not counted). A call whose workspace
 * would exceed the cap fails with HH_ERR_OOM before allocating and leaves the
 * context usable; batched solves size their waves of subimages to 3/4 of the
 * cap. Setting a cap releases the workspace the context holds (it is
 * reallocated on demand). 0 (the default) = no cap. Errors: HH_ERR_ARG
 * (bytes < 0), HH_ERR_CUDA. */
hh_status hh_set_memory_limit(hh_ctx *ctx, int64_t bytes);

/* Direct (brute-force) homogenization of a whole periodic image: the six load
 * cases of Section 4 on the full grid, averages over the whole grid, C =
 * Sigma Eps^-1 (Section 5: the reference M_N). `out` receives C, K, G. */
hh_status hh_homogenize_direct(hh_ctx *ctx, const uint8_t *img, int nx, int ny, int nz,
                               int img_on_device, const hh_phase *phases, int nphase,
                               const hh_options *opt, hh_result *out);

/* Two-level hierarchical homogenization with a uniform partition (Section 3,
 * Fig. 2; Section 4, Fig. 4): cores of edge n (n divides nx, ny, nz), buffer
 * b >= 0 voxels wrapped periodically at the image edge, C_R = Sigma Eps^-1
 * over each core, assembly of sym(C_R) into an (nx/n, ny/n, nz/n) image,
 * second solve. `per_sub_C` (caller-owned, may be NULL) receives the raw 36
 * values of every subimage, subimages ordered x fastest then y then z;
 * `per_sub_iters` (may be NULL) receives the 6 iteration counts of each. */
hh_status hh_homogenize_hierarchical(hh_ctx *ctx, const uint8_t *img, int nx, int ny, int nz,
                                     int img_on_device, const hh_phase *phases, int nphase,
                                     int n, int b, const hh_options *opt, hh_result *out,
                                     double *per_sub_C, int *per_sub_iters);

/* Two-level scheme on an arbitrary partition. `boxes` holds nbox rows of 7
 * int32 (ox, oy, oz, cnx, cny, cnz, b): core origin, core size, buffer width.
 * Every core edge and origin must be a multiple of `unit` (unit <= 0: the
 * largest unit that divides every core origin and edge), and the cores must
 * tile a box-shaped region of the image (normally the whole image). The
 * coarse image covers that region with unit-size voxels, each subimage
 * filling its block; buffers always wrap periodically in the whole image.
 * Outputs as above, in box order. */
hh_status hh_homogenize_partition(hh_ctx *ctx, const uint8_t *img, int nx, int ny, int nz,
                                  int img_on_device, const hh_phase *phases, int nphase,
                                  const int32_t *boxes, int nbox, int unit,
                                  const hh_options *opt, hh_result *out,
                                  double *per_sub_C, int *per_sub_iters);

/* Level-1 only: the subimage stiffnesses of a partition (Section 4), without
 * assembly or second solve. `boxes` as above (no tiling requirement, unit
 * ignored). Outputs per box: raw C (36), Sigma and Eps (36 each, columns =
 * load cases, may be NULL), iterations (6), final residuals (6, may be NULL). */
hh_status hh_solve_subimages(hh_ctx *ctx, const uint8_t *img, int nx, int ny, int nz,
                             int img_on_device, const hh_phase *phases, int nphase,
                             const int32_t *boxes, int nbox, const hh_options *opt,
                             double *C_out, double *Sigma_out, double *Eps_out,
                             int *iters_out, double *resid_out);

/* Homogenization of an anisotropic image (Section 3: the assembled
 * intermediate image; Section 4: fully anisotropic voxels). `C21` holds the
 * upper triangle of each voxel's 6x6 Voigt stiffness, component-major:
 * C21[k * V + voxel], k over (00 01 02 03 04 05 11 12 ... 55). Every voxel
 * stiffness must be symmetric positive definite (checked: HH_ERR_BAD_STIFFNESS). */
hh_status hh_homogenize_aniso(hh_ctx *ctx, const double *C21, int nx, int ny, int nz,
                              int c21_on_device, const hh_options *opt, hh_result *out);

/* One application of the discrete operator of Appendix A to a strain field:
 * q = G * (C : p), with C from labels + phases (C21 == NULL) or from C21
 * (labels ignored). p and q are host doubles [6][nz][ny][nx] (tensor
 * components 11 22 33 23 13 12). Runs in the requested precision. */
hh_status hh_apply_operator(hh_ctx *ctx, const uint8_t *labels, const hh_phase *phases,
                            int nphase, const double *C21, int nx, int ny, int nz,
                            const double *p, double *q, const hh_options *opt);

/* Extraction of the buffered subimages (Section 4, Fig. 4) exactly as the
 * solver sees them: out receives the concatenated Omega_B label arrays of all
 * boxes (each (cnz+2b)(cny+2b)(cnx+2b), x fastest), indices wrapped
 * periodically. `out_len` is the capacity of out in bytes. */
hh_status hh_extract_subimages(hh_ctx *ctx, const uint8_t *img, int nx, int ny, int nz,
                               int img_on_device, const int32_t *boxes, int nbox,
                               uint8_t *out, int64_t out_len);

/* Hierarchical homogenization for each subimage edge in ns[0..count) (buffer
 * b), then the least-squares fit M(n) = M_inf + C / n (Section 5, Eq.
 * fit_power_law; with two sizes this is Richardson extrapolation) for K and G.
 * `per_n` (caller-owned [count] or NULL) receives each hierarchical result. */
hh_status hh_extrapolate(hh_ctx *ctx, const uint8_t *img, int nx, int ny, int nz,
                         int img_on_device, const hh_phase *phases, int nphase,
                         const int *ns, int count, int b, const hh_options *opt,
                         double *K_inf, double *C_K, double *G_inf, double *C_G,
                         hh_result *per_n);

/* Copy up to `cap` per-kernel statistics gathered since the last reset;
 * *count receives the number available. */
hh_status hh_profile_read(hh_ctx *ctx, hh_kernel_stat *out, int cap, int *count);

/* Clear the per-kernel statistics. */
hh_status hh_profile_reset(hh_ctx *ctx);

/* Least-squares fit of M(n) = M_inf + C / n over count >= 2 points (Section 5,
 * Eq. fit_power_law), evaluated in FP64 on the context's device. */
hh_status hh_fit_inverse_n(hh_ctx *ctx, const int *ns, const double *M, int count,
                           double *M_inf, double *C);

/* ---------------------------------------------------------------------------
 * Subimage surrogate (not in the paper; a learned shortcut for the first
 * hierarchical level). A small 3D CNN maps a buffered subimage (Omega_B) of
 * phase labels (0, 1, 2) with its core (Omega_R) to the 21 upper-triangle
 * components of the core's effective Voigt stiffness (row-major i <= j,
 * engineering shear), divided by a caller-chosen scale. Input channels: the
 * one-hot labels and the core mask (1 in the core, 0 in the buffer; a label
 * >= 3 contributes no phase channel). Layers: conv3^3 4->16 -> ReLU -> conv
 * 16->32 stride 2 -> ReLU -> conv 32->64 stride 2 -> ReLU -> conv 64->64 ->
 * ReLU -> mean pool over the voxels -> fc 64->128 -> ReLU -> fc 128->21; zero
 * padding 1, so any box shape runs through the same network.
 *
 * A call takes `count` subimages: boxes[count][9] int32 rows (nx, ny, nz, ox,
 * oy, oz, cnx, cny, cnz) give each box (every edge 8..256) and its core
 * (origin and size inside the box, at least one voxel); `labels` holds the
 * boxes' labels one after the other, each x fastest. Subimages of one box
 * shape are batched together.
 * Parameters are one flat FP32 vector of hh_cnn_num_params() values: per conv
 * layer W[tap][ci][co] (tap = (kz*3+ky)*3+kx) then bias[co]; per fc layer
 * W[in][out] then bias[out]. The convolutions run on BF16 tensor cores with
 * FP32 accumulation. All buffers below are host memory owned by the caller;
 * errors: HH_ERR_ARG (count < 1, a box or core outside the limits, NULL
 * pointers), HH_ERR_OOM, HH_ERR_CUDA. */
int64_t hh_cnn_num_params(void);

/* He-uniform initial parameters (params[hh_cnn_num_params()], host memory):
 * every weight of a layer with fan-in f (27 x input channels for a
 * convolution, the input width for a fully connected layer) is
 * (2 u_i - 1) sqrt(6 / f) and every bias 0, where u_i is the i-th output (i
 * the flat parameter index, from 0) of the SplitMix64 generator seeded with
 * `seed`, as a double in [0, 1) from its top 53 bits (the draws of the audit
 * below). Host only; HH_ERR_ARG for a NULL pointer. */
hh_status hh_cnn_init_params(uint64_t seed, float *params);

/* Network outputs out[count][21]. */
hh_status hh_cnn_forward(hh_ctx *ctx, const uint8_t *labels, int count, const int32_t *boxes,
                         const float *params, float *out);

/* Mean squared error over the count x 21 outputs against targets[count][21]
 * (*loss) and its gradient with respect to the parameters (grad[n_params]). */
hh_status hh_cnn_loss_grad(hh_ctx *ctx, const uint8_t *labels, int count, const int32_t *boxes,
                           const float *params, const float *targets, double *loss, float *grad);

/* Trains one network from `init` with Adam (beta 0.9/0.999, eps 1e-8; step
 * size lr with cosine decay to 0 over the run). Every epoch draws a seeded
 * permutation of each box shape's subimages, cuts it into whole minibatches of
 * min(batch, subimages of that shape), and takes the epoch's minibatches of all
 * shapes in a seeded order (SplitMix64 from `seed`); the final parameters go
 * to params_out. loss_history (epochs values, may be NULL) receives each
 * epoch's mean training loss. */
hh_status hh_surrogate_train(hh_ctx *ctx, const uint8_t *labels, int count, const int32_t *boxes,
                             const float *targets, const float *init, int epochs, int batch,
                             double lr, uint64_t seed, float *params_out, double *loss_history);

/* Predictions of an ensemble (params[ensemble][n_params]) in GPa:
 * out[count][ensemble][21] = network output * scale. */
hh_status hh_surrogate_predict(hh_ctx *ctx, const uint8_t *labels, int count, const int32_t *boxes,
                               const float *params, int ensemble, double scale, float *out);

/* Ensemble files. hh_surrogate_save writes params[ensemble][n_params]
 * (n_params = hh_cnn_num_params()) and the output scale to `path`; the file
 * is little-endian: the 8 bytes "HHSURR01", int32 ensemble, int32 0,
 * int64 n_params, float64 scale, uint64 FNV-1a (64-bit) hash of the
 * parameter bytes, then the FP32 parameters. hh_surrogate_load reads it back
 * bit for bit into params (capacity = floats available) and sets *ensemble
 * and *scale; with params NULL it only reads the header and sets both, so
 * the caller can size the buffer. Host-only calls (no context, no GPU).
 * Errors (text via hh_last_error(NULL)): HH_ERR_ARG for NULL pointers,
 * ensemble < 1, a scale that is not finite and > 0, a file that cannot be
 * opened, written or read, a wrong magic, n_params or length, a hash that
 * does not match, or a capacity below ensemble * n_params. */
hh_status hh_surrogate_save(const char *path, const float *params, int ensemble, double scale);
hh_status hh_surrogate_load(const char *path, float *params, int64_t capacity, int *ensemble,
                            double *scale);

/* The gate: accept[i] = 1 when every member's Voigt-projected K and G lie in
 * the Reuss..Voigt bounds of the phase moduli over the subimage's core (from
 * the core's phase fractions), the relative spread (max - min) / mean over the
 * members of K and of G is <= spread, and the members' mean stiffness is
 * positive definite; else 0 (the subimage goes to the FFT solver). c21[count][21]
 * receives the members' mean. members[count][ensemble][21] in GPa. */
hh_status hh_surrogate_gate(hh_ctx *ctx, const uint8_t *labels, int count, const int32_t *boxes,
                            const hh_phase *phases, int nphase, const float *members,
                            int ensemble, double spread, int *accept, double *c21);

/* Correlation length (Section 2, Eq. eq_correlation): with M = 1 on every
 * voxel whose label is not pore_label (mineral) and 0 on the pore,
 * counts[a][l] = sum of M(v) M(v + l e_a) over the voxel pairs inside the
 * image (a = 0, 1, 2 for x, y, z; l = 0..lmax; exact integers),
 * corr[a][l] = (<M M_l> - <M>^2) / (<M^2> - <M>^2) with the pair average over
 * those pairs and <M> = <M^2> over all voxels, and xi[a] the least-squares
 * fit of exp(-l / xi) to corr[a][0..L], L the first l where corr < 0.05. The
 * paper takes subimages of at least 3 xi (Section 2): *n_min (may be NULL)
 * receives ceil(3 max_a xi[a]), the smallest cubic subimage edge by that
 * rule. Buffers counts[3][lmax+1], corr[3][lmax+1], xi[3] are host memory
 * owned by the caller. Errors: HH_ERR_ARG (lmax outside 1..4096, pore_label
 * outside 0..255, a dimension < 2), HH_ERR_CUDA. */
hh_status hh_correlation(hh_ctx *ctx, const uint8_t *img, int nx, int ny, int nz, int img_on_device,
                         int pore_label, int lmax, int64_t *counts, double *corr, double *xi, int *n_min);

/* Hierarchical homogenization over several levels (Section 3: the coarse
 * image is renormalised again until it is small). Level 1 cuts the image
 * into cubes of edge ns[0] with buffer bs[0] (as hh_homogenize_hierarchical);
 * each further level l cuts the previous coarse anisotropic image into cubes
 * of ns[l] coarse cells with buffer bs[l], solves them with the anisotropic
 * medium and assembles their symmetric stiffnesses (raised to the stiffness
 * floor) into the next coarse image; the last coarse image is solved whole
 * by CG. Every ns[l] must divide the grid of its level. out receives the
 * final stiffness, K and G (K_am, G_am and the per-subimage arrays are not
 * filled). Errors as hh_homogenize_hierarchical. */
hh_status hh_homogenize_multilevel(hh_ctx *ctx, const uint8_t *img, int nx, int ny, int nz, int img_on_device,
                                   const hh_phase *phases, int nphase, const int *ns, const int *bs,
                                   int nlevels, const hh_options *opt, hh_result *out);

/* Choice of the subimage edge n and buffer width b (Section 2: n at least
 * 3 xi, see hh_correlation; Section 3, Eq. 2: the cost of the level-1
 * solves; Section 5: the HH error falls as C_b / n, with a constant C_b for
 * each buffer width, Table fit_pad). No GPU and no context needed.
 *
 * Candidates: every n with max(n_min, 1) <= n <= min(nx, ny, nz) that
 * divides nx, ny and nz, combined with every bs[i] (i < nb) such that the
 * buffered box edge n + 2 bs[i] has no prime factor above 31 (the FFT lengths
 * the solver takes). For each: predicted relative error c_rel[i] / n, where
 * c_rel[i] = |C_b| / M_inf is the fitted constant of buffer bs[i] (for
 * example from hh_extrapolate at that buffer), and predicted cost
 * (nx ny nz / n^3) (n + 2 bs[i])^a, in units of one solve of a 1-voxel box,
 * with a the exponent of the single-solve time against the edge (the paper
 * measured 3.66). The cheapest candidate whose error is <= eps is returned;
 * equal costs go to the smaller error, then the larger n, then the smaller
 * b. If no candidate meets eps, the one with the least error (then the
 * least cost) is returned with HH_WARN_TARGET_UNMET.
 * Outputs (host): *n_out, *b_out, *err_out and *cost_out (the last two may
 * be NULL). Errors: HH_ERR_ARG (a dimension < 1, NULL bs, c_rel, n_out or
 * b_out, nb < 1, a buffer < 0, a constant negative or not finite, a <= 0,
 * eps <= 0, or no candidate at all). */
hh_status hh_plan_partition(int nx, int ny, int nz, int n_min, const int *bs, const double *c_rel, int nb,
                            double a, double eps, int *n_out, int *b_out, double *err_out, double *cost_out);

/* Two-level scheme on a partition (as hh_homogenize_partition) where every
 * subimage whose buffered box has edges 8..256 is first offered, with its
 * buffer and its core, to the surrogate ensemble (params[ensemble][n_params],
 * outputs * scale = GPa) and its gate (spread as in hh_surrogate_gate):
 * accepted subimages take the ensemble's mean stiffness (raised to the
 * stiffness floor like FFT results) and skip the FFT solve; every other
 * subimage is solved by the FFT solver with `opt`.
 *
 * Audit: the FFT solver also checks a random sample of the accepted
 * subimages. Accepted subimage i is audited when u_i < audit_fraction, where
 * u_i is the top 53 bits (times 2^-53) of the i-th output (i from 0) of the
 * SplitMix64 generator (Steele, Lea and Flood, 2014) seeded with audit_seed:
 * u_i = mix(audit_seed + (i + 1) * 0x9E3779B97F4A7C15), mix(z) = z3 ^ (z3 >> 31)
 * with z2 = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9 and
 * z3 = (z2 ^ (z2 >> 27)) * 0x94D049BB133111EB (64-bit wrap-around). An
 * audited subimage is solved by the FFT solver, which supplies its stiffness
 * for the assembly, and audit_err[i] (may be NULL; -1 elsewhere) receives the
 * ensemble mean's error against it: max(|K_p - K|/K, |G_p - G|/G) of the
 * isotropic Voigt projections of the ensemble mean as gated and of the FFT
 * solver's (C + C^T) / 2.
 * audit_fraction 0 audits nothing, 1 every accepted subimage.
 *
 * accepted[nbox] (may be NULL): 0 rejected by the gate (or not a candidate),
 * 1 accepted (the ensemble's stiffness is used), 2 accepted and audited.
 * out->n_surrogate_accepted counts the subimages the gate accepted, audited
 * ones included. out->device_ms covers the FFT solves, the assembly and
 * level 2, not the network's inference. */
hh_status hh_homogenize_partition_surrogate(hh_ctx *ctx, const uint8_t *img, int nx, int ny, int nz,
                                            int img_on_device, const hh_phase *phases, int nphase,
                                            const int32_t *boxes, int nbox, int unit, const float *params,
                                            int ensemble, double scale, double spread, double audit_fraction,
                                            uint64_t audit_seed, const hh_options *opt, hh_result *out,
                                            double *per_sub_C, int *accepted, double *audit_err);

/* ---------------------------------------------------------------------------
 * Operator application without allocation. The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory (code
 * that runs inside a memory pool or arena it does not own, allocation-free
 * real-time loops, hosts whose allocator must not be re-entered).
 *
 * q = G * (C : p) as hh_apply_operator computes it, in FP32, on device
 * buffers the caller owns: labels (uint8 [nz][ny][nx], every label < nphase:
 * checked on the device before the operator runs, HH_ERR_ARG otherwise), p
 * and q (float [6][nz][ny][nx], tensor components 11 22 33 23 13 12).
 * `phases` is a host table. Work is enqueued on `cuda_stream` (NULL = legacy
 * default stream) of the current device; the call synchronizes that stream
 * twice (after the label check and at the end) before returning.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine. Its scratch
 * is one fixed device array of HH_NOALLOC_SCRATCH_BYTES inside the library,
 * held by every GPU that loads the library until the process exits; each
 * edge is limited to HH_NOALLOC_MAX_EDGE and the half spectrum must fit the
 * array, else HH_ERR_ARG. The first call on a device looks the array's
 * device address up (cudaGetSymbolAddress) and raises the kernels'
 * shared-memory limit, with that device current: make that first call
 * before any stream capture. Every call shares the array and overwrites
 * what it reads there (the label check's flag, the one value that must
 * start at zero, is cleared by each call's copy of its tables), so calls
 * that overlap on the GPU race; serialize them.
 * Errors: HH_ERR_ARG, HH_ERR_UNSUPPORTED, HH_ERR_CUDA; text via
 * hh_last_error(NULL). */
#define HH_NOALLOC_SCRATCH_BYTES (16u << 20)
#define HH_NOALLOC_MAX_EDGE 80
hh_status hh_apply_operator_noalloc(const uint8_t *labels, const hh_phase *phases, int nphase,
                                    int nx, int ny, int nz, const float *p, float *q,
                                    int nyquist, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* HH_H */
