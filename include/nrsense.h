/*
 * nrsense.h - C ABI of the GB300 (sm_103a) nonrigid SENSE operator library.
 *
 * The library applies the nonrigid SENSE operator of Jang, Malave & Nishimura,
 * "Image-Space Gridding for Nonrigid Motion-Corrected MR Image Reconstruction"
 * (arXiv 2501.16713), section "Nonrigid SENSE Operators":
 *
 *     A_j = G_j S T_j,   A_j^H = T_j^H S^H G_j^H,   j = 0 .. P-1,
 *
 * stacked over motion states (respiratory phases) as in the stacked SENSE
 * equation, and the Tikhonov-regularised normal equations of the
 * reconstruction problem.  T_j is image-space gridding (section "Image-space
 * Gridding", forward and adjoint process diagrams), S the coil sensitivities,
 * G_j inverse k-space gridding (section "k-space Gridding", inverse gridding
 * diagram) and G_j^H k-space gridding (gridding process diagram).
 *
 * Conventions (all entry points):
 *   - Complex data are interleaved single precision (nrsense_c64).
 *   - Images are C-order arrays of shape (n[0], n[1], n[2]) (axis 2 fastest).
 *   - Displacements are float32, shape (P, 3, n0, n1, n2): component a moves
 *     along image axis a, in voxels; the warp pulls: m_j[r] = m(r + d_j[r])
 *     (displacement-field equation).  Boundaries are periodic.
 *   - k-space coordinates are float32 radians, shape (sum_j M_j, 3),
 *     phase-major; column a is the angular frequency along image axis a; any
 *     finite value is accepted and wrapped to [-pi, pi).
 *   - k-space data are phase-major, sample-major, coil fastest: the value of
 *     coil c at sample s of phase j sits at row off_j + s, column c of a
 *     (sum_j M_j) x C array, off_j = M_0 + ... + M_{j-1}.
 *   - Coil sensitivities are (C, n0, n1, n2) complex.
 *   - Every pointer argument named *_dev is a CUDA device pointer owned by the
 *     caller; the plan copies what it keeps during nrsense_plan_create.
 *     Pointers named *_host are host memory.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Apply calls
 *     are stream-ordered and asynchronous; they never synchronise the device
 *     except where stated.
 *   - A plan is not thread-safe: calls on one plan must be serialised (they
 *     share internal work buffers), and work launched on different streams
 *     with the same plan must not overlap.
 *   - Return values: NRSENSE_OK or a negative nrsense_status; on error nothing
 *     is written to outputs unless stated.  Errors detected inside kernels
 *     (bounded waits, bounds checks) are latched into a device status word
 *     readable with nrsense_device_status.
 */
#ifndef NRSENSE_H
#define NRSENSE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t nrsense_status;
#define NRSENSE_OK                 0
#define NRSENSE_ERR_ARG           -1  /* invalid argument or descriptor */
#define NRSENSE_ERR_OOM           -2  /* device or host allocation failed */
#define NRSENSE_ERR_CUFFT         -3  /* cuFFT plan or execution failed */
#define NRSENSE_ERR_CUDA          -4  /* CUDA runtime error (launch, copy) */
#define NRSENSE_ERR_BREAKDOWN     -5  /* CG: non-positive curvature or non-finite scalar */
#define NRSENSE_ERR_NOT_CONVERGED -6  /* CG: maxit reached above tolerance */
#define NRSENSE_ERR_TIMEOUT       -7  /* a bounded device wait expired */
#define NRSENSE_ERR_BOUNDS        -8  /* a device bounds check fired */
#define NRSENSE_ERR_STATE         -9  /* call not valid for this plan (e.g. no coils) */

typedef struct { float re, im; } nrsense_c64;

typedef struct nrsense_plan_s* nrsense_plan_t;

/* precision of the gridding grids (desc.precision) */
#define NRSENSE_FP32            0  /* FP32 storage and accumulation */

/* desc.flags */
#define NRSENSE_IDENTITY_WARP   (1u << 0)  /* T_j = I for every phase (plain SENSE) */

typedef struct {
  int32_t n[3];        /* image size per axis; each even and >= 4 */
  int32_t osf;         /* oversampling sigma, integer >= 2 (grid G = osf * n) */
  int32_t kb_width;    /* kernel width W in oversampled-grid units: 4 or 6 */
  double  kb_beta;     /* Kaiser-Bessel beta; 0 selects Beatty's formula */
  int32_t n_phases;    /* P >= 1 */
  int32_t n_coils;     /* C >= 0; 0 = image-space warp only (no S, no G_j) */
  int32_t precision;   /* NRSENSE_FP32 */
  uint32_t flags;      /* NRSENSE_* flags */
  int32_t phase_chunk; /* phases processed per launch (1..16); 0 = as many as half of the
                          free device memory at plan time allows */
} nrsense_desc;

/* Plan-time facts, for benchmarking and tests. */
typedef struct {
  int32_t grid[3];           /* oversampled grid size G per axis */
  double  kb_beta;           /* beta actually used */
  double  kernel_poly_err;   /* max |poly - c| / c(0) of the FP32 kernel polynomials */
  int64_t total_samples;     /* sum_j M_j */
  int32_t tile[3];           /* spreading tile (grid points per axis) */
  int64_t n_tiles;           /* tiles of one grid */
  double  occupied_fraction; /* fraction of (phase, tile) pairs holding samples */
  int64_t spread_items;      /* work items of the k-space spread (all phases) */
  int64_t split_tiles;       /* tiles split across several work items */
  int64_t device_bytes;      /* device memory held by the plan (excl. cuFFT work) */
  int32_t phase_chunk;       /* phases per launch actually used */
} nrsense_info;

/*
 * nrsense_plan_create - build an operator for one acquisition.
 *   desc           geometry and options (host).
 *   n_samples_host M_j for j = 0..P-1 (host, length P); ignored if n_coils == 0.
 *   coords_dev     (sum_j M_j, 3) float32 radians (device), or NULL if n_coils == 0.
 *   disp_dev       (P, 3, n0, n1, n2) float32 voxels (device); may be NULL when
 *                  desc->flags has NRSENSE_IDENTITY_WARP.
 *   smaps_dev      (C, n0, n1, n2) complex (device), or NULL if n_coils == 0.
 *   stream         stream for the plan's uploads and set-up kernels; the call
 *                  synchronises this stream before returning.
 *   out            receives the plan handle (host).
 * The plan copies coords, displacements and maps (the caller may free them
 * afterwards), computes the kernel and deapodization tables in FP64 on the
 * host, sorts each phase's samples into spreading tiles and creates cuFFT
 * plans.  Errors: ERR_ARG (bad descriptor, NaN/Inf coordinates or
 * displacements), ERR_OOM, ERR_CUFFT, ERR_CUDA.
 */
nrsense_status nrsense_plan_create(const nrsense_desc* desc,
                                   const int64_t* n_samples_host,
                                   const float* coords_dev,
                                   const float* disp_dev,
                                   const nrsense_c64* smaps_dev,
                                   void* stream,
                                   nrsense_plan_t* out);

/* Release every resource of a plan (synchronises the device).  NULL is a no-op. */
nrsense_status nrsense_plan_destroy(nrsense_plan_t plan);

/* Plan facts (host struct). */
nrsense_status nrsense_plan_info(nrsense_plan_t plan, nrsense_info* out);

/*
 * nrsense_apply_forward - y = [A_0; ...; A_{P-1}] x (stacked SENSE equation).
 *   x_dev  image (n0, n1, n2) complex (device, read only).
 *   y_dev  with coils: (sum_j M_j, C) complex (device, overwritten);
 *          without coils (n_coils == 0): the warped images T_j x as
 *          (P, n0, n1, n2) complex.
 */
nrsense_status nrsense_apply_forward(nrsense_plan_t plan, const nrsense_c64* x_dev,
                                     nrsense_c64* y_dev, void* stream);

/*
 * nrsense_apply_adjoint - x = sum_j A_j^H y_j (or sum_j T_j^H m_j without coils).
 *   y_dev  layout as the output of nrsense_apply_forward (device, read only).
 *   x_dev  image (n0, n1, n2) complex (device, overwritten).
 */
nrsense_status nrsense_apply_adjoint(nrsense_plan_t plan, const nrsense_c64* y_dev,
                                     nrsense_c64* x_dev, void* stream);

/*
 * nrsense_apply_normal - out = sum_j A_j^H A_j x + lambda x (normal operator of
 * the Tikhonov-regularised reconstruction problem; without coils the sum is
 * over T_j^H T_j).  x_dev and out_dev are (n0, n1, n2) complex device arrays
 * and must not alias.
 */
nrsense_status nrsense_apply_normal(nrsense_plan_t plan, const nrsense_c64* x_dev,
                                    double lambda, nrsense_c64* out_dev, void* stream);

/*
 * Stage entry points (same operator, one factor at a time).
 * nrsense_warp_forward:  m_dev (P, n0, n1, n2) = T_j x for every phase j.
 * nrsense_warp_adjoint:  x_dev = sum_j T_j^H m_j.
 * nrsense_kspace_forward: y_dev (M_j, C) = G_j v for coil images v_dev (C, n0, n1, n2).
 * nrsense_kspace_adjoint: v_dev (C, n0, n1, n2) = G_j^H y for y_dev (M_j, C).
 * The k-space calls need n_coils >= 1 (ERR_STATE otherwise) and 0 <= phase < P.
 */
nrsense_status nrsense_warp_forward(nrsense_plan_t plan, const nrsense_c64* x_dev,
                                    nrsense_c64* m_dev, void* stream);
nrsense_status nrsense_warp_adjoint(nrsense_plan_t plan, const nrsense_c64* m_dev,
                                    nrsense_c64* x_dev, void* stream);
nrsense_status nrsense_kspace_forward(nrsense_plan_t plan, int32_t phase,
                                      const nrsense_c64* v_dev, nrsense_c64* y_dev,
                                      void* stream);
nrsense_status nrsense_kspace_adjoint(nrsense_plan_t plan, int32_t phase,
                                      const nrsense_c64* y_dev, nrsense_c64* v_dev,
                                      void* stream);

/*
 * nrsense_solve_cg - conjugate gradients on the Tikhonov-regularised normal
 * equations (sum_j A_j^H A_j + lambda I) x = sum_j A_j^H y_j, the regularised
 * least-squares form of the reconstruction problem (reconstruction
 * optimisation equation, with lambda ||x||^2 in place of the wavelet L1 term).
 *   y_dev        k-space data, layout of nrsense_apply_forward's output (device).
 *   lambda       Tikhonov weight (>= 0; > 0 makes the system positive definite).
 *   tol          stop when ||r_k|| <= tol ||b|| (recursive residual, x0 = 0 unless
 *                NRSENSE_CG_X0).
 *   maxit        iteration limit (0 .. 2^20).
 *   flags        NRSENSE_CG_X0: x_dev holds the initial guess; NRSENSE_CG_GRAPH:
 *                iterations are captured once as a CUDA graph (per plan, x_dev,
 *                lambda) and replayed.
 *   x_dev        image (device): initial guess (with NRSENSE_CG_X0) and solution.
 *   iters_host   receives the number of iterations (may be NULL).
 *   res_hist_host receives ||r_k|| / ||b|| for k = 0 .. iters (maxit + 1 doubles
 *                of room; may be NULL).
 *   true_res_host receives ||b - E x|| / ||b||, recomputed once at exit (may be NULL).
 * Inner products, alpha, beta and norms are FP64 on the device; vectors are FP32.
 * The first call allocates the plan's CG workspace (four image vectors, an
 * internal stream).  The call synchronises the device at chunk boundaries and
 * at exit.  Returns NRSENSE_ERR_BREAKDOWN on non-positive curvature or
 * non-finite scalars, NRSENSE_ERR_NOT_CONVERGED if maxit is reached above tol.
 */
#define NRSENSE_CG_X0     (1u << 0)
#define NRSENSE_CG_GRAPH  (1u << 1)
nrsense_status nrsense_solve_cg(nrsense_plan_t plan, const nrsense_c64* y_dev, double lambda,
                                double tol, int32_t maxit, uint32_t flags, nrsense_c64* x_dev,
                                int32_t* iters_host, double* res_hist_host, double* true_res_host,
                                void* stream);

/*
 * nrsense_dot_noalloc - <x, y> = sum_i conj(x_i) y_i in FP64, for callers that
 * cannot allocate device memory.  The paper has no counterpart: this is a
 * variant of the CG solver's inner-product kernel that needs no plan and
 * calls no allocator.  Some callers may not call cudaMalloc (their device
 * memory belongs to another allocator or a fixed pool, or they run where an
 * allocation could block), so they can create no plan; they pass the inputs
 * and the output, and the block partial sums go to a fixed 256 KB array that
 * the library holds on every GPU where it is loaded, until the process exits.
 *   x_dev, y_dev  n complex values each (device, read only).
 *   n             0 <= n <= NRSENSE_DOT_NOALLOC_MAX_N; larger n is rejected
 *                 with NRSENSE_ERR_ARG before anything is launched.
 *   out_dev       two doubles (device): real and imaginary part of the sum.
 *   stream        stream for the two kernels; asynchronous.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  All calls
 * on a device share the one array: calls that overlap on the GPU (different
 * streams, no ordering) race and must not be issued.  Returns NRSENSE_ERR_CUDA
 * if the address lookup or a launch fails.
 */
#define NRSENSE_DOT_NOALLOC_MAX_N (16384LL * 4096LL)
nrsense_status nrsense_dot_noalloc(const nrsense_c64* x_dev, const nrsense_c64* y_dev, int64_t n,
                                   double* out_dev, void* stream);

/*
 * nrsense_device_status - read (and with clear != 0, reset) the plan's
 * latched device status word; synchronises `stream`.  *out_host receives
 * NRSENSE_OK or the first device-side error (ERR_BOUNDS, ERR_TIMEOUT).
 */
nrsense_status nrsense_device_status(nrsense_plan_t plan, int32_t clear, int32_t* out_host,
                                     void* stream);

/*
 * Stage profiling.  Between nrsense_profile_start and nrsense_profile_stop the
 * plan records a CUDA event pair around every stage it launches (on the
 * launching stream), for at most max_launches stages.  nrsense_profile_stop
 * synchronises the device and writes, per stage s < NRSENSE_NUM_STAGES, the
 * summed device time ms_host[s] and the number of recorded launches
 * count_host[s]; *own_kernels_host receives the number of the library's own
 * CUDA kernels launched in the window (cuFFT kernels excluded).
 */
#define NRSENSE_NUM_STAGES 13
#define NRSENSE_STAGE_FFT_N          0  /* cuFFT, N^3 */
#define NRSENSE_STAGE_FFT_G          1  /* cuFFT, G^3 single grid */
#define NRSENSE_STAGE_FFT_GC         2  /* cuFFT, G^3 x C batched */
#define NRSENSE_STAGE_DEAPOD_PAD     3  /* K1 */
#define NRSENSE_STAGE_INTERP_IMAGE   4  /* K2 */
#define NRSENSE_STAGE_SPREAD_IMAGE   5  /* K3 (+ partial-tile reduction) */
#define NRSENSE_STAGE_CROP_DEAPOD    6  /* K4 */
#define NRSENSE_STAGE_COIL_FANOUT    7  /* K5 */
#define NRSENSE_STAGE_INTERP_KSPACE  8  /* K6 */
#define NRSENSE_STAGE_SPREAD_KSPACE  9  /* K7 (+ partial-tile reduction) */
#define NRSENSE_STAGE_CROP_COILSUM  10  /* K8 */
#define NRSENSE_STAGE_VECTOR        11  /* elementwise vector kernels */
#define NRSENSE_STAGE_SOLVER        12  /* CG reductions and updates */
nrsense_status nrsense_profile_start(nrsense_plan_t plan, int32_t max_launches);
nrsense_status nrsense_profile_stop(nrsense_plan_t plan, double* ms_host, int64_t* count_host,
                                    int64_t* own_kernels_host);
const char* nrsense_stage_name(int32_t stage);

/* Static description of a status code. */
const char* nrsense_status_string(nrsense_status status);

#ifdef __cplusplus
}
#endif

#endif /* NRSENSE_H */
