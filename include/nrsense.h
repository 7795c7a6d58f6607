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
/* -8 is not used */
#define NRSENSE_ERR_STATE         -9  /* call not valid for this plan (e.g. no coils) */

typedef struct { float re, im; } nrsense_c64;

typedef struct nrsense_plan_s* nrsense_plan_t;
typedef struct nrsense_cnn_s* nrsense_cnn_t;

/* precision of the gridding grids (desc.precision) */
#define NRSENSE_FP32             0  /* FP32 storage and accumulation */
#define NRSENSE_BF16_STORE       1  /* k-space coil grids stored as complex BF16 (round to
                                       nearest even), FP32 arithmetic in every kernel, cuFFT
                                       BF16 transforms of the coil grids; every oversampled
                                       grid size must be a power of two */
#define NRSENSE_FP32_COMPENSATED 2  /* FP32 storage; spreading (W = 4 only) accumulates with
                                       compensated summation (FMA residual + TwoSum per
                                       update, compensation added at write-out) */

/* desc.flags */
#define NRSENSE_IDENTITY_WARP   (1u << 0)  /* T_j = I for every phase (plain SENSE) */

typedef struct {
  int32_t n[3];        /* image size per axis; each even and >= 4 */
  int32_t osf;         /* oversampling sigma, integer 2..4 (grid G = osf * n) unless grid[]
                          is given */
  int32_t kb_width;    /* kernel width W in oversampled-grid units: 4 or 6 */
  double  kb_beta;     /* Kaiser-Bessel beta; 0 selects Beatty's formula */
  int32_t n_phases;    /* P >= 1 */
  int32_t n_coils;     /* C >= 0; 0 = image-space warp only (no S, no G_j) */
  int32_t precision;   /* NRSENSE_FP32, NRSENSE_BF16_STORE or NRSENSE_FP32_COMPENSATED */
  uint32_t flags;      /* NRSENSE_* flags */
  int32_t phase_chunk; /* phases processed per launch (1..16); 0 = as many as half of the
                          free device memory at plan time allows */
  int32_t grid[3];     /* oversampled grid G per axis, overriding osf when all three are
                          > 0: sigma = G / n, the same ratio on every axis, 1.25 <= sigma
                          <= 4, G <= 1024 (a rational sigma such as 1.5 or 1.25, with a wider
                          kernel for the same aliasing error; the pruned coil-grid transforms
                          need sigma 2 and the tensor-core and TMA kernels W = 4, so other
                          choices run the generic kernels); all 0: G = osf * n */
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
  double  union_fraction;    /* fraction of tiles in the union over phases (the tiles the
                                k-space spread writes; the rest of a coil grid stays zero) */
  double  union_columns;     /* fraction of (axis 1, axis 2) tile columns holding a union tile:
                                the pruned transforms' axis-0 passes touch only those */
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
 * displacements), ERR_OOM, ERR_CUFFT, ERR_CUDA; on any error every resource
 * the call had taken is released.
 * Test-only environment variables, read at plan creation: NRSENSE_FAULT =
 * alloc | cufft | upload makes the first device allocation, cuFFT plan
 * creation or host-to-device upload fail (ERR_OOM, ERR_CUFFT, ERR_CUDA);
 * NRSENSE_TMA_POLL_LIMIT = n bounds the TMA halo wait of the k-space
 * interpolation to n polls (0: every TMA-staged CTA records ERR_TIMEOUT,
 * waits for its copy to land and returns without computing).
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
 *                lambda) and replayed: with tol = 0 (a fixed iteration count)
 *                min(maxit, 64) iterations form one graph, otherwise 2, with
 *                the converged flag read between graph launches.
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
#define NRSENSE_CG_CIRCULANT (1u << 2)  /* nrsense_solve_fcg: precondition by the plan's
                                            circulant preconditioner (nrsense_set_circulant),
                                            before the network when one is given */
#define NRSENSE_CG_DEFLATE   (1u << 3)  /* nrsense_solve_fcg: deflate the plan's recycled
                                            subspace (nrsense_set_deflation) */
#define NRSENSE_DEFLATE_LARGEST (1u << 4)  /* nrsense_deflation_from_solve: the Ritz vectors
                                               of the k largest Ritz values, not the smallest */
nrsense_status nrsense_solve_cg(nrsense_plan_t plan, const nrsense_c64* y_dev, double lambda,
                                double tol, int32_t maxit, uint32_t flags, nrsense_c64* x_dev,
                                int32_t* iters_host, double* res_hist_host, double* true_res_host,
                                void* stream);

/*
 * nrsense_solve_cg_record - nrsense_solve_cg that also records iterates, to
 * generate training pairs for the preconditioner network.  Before iteration
 * k = 0, 1, ... (while k < capacity and the solve has not converged) it
 * stores the recursive residual r_k in rec_r_dev[k] and, at exit, the error
 * x_final - x_k in rec_e_dev[k]; since E (x* - x_k) = r_k, a converged x_final
 * makes (r_k, e_k) an input/target pair of the preconditioner.
 *   rec_r_dev, rec_e_dev  capacity x (n0 n1 n2) complex each (device, written).
 *   capacity              >= 0 (0 records nothing).
 *   rec_count_host        receives the number of recorded pairs.
 * NRSENSE_CG_GRAPH is not accepted here (ERR_ARG): recording synchronises the
 * host once per iteration.  Other arguments, results and errors as
 * nrsense_solve_cg.
 */
nrsense_status nrsense_solve_cg_record(nrsense_plan_t plan, const nrsense_c64* y_dev, double lambda,
                                       double tol, int32_t maxit, uint32_t flags,
                                       nrsense_c64* x_dev, int32_t* iters_host,
                                       double* res_hist_host, double* true_res_host,
                                       nrsense_c64* rec_r_dev, nrsense_c64* rec_e_dev,
                                       int32_t capacity, int32_t* rec_count_host, void* stream);

/*
 * nrsense_solve_fcg - flexible conjugate gradients (FCG(1), Polak-Ribiere
 * coefficient) on the same normal equations, preconditioned by the network
 * `net` (z_k = M(r_k)); net = NULL gives the unpreconditioned iteration in
 * the same form.  The paper has no preconditioner: this is the learned
 * preconditioner added to the Tikhonov CG solve.
 *   alpha = Re<r, z> / Re<p, E p>,  beta = -alpha Re<z_new, E p> / Re<z, r>.
 * A network output with Re<r, z> <= 0 or non-finite falls back to z = r and
 * restarts (beta = 0); *fallbacks_host (may be NULL) receives how often.
 * net must have the plan's image shape (ERR_ARG otherwise) and is used, not
 * modified; its activation buffers are shared, so no other call on net may
 * overlap the solve.  Arguments, flags (NRSENSE_CG_X0, NRSENSE_CG_GRAPH),
 * results and errors as nrsense_solve_cg; the convergence test uses the
 * recursive residual ||r_k|| <= tol ||b||.
 */
nrsense_status nrsense_solve_fcg(nrsense_plan_t plan, nrsense_cnn_t net, const nrsense_c64* y_dev,
                                 double lambda, double tol, int32_t maxit, uint32_t flags,
                                 nrsense_c64* x_dev, int32_t* iters_host, double* res_hist_host,
                                 double* true_res_host, int32_t* fallbacks_host, void* stream);

/*
 * Preconditioner network M (no counterpart in the paper).  For a residual
 * image r (n0, n1, n2) complex:
 *   s = sqrt(mean |r|^2),  u0 = [Re r, Im r] / s  (2 channels),
 *   h_l = relu(conv_l(h_{l-1})), l = 1..4 (16 channels),  o = conv_5(h_4),
 *   z = u0 + o read as a complex image (z = 0 when r = 0),
 * conv_l: 3x3x3 cross-correlation with zero padding plus a bias, channels
 * 2 -> 16 -> 16 -> 16 -> 16 -> 2.  Training loss for a target e:
 *   L = 1 - Re<z, e> / (||z|| ||e||)  (L = 1 and no gradient if z or e is 0).
 * Weights and activations are BF16 on the device with FP32 accumulation
 * (tensor cores); master weights, gradients and Adam moments are FP32; the
 * input scale and the loss are FP64 reductions.
 *
 * Parameter layout (host arrays of nrsense_cnn_num_params() floats): layer by
 * layer, W_l as C-order (Cout, Cin, 3, 3, 3) with W[o, c, tz, ty, tx]
 * multiplying input voxel (z + tz - 1, y + ty - 1, x + tx - 1), then b_l (Cout).
 *
 * nrsense_cnn_create     network for images of shape n_host[3] (each 1..4096),
 *                        all parameters zero; allocates its activations
 *                        (7 x 32 bytes + 8 bytes per voxel, 13 x 32 + 8 in the
 *                        symmetric form); synchronises stream.  flags:
 *                        NRSENSE_CNN_SYMMETRIC selects the symmetric form
 *                          z = u0 + N4^T (I + W5^T W5) N4 u0,
 *                        N4 = D_4 W_4 D_3 W_3 D_2 W_2 D_1 W_1 the first four
 *                        convolutions without biases (D_l: ReLU masks of the
 *                        forward pass), W_5 the fifth, ^T the transposed
 *                        convolutions in reverse order with the same masks: for
 *                        fixed masks z = (I + A^T A) u0, A = [N4; W_5 N4],
 *                        symmetric positive definite in u0, as CG-type methods
 *                        expect of a preconditioner.
 *                        Biases are ignored and never updated in this form.
 * nrsense_cnn_init_params He initialisation from a seeded generator
 *                        (splitmix64 + Box-Muller), last layer scaled by 0.1,
 *                        biases zero; resets the Adam state.
 * nrsense_cnn_set_params / get_params  host copies in the layout above
 *                        (count must equal nrsense_cnn_num_params(); set rejects
 *                        non-finite values and resets the Adam state).
 * nrsense_cnn_apply      z_dev = M(r_dev), both (n0, n1, n2) complex device
 *                        arrays; asynchronous.
 * nrsense_cnn_gradients  forward + backward for one pair (r_dev, e_dev); the
 *                        parameter gradients are written (accumulate = 0) or
 *                        added (accumulate != 0) to the device gradient buffer;
 *                        *loss_host (may be NULL; then asynchronous) receives L.
 *                        plan == NULL: the cosine loss above.  plan != NULL
 *                        (same image shape, else ERR_ARG): the energy loss
 *                          L = 1 - c|c| / (<z, E z> <e, r>),  c = Re<z, r>,
 *                        E = sum_j A_j^H A_j + lambda I of the plan, the error
 *                        energy left after a line search along z when E e = r
 *                        (one nrsense_apply_normal per call; the first such
 *                        call allocates an image buffer).
 * nrsense_cnn_get_grads  host copy of the gradient buffer (layout above).
 * nrsense_cnn_adam_step  one Adam update with gradient grad_scale * buffer
 *                        (e.g. 1 / pairs accumulated); asynchronous.  flags:
 *                        NRSENSE_CNN_FREEZE_BIAS leaves the biases unchanged.
 * nrsense_cnn_launches   the network's own kernel launches so far.
 * Errors: ERR_ARG (null handle or pointer, bad shape or count, bad Adam
 * constants), ERR_OOM, ERR_CUDA.  A handle is not thread-safe.
 */
#define NRSENSE_CNN_SYMMETRIC (1u << 0)
nrsense_status nrsense_cnn_create(const int32_t* n_host, uint32_t flags, void* stream,
                                  nrsense_cnn_t* out);
nrsense_status nrsense_cnn_destroy(nrsense_cnn_t net);
int64_t nrsense_cnn_num_params(void);
nrsense_status nrsense_cnn_init_params(nrsense_cnn_t net, uint64_t seed, void* stream);
nrsense_status nrsense_cnn_set_params(nrsense_cnn_t net, const float* params_host, int64_t count,
                                      void* stream);
nrsense_status nrsense_cnn_get_params(nrsense_cnn_t net, float* params_host, int64_t count,
                                      void* stream);
nrsense_status nrsense_cnn_apply(nrsense_cnn_t net, const nrsense_c64* r_dev, nrsense_c64* z_dev,
                                 void* stream);
nrsense_status nrsense_cnn_gradients(nrsense_cnn_t net, nrsense_plan_t plan, double lambda,
                                     const nrsense_c64* r_dev, const nrsense_c64* e_dev,
                                     int32_t accumulate, double* loss_host, void* stream);
nrsense_status nrsense_cnn_get_grads(nrsense_cnn_t net, float* grads_host, int64_t count,
                                     void* stream);
#define NRSENSE_CNN_FREEZE_BIAS (1u << 0)
nrsense_status nrsense_cnn_adam_step(nrsense_cnn_t net, float lr, float grad_scale, float beta1,
                                     float beta2, float eps, uint32_t flags, void* stream);
nrsense_status nrsense_cnn_launches(nrsense_cnn_t net, int64_t* out_host);

/*
 * nrsense_cnn_set_conv - the kernel behind the network's 3x3x3 convolutions:
 * NRSENSE_CNN_CONV_MMA (mma.sync m16n8k16 BF16, operands fed by ldmatrix; the
 * default) or NRSENSE_CNN_CONV_TCGEN05 (fifth-generation tensor cores: per
 * 4 x 8 x 16 output block four M = 128, N = 16 accumulator tiles in tensor
 * memory, 27 K = 16 BF16 products each issued by one thread, operands in
 * shared memory in the canonical no-swizzle K-major layout).  Both compute the
 * same sums in FP32 (in a different order: results agree to FP32 rounding,
 * and stored BF16 activations to about one BF16 ulp).  The tcgen05 kernel
 * loads each block's input halo by bulk tensor copies (tensor maps of the
 * network's activation buffers, built at creation).  Errors: ERR_ARG,
 * ERR_STATE (tcgen05 asked but the tensor maps could not be built).
 * nrsense_cnn_device_status - the network's device status word: 0, or
 * NRSENSE_ERR_TIMEOUT when a tcgen05 convolution's bounded wait for its
 * products expired (that block stored nothing); clear != 0 resets it.
 * Synchronises the stream.
 */
#define NRSENSE_CNN_CONV_MMA      0
#define NRSENSE_CNN_CONV_TCGEN05  1
nrsense_status nrsense_cnn_set_conv(nrsense_cnn_t net, int32_t kind);
nrsense_status nrsense_cnn_device_status(nrsense_cnn_t net, int32_t clear, int32_t* out_host,
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
 * streams, no ordering) race and must not be issued.  The looked-up address
 * is cached per device for the life of the process; after a cudaDeviceReset
 * of that device the cache is stale and the call must not be used again in
 * that process.  Returns NRSENSE_ERR_CUDA if a CUDA error from earlier work is
 * pending when it is called (nothing is launched then), or if the address
 * lookup or a launch fails.
 */
#define NRSENSE_DOT_NOALLOC_MAX_N (16384LL * 4096LL)
nrsense_status nrsense_dot_noalloc(const nrsense_c64* x_dev, const nrsense_c64* y_dev, int64_t n,
                                   double* out_dev, void* stream);

/*
 * Phase sharding over several GPUs (one process per GPU).  The stacked SENSE
 * equation sums the motion states ("Nonrigid SENSE Operators": A^H y =
 * sum_j A_j^H y_j, E = sum_j A_j^H A_j + lambda I), so a rank can hold a plan
 * of its own states j in J_r only and the ranks' partial sums add up to the
 * whole.  nrsense_plan_set_reduce registers the step that adds them: the
 * library calls fn(user, image_dev, n, stream) right after it has formed this
 * plan's phase sum of an adjoint (nrsense_apply_adjoint, and so every solver's
 * right-hand side) or of a normal-operator application (nrsense_apply_normal,
 * before lambda x is added), with image_dev the n = n0 n1 n2 complex values
 * (device) and `stream` the stream the sum was formed on.  fn must replace the
 * image, in stream order, by the sum of every rank's image (an all-reduce, e.g.
 * ncclAllReduce on `stream`) and return NRSENSE_OK; any other return makes the
 * calling entry point fail with ERR_CUDA.  Every rank then holds the same
 * vectors, so the CG, flexible-CG and FISTA iterations and their FP64
 * reductions run unchanged and identically on every rank; only images are
 * exchanged.  fn = NULL removes the hook.  With a hook, graph capture of a
 * solve (NRSENSE_CG_GRAPH) requires fn's work to be capturable on `stream`.
 * As for every call of this library, the calling thread must have the plan's
 * device current (cudaSetDevice) before it calls in.
 * nrsense_copy_c64 copies n complex values device to device on `stream` (for
 * reduction hooks that stage the image in their own buffer).
 */
typedef nrsense_status (*nrsense_reduce_fn)(void* user, nrsense_c64* image_dev, int64_t n,
                                            void* stream);
nrsense_status nrsense_plan_set_reduce(nrsense_plan_t plan, nrsense_reduce_fn fn, void* user);
nrsense_status nrsense_copy_c64(nrsense_c64* dst_dev, const nrsense_c64* src_dev, int64_t n,
                                void* stream);

/*
 * Circulant preconditioner (not in the paper; serves the Tikhonov CG solve).
 * nrsense_set_circulant computes the point-spread function of the plan's
 * normal operator, h = E0 delta at the image centre (E0 with lambda = 0, one
 * application), and keeps d[k] = 1 / (max(Re DFT(h with the centre moved to
 * the origin)[k], 0) + lambda): the inverse of the circulant (shift-invariant)
 * approximation of E0 + lambda I, Hermitian positive definite.  enable = 0
 * switches it off (buffers are kept).  Synchronises the stream.  Errors:
 * ERR_ARG (lambda < 0 or not finite), ERR_OOM, ERR_CUFFT.
 * nrsense_apply_circulant: z = IDFT(d . DFT(r)) for image-shaped device
 * vectors (z may equal r); ERR_STATE before nrsense_set_circulant.
 * nrsense_solve_fcg with NRSENSE_CG_CIRCULANT uses z = M(M_c r) (network
 * given) or z = M_c r (net = NULL: preconditioned CG).
 */
nrsense_status nrsense_set_circulant(nrsense_plan_t plan, double lambda, int32_t enable,
                                     void* stream);
nrsense_status nrsense_apply_circulant(nrsense_plan_t plan, const nrsense_c64* r_dev,
                                       nrsense_c64* z_dev, void* stream);

/*
 * Deflation with a recycled subspace (not in the paper; serves the Tikhonov CG
 * solve of its reconstruction problem when the same operator is solved for
 * several right-hand sides).  The method is the A-DEF2 deflated preconditioned
 * CG of Tang, Nabben and Vuik (J. Sci. Comput. 39, 2009) with a basis W of k
 * image vectors: E_c = W^H E W, x_0 = x_init + W E_c^-1 W^H r_init, and every
 * search direction is projected by P^T z = z - W E_c^-1 (E W)^H z, so each
 * residual stays orthogonal to W and the iteration runs on the spectrum of
 * M E without W's part.
 *
 * nrsense_set_deflation copies W (w_dev: k consecutive image-shaped device
 * vectors), orthonormalises it (modified Gram-Schmidt, twice per vector, FP64
 * inner products; a vector with less than 1 % of its norm outside the span of
 * the earlier kept ones is dropped, so the space depends only on span(W) and
 * repeated vectors cost nothing), applies E0 (lambda = 0) to each kept vector
 * and keeps W^H E0 W and W^H W in FP64 on the host; kept_host (may be NULL)
 * receives the number of kept vectors.  A solve with lambda forms
 * E W = E0 W + lambda W and inverts E_c = W^H E0 W + lambda W^H W (FP64, on the
 * host; a pseudo-inverse that drops eigenvalues below 1e-10 of the largest, so
 * nearly dependent basis vectors do not amplify rounding) when lambda changes.
 * k = 0 switches deflation off and frees the space.
 * Memory: 3 k image vectors.  Synchronises the stream.  Errors: ERR_ARG (k < 0,
 * k > 64, w_dev NULL with k > 0), ERR_BREAKDOWN (no vector kept: W zero or
 * not finite), ERR_OOM, ERR_CUDA.
 *
 * nrsense_deflation_from_solve builds W from a solve: `steps` iterations of CG
 * (preconditioned by the circulant preconditioner with NRSENSE_CG_CIRCULANT,
 * else none) from x = 0 on E x = sum_j A_j^H y_j, recording z_j / sqrt(rho_j)
 * (z_j the preconditioned residual, rho_j = Re<r_j, z_j>) and the step sizes;
 * the CG-Lanczos tridiagonal T (T[j][j] = 1/alpha_j + beta_{j-1}/alpha_{j-1},
 * T[j][j+1] = -sqrt(beta_j)/alpha_j, beta_j = rho_{j+1}/rho_j) is
 * diagonalised on the host (FP64 Jacobi rotations); the Ritz vectors of the k
 * smallest Ritz values (estimates of the smallest eigenvalues of M E), or with
 * NRSENSE_DEFLATE_LARGEST of the k largest, become W as by
 * nrsense_set_deflation.  ritz_host receives those k Ritz values in the order
 * taken (ascending, or descending with NRSENSE_DEFLATE_LARGEST; may be NULL)
 * and kept_host (may be NULL) the number of basis vectors kept (repeated Ritz
 * vectors, which a long run in finite precision produces, are dropped).
 * Which end pays depends on the spectrum: with the circulant preconditioner
 * built for a larger lambda than the solve's, the low end of M E is a large
 * cluster (every poorly sampled frequency) that k vectors cannot remove, and
 * the high end holds the outliers.  A run that converges before `steps` uses
 * the iterations it made (k is then clipped to them).  Temporary memory:
 * `steps` image vectors.  Errors: ERR_ARG (steps < 1 or > 256, k < 1,
 * k > min(steps, 64), flags other than NRSENSE_CG_CIRCULANT and
 * NRSENSE_DEFLATE_LARGEST), ERR_STATE (circulant flag before
 * nrsense_set_circulant), ERR_BREAKDOWN, ERR_OOM, ERR_CUDA.
 *
 * nrsense_solve_fcg with NRSENSE_CG_DEFLATE runs the deflated iteration
 * (circulant and network preconditioning as without it; a network step that
 * falls back to z = r is not projected); ERR_STATE without a space.
 */
nrsense_status nrsense_set_deflation(nrsense_plan_t plan, const nrsense_c64* w_dev, int32_t k,
                                     int32_t* kept_host, void* stream);
nrsense_status nrsense_deflation_from_solve(nrsense_plan_t plan, const nrsense_c64* y_dev,
                                            double lambda, int32_t steps, int32_t k,
                                            uint32_t flags, double* ritz_host,
                                            int32_t* kept_host, void* stream);

/*
 * nrsense_symmetric_eigen - the host eigen-solver nrsense_deflation_from_solve
 * uses: eigenvalues (ascending, vals_host[m]) and eigenvectors (column i of
 * the row-major m x m vecs_host belongs to vals_host[i]) of the real
 * symmetric m x m matrix a_host (row-major; only its symmetric part is
 * meaningful), by cyclic Jacobi rotations in FP64.  Host only: needs no
 * device.  Errors: ERR_ARG (m < 1 or > 256, NULL pointers).
 */
nrsense_status nrsense_symmetric_eigen(int32_t m, const double* a_host, double* vals_host,
                                       double* vecs_host);

/*
 * Autotuning of the launch choices of a plan (no counterpart in the paper).
 * nrsense_plan_autotune times, on the plan's own k-space point sets (first
 * phase chunk) and internal buffers, the k-space spreading kernel with
 * register accumulation (a CTA per tile or per tile plane), with
 * shared-memory accumulation and with tensor-core accumulation, the image-space spreading kernel with a CTA
 * per tile or per plane pair, the k-space
 * interpolation with 8 and with 4 coils per CTA, its tile halos staged per
 * value or by one tensor-memory-accelerator copy, and the coil-grid
 * transforms (cuFFT or the own pruned passes) (reps launches each, after
 * one warm-up launch, CUDA events on `stream`; synchronises), keeps the
 * faster of each in the plan and reports times and choices in *out (host).
 * The compensated precision always uses shared-memory accumulation for k
 * space; plans without coils tune only the image-space spread.
 * nrsense_plan_set_tuning applies stored choices (e.g. a cache keyed by the
 * geometry).  Both change only speed: every choice computes the same values
 * (bitwise, except the tensor-core spread and the pruned transforms, which
 * agree to FP32 rounding).
 * Errors: ERR_ARG (null, reps outside 1..100, unknown choice), ERR_CUDA.
 */
#define NRSENSE_TUNE_SPREAD_REGISTER      1  /* register accumulation, CTA per tile */
#define NRSENSE_TUNE_SPREAD_SHARED        2  /* shared-memory accumulation */
#define NRSENSE_TUNE_SPREAD_REGISTER_WARP 3  /* register accumulation, CTA per tile plane */
#define NRSENSE_TUNE_SPREAD_MMA           4  /* tensor-core accumulation (TF32 split in three
                                                products), a warp per tile plane or per 4^3
                                                sub-block, 8-coil chunks
                                                (fewer coils: as REGISTER_WARP); within FP32
                                                rounding of, not bitwise equal to, the others */
typedef struct {
  int32_t spread_variant;  /* NRSENSE_TUNE_SPREAD_* */
  int32_t interp_coils;    /* coils per interpolation CTA: 8, 4 or 2 (2 with TMA staging; the
                              per-value staging then takes 4) */
  int32_t interp_tma;      /* 1: tile halos loaded by the tensor memory accelerator */
  double  spread_ms[3];    /* measured: register, shared, register per plane */
  double  interp_ms[2];    /* measured, per-value staging: 8 coils, 4 coils */
  double  interp_tma_ms[2];/* measured, TMA staging: 8 coils, 4 coils (-1: not available) */
  int32_t spread_image_warp;   /* image-space spread: 0 CTA per tile, 1 CTA per plane pair
                                  (both over per-tile halo lists), 2 home tiles (every displaced
                                  voxel spread once by the warp of the 8^3 tile holding its first
                                  tap, super-tile rims summed by a second kernel; W = 4 and not
                                  compensated; set_tuning rejects 2 elsewhere) */
  double  spread_image_ms[3];  /* measured: CTA per tile, CTA per plane pair, home tiles
                                  (-1: n/a) */
  int32_t fft_pruned;          /* 1: own pruned coil-grid transforms with the coil fan-out and
                                  combination fused (sigma 2, power-of-two grid sizes 32..256,
                                  FP32 grids); 0: cuFFT plus the fan-out / combination kernels */
  double  fft_ms[2];           /* measured forward + adjoint of the first phase chunk:
                                  cuFFT path, pruned path (-1: not available) */
  double  spread_mma_ms;       /* measured tensor-core spread, best geometry and warps per CTA
                                  (-1: n/a) */
  int32_t spread_mma_wpc;      /* warps per CTA of the tensor-core spread: 1, 2 or 4
                                  (set_tuning: other values mean 1) */
  int32_t spread_mma_cube;     /* tensor-core spread geometry: 0 a warp per tile plane (1 x 8 x 8
                                  grid points), 1 a warp per 4 x 4 x 4 sub-block of the tile
                                  (points staged once per sub-block they meet: 5.4 times on
                                  average against 7.6 tile planes) */
  double  spread_mma_geo_ms[2];/* measured, best warps per CTA: planes, sub-blocks (-1: n/a) */
  double  interp_tma2_ms;      /* measured, TMA staging with 2 coils per CTA (-1: n/a) */
  int32_t spread_max_item;     /* list entries per k-space spreading work item: heavier tiles
                                  are split into items this long whose partial tiles are summed
                                  in a fixed order (512, 1024 or 2048; longer items lengthen the
                                  FP32 accumulation chains past the 1e-5 bound on dense
                                  trajectories; set_tuning: 0 keeps the plan's, another value
                                  re-tiles the plan, synchronising) */
  double  spread_item_ms[3];   /* measured k-space spread with the chosen kernel at 512, 1024,
                                  2048 entries per item (-1: n/a) */
  int32_t interp_image_home;   /* image-space interpolation: 0 a thread per displaced voxel
                                  gathering from global memory, 1 super-tiles of the upsampled
                                  image staged in shared memory (W = 4, not compensated) */
  double  interp_image_ms[2];  /* measured: per voxel, super-tiles (-1: n/a) */
  int32_t image_fft_pruned;    /* image-space G^3 transforms of T and T^H: 1 own pruned passes
                                  (data half of every axis loaded or stored, deapodization and
                                  zero-padding / cropping fused into the x passes; sigma 2,
                                  power-of-two grid sizes 32..256, not with the compensated
                                  precision; set_tuning rejects 1 elsewhere), 0 cuFFT plus the
                                  deapodization kernels */
  double  image_fft_ms[2];     /* measured forward + adjoint G^3 transforms with their
                                  deapodization: cuFFT path, pruned path (-1: n/a) */
} nrsense_tuning;
nrsense_status nrsense_plan_autotune(nrsense_plan_t plan, int32_t reps, nrsense_tuning* out_host,
                                     void* stream);
nrsense_status nrsense_plan_set_tuning(nrsense_plan_t plan, const nrsense_tuning* tuning_host);

/*
 * Wavelet-FISTA (reconstruction optimisation equation; wavelet-FISTA as in
 * the in-vivo study and Appendix 1).  The problem
 *     minimise  ||y - A x||_2^2 + lambda ||W x||_1,   A = [A_0; ...; A_{P-1}]
 * (without coils A = [T_0; ...; T_{P-1}], the warp-only inversion of Appendix
 * 1) is solved by Beck and Teboulle's constant-step FISTA:
 *     x_k = W^H soft(W (z_k - (2/L)(E0 z_k - b)), lambda / L),
 *     z_{k+1} = x_k + ((t_k - 1) / t_{k+1}) (x_k - x_{k-1}),
 *     t_1 = 1, t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,  z_1 = x_0,
 * E0 = sum_j A_j^H A_j, b = sum_j A_j^H y_j, L >= 2 lambda_max(E0) (the
 * Lipschitz constant of the gradient of ||y - A x||^2).  W is the orthonormal
 * separable 3D Haar transform with `levels` levels (0 .. 4; 0 = identity)
 * applied to real and imaginary parts; every image axis must be divisible by
 * 2^levels (ERR_ARG otherwise).  soft(c, tau) = c max(0, 1 - tau / |c|) on
 * every coefficient, the coarsest approximation included.
 *
 * nrsense_wavelet_forward - c = W x in the Mallat layout: level 1 details
 *   fill the seven high-pass octants of the volume, level 2 details the
 *   octants of the low-pass corner, and so on; the approximation sits in the
 *   corner (n0, n1, n2) / 2^levels.  n_host: image shape (host, 3 values, each
 *   >= 1).  x_dev, c_dev: (n0, n1, n2) complex device arrays; they must not
 *   alias (ERR_ARG).
 * nrsense_wavelet_inverse - x = W^H c (c in the Mallat layout); no aliasing.
 * nrsense_wavelet_shrink  - u = W^H soft(W v, tau), the proximal map of
 *   tau ||W .||_1; tau >= 0; u_dev may equal v_dev (in place).
 *   All three are stream-ordered and need no plan.
 *
 * nrsense_normal_max_eig - power iteration on E0 (the plan's normal operator
 *   with lambda = 0): v <- v / |v|, then `iters` times w = E0 v,
 *   q = Re<v, w>, v <- w / |w|.  v_dev (plan image shape, device): the start
 *   vector on entry (caller-chosen, e.g. random), the last normalised iterate
 *   on exit.  *eig_host receives the last q (a lower bound of lambda_max that
 *   converges to it).  Synchronises the call's stream.
 *
 * nrsense_fista_lipschitz - the step bound L = 2 margin q of the FISTA
 *   iteration, q from nrsense_normal_max_eig(plan, v_dev, iters) (same
 *   arguments and behaviour, v_dev overwritten).  The gradient of
 *   ||y - A x||^2 is 2 (E0 x - b), so its Lipschitz constant is 2 lambda_max(E0);
 *   q approaches lambda_max from below and margin >= 1 (e.g. 1.02) covers the
 *   rest.  *lipschitz_host receives L.  ERR_ARG: margin < 1 or not finite,
 *   or an argument nrsense_normal_max_eig rejects.
 *
 * nrsense_solve_fista - `maxit` FISTA iterations (0 .. 2^20).
 *   y_dev      data, layout of nrsense_apply_forward's output (device).
 *   lambda     L1 weight (>= 0).
 *   lipschitz  L (> 0); a value below 2 lambda_max(E0) may diverge.
 *   flags      NRSENSE_CG_X0: x_dev holds x_0 (else x_0 = 0);
 *              NRSENSE_CG_GRAPH: iterations run as a captured CUDA graph of 32
 *              iterations, replayed (captured once per plan, x_dev, levels,
 *              lambda and L), the remainder eagerly.
 *   x_dev      image (device): x_0 on entry with NRSENSE_CG_X0, x_maxit on exit.
 *   hist_host  receives ||x_k - x_{k-1}|| / ||x_k|| for k = 1 .. maxit (maxit
 *              doubles; may be NULL).
 *   The first call allocates the plan's FISTA workspace (three image
 *   vectors, an internal stream).  Vectors are FP32, reductions FP64; the
 *   call synchronises its stream at exit.
 */
nrsense_status nrsense_wavelet_forward(const nrsense_c64* x_dev, nrsense_c64* c_dev,
                                       const int32_t* n_host, int32_t levels, void* stream);
nrsense_status nrsense_wavelet_inverse(const nrsense_c64* c_dev, nrsense_c64* x_dev,
                                       const int32_t* n_host, int32_t levels, void* stream);
nrsense_status nrsense_wavelet_shrink(const nrsense_c64* v_dev, nrsense_c64* u_dev,
                                      const int32_t* n_host, int32_t levels, double tau,
                                      void* stream);
nrsense_status nrsense_normal_max_eig(nrsense_plan_t plan, nrsense_c64* v_dev, int32_t iters,
                                      double* eig_host, void* stream);
nrsense_status nrsense_fista_lipschitz(nrsense_plan_t plan, nrsense_c64* v_dev, int32_t iters,
                                      double margin, double* lipschitz_host, void* stream);
nrsense_status nrsense_solve_fista(nrsense_plan_t plan, const nrsense_c64* y_dev, double lambda,
                                   int32_t levels, double lipschitz, int32_t maxit,
                                   uint32_t flags, nrsense_c64* x_dev, double* hist_host,
                                   void* stream);

/*
 * Motion capture for segmented acquisitions (section "Motion Capturing for
 * Segmented Data Acquisitions"; phase binning in "Nonrigid Respiratory Motion
 * Correction").  A heartbeat's low-resolution iNAV is the gridding
 * reconstruction of its density-corrected data; translations come from
 * correlations with a reference iNAV and are removed by linear phase shifts
 * of the k-space data; k-means on the translations gives the respiratory
 * phases, the least-variance cluster being the reference.
 *
 * nrsense_dcf - Pipe-Menon density compensation of phase `phase`'s samples:
 *   w = 1, then `iters` times w <- w / (B P w), P the k-space spread of w onto
 *   the oversampled grid and B the interpolation back to the samples, both
 *   with the plan's gridding kernel (no FFT).  w_dev: M_phase floats (device,
 *   overwritten).  Needs n_coils >= 1 and FP32 grids (ERR_STATE otherwise);
 *   0 <= iters <= 10000.  Stream-ordered; uses the plan's k-space grid
 *   buffers (so it must not overlap other calls on the plan).
 * nrsense_apply_adjoint_weighted - x = sum_j A_j^H (w . y_j): the adjoint of
 *   nrsense_apply_adjoint with every row (sample) of y scaled by w (one float
 *   per sample, shared by the coils; rows as y).  The first call allocates a
 *   copy of y's size in the plan.  Needs n_coils >= 1.
 * nrsense_translation_xcorr - for b < count: c_b[t] = sum_n |ref[n]| |img_b[n + t]|
 *   (circular), t_b = argmax (first in C order on ties) refined per axis by
 *   the vertex of the parabola through c at t - 1, t, t + 1 (kept when that
 *   parabola is not concave) and wrapped to (-n/2, n/2]; img_b[n] = ref[n - t]
 *   gives t_b = t.  ref_dev: (n0, n1, n2) complex; imgs_dev: count images of
 *   that shape, consecutive (device).  shifts_host: count x 3 doubles.  FP32
 *   magnitudes and cuFFT real transforms; allocates its buffers and cuFFT
 *   plans per call and synchronises the stream.  Each n >= 2, n0 n1 n2 <= 2^28.
 * nrsense_phase_ramp - y[r][c] *= exp(+i omega_r . t_s) for every row r of
 *   segment s, rows seg_off[s] <= r < seg_off[s + 1] (undoes a translation of
 *   the image by +t_s).  coords_dev: rows_total x 3 float radians; y_dev:
 *   rows_total x n_coils complex, in place (device).  seg_off_host: nseg + 1
 *   non-decreasing int64 within [0, rows_total] (ERR_ARG otherwise);
 *   shifts_host: nseg x 3 finite doubles (voxels).  Synchronises the stream.
 * nrsense_kmeans - k-means (Lloyd) of n points in 3D (host memory, n x 3
 *   doubles): start from the points at the positions (j + 1/2) n / k of the
 *   order along the first principal axis (sign: largest-magnitude entry
 *   positive; stable order), then assign each point to the nearest centre
 *   (ties to the lower index) and move each centre to its members' mean (an
 *   empty cluster keeps its centre) until the assignment repeats or max_iter
 *   assignments.  labels_host: n int32; centres_host: k x 3; inertia_host,
 *   iters_host, reference_host (the cluster of least mean squared distance to
 *   its centre) may be NULL.  Host only; 1 <= k <= n.
 */
nrsense_status nrsense_dcf(nrsense_plan_t plan, int32_t phase, int32_t iters, float* w_dev,
                           void* stream);
nrsense_status nrsense_apply_adjoint_weighted(nrsense_plan_t plan, const nrsense_c64* y_dev,
                                              const float* w_dev, nrsense_c64* x_dev,
                                              void* stream);
nrsense_status nrsense_translation_xcorr(const nrsense_c64* ref_dev, const nrsense_c64* imgs_dev,
                                         const int32_t* n_host, int32_t count,
                                         double* shifts_host, void* stream);
nrsense_status nrsense_phase_ramp(const float* coords_dev, nrsense_c64* y_dev, int64_t rows_total,
                                  int32_t n_coils, int32_t nseg, const int64_t* seg_off_host,
                                  const double* shifts_host, void* stream);
nrsense_status nrsense_kmeans(const double* points_host, int64_t n, int32_t k, int32_t max_iter,
                              int32_t* labels_host, double* centres_host, double* inertia_host,
                              int32_t* iters_host, int32_t* reference_host);

/*
 * nrsense_device_status - read (and with clear != 0, reset) the plan's
 * latched device status word; synchronises `stream`.  *out_host receives
 * NRSENSE_OK or the first device-side error (ERR_TIMEOUT: a bounded wait of
 * the TMA-staged k-space interpolation expired).
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
#define NRSENSE_NUM_STAGES 16
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
#define NRSENSE_STAGE_CNN           13  /* preconditioner network inside flexible CG */
#define NRSENSE_STAGE_FISTA         14  /* wavelet FISTA steps and power iteration */
#define NRSENSE_STAGE_FFT_PRUNED    15  /* own pruned coil-grid transforms, K5 and K8 fused */
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
