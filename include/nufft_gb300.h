/*
 * nufft_gb300.h - C ABI of the GB300 (sm_103a) min-max NUFFT library.
 *
 * The library implements the NUFFT operator chain of PyNUFFT
 * (J.-M. Lin, "Python Non-Uniform Fast Fourier Transform (PyNUFFT)",
 * arXiv:1710.03197): the forward operator A = V F S (Section 2.1, Eq. 1),
 * the adjoint A^H = S^H F^H V^H (Section 2.1.4, Eq. 2), the self-adjoint
 * normal operator A^H A (Section 2.1.5), and the solvers of Section 2.2
 * (conjugate gradient, L1TV-OLS Eqs. 11-20, L1TV-LAD Eqs. 21-31).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Complex data are interleaved float pairs (re, im), i.e. complex64.
 *   An "image" is N_0 x ... x N_{d-1} complex values in C (row-major) order,
 *   the order the paper uses for its interpolation matrix (Section 2.1.3).
 *   "k-space data" y is M complex values in trajectory order.
 *   The "grid" is K_0 x ... x K_{d-1} complex values in C order.
 * - The trajectory om is M x d float32, row-major, in radians; column i pairs
 *   with image axis i.  Sample m measures
 *       y_m ~= sum_n x[n] exp(-i sum_i om[m,i] (n_i - N_i/2)).
 * - Pointers named *_dev are CUDA device pointers; *_host are host pointers.
 *   The caller owns every buffer it passes; no call uses a caller buffer
 *   after its work completes (a recorded graph, below, refers to the buffers
 *   of the call that recorded it and runs again only for a call with the same
 *   buffers).  The plan owns everything it allocates.
 * - Calls on device buffers are asynchronous and ordered on the plan's
 *   stream (set at plan creation, changeable with nufft_set_stream).  Input
 *   buffers must stay valid and unmodified until the work completes.
 * - Calls on host buffers (*_host) are synchronous.
 * - Every call returns a status; on failure nufft_last_error() describes it.
 * - A plan is not thread-safe: do not call into one plan from two host
 *   threads at once.  Distinct plans are independent.
 * - Results are bit-identical from run to run for the same plan, inputs and
 *   call: the gridding V^H accumulates each chunk of points in fixed point
 *   (integer atomics under a per-chunk power-of-two scale), and every sum
 *   across threads (tile reduction, solver inner products) has a fixed order.
 * - CUDA graphs: nufft_forward, nufft_adjoint, nufft_selfadjoint, their
 *   host-buffer forms (copies included when both host buffers are
 *   page-locked; other host memory runs eagerly), the stage calls, the batch and
 *   multi-coil calls, density compensation, the gridding reconstruction, the
 *   trajectory gradient and the solvers record their launch sequence into a
 *   CUDA graph on the second
 *   call with the same buffers, parameters and stream, and replay it
 *   afterwards (one launch instead of up to a dozen per operator, and
 *   hundreds per solve).  The first call runs eagerly and does any lazy
 *   allocation.  When the stream is already being captured by the caller,
 *   the calls launch normally into the caller's capture.
 *   nufft_set_graphs(plan, 0) turns recording off.
 */
#ifndef NUFFT_GB300_H
#define NUFFT_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define NUFFT_OK        0
#define NUFFT_EINVAL    1  /* bad argument (sizes, pointers, non-finite om, ...) */
#define NUFFT_ENOMEM    2  /* a device or host allocation failed               */
#define NUFFT_ECUDA     3  /* a CUDA runtime call or kernel launch failed       */
#define NUFFT_ETIMEOUT  4  /* reserved: no call of this library waits on device */

typedef struct nufft_plan nufft_plan_t;

/*
 * nufft_plan - precompute the min-max interpolator for one trajectory.
 *
 * Section 2.1 (Eq. 1) and Section 2.1.3: the interpolation V uses the min-max
 * interpolator of Fessler and Sutton (the paper's default kernel), whose
 * scaling S is chosen together with it to keep the off-grid error small.  The
 * plan computes, in FP64 on the GPU: the per-dimension scaling factors s_i
 * (reciprocal Kaiser-Bessel transform, alpha = 2.34 J), the J x J min-max
 * matrix inverse per dimension, and per point and dimension the first
 * neighbour and the J interpolation coefficients (stored as complex64).
 * Points are then sorted by grid tile (stable radix sort by tile), each tile's
 * points are cut into chunks, and the points inside a chunk are reordered so
 * that the points sharing a warp instruction in the gridding kernel hit
 * disjoint shared-memory banks.  This replaces the paper's CSR matrix and
 * pre-indexes (Section 2.1.2, Section 2.2.3) with per-point records.
 *
 *   d       number of dimensions, 1..3
 *   Nd      image size per dimension (d ints): even, 2 <= N_i <= K_i
 *   Kd      oversampled grid per dimension (d ints): even, 16..1024, with no
 *           prime factor other than 2, 3 and 5 (e.g. 1.25x / 1.5x grids such
 *           as 80, 320, 384); powers of two take the register-resident FFT
 *           passes, the other sizes a mixed-radix pass through shared memory.
 *           The gridding tile edge is the largest divisor of K_i up to 16
 *           (2D, 3D) or 1024 (1D), or, if that is below J_i - 1, the smallest
 *           divisor of K_i from J_i - 1 up.
 *   Jd      neighbours per dimension (d ints): 1 <= J_i <= 16
 *   M       number of k-space points, 0 <= M < 2^31
 *   om_dev  M x d float32 device array (may be NULL when M == 0); every value
 *           finite with |om| <= 2^20.  Read during the call only.
 *   stream  cudaStream_t to order all work of this plan on (NULL = legacy
 *           default stream).  The plan creation itself synchronizes it.
 *   out     receives the new plan; set to NULL on failure.
 *
 * Errors: NUFFT_EINVAL (sizes out of range, om non-finite or too large),
 * NUFFT_ENOMEM, NUFFT_ECUDA.  nufft_last_error(NULL) describes a failure.
 */
int nufft_plan(int d, const int* Nd, const int* Kd, const int* Jd, int64_t M,
               const float* om_dev, void* stream, nufft_plan_t** out);

/*
 * nufft_plan_tuned - nufft_plan with the gridding tile edge chosen by
 * measurement (the paper has no counterpart: it is a property of this
 * implementation's bin-tiled V^H).  One plan is built per candidate edge
 * (1D: 256, 512, 1024; 2D: 8, 16, 32; 3D: 8, 16; each clipped to K, edges
 * whose padded tile does not fit shared memory skipped), each is timed on a
 * forward + adjoint pair of zero data on `stream` (CUDA events around five
 * replays of the recorded calls), and the fastest plan is returned; the
 * others are destroyed.  Same arguments, results (to rounding) and errors as
 * nufft_plan; nufft_plan_info [14..15] report the chosen edge.  Takes a few
 * plan builds' time and synchronizes the stream.
 */
int nufft_plan_tuned(int d, const int* Nd, const int* Kd, const int* Jd, int64_t M,
                     const float* om_dev, void* stream, nufft_plan_t** out);

/* Release every device and host buffer the plan owns.  NULL is a no-op.
 * Synchronizes the plan's stream first. */
int nufft_plan_destroy(nufft_plan_t* plan);

/* Message for the last failure on this plan (plan == NULL: last failure of a
 * plan-less call on this host thread).  Never NULL; valid until the next call. */
const char* nufft_last_error(const nufft_plan_t* plan);

/*
 * nufft_plan_set_trajectory - give the plan a new trajectory of the same M
 * points (om_dev: M x d float32 row-major radians, as for nufft_plan; the
 * caller keeps it).  Only what depends on the points is redone (Section
 * 2.1.3's interpolator: the tile sort, the chunk list, the per-point
 * coefficients, and their trajectory derivative if the plan has computed it);
 * the scaling factors, the min-max inverses, their Chebyshev expansions and
 * the work space are kept, the chunk list and partial tiles grow when the new
 * points need more, and the gridding tile edge stays (a tuned plan keeps its
 * tuned edge).  Recorded graphs are dropped (frame sets over the plan
 * re-record), a Toeplitz kernel is discarded (the solvers' normal operator
 * goes back to V^H V until nufft_toeplitz_init is called again).
 * Synchronizes the stream.  Errors: NUFFT_EINVAL for a NULL argument or a
 * non-finite / out-of-range om, with the plan unchanged; NUFFT_ECUDA /
 * NUFFT_ENOMEM leave the plan unusable (destroy it).
 */
int nufft_plan_set_trajectory(nufft_plan_t* plan, const float* om_dev);

/* Change the stream the plan's work is ordered on (cudaStream_t as void*). */
int nufft_set_stream(nufft_plan_t* plan, void* stream);

/* Turn graph recording and replay on (1, the default) or off (0, also drops
 * the recorded graphs).  See "CUDA graphs" above. */
int nufft_set_graphs(nufft_plan_t* plan, int enable);

/*
 * Plan description.  info receives 16 int64 values:
 *   [0] d, [1] M, [2..4] N_i, [5..7] K_i, [8..10] J_i,
 *   [11] number of tiles (bins), [12] number of gridding chunks,
 *   [13] device bytes owned by the plan, [14..15] tile edge for dims 0 and d-1.
 */
int nufft_plan_info(const nufft_plan_t* plan, int64_t* info);

/*
 * Copy the plan's per-point interpolator back to the host, in trajectory
 * order (Section 2.1.3; the min-max coefficients of Fessler and Sutton):
 *   kfirst_host  M x d int32: grid index of the first neighbour,
 *                (floor-based offset + 1) mod K_i; neighbours are
 *                kfirst + j mod K_i, j = 0..J_i-1.
 *   coef_host    for i = 0..d-1 in turn, M x J_i complex64 coefficients
 *                (float pairs), i.e. sum_i M*J_i*2 floats in total.
 *   s_host       for i = 0..d-1 in turn, the N_i scaling factors (float).
 *   perm_host    M int32: perm[r] = trajectory index of the r-th point in
 *                tile-sorted order (may be NULL to skip).
 * Any output pointer may be NULL to skip it.  Synchronous.
 */
int nufft_plan_get_interpolator(const nufft_plan_t* plan, int32_t* kfirst_host,
                                float* coef_host, float* s_host, int32_t* perm_host);

/* y = A x = V F S x (Section 2.1, Eq. 1).  x_dev: image, y_dev: M values.
 * x is not modified.  No allocation. */
int nufft_forward(nufft_plan_t* plan, const float* x_dev, float* y_dev);

/* x = A^H y = S^H F^H V^H y (Section 2.1.4, Eq. 2): the exact conjugate
 * transpose of nufft_forward (no 1/K normalisation).  No allocation. */
int nufft_adjoint(nufft_plan_t* plan, const float* y_dev, float* x_dev);

/* out = A^H A x (Section 2.1.5, the normal operator of Eq. 4), computed as
 * S^H F^H (V^H V) F S x with V^H V applied per grid tile.  x and out may not
 * alias.  No allocation. */
int nufft_selfadjoint(nufft_plan_t* plan, const float* x_dev, float* out_dev);

/* Host-buffer forms of nufft_forward / nufft_adjoint; they return after the
 * result is in host memory (the plan's stream is synchronized).  With
 * page-locked host buffers (cudaHostAlloc, cudaHostRegister) the FFT reads or
 * writes the image in host memory directly and only the k-space samples are
 * copied (by a copy kernel through the buffer's device address, not a
 * copy-engine transfer); any other host memory is copied through the plan's device staging
 * buffers.  The buffers must stay valid and, if page-locked, stay page-locked
 * until the call returns. */
int nufft_forward_host(nufft_plan_t* plan, const float* x_host, float* y_host);
int nufft_adjoint_host(nufft_plan_t* plan, const float* y_host, float* x_host);

/*
 * Stage calls (the pieces nufft_forward / nufft_adjoint are made of):
 *   nufft_scale_pad_fft      grid = F pad(S x)  (Sections 2.1.1-2.1.2)
 *   nufft_interp             y = V grid         (Section 2.1.3)
 *   nufft_gridding           grid = V^H y       (Section 2.1.3, "gridding")
 *   nufft_ifft_crop_rescale  x = S^H crop(F^H grid) (Section 2.1.2, Table 1
 *                            "IFFT" and "Rescaling"); grid_dev is used as
 *                            work space and left undefined.
 * grid_dev is K_0 x ... x K_{d-1} complex64.  The transforms are pruned
 * (zero lines of the padded image are never read, lines outside the crop are
 * never written back) but nufft_scale_pad_fft leaves every grid cell holding
 * F pad(S x), and nufft_gridding writes every grid cell.
 */
int nufft_scale_pad_fft(nufft_plan_t* plan, const float* x_dev, float* grid_dev);
int nufft_interp(nufft_plan_t* plan, const float* grid_dev, float* y_dev);
int nufft_gridding(nufft_plan_t* plan, const float* y_dev, float* grid_dev);
int nufft_ifft_crop_rescale(nufft_plan_t* plan, float* grid_dev, float* x_dev);

/*
 * nufft_gridding_static - grid = V^H y exactly as nufft_gridding, for callers
 * that cannot allocate device memory at call time (for example code running
 * under a memory budget that forbids cudaMalloc, or inside a framework whose
 * allocator must not be entered from this point).  The paper has no
 * counterpart: this is a library-usage variant, not a step of the method.
 *
 * The per-chunk partial tiles that nufft_gridding keeps in plan-owned memory
 * live here in one fixed device array of 16 MiB that every GPU loading this
 * library holds until the process exits.  The call allocates nothing and
 * frees nothing.  Plans whose partial tiles need more than 16 MiB
 * (nchunks * padded-tile bytes, nufft_plan_info [12]) are rejected with
 * NUFFT_EINVAL; the 2D 256^2 / 512^2 workloads fit, large 3D grids do not.
 * The call runs on the plan's device (the device current when the plan was
 * made): it makes that device current for its duration and restores the
 * caller's current device before returning.  The first call on a device looks
 * up the array's device address there (once per device, with that device
 * current): make that first call before any stream capture.  Every call
 * shares the one array, and each call overwrites the
 * part it uses before reading it, so nothing needs clearing; calls that can
 * overlap on the GPU (other streams, other plans, other threads) race on it
 * and must be serialised by the caller.
 */
int nufft_gridding_static(nufft_plan_t* plan, const float* y_dev, float* grid_dev);

/*
 * solve_cg - conjugate gradient on the normal equation A^H A x = A^H y
 * (Section 2.1.5 Eq. 4; Section 2.2.2 Eqs. 7-9 give the paper's k-space form,
 * this is the image-domain form).  Exactly maxiter iterations, no early exit;
 * inner products accumulated in FP64 with a fixed reduction order.
 *   y_dev  M k-space values; x_dev in: initial image x0, out: the result.
 * Allocates the solver work space on first use (kept by the plan).
 */
int solve_cg(nufft_plan_t* plan, const float* y_dev, float* x_dev, int maxiter);

/*
 * solve_l1tv_ols - L1 total-variation regularised least squares by variable
 * splitting (Section 2.2.3, Eqs. 11-20):
 *   K = mu A^H A + lambda sum_i grad_i^T grad_i;
 *   per inner iteration: rhs = mu A^H y^k + lambda sum_i grad_i^T (d_i - b_i),
 *   x = K^{-1} rhs (cg_iters CG steps warm-started from x),
 *   d_i = shrink(grad_i x + b_i, 1/lambda), b_i += grad_i x - d_i;
 *   per outer iteration: A^H y^{k+1} = A^H y^k + A^H y - A^H A x.
 * grad_i is the periodic forward difference along image axis i (every axis).
 *   maxiter  outer iterations (>= 0), inner: split iterations per outer (>= 1),
 *   cg_iters CG steps per K-solve (>= 1), mu > 0, lambda > 0.
 *   x_dev in: initial image, out: result.  d_i = b_i = 0 at the start.
 */
int solve_l1tv_ols(nufft_plan_t* plan, const float* y_dev, float* x_dev, int maxiter,
                   int inner, int cg_iters, double mu, double lambda);

/*
 * solve_l1tv_lad - L1 total-variation regularised least absolute deviation
 * (Section 2.2.3, Eqs. 21-31): as solve_l1tv_ols with the data term split
 * too: rhs adds mu (d_f - b_f); after the shrink steps,
 *   d_f = shrink(A^H A x - A^H y + b_f, 1/mu), b_f += A^H A x - A^H y - d_f
 * (the printed "+ b_y" of Eq. 26 is read as b_f).
 */
int solve_l1tv_lad(nufft_plan_t* plan, const float* y_dev, float* x_dev, int maxiter,
                   int inner, int cg_iters, double mu, double lambda);

/*
 * Batched operators: nb independent transforms with one plan (one trajectory),
 * e.g. the coil images of one frame.  x_dev: nb images back to back, y_dev:
 * nb x M complex64 (element b at y_dev + 2 b M floats).  Each stage runs as
 * one launch for the whole batch.  The first call with a given nb allocates
 * (and keeps) nb-sized work space: nb grids, nb sets of gridding partial
 * tiles, nb x M samples and nb images.  Results equal nb single calls.
 *   nufft_forward_batch      y_b = A x_b        (Section 2.1, Eq. 1)
 *   nufft_adjoint_batch      x_b = A^H y_b      (Section 2.1.4, Eq. 2)
 *   nufft_selfadjoint_batch  out_b = A^H A x_b  (Section 2.1.5); x and out
 *                            may not alias
 */
int nufft_forward_batch(nufft_plan_t* plan, int nb, const float* x_dev, float* y_dev);
int nufft_adjoint_batch(nufft_plan_t* plan, int nb, const float* y_dev, float* x_dev);
int nufft_selfadjoint_batch(nufft_plan_t* plan, int nb, const float* x_dev, float* out_dev);

/*
 * nufft_density_compensation - sampling density compensation by the
 * Pipe-Menon iteration (Section 2.2.1, Eq. 5): iters times
 *   w <- w / |A A^H w|
 * (A A^H w is complex for real w; its magnitude is used, keeping w real and
 * positive).  w_dev: M float32 weights, in: the starting weights (usually all
 * 1), out: the result.  A point whose |A A^H w| is 0 keeps its weight.  On
 * radial trajectories the iteration with the exact operator improves for a
 * few steps and then oscillates; a handful of iterations is the intended use.
 */
int nufft_density_compensation(nufft_plan_t* plan, float* w_dev, int iters);

/* x = A^H (y . w), the density-compensated gridding reconstruction
 * (Section 2.2.1, Eq. 6).  y_dev: M complex64, w_dev: M float32, x_dev: image. */
int nufft_gridding_recon(nufft_plan_t* plan, const float* y_dev, const float* w_dev, float* x_dev);

/*
 * solve_cg_kspace - the paper's two-step least squares (Section 2.2.2,
 * Eqs. 7-9): CG (maxiter iterations, from k = 0) on the oversampled k-space
 * normal equation V^H V k = V^H y, then x = S^{-1} F^{-1} k (normalised
 * inverse FFT, crop to N^d, divide by the scaling factors).  x_dev: output
 * image.  Allocates five grid-sized work vectors on first use.
 */
int solve_cg_kspace(nufft_plan_t* plan, const float* y_dev, float* x_dev, int maxiter);

/*
 * Multi-coil operators (Section 2.2.3, Eqs. 32-33) for nc coil maps c_i
 * (coils_dev: nc images, complex64, coil-major), with k-space data stacked
 * coil by coil (nc x M complex64):
 *   nufft_forward_multicoil      y_i = A (c_i . x)
 *   nufft_adjoint_multicoil      x = sum_i conj(c_i) . A^H y_i
 *   nufft_selfadjoint_multicoil  out = sum_i conj(c_i) . A^H A (c_i . x)
 *   solve_cg_multicoil           CG on A_multi^H A_multi x = A_multi^H y
 *                                (x_dev in: x0, out: result)
 * nc >= 1.  The nc coils run as one batch (see nufft_forward_batch); the
 * batched work space is allocated on first use with a given nc.
 */
int nufft_forward_multicoil(nufft_plan_t* plan, const float* coils_dev, int nc, const float* x_dev, float* y_dev);
int nufft_adjoint_multicoil(nufft_plan_t* plan, const float* coils_dev, int nc, const float* y_dev, float* x_dev);
int nufft_selfadjoint_multicoil(nufft_plan_t* plan, const float* coils_dev, int nc, const float* x_dev,
                                float* out_dev);
int solve_cg_multicoil(nufft_plan_t* plan, const float* coils_dev, int nc, const float* y_dev, float* x_dev,
                       int maxiter);

/*
 * Frame sets - a dynamic series (Section 2.2.3, Eqs. 32-33 per frame): frames
 * with the same image geometry N^d and their own trajectories (one plan each,
 * any number of points), sharing the coil maps.
 *
 *   nufft_frames_create   the set over plans[0..nframes-1] (distinct plans of
 *                         equal d and N^d; the set does not own them and they
 *                         must outlive it); work is ordered on `stream`.
 *   nufft_frames_selfadjoint_multicoil
 *                         out_f = sum_i conj(c_i) . A_f^H A_f (c_i . x_f) for
 *                         every frame f.  x_dev, out_dev: nframes x N^d
 *                         complex64 (frame-major, may not alias); coils_dev:
 *                         nc x N^d.  The first call with a buffer set runs
 *                         eagerly; the second records all frames as concurrent
 *                         branches of one CUDA graph, replayed afterwards as one
 *                         launch.  Frame plans may not be used on other streams
 *                         while a call is in flight.
 *   nufft_frames_set_stream / nufft_frames_destroy (synchronizes the stream).
 *
 * Errors: NUFFT_EINVAL (NULL arguments, nc < 1, mismatched or repeated plans),
 * NUFFT_ENOMEM, NUFFT_ECUDA; nufft_last_error(NULL) or the frame's plan
 * describes a failure.
 */
typedef struct nufft_frames nufft_frames_t;
int nufft_frames_create(nufft_plan_t* const* plans, int nframes, void* stream, nufft_frames_t** out);
int nufft_frames_destroy(nufft_frames_t* frames);
int nufft_frames_set_stream(nufft_frames_t* frames, void* stream);
int nufft_frames_selfadjoint_multicoil(nufft_frames_t* frames, const float* coils_dev, int nc, const float* x_dev,
                                       float* out_dev);

/*
 * Toeplitz-embedded normal operator (Section 2.1.5: the paper precomputes
 * A^H A for its iterative solvers, citing Fessler et al.'s Toeplitz method).
 * A^H A is a convolution with t[D] = sum_m exp(i om_m . D), D in (-N, N)^d;
 * embedded circularly in a grid of period P_i (2 N_i rounded up to a power of
 * two) it becomes FFT, pointwise product, inverse FFT.
 *   nufft_toeplitz_init         computes the kernel: the adjoint NUFFT of
 *                               all-ones on a P image (grid 2P, same J), then
 *                               its DFT.  Needs 2 P_i <= 1024.  Allocates the
 *                               P^d spectrum; synchronous.  The kernel carries
 *                               the NUFFT's accuracy (~1e-6 relative).
 *   nufft_selfadjoint_toeplitz  out = A^H A x through the embedding.
 *   nufft_set_normal_operator   mode 0: the solvers (solve_cg, solve_l1tv_*,
 *                               solve_cg_multicoil) apply V^H V through the
 *                               grid (default); mode 1: the Toeplitz form
 *                               (after nufft_toeplitz_init).  nufft_selfadjoint
 *                               always uses V^H V.
 */
int nufft_toeplitz_init(nufft_plan_t* plan);
int nufft_selfadjoint_toeplitz(nufft_plan_t* plan, const float* x_dev, float* out_dev);
int nufft_set_normal_operator(nufft_plan_t* plan, int mode);

/*
 * nufft_trajectory_gradient - gradient of a real loss L(y), y = A(om) x, with
 * respect to the trajectory (the forward operator of Section 2.1, Eq. 1,
 * differentiated through the min-max coefficients of Section 2.1.3; the paper
 * itself has no derivative):
 *   gom[m, a] = Re(conj(g_m) d y_m / d om[m, a]),  g = dL/dRe(y) + i dL/dIm(y),
 * with d c / d om = G^{-1} d r / d om and the neighbourhood held fixed (the
 * interpolator is discontinuous where a point crosses a grid-cell boundary).
 *   x_dev    image the forward operator was applied to
 *   g_dev    M complex64
 *   gom_dev  M x d float32, row-major, trajectory order
 * The derivative coefficients are computed (FP64, stored complex64) on the
 * first call and kept by the plan.  The image gradient is nufft_adjoint(g).
 */
int nufft_trajectory_gradient(nufft_plan_t* plan, const float* x_dev, const float* g_dev, float* gom_dev);

/*
 * nufft_trajectory_gradient_grid - the same gradient from the oversampled
 * spectrum Y = F S x instead of the image (Section 2.1, Eq. 1: the grid the
 * interpolation reads), e.g. the grid nufft_scale_pad_fft wrote for the
 * forward pass, so that a backward pass needs no second FFT.
 *   grid_dev K^d complex64 in the plan's grid layout (as nufft_scale_pad_fft writes it)
 *   g_dev, gom_dev as for nufft_trajectory_gradient
 * Bit-identical to nufft_trajectory_gradient(x) when grid_dev holds
 * nufft_scale_pad_fft(x).
 */
int nufft_trajectory_gradient_grid(nufft_plan_t* plan, const float* grid_dev, const float* g_dev, float* gom_dev);

/*
 * Fault injection for tests (no counterpart in the paper).  Every device
 * buffer the library owns is allocated through one wrapper.
 *
 * nufft_debug_fail_allocation - arm a one-shot failure: the n-th device
 *   allocation the library makes from now on (n = 0: the next one) fails as
 *   if the device were out of memory, without calling CUDA, so the call that
 *   makes it returns NUFFT_ENOMEM and no CUDA error is left behind.  n < 0
 *   disarms.  Process-wide; returns NUFFT_OK.
 * nufft_debug_device_bytes - bytes of device memory the library holds now,
 *   over all plans, frame sets and work spaces (the static scratch of
 *   nufft_gridding_static not included).  A call that fails must leave this
 *   where it was before the call, apart from work space it keeps by design.
 */
int nufft_debug_fail_allocation(int64_t n);
int64_t nufft_debug_device_bytes(void);

#ifdef __cplusplus
}
#endif

#endif /* NUFFT_GB300_H */
