/*
 * wc4d -- GB300 (sm_103a) inner loop of forcing-formulation weak-constraint
 * 4D-Var with randomised spectral limited-memory preconditioning.
 *
 * Method: Dauzickaite, Lawless, Scott, van Leeuwen, "Randomised
 * preconditioning for the forcing formulation of weak constraint 4D-Var".
 *
 * The library solves A x = b for the first-level preconditioned Hessian
 *     A = I + D^{1/2} L^{-T} H^T R^{-1} H L^{-1} D^{1/2}          (eq. 10)
 * with D = diag(B, Q_1..Q_N), L^{-1} the block lower-triangular product of
 * the linearised model over the N subwindows (eq. 5), H the observation
 * operator and R = sigma_o^2 I.  It applies A to blocks of probe vectors,
 * builds Ritz pairs with REVD (Alg. 3, plus power iterations), randomised
 * Nystrom (Alg. 4) or REVD_ritzit (Alg. 5), forms the spectral LMP factor
 * C = I - sum_i (1 - theta_i^{-1/2}) u_i u_i^T (eq. 15-16) and runs split-
 * preconditioned CG (Alg. 1).
 *
 * Conventions (every entry point):
 *  - A control-space block of K vectors (dimension nA = n (N+1)) is a
 *    column-major nA x K matrix with leading dimension ld >= nA; row t*n + s
 *    holds grid point s of time block t (t = 0: x_0, t >= 1: eta_t).
 *  - "device" pointers are CUDA global-memory pointers of the current
 *    device; "host" pointers are ordinary memory.  The caller owns every
 *    pointer it passes; the library owns its workspaces (allocated on
 *    demand, freed by wc4d_destroy).
 *  - All work is queued on the context's stream.  Calls that return
 *    scalars to host memory (theta, iters, relres, histories) synchronise
 *    that stream before returning.
 *  - Errors are returned as wc4d_status; wc4d_last_error() gives a message.
 *    Nothing traps: device-side failures (non-SPD Gram, CG breakdown,
 *    non-finite values) come back as statuses.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef WC4D_H
#define WC4D_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wc4d_ctx wc4d_ctx;

typedef enum {
    WC4D_OK = 0,
    WC4D_EINVAL = -1,      /* bad argument or unsupported size                  */
    WC4D_ENOMEM = -2,      /* device allocation failed                          */
    WC4D_ECUDA = -3,       /* a CUDA runtime call failed                        */
    WC4D_ENOTSPD = -4,     /* Cholesky of a Gram matrix broke down              */
    WC4D_EBREAKDOWN = -5,  /* CG: p^T A p <= 0 or not finite                    */
    WC4D_ENOCONV = -6,     /* CG: maxit reached before the tolerance            */
    WC4D_ETIMEOUT = -7,    /* an iteration limit inside the library was hit     */
    WC4D_ENAN = -8,        /* a non-finite value was produced                   */
    WC4D_ESTATE = -9       /* a required set-up call has not been made          */
} wc4d_status;

typedef enum { WC4D_FP64 = 0, WC4D_MIXED = 1 } wc4d_precision;
typedef enum { WC4D_REVD = 0, WC4D_NYSTROM = 1, WC4D_RITZIT = 2, WC4D_NYSTROM1 = 3 } wc4d_method;
typedef enum { WC4D_MODEL_DENSE = 0, WC4D_MODEL_L96 = 1 } wc4d_model;
typedef enum { WC4D_CORR_SOAR = 0, WC4D_CORR_GAUSS = 1, WC4D_CORR_DIAG = 2 } wc4d_corr;

/* Problem statement (Section 2; Section 5 for the two model families).
 *  n, N        grid points per time block and number of subwindows; nA = n (N+1).
 *  model       WC4D_MODEL_DENSE: a linear model given as one dense n x n
 *              propagator M_t per subwindow (or one shared by all);
 *              WC4D_MODEL_L96: Lorenz-96 (eq. 22 of the paper) integrated by RK4,
 *              with tangent-linear and adjoint sweeps along the stored
 *              nonlinear trajectory.
 *  steps, dt   RK4 steps per subwindow and step size (Lorenz-96 only).
 *  F           Lorenz-96 forcing.
 *  sigma_o2    R_t = sigma_o2 * I.
 *  obs_stride  H_t observes the points s = 0, obs_stride, 2 obs_stride, ...
 *  obs_t0, obs_tstride  observed times t = obs_t0, obs_t0 + obs_tstride, ... <= N.
 *  M_shared    dense model: 1 = one propagator used for every subwindow. */
typedef struct {
    int32_t n, N;
    int32_t model;
    int32_t steps;
    double dt;
    double F;
    double sigma_o2;
    int32_t obs_stride, obs_t0, obs_tstride;
    int32_t M_shared;
} wc4d_problem;

/* Create a context bound to the current CUDA device and the given stream
 * (a cudaStream_t; NULL = the legacy default stream).  Fails with
 * WC4D_EINVAL for n < 2, N < 1, n > 8192 or a non-positive sigma_o2. */
wc4d_status wc4d_create(wc4d_ctx **ctx, const wc4d_problem *prob, void *cuda_stream);
void        wc4d_destroy(wc4d_ctx *ctx);
const char *wc4d_last_error(const wc4d_ctx *ctx);
wc4d_status wc4d_set_stream(wc4d_ctx *ctx, void *cuda_stream);

/* ---- problem set-up (not part of the timed inner loop) ---------------- */

/* Linearised model M_t (eq. 5): copy a dense row-major n x n propagator from
 * device memory into the context.  t in [0, N) sets subwindow t; t = -1 sets
 * every subwindow (or the shared one when M_shared).  The library keeps
 * FP64, FP32 and BF16 copies and their transposes (for L^{-T}). */
wc4d_status wc4d_set_propagator(wc4d_ctx *ctx, int32_t t, const double *M_device);

/* Build the propagator of `steps` Crank-Nicolson steps of periodic
 * advection-diffusion u_t + c u_z = kappa u_zz on [0,1) with n points and
 * centred differences, on the device, from the closed-form Fourier symbol
 * of one step ((1 + dt/2 k_m)/(1 - dt/2 k_m), k_m the symbol of the centred
 * operator), and store it for every subwindow. */
wc4d_status wc4d_build_advdiff_propagator(wc4d_ctx *ctx, double kappa, double c, double dt, int32_t steps);

/* Covariance blocks of D (Section 5): block 0 = B, block 1 = Q_t (all
 * subwindows).  Circulant on the periodic grid with first row
 * variance * rho(r), r the periodic distance in grid points:
 * SOAR (1 + r/L) e^{-r/L}, Gaussian e^{-r^2/(2 L^2)}, or DIAG (variance * I).
 * The symmetric square root D^{1/2} is formed on the device from the
 * eigenvalues of the circulant, computed in closed form so that the smallest
 * keep their relative accuracy (SOAR: finite geometric sums; Gaussian: the
 * Poisson summation formula less the images the periodic row omits):
 * sqrt(lambda) for lambda >= 0, and zero for the negative eigenvalues that a
 * periodically wrapped correlation function can have.  EINVAL for a block
 * outside {0, 1}, an unknown corr, a negative variance or L <= 0. */
wc4d_status wc4d_set_covariance(wc4d_ctx *ctx, int32_t block, int32_t corr, double variance, double length);
/* Same, from an explicit first row (host, n values, symmetric): eigenvalues
 * by an FP64 DFT of the row (errors ~1e-16 of the largest eigenvalue, which
 * the square root amplifies where the spectrum is tiny), negative ones
 * clamped to zero. */
wc4d_status wc4d_set_covariance_row(wc4d_ctx *ctx, int32_t block, const double *row_host);

/* A covariance block of D given by its square root (Section 2.2, eq. 10
 * needs only D^{1/2}): block 0 = B, 1 = Q_t (all subwindows).
 *   kind 0: circulant, data = first row of the symmetric square root (host,
 *           n values; applied by FFT for power-of-two n, directly otherwise);
 *   kind 1: dense, data = the n x n square root (device, row-major; applied
 *           by one n x n by n x K product per time block; FP32 copy for the
 *           mixed path);
 *   kind 2: scalar, data = sigma (host, one value >= 0): the block is
 *           sigma^2 I, applied by scaling.
 * EINVAL for an unknown kind, a negative or non-finite sigma. */
wc4d_status wc4d_set_cov_sqrt(wc4d_ctx *ctx, int32_t block, int32_t kind, const double *data);

/* Outer-loop quantities (Section 2.1): run the model from the background
 * xb (host, n values) over the window (the nonlinear RK4 model for
 * Lorenz-96, which also stores the linearisation trajectory in FP64 and
 * FP32; the linear propagators otherwise), form the innovations
 * d_t = y_t - H_t x_t (y: host, nobs values, time-major over the observed
 * times) and the right-hand side of eq. 10, rhs = D^{1/2} L^{-T} H^T R^{-1} d
 * (+ D^{-1/2} b when Dm12b_host is not NULL). */
wc4d_status wc4d_set_background_obs(wc4d_ctx *ctx, const double *xb_host, const double *y_host,
                                    const double *Dm12b_host);
/* Next outer loop (Section 2.1, eq. 3): x_device (nA values, FP64) is the
 * inner-loop solution of eq. 10, i.e. the preconditioned increment
 * D^{-1/2} dp.  The linearisation point p = (x_0, eta_1..eta_N) becomes
 * p + D^{1/2} x, D^{-1/2} b becomes D^{-1/2} b - x (b = p^b - p), and the
 * model is re-run from the new point with the forcing eta added at the end
 * of every subwindow (eq. 1); innovations and rhs are recomputed from the
 * observations given to wc4d_set_background_obs.  WC4D_ESTATE before
 * wc4d_set_background_obs. */
wc4d_status wc4d_outer_update(wc4d_ctx *ctx, const double *x_device);
/* The linearisation trajectory of a Lorenz-96 context given by the caller
 * (its own nonlinear run, eq. 1), in place of the library's run from the
 * background: X (device) holds the N steps + 1 states x_0 .. x_{N steps},
 * n values each; the RK4 stage states of every step are recomputed from
 * them for the tangent-linear and adjoint sweeps.  EINVAL for a dense model.
 * wc4d_set_innovation then supplies the innovations d (device, nobs values,
 * time-major over the observed times) and optionally D^{-1/2} b (device,
 * nA values, or NULL), and forms the right-hand side of eq. 10,
 * D^{1/2} L^{-T} H^T R^{-1} d (+ D^{-1/2} b), with the current operator. */
wc4d_status wc4d_set_trajectory(wc4d_ctx *ctx, const double *X_device);
wc4d_status wc4d_set_innovation(wc4d_ctx *ctx, const double *d_device, const double *Dm12b_device);
/* Number of observations q of the problem. */
int64_t     wc4d_nobs(const wc4d_ctx *ctx);
/* Dimension n_A = n (N + 1) of the control vector (eq. 10's A is n_A x n_A):
   the length of every control-space vector and the least leading dimension
   of every block passed to the library; -1 for a null context. */
int64_t     wc4d_control_dim(const wc4d_ctx *ctx);
/* The problem statement the context was created with (host copy). */
wc4d_status wc4d_get_problem(const wc4d_ctx *ctx, wc4d_problem *out);
/* Number of Ritz pairs currently installed (what wc4d_get_ritz copies:
   n_A x count values and count Ritz values); -1 for a null context. */
int32_t     wc4d_ritz_count(const wc4d_ctx *ctx);
/* Copy the right-hand side (nA values) to device memory. */
wc4d_status wc4d_get_rhs(wc4d_ctx *ctx, double *rhs_device);

/* ---- the hot path ------------------------------------------------------ */

/* Y = A X for a block of K vectors (eq. 10): D^{1/2} by FFT (n a power of
 * two) or direct circulant products, the forward sweep L^{-1}, H^T R^{-1} H,
 * the adjoint sweep L^{-T}, then X + D^{1/2}(.).  X and Y are device,
 * column-major, leading dimension ld; they must not overlap.
 * WC4D_FP64: double in/out.  WC4D_MIXED: float in/out, FP32 operators and
 * FP32 accumulation (tensor cores for K >= 16 on dense models). */
wc4d_status wc4d_hvp(wc4d_ctx *ctx, const void *X, void *Y, int32_t K, int64_t ld, int32_t precision);

/* Gaussian probe block (Alg. 3-5, step 1): G (device, rows x cols,
 * column-major, ld) from Philox4x32-10 keyed by seed (Salmon et al. 2011),
 * element e = col*rows + row taking Box-Muller output (e & 1) of counter
 * e >> 1, with uniforms (hi27:lo26 of two words + 1) / 2^53. */
wc4d_status wc4d_gaussian(wc4d_ctx *ctx, uint64_t seed, int64_t rows, int32_t cols, int64_t ld, double *G);
/* The same probes computed in FP32 arithmetic (the mixed sketch's own
   probes): the same Philox counters and 53-bit uniforms, each rounded once
   to FP32, Box-Muller in FP32; equal to the FP64 probes to FP32 rounding
   of log, sqrt, sin and cos (an absolute ~1e-4 where u1 is within a few
   FP32 ulp of 1).  G: device FP32, column-major rows x cols, ld >= rows. */
wc4d_status wc4d_gaussian_f32(wc4d_ctx *ctx, uint64_t seed, int64_t rows, int32_t cols, int64_t ld, float *G);

/* Randomised Ritz pairs of A (Section 4) kept in the context for the LMP:
 * method REVD (Alg. 3 with q_power extra products and orthonormalisations),
 * NYSTROM (Alg. 4), RITZIT (Alg. 5) or NYSTROM1 (single-pass Nystrom, the
 * one-product method Section 6 names as future work, after Tropp, Yurtsever,
 * Udell and Cevher 2017: Omega = orth(G), Y = A Omega, shift nu = s ||Y||_F
 * with s = sqrt(nA) 2^-52 (FP64) or 2^-22 (mixed), Omega^T (Y + nu Omega) =
 * C^T C, (Y + nu Omega) C^{-1} = U Sigma V^T, theta = max(Sigma^2 - nu, 0)),
 * target rank k, oversampling l.
 * G_device: explicit probes (nA x (k+l), ld = nA, FP64) or NULL to draw
 * them with wc4d_gaussian(seed).  theta_host: k Ritz values, decreasing.
 * Orthonormalisation is CholeskyQR2 with an FP64-accurate Gram (double-float
 * for FP32 blocks; shifted CholeskyQR3 when the Gram is singular to working
 * precision); the small eigenproblems are solved by one-sided Jacobi, in FP64
 * for the result, after FP32 pre-rotation sweeps for the SPD ones (REVD's K_1,
 * Nystrom's F^T F). */
wc4d_status wc4d_sketch(wc4d_ctx *ctx, int32_t method, int32_t k, int32_t l, int32_t q_power,
                        uint64_t seed, const double *G_device, double *theta_host, int32_t precision);
/* Copy the current Ritz vectors (nA x k, column-major, FP64) and values. */
wc4d_status wc4d_get_ritz(wc4d_ctx *ctx, double *U_device, double *theta_host);
/* Install explicit pairs (orthonormal U, device nA x k; theta host). */
wc4d_status wc4d_set_ritz(wc4d_ctx *ctx, int32_t k, const double *U_device, const double *theta_host);

/* y = C v (transpose = 0) or C^T v for the spectral-LMP factor of the
 * current Ritz pairs (eq. 16 in its closed form for orthonormal U; C is
 * symmetric then).  v, y: device, nA doubles. */
wc4d_status wc4d_lmp_apply(wc4d_ctx *ctx, const double *v, double *y, int32_t transpose);

/* Split-preconditioned CG (Alg. 1) on A x = rhs from x_0 = 0.  use_lmp: 1 =
 * precondition with the current Ritz pairs.  Stops when |rhs - A x| / |rhs|
 * <= tol (the unpreconditioned residual carried by recurrence) or after
 * maxit iterations (WC4D_ENOCONV); force_iters > 0 runs exactly that many.
 * WC4D_MIXED: FP32 vectors and operators with FP64 scalars, wrapped in FP64
 * true-residual refinement until the FP64 residual meets tol.
 * x_device: nA doubles (output).  iters/relres may be NULL; relres is the
 * final true relative residual, computed in FP64.  qcf_drop_host (maxit
 * doubles or NULL): alpha_j rho_{j-1} / 2 per iteration, the decrease of
 * the quadratic cost (eq. 4). */
wc4d_status wc4d_pcg(wc4d_ctx *ctx, double *x_device, double tol, int32_t maxit, int32_t use_lmp,
                     int32_t force_iters, int32_t precision, int32_t *iters, double *relres,
                     double *qcf_drop_host);

/* The inner loop of Section 4: Ritz pairs by `method`, spectral LMP, PCG
 * on the exact A to tol.  Equivalent to wc4d_sketch + wc4d_pcg(use_lmp=1). */
wc4d_status wc4d_inner_loop(wc4d_ctx *ctx, int32_t method, int32_t k, int32_t l, int32_t q_power,
                            uint64_t seed, double tol, int32_t maxit, int32_t precision,
                            double *x_device, int32_t *iters, double *relres);

/* A non-blocking CUDA stream owned by the caller (wc4d_stream_destroy frees
   it after the contexts using it are destroyed): one per batched instance.
   ECUDA when the runtime refuses. */
wc4d_status wc4d_stream_create(void **stream);
wc4d_status wc4d_stream_destroy(void *stream);
/* Batched inner loops of `count` independent problems (windows of different
 * sizes; the paper solves one window at a time, this is a throughput
 * wrapper): instance i runs wc4d_inner_loop(ctxs[i], method, k[i], l[i],
 * q_power, seeds[i], tol, maxit, precision, x[i], iters + i, relres + i) on
 * its context's stream, driven by one of `workers` host threads (<= 0: 16),
 * so that the instances' kernels overlap on the GPU.  Every context must have
 * its own stream (WC4D_EINVAL otherwise); while in the batch a context uses
 * the per-launch forms of its grid-synchronised kernels and one CG graph
 * launch per iteration (not the device-side loop).  status[i] receives
 * each instance's status; the call returns the first non-OK one. */
wc4d_status wc4d_batch_inner_loop(wc4d_ctx *const *ctxs, int32_t count, int32_t method, const int32_t *k,
                                  const int32_t *l, int32_t q_power, const uint64_t *seeds, double tol,
                                  int32_t maxit, int32_t precision, double *const *x_device, int32_t *iters,
                                  double *relres, int32_t *status, int32_t workers);

/* Learned sketch proposal (the paper has none: an aid to the randomised
 * range finder, whose Alg. 3 input it becomes together with Gaussian
 * columns).  A fixed 4-layer 1D convolutional encoder over the periodic
 * Lorenz-96 grid maps the current linearisation trajectory (states at the
 * subwindow boundaries, divided by F) and the observation mask of every time
 * to m columns S (device, nA x m, column-major, ld >= nA, FP64 output):
 *   layer 0: 2(N+1) -> 64 channels, width 5, ReLU; layers 1, 2: 64 -> 64,
 *   width 5, ReLU; layer 3: 64 -> m(N+1), width 1; output channel
 *   j(N+1) + t is time block t of column j.
 * w_bf16 (device): BF16 weights W0|W1|W2|W3, each [out][in][width]; bias
 * (device): FP32 b0|b1|b2|b3.  Sums in FP32.  Lorenz-96 contexts after
 * wc4d_set_background_obs only (WC4D_EINVAL / WC4D_ESTATE otherwise). */
wc4d_status wc4d_learned_probes(wc4d_ctx *ctx, const uint16_t *w_bf16_device, const float *bias_device, int32_t m,
                                double *S_device, int64_t ld);

/* ---- small building blocks, exported for verification ------------------ */

/* CholeskyQR2 in place (the orthonormalisation of Alg. 3-5): Y (device,
 * rows x m, ld; double for WC4D_FP64, float for WC4D_MIXED) becomes Z with
 * orthonormal columns and span(Z) = span(Y); R_host (m x m column-major,
 * may be NULL) receives the upper-triangular factor with Y = Z R, positive
 * diagonal.  Both precisions form the Gram matrix Y^T Y to about 48
 * significant bits or more (FP64 accumulation; for float data, exact
 * products with double-float sums) and factor it in FP64.
 * WC4D_ENOTSPD when the Gram matrix is not numerically positive definite. */
wc4d_status wc4d_orthonormalize(wc4d_ctx *ctx, void *Y, int64_t rows, int32_t m, int64_t ld, double *R_host,
                                int32_t precision);
/* Eigen-decomposition of a symmetric positive semi-definite m x m matrix
 * (device, column-major) by one-sided Jacobi: w_host decreasing, V_device
 * (m x m column-major) the eigenvectors. */
wc4d_status wc4d_symeig(wc4d_ctx *ctx, int32_t m, const double *S_device, double *w_host, double *V_device);
/* Pieces of the Hessian product (eq. 5, eq. 10), for verification and for
 * callers that compose their own operators.  Blocks as for wc4d_hvp.
 *   wc4d_apply_dsqrt: Y = D^{1/2} X.
 *   wc4d_apply_linv : W <- L^{-1} W in place (w_{t+1} += M_t w_t).
 *   wc4d_apply_linvT: W <- L^{-T} W in place (w_t += M_t^T w_{t+1}). */
wc4d_status wc4d_apply_dsqrt(wc4d_ctx *ctx, const void *X, void *Y, int32_t K, int64_t ld, int32_t precision);
wc4d_status wc4d_apply_linv(wc4d_ctx *ctx, void *W, int32_t K, int64_t ld, int32_t precision);
wc4d_status wc4d_apply_linvT(wc4d_ctx *ctx, void *W, int32_t K, int64_t ld, int32_t precision);
/* Pieces of the orthonormalisation (CholeskyQR) and Rayleigh-Ritz steps of
 * Alg. 3-5, for callers that distribute the rows of a block over several
 * devices and sum the partial Gram matrices themselves (the column-sharded
 * sketch; the paper notes that the products with A and the block work can be
 * parallelised).  All pointers are device memory of the context's device;
 * blocks are column-major.
 *   wc4d_gram: C = A^T B (ma x mb, ld ma, FP64) for A (rows x ma, lda) and B
 *     (rows x mb, ldb): FP64 data with FP64 sums (WC4D_FP64), or FP32 data
 *     with exact products and double-float sums (WC4D_MIXED; entries of
 *     magnitude up to ~2^60, so that products and partial sums stay finite
 *     in FP32's exponent range).
 *   wc4d_chol_inverse: G = R^T R (m x m SPD, FP64) and Rinv = R^{-1} (upper
 *     triangular, m x m, ld m); ENOTSPD when G is not numerically positive
 *     definite.
 *   wc4d_tall_times_small: Z = Y W for Y (rows x m, ldy; FP64, or FP32 with
 *     WC4D_MIXED) and W (m x k FP64, ld m); Z (rows x k, ldz) in Y's
 *     precision (FP32 data: W rounded to FP32, the FP32 pipe); Z must not
 *     overlap Y; rows < 2^31. */
wc4d_status wc4d_gram(wc4d_ctx *ctx, const void *A, int64_t lda, const void *B, int64_t ldb, int64_t rows, int32_t ma,
                      int32_t mb, double *C, int32_t precision);
/* C = A^T B (m x m, FP64, column-major) for products known to be symmetric
   -- a Gram matrix (B = A) or Z^T (A Z) -- from the upper 64 x 64 tiles,
   mirrored (paper Alg. 3 step 4; CholeskyQR Grams of Alg. 3-5).  A and B
   column-major (rows x m, leading dimensions lda, ldb >= rows), FP64 or --
   precision WC4D_MIXED -- FP32, on the device.  FP32 blocks take the path
   wc4d_set_gram_path selects.  Synchronises the context's stream.  EINVAL
   for bad arguments, ETIMEOUT if a bounded device wait ran out. */
wc4d_status wc4d_gram_sym(wc4d_ctx *ctx, const void *A, int64_t lda, const void *B, int64_t ldb, int64_t rows,
                          int32_t m, double *C, int32_t precision);
wc4d_status wc4d_chol_inverse(wc4d_ctx *ctx, int32_t m, const double *G, double *Rinv);
wc4d_status wc4d_tall_times_small(wc4d_ctx *ctx, const void *Y, int64_t ldy, int64_t rows, int32_t m, const double *W,
                                  int32_t k, void *Z, int64_t ldz, int32_t precision);
/* Copy the FP64 propagator of subwindow t (dense model) to device memory. */
wc4d_status wc4d_get_propagator(wc4d_ctx *ctx, int32_t t, double *M_device);
/* Kernel launches issued by the library in this process (all contexts). */
int64_t     wc4d_launch_count(int32_t reset);
/* Optional CUDA-event timing of kernel classes on the context's stream:
 * wc4d_profile(ctx, 1) clears the log and starts recording an event pair
 * around every launch group of the classes below; wc4d_profile_read
 * synchronises and returns the summed device time (ms) and the number of
 * timed groups of one class.  Classes: 0 FP32 one-column sweep (all N
 * subwindow GEMVs of L^{-1} or L^{-T} in one group), 1 sweep SIMT GEMM,
 * 2 sweep tensor-core GEMM (one subwindow), 3 D^{1/2} circulant, 4 LMP
 * application, 5 Gram products, 6 tall-skinny products Y R^{-1} and Z W,
 * 7 Lorenz-96 tangent-linear sweep, 8 Lorenz-96 adjoint sweep, 9 PCG vector
 * kernels, 10 FP64 one-column sweep, 11 Jacobi EVD/SVD, 12 Cholesky and
 * triangular inverse. */
wc4d_status wc4d_profile(wc4d_ctx *ctx, int32_t enable);
wc4d_status wc4d_profile_read(wc4d_ctx *ctx, int32_t cls, double *total_ms, int64_t *launch_groups);
/* Allocation-free spectral-LMP application, y = C v (the paper has no
 * counterpart: it is an integration aid).  For callers that cannot allocate
 * device memory where they apply the preconditioner: systems that reserve
 * their whole device memory budget up front and forbid later allocations,
 * code that must not take the device-wide synchronisation an allocation or
 * free can cause in the middle of a solve, and callers without a library
 * context.  U (device, nA x k column-major, orthonormal columns), theta
 * (device, k values), v and y (device, nA doubles, distinct); queued on
 * cuda_stream.  Creates no context and allocates nothing: its scratch
 * (weighted coefficients and partial dot products) is one fixed
 * 1 MiB + 8 KiB device array in the library, held by every GPU that loads it
 * until exit.  k > 1024 returns WC4D_EINVAL.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) and caches it,
 * so make that first call before any stream capture; resetting the device
 * (cudaDeviceReset) after it is not supported.  All calls share the array,
 * which keeps the last call's contents: calls that overlap on the GPU
 * (other streams, other host threads) race and must be serialised by the
 * caller. */
wc4d_status wc4d_lmp_apply_static(const double *U, const double *theta, int32_t k, int64_t nA, const double *v,
                                  double *y, void *cuda_stream);
/* Ritz pairs from CG (Section 3.3, eq. 18-20), the deterministic LMP built
 * from the previous inner loop.  wc4d_lanczos_cg runs FP64 CG without a
 * preconditioner (Alg. 1 with C = I) on the context's A x = rhs from x = 0
 * until the relative residual reaches tol or maxit iterations, keeping
 * alpha_j, beta_j and the Lanczos vectors f_j = (-1)^j r_j / |r_j| (nA x
 * (maxit + 1) FP64 in the context); reorth != 0 reorthogonalises every new
 * residual against all previous f (classical Gram-Schmidt twice).  iters,
 * relres: iterations J and the recursive relative residual.
 * wc4d_lanczos_tridiag: gamma_1..gamma_J, tau_1..tau_{J-1} of T_J.
 * wc4d_lanczos_ritz: the k largest eigenpairs of T_J, u_i = F_J w_i,
 * installed as the context's Ritz pairs (as wc4d_set_ritz); theta_host may
 * be NULL.  ESTATE without Lanczos data; EINVAL for k > J. */
wc4d_status wc4d_lanczos_cg(wc4d_ctx *ctx, double *x_device, double tol, int32_t maxit, int32_t reorth,
                            int32_t *iters, double *relres);
wc4d_status wc4d_lanczos_tridiag(wc4d_ctx *ctx, double *gamma_host, double *tau_host);
wc4d_status wc4d_lanczos_ritz(wc4d_ctx *ctx, int32_t k, double *theta_host);
/* Products with A issued so far (block products count once). */
int64_t     wc4d_hvp_count(wc4d_ctx *ctx, int32_t reset);
/* One-sided Jacobi sweeps used by the last small eigensolve or SVD of the
   context (Alg. 2 EVD of K, Alg. 4 SVD of F, Alg. 5 SVD of R_3, or
   wc4d_symeig), counting a final sweep without rotations when the solve ran
   to convergence; -1 for a null context.  In a mixed-precision sketch the
   solve stops after a sweep whose largest rotation had |cos| <= 1e-5. */
int32_t     wc4d_jacobi_sweeps(const wc4d_ctx *ctx);
/* FP32 pre-rotation sweeps that preceded the last FP64 eigensolve of an SPD
   matrix (0 when none ran; negative when it stopped at its sweep limit). */
int32_t     wc4d_jacobi_sweeps_fp32(const wc4d_ctx *ctx);
/* Which kernel ran those FP32 sweeps: 1 = one 16-CTA thread-block cluster
   (distributed shared memory), 2 = the cooperative whole-grid form (used when
   the device cannot co-schedule such a cluster), 0 = none; -1 for a null
   context. */
int32_t     wc4d_jacobi_fp32_kernel(const wc4d_ctx *ctx);
/* CUDA graphs for the CG iterations (Alg. 1's loop body: the product with A,
   the LMP step and the direction update), built once per solve after one
   eager iteration; the results are bitwise those of eager launches.
   enable = 1 (default): one graph whose conditional WHILE node runs the
   iterations on the device, the host waking only when CG stops, the limit is
   reached or a reliable update is due (falls back to the next form if the
   driver refuses it); 2: one graph launch per iteration, the host reading
   the stopping flags after each; 0: every iteration eager.  The graphs are
   captured on a private stream of the context and launched on its stream.
   EINVAL for a null context or enable outside 0..2. */
wc4d_status wc4d_set_graphs(wc4d_ctx *ctx, int32_t enable);
/* How the last wc4d_pcg / wc4d_inner_loop solve ran the CG iterations after
   the first: 0 = eager launches (graphs off, profiling on, or both graph
   forms refused), 1 = one graph launch per iteration, the host reading the
   stopping flags after each, 2 = a graph with a conditional WHILE node that
   runs iterations on the device until CG stops, the iteration limit is
   reached or (mixed path) a reliable update is due.  If the WHILE-node graph
   could not be built, note (when not NULL; note_len bytes, NUL-terminated,
   truncated) receives the failing CUDA call and its error, else "".
   -1 for a null context. */
int32_t     wc4d_iteration_mode(const wc4d_ctx *ctx, char *note, int32_t note_len);
/* Dense FP32 contractions of the mixed path's sketch.  (1) Gram-type
   products -- the CholeskyQR Gram Y^T Y (Alg. 3-5, orthonormalisation), the
   Rayleigh-Ritz matrix Z^T (A Z) (Alg. 3 step 4, Alg. 4 step 4) and the
   Nystrom products -- computed to FP64-class accuracy.  (2) The tall
   product Y R^{-1} of CholeskyQR in 3xTF32: Y and R^{-1} each split into a
   TF32 value and a TF32 remainder, three products summed in FP32 tensor
   memory (about 2^-21 relative; the second CholeskyQR pass restores the
   orthogonality), when m is a multiple of 32 up to 256 and there are at
   least 128 rows.  tensor_cores = 1 (default), Gram products: when the
   block has a multiple of 128 columns and at least 512 rows, each FP32
   column is split (scaled by a power of two) into six 7-bit integer slices
   held exactly in BF16, the 21 slice products that matter are summed
   exactly by tcgen05 BF16 MMAs in FP32 tensor memory over 512-row chunks,
   and the chunks are combined in double-float and FP64 (relative accuracy
   about 2^-41 of the largest entries); 0: the FP32-pipe double-float
   product (about 2^-44) and the FP32-pipe tall product for every shape.
   EINVAL for a null context. */
wc4d_status wc4d_set_gram_path(wc4d_ctx *ctx, int32_t tensor_cores);
/* Polls of a bounded device-side wait before it gives up, for the grid
   barriers of the persistent one-column sweeps (the FP64 sweep, and the FP32
   sweep when n is not a multiple of 2048) and for the waits of the FP32
   Lorenz-96 sweeps on their staged stage-state copies.  A kernel whose wait
   gives up records the failure and returns (a Lorenz-96 sweep first waits,
   bounded, for its copies still in flight), and the call that ran it
   (wc4d_hvp, wc4d_pcg, wc4d_inner_loop, wc4d_sketch) returns WC4D_ETIMEOUT
   with the context still usable.  polls < 0 restores the default (2^22,
   seconds); 0 makes a grid barrier that is not already complete at its first
   poll, and every staged-copy wait, fail at once, which exercises the timeout
   path.  EINVAL for a null context or polls >= 2^32. */
wc4d_status wc4d_set_wait_limit(wc4d_ctx *ctx, int64_t polls);
/* Synchronise the context's stream and report a device-side failure of the
   work queued on it that no call has reported yet: WC4D_ETIMEOUT when a
   bounded wait of a product queued by wc4d_hvp (a persistent sweep's grid
   barrier, a staged-copy wait of an FP32 Lorenz-96 sweep, a tensor-core
   kernel's wait) gave up; WC4D_ECUDA for a CUDA error; else WC4D_OK.  The
   solves and sketches report these failures themselves.  EINVAL for a null
   context. */
wc4d_status wc4d_sync(wc4d_ctx *ctx);
/* Mixed-precision CG (reliable updates): the FP32 recurrence residual must
   fall by the factor delta (0 < delta <= 1, default 1e-3) since the last
   update, or claim convergence, before the FP64 true residual replaces it.
   EINVAL outside (0, 1]. */
wc4d_status wc4d_set_reliable_delta(wc4d_ctx *ctx, double delta);
/* Autotuned tile shapes of the SIMT propagator GEMMs (process-wide, default
   on): the first product of a shape times every candidate tile (scratch
   output) and keeps the fastest.  wc4d_autotune_choice returns the tile index
   chosen for (kind, rows, cols, kdim), or -1 if that shape was not tuned;
   kind bit 0: FP64, bit 1: the tall-skinny products (A row-contiguous)
   rather than the propagator sweeps. */
void        wc4d_set_autotune(int32_t enable);
int32_t     wc4d_autotune_choice(int32_t fp64, int32_t rows, int32_t cols, int32_t kdim);

#ifdef __cplusplus
}
#endif
#endif
