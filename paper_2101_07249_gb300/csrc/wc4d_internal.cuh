// Internal declarations of libwc4d (GB300 / sm_103a).  Not part of the ABI.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "wc4d.h"

#define WC4D_FFT_MAX_N 8192   // largest power-of-two n handled by the on-chip FFT

// ------------------------------------------------------------------ buffers
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Epilogue of the sweep products.  mode 0: C = alpha*acc + beta*C_old
// (C_old not read when beta == 0).  mode 1 (adjoint with observations):
// C = acc + obs(C_old), obs(v)[s] = obs_scale * v[s] on observed points
// s % obs_stride == 0, zero elsewhere.
struct Epi {
    int mode;
    double alpha, beta;
    double obs_scale;
    int obs_stride;
};

// Kernel classes timed with CUDA events when profiling is enabled.
enum ProfId {
    PROF_GEMV = 0,   // FP32 one-column sweeps (dense propagators)
    PROF_GEMM,       // sweep SIMT GEMM (probe blocks)
    PROF_TC,         // sweep tensor-core GEMM
    PROF_CIRC,       // D^{1/2} circulant (FFT or direct)
    PROF_LMP,        // spectral-LMP application
    PROF_GRAM,       // A^T B Gram products
    PROF_LA,         // tall-skinny products Y R^{-1}, Z W (and Nystrom F)
    PROF_L96_TLM,    // Lorenz-96 tangent-linear sweep
    PROF_L96_ADJ,    // Lorenz-96 adjoint sweep
    PROF_VEC,        // PCG vector kernels
    PROF_GEMV64,     // FP64 one-column sweeps (true residuals, set-up)
    PROF_JACOBI,     // one-sided Jacobi EVD / SVD of the small matrices
    PROF_CHOL,       // Cholesky and triangular inverse of the small matrices
    PROF_N
};
struct ProfEntry {
    int id;
    cudaEvent_t e0, e1;
};

// ------------------------------------------------------------------ context
struct wc4d_ctx {
    wc4d_problem prob{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    std::string err;
    int64_t nA = 0;
    int64_t nobs = 0;
    int obs_per_time = 0;
    std::vector<int> obs_times;     // observed time indices

    // linear model: nM blocks of n*n (1 when shared), FP64 master + derived
    int nM = 0;
    bool have_M = false;
    DevBuf M64, MT64, M32, MT32;
    bool have_M32 = false;

    // Lorenz-96: nonlinear states (N*steps+1) x n and the four RK4 stage
    // states of every step, stages[(4 g + i) n + j] (i = 0 is the state itself)
    DevBuf traj64, stage64, stage32;
    bool have_traj = false;

    // covariance square roots: [0] = B, [1] = Q
    bool have_cov[2] = {false, false};
    bool fft = false;               // n is a power of two <= WC4D_FFT_MAX_N
    int logn = 0;
    DevBuf spec64[2], spec32[2];    // FFT path: sqrt spectrum in bit-reversed order, / n
    DevBuf row64[2], row32[2];      // direct path: first row of the square root
    DevBuf tw64, tw32;              // FFT twiddles e^{-2 pi i j / n}, j < n/2
    DevBuf twp64, twp32;            // per-pass twiddles of the radix-16 Stockham FFT (n entries)
    DevBuf cosn;                    // cos/sin table e^{2 pi i j/n}, j < n (set-up DFTs)
    double cov_sd[2] = {-1.0, -1.0};  // sqrt(variance) of a block that is variance * I, else -1
    bool cov_dense[2] = {false, false};   // dense square root given (wc4d_set_cov_sqrt kind 1)
    DevBuf dense64[2], dense32[2];        // its n x n row-major FP64 and FP32 copies

    // observations and right-hand side
    DevBuf d, rhs, Dm12b;
    bool have_rhs = false;
    // outer loop (Section 2.1): linearisation point p = (x_0, eta_1..eta_N)
    // (lin: (N+1) x n, block 0 = x_0), observations y, and whether D^{-1/2} b
    // is non-zero
    DevBuf lin, ydev;
    // per-call scratch kept across calls (a cudaFree would synchronise the
    // whole device): sketch small matrices, EVD factor, CG cost history
    DevBuf sk_k, sk_w, sk_r, evd_r, qcf;
    DevBuf learn_buf;               // learned-probe network activations
    bool have_lin = false, have_Dm12b = false;

    // workspaces
    DevBuf work64, work32;          // sweep workspace nA x K
    DevBuf blkA, blkB, blkC, blkD;  // nA x m blocks for the eigensolvers
    DevBuf small0, small1, small2, small3;  // m x m FP64
    DevBuf part;                    // partial sums
    DevBuf scal;                    // device scalars (PCG)
    DevBuf counter;                 // int counters
    DevBuf pinned;                  // pinned host staging

    // PCG vectors
    DevBuf pcg64[8], pcg32[8];

    // tensor-core sweeps: split partials and the error flag of bounded waits
    DevBuf tc_part, tc_err;
    bool tc_err_zeroed = false;
    bool gram_tc = true;        // FP32 Gram and tall products on the tensor cores when the shape allows (wc4d_set_gram_path)
    bool tc_err_pending = false;  // a kernel with bounded copy waits (tensor-core Gram or tall product, FP32
                                  // Lorenz-96 sweep) ran since tc_err was last read
    DevBuf oz_slices, oz_work;
    DevBuf chol_bar;            // grid-barrier counter of the cooperative Cholesky
    DevBuf tall_ys, tall_ws;    // TF32 hi / lo halves of the tall product's operands
    DevBuf Mlo, MTlo;           // FP32 remainders M - M32, M^T - MT32 (double-float true-residual sweeps)
    bool have_Mlo = false;
    bool sweep_df = false;      // one-column FP64 sweeps in double-float (set around the mixed CG's true residual)
    DevBuf df_vec;              // hi / lo FP32 halves of the swept FP64 vector  // BF16 slices of the Gram operands; column maxima and exponents
    // tensor-core operands rounded to TF32 (nearest): the propagators, and
    // the probe block as the sweep produces it (nA x K, ld nA)
    DevBuf Mtf, MTtf, tc_round;
    bool have_Mtf = false;

    // persistent one-column sweeps: grid barrier words and error flag
    DevBuf sweep_bar;
    bool sweep_bar_zeroed = false;
    unsigned wait_limit = 1u << 22;   // polls of the persistent sweeps' grid barriers (wc4d_set_wait_limit)

    // Ritz pairs
    int kU = 0;
    int kp = 0;                     // kU rounded up to a multiple of 4
    DevBuf U64, U32, theta64, c64, c32;
    DevBuf Urm64, Urm32;            // row-major nA x kp copies for the LMP kernels
    bool have_U32 = false;
    std::vector<double> theta_host;

    int64_t hvp_count = 0;

    // profiling (CUDA events per launch group)
    // cooperative (grid-synchronised) kernels need the whole GPU; off while
    // the context runs concurrently with others (wc4d_batch_inner_loop)
    // Lanczos data of the last wc4d_lanczos_cg: F (nA x (J + 1)), alpha/beta pairs
    DevBuf lz_F, lz_ab, lz_h;
    int lz_J = 0;
    bool use_graphs = true;         // CG iterations replayed as a CUDA graph (wc4d_set_graphs)
    bool use_loop_graph = true;     // ... as one graph with a device-side WHILE loop
    cudaStream_t cap_stream = nullptr;   // private stream CUDA-graph captures run on
    int iter_mode = 0;              // how the last solve ran its iterations (wc4d_iteration_mode)
    std::string loop_note;          // why the device-side loop graph could not be built ("" if it could)
    double reliable_delta = 1e-3;   // mixed CG: residual reduction between FP64 true-residual updates
    double jacobi_stop2 = 0.0;      // early stop of the small eigensolves (0: run to a sweep without rotations)
    int jacobi_sweeps = 0;          // sweeps used by the last one
    int jacobi_sweeps32 = 0;        // FP32 pre-rotation sweeps before it (0: none)
    int jacobi_kernel32 = 0;        // its kernel: 1 one 16-CTA cluster, 2 cooperative grid (0: none)
    DevBuf jq32;                    // FP32 pre-rotation workspace
    bool allow_coop = true;
    bool prof_on = false;
    std::vector<ProfEntry> prof_log;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
};

// ------------------------------------------------------------------ launch accounting
// Every kernel launch of the library goes through WC4D_LAUNCH, which counts
// it (wc4d_launch_count).  Usage: WC4D_LAUNCH(kernel<<<g, b, smem, s>>>(args)).
void wc4d_note_launch();
#define WC4D_LAUNCH(...) (wc4d_note_launch(), __VA_ARGS__)

// RAII: records an event pair around the launches in scope (no-op when
// profiling is off).
struct ProfScope {
    wc4d_ctx *c;
    int id;
    int slot;
    ProfScope(wc4d_ctx *ctx, int pid);
    ~ProfScope();
};

// ------------------------------------------------------------------ helpers
wc4d_status set_err(wc4d_ctx *c, wc4d_status s, const char *fmt, ...);
wc4d_status ensure(wc4d_ctx *c, DevBuf &b, size_t bytes);
wc4d_status check_launch(wc4d_ctx *c, const char *what);
void free_buf(DevBuf &b);

#define WC4D_TRY(expr)                              \
    do {                                            \
        wc4d_status _s = (expr);                    \
        if (_s != WC4D_OK) return _s;               \
    } while (0)

#define WC4D_CUDA(c, call)                                                              \
    do {                                                                                \
        cudaError_t _e = (call);                                                        \
        if (_e != cudaSuccess)                                                          \
            return set_err((c), WC4D_ECUDA, "%s: %s", #call, cudaGetErrorString(_e));   \
    } while (0)

static inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ------------------------------------------------------------------ kernels (launchers)
// set-up
void launch_gaussian(cudaStream_t s, uint64_t seed, int64_t rows, int64_t cols, int64_t ld, double *G);
void launch_gaussian_f32(cudaStream_t s, uint64_t seed, int64_t rows, int64_t cols, int64_t ld, float *G);
void launch_twiddles(cudaStream_t s, int n, double2 *tab_full, double2 *tw64, float2 *tw32);
void launch_pass_twiddles(cudaStream_t s, int n, double2 *twp64, float2 *twp32);
void launch_cov_sqrt(cudaStream_t s, int n, int logn, bool fft, int kind, double L, double var, const double *row,
                     const double2 *tab, double *lam_tmp, double *spec64, float *spec32, double *row64, float *row32,
                     bool root_given = false);
void launch_advdiff_column(cudaStream_t s, int n, double kappa, double c, double dt, int steps,
                           const double2 *tab, double2 *sym_tmp, double *col);
void launch_expand_circulant(cudaStream_t s, int n, const double *col, double *M, double *MT);
void launch_convert_f64_f32(cudaStream_t s, int64_t count, const double *a, float *b);
void launch_convert_f32_f64(cudaStream_t s, int64_t count, const float *a, double *b);
void launch_transpose_f64(cudaStream_t s, int n, const double *A, double *AT);

// sweeps
// skip: bit 0 leaves block 0 (B) untouched, bit 1 blocks 1..N (Q) -- blocks
// whose square root is dense and applied by GEMMs instead.
template <typename T>
void launch_circulant(cudaStream_t s, const wc4d_ctx *c, int K, const T *X, int64_t ldx, T *Y, int64_t ldy,
                      const T *addX, int64_t ld_add, bool fft, const T *specB, const T *specQ,
                      const T *rowB, const T *rowQ, const void *tw, int skip = 0);
template <typename T>
void launch_sweep_gemm(cudaStream_t s, int n, int K, const T *M, const T *B, int64_t ldb, T *C, int64_t ldc,
                       const Epi &e);
// Persistent one-column sweep over all subwindows (cooperative launch);
// bar: N zeroed unsigned (one arrival counter per step); err set on a timeout
// (a grid barrier that stays incomplete for wait_limit polls; the staged FP32
// form keeps its own limit).
template <typename T>
bool launch_gemv_sweep(cudaStream_t s, int num_sms, int n, int N, const T *M0, int64_t mstride, T *W, int mode,
                       double obs_inv, int obs_stride, int t0, int ts, unsigned *bar, int *err, unsigned wait_limit);
bool launch_gemv_sweep_df(cudaStream_t s, int num_sms, int n, int N, const float *Mh0, const float *Ml0,
                          int64_t mstride, double *W, float *Wh, float *Wl, int mode, double obs_inv, int obs_stride,
                          int t0, int ts, unsigned *bar, int *err, unsigned wait_limit);
template <typename T>
void launch_obs_block(cudaStream_t s, int n, int K, T *W, int64_t ld, double scale, int stride);

// generic products: C(i,j) = epi(sum_k A(i,k) B(k,j)), A(i,k) = A[i*sam + k*sak],
// B(k,j) = B[k + j*ldb], C column-major ldc.
template <typename T>
void launch_gemm(cudaStream_t s, int Mrows, int Ncols, int Kdim, const T *A, int64_t sam, int64_t sak,
                 const T *B, int64_t ldb, T *C, int64_t ldc, const Epi &e);

// linear algebra
// C = A^T B with FP64 accumulation; `upper` (square products known to be
// symmetric) computes the upper tiles only and mirrors them.  part must hold
// atb_part_doubles(...) doubles; returns -1 without launching otherwise.
size_t atb_part_doubles(int num_sms, int64_t rows, int ma, int mb, int upper);
template <typename T>
int launch_atb(cudaStream_t s, int num_sms, int64_t rows, int ma, int mb, const T *A, int64_t lda, const T *B,
               int64_t ldb, double *part, size_t part_capacity, int *splits_out, double *C, int upper);
void launch_chol_upper(cudaStream_t s, int m, const double *A, double *R, int *info);
bool launch_chol_upper_coop(cudaStream_t s, int num_sms, int m, const double *A, double *R, int *info, unsigned *bar);
void launch_shift_diag(cudaStream_t s, int m, double *A, double factor);   // A_ii += factor * trace(A)
// Y (FP32, rows x m, ld) *= 2^-e when max |Y| is outside [2^-24, 2^24] (e kept
// in work[1]); launch_unscale_R: R *= 2^e.  work: 2 device words.
void launch_range_scale_f32(cudaStream_t s, int num_sms, int64_t rows, int m, int64_t ld, float *Y, unsigned *work);
void launch_unscale_R(cudaStream_t s, int m, double *R, const unsigned *work);
void launch_trinv_upper(cudaStream_t s, int m, const double *R, double *Rinv);
void launch_jacobi_init(cudaStream_t s, int m, int mp, const double *S, double *X, double *V);
void launch_jacobi_round(cudaStream_t s, int mp, double *X, double *V, int round, double tol, int *rot);
// One-launch cooperative FP64 Jacobi for 2 <= m <= 256 (P = jacobi_coop_size(m),
// 0 otherwise): XV holds jacobi_coop_doubles(m) doubles, the result is
// X = XV[0, P^2), V = XV[P^2, 2 P^2); rot holds max_sweeps ints, bar one
// counter (zeroed by the launcher), err is set to 1 on a barrier timeout,
// status receives the sweeps used or -1; false when the cooperative launch
// is refused (nothing runs).
int jacobi_coop_size(int m);
size_t jacobi_coop_doubles(int m);
bool launch_jacobi_coop(cudaStream_t s, int m, const double *X0, double *XV, double tol, int max_sweeps, int *rot,
                        unsigned *bar, int *err, int *status, bool want_v, double stop2, unsigned long long *maxm);
bool launch_jacobi_coop_f32(cudaStream_t s, int m, const double *X0, float *XV32, double tol, int max_sweeps,
                            int *rot, unsigned *bar, int *err, int *status, double stop2, unsigned long long *maxm,
                            double *scale_work);
// FP32 pre-rotation on one 16-CTA cluster; V (P x P FP32) and sweeps in *status
// (-1: not converged).  false when the cluster launch is unavailable.
bool launch_jacobi_cluster_f32(cudaStream_t s, int m, const double *X0, float *Vout, double tol, int max_sweeps,
                               int *status, double stop2, double *scale_work);
void launch_small_gemm64(cudaStream_t s, int m, const double *A, int lda, bool transA, const double *B, int ldb,
                         double *C, int ldc, double alpha, double beta);
void launch_orthogonalise_ns(cudaStream_t s, int m, double *V, int ldv, double *tmp);
void launch_jacobi_finish_left(cudaStream_t s, int m, int mp, const double *X, double *w, double *Vout);
void launch_jacobi_finish(cudaStream_t s, int m, int mp, const double *X, const double *V, double *w, double *Vout);
void launch_rrt(cudaStream_t s, int m, const double *R, double *RT);
void launch_symmetrize(cudaStream_t s, int m, double *S);
void launch_scale_cols(cudaStream_t s, int64_t rows, int m, double *A, int64_t lda, const double *w, int inv_sqrt);
// number of row chunks (partial sums per column) of launch_utv
int utv_splits(int64_t nA);
template <typename T>
void launch_utv(cudaStream_t s, int num_sms, int64_t nA, int k, const T *U, const T *v, double *part, int *splits);
template <typename T>
void launch_lmp_combine(cudaStream_t s, int64_t nA, int k, const T *U, const double *part, int splits,
                        const double *cvec, double coef, const T *v, T *y, const T *add, const double *beta_dev,
                        const int *skip);
void launch_lmp_coeffs(cudaStream_t s, int k, const double *theta, double *c);
template <typename T> void launch_axpy_block(cudaStream_t s, int num_sms, int64_t count, double alpha, const T *x, T *y);
void launch_theta_unshift(cudaStream_t s, int k, const double *w, double nu, double *theta);
void launch_lanczos_first(cudaStream_t s, int grid, int64_t n, const double *b, const double *scal, double *F);
void launch_lanczos_record(cudaStream_t s, int grid, int64_t n, const double *r, const double *scal, const int *flags,
                           double *F, double *ab, int cap);
template <typename T>
void launch_to_rowmajor(cudaStream_t s, int64_t nA, int k, int kp, const T *U, T *Urm);
int utv_rm_splits(int64_t nA);
template <typename T>
void launch_utv_rm(cudaStream_t s, int64_t nA, int kp, const T *Urm, const T *v, double *part, int *splits);
template <typename T>
void launch_lmp_combine_rm(cudaStream_t s, int num_sms, int64_t nA, int k, int kp, const T *Urm, const double *t,
                           const double *cvec, const T *v, T *y, const int *skip);

// PCG vector kernels
template <typename T>
void launch_dot_partial(cudaStream_t s, int grid, int64_t n, const T *a, const T *b, double *part);
template <typename T>
void launch_pcg_xr(cudaStream_t s, int grid, int64_t n, const double *scal, T *x, T *r, const T *p, const T *q,
                   double *part);
template <typename T>
void launch_pcg_rh(cudaStream_t s, int grid, int64_t n, const double *scal, T *rh, const T *t, double *part);
template <typename T>
void launch_pcg_p(cudaStream_t s, int grid, int64_t n, const double *scal, T *p, const T *t);
void launch_pcg_alpha(cudaStream_t s, int grid, const double *part, double *scal, int *flags);
// One fused split-preconditioned CG iteration after q = A p (two passes
// over the row-major Ritz vectors Urm, the second from the end of each CTA's
// rows so that it starts on rows still in L2; for kp > 256 the second pass
// reads the column-major copy Ucm, ld nA):
// alpha in scal[1], rhat, t = C rhat, x, r updated, then (last CTA of the
// second pass) the CG beta step: beta, rho, relative residual, QCF decrease,
// flags.  partB: 2 max(lmp_pass_b_grid(nA), lmp_pass_a_splits(nA, num_sms))
// doubles of partial sums; partA:
// lmp_pass_a_splits(nA, num_sms) x (2 kp + 1) doubles; w: 4 kp + 1 doubles;
// done: two counters that are zero on entry (and are left at zero).
int lmp_pass_a_splits(int64_t nA, int num_sms);
int lmp_pass_b_grid(int64_t nA);
template <typename T>
void launch_lmp_fused(cudaStream_t s, int num_sms, int64_t nA, int k, int kp, const T *Urm, const T *Ucm,
                      const double *cvec, const T *q, const T *p, T *rh, T *t, T *x, T *r, double *scal, int *flags,
                      double *partA, double *w, double *partB, unsigned *done, double tol, double *qcf_drop);
void launch_pcg_restart(cudaStream_t s, int grid, const double *part_rh, const double *part_r, double *scal,
                        int *flags);
void launch_pcg_beta(cudaStream_t s, int grid, const double *part_rh, const double *part_r, double *scal,
                     int *flags, double tol, double *qcf_drop);
void launch_pcg_init(cudaStream_t s, int grid, const double *part_b, const double *part_rh, double *scal,
                     int *flags);
template <typename T>
void launch_copy(cudaStream_t s, int64_t n, const T *a, T *b);
template <typename T>
void launch_axpby(cudaStream_t s, int64_t n, double alpha, const T *x, double beta, T *y);
void launch_sub_f64(cudaStream_t s, int64_t n, const double *a, const double *b, double *out);
void launch_add_f32_to_f64(cudaStream_t s, int64_t n, const float *a, double *b);

// Lorenz-96 sweeps (state kept on chip).  The FP32 register-blocked form
// bounds its waits on the staged stage states by wait_limit polls and sets
// *err (when err is not null) if one gives up; the other forms have no waits
// and ignore both.
template <typename T>
void launch_l96_tlm_sweep(cudaStream_t s, int n, int N, int steps, double dt, const T *stages, int K, T *W,
                          int64_t ld, int *err, unsigned wait_limit);
template <typename T>
void launch_l96_adj_sweep(cudaStream_t s, int n, int N, int steps, double dt, const T *stages, int K, T *W,
                          int64_t ld, int obs_mode, double obs_scale, int obs_stride, int obs_t0, int obs_tstride,
                          int *err, unsigned wait_limit);
void launch_l96_run(cudaStream_t s, int n, int nsteps, double F, double dt, double *traj, double *stages,
                    const double *eta, int steps);
void launch_l96_stages(cudaStream_t s, int n, int nsteps, double F, double dt, const double *traj, double *stages);
