/*
 * FP64 CPU oracle for the inner loop of forcing-formulation weak-constraint
 * 4D-Var with randomised spectral-LMP preconditioning (Dauzickaite, Lawless,
 * Scott, van Leeuwen, "Randomised preconditioning for the forcing formulation
 * of weak constraint 4D-Var").
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the plain, slow reference that the
 * CUDA library is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code with
 * the CUDA library.
 *
 * Conventions
 *   - A block of K vectors of the control space (dimension nA = n*(N+1)) is a
 *     column-major nA x K matrix with leading dimension ld >= nA.  Row
 *     t*n + s holds grid point s of time block t (t = 0 is x_0, t >= 1 is
 *     eta_t).
 *   - Dense propagators are row-major n x n.
 *   - Everything is double precision, except the covariance eigenvalue sums
 *     (long double, so that eigenvalues far below the largest stay accurate).
 */
#ifndef WC4D_ORACLE_H
#define WC4D_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { O_MODEL_DENSE = 0, O_MODEL_ADVDIFF = 1, O_MODEL_L96 = 2 };

typedef struct {
    int32_t n;          /* grid points per time block                          */
    int32_t N;          /* subwindows; control dimension nA = n*(N+1)          */
    int32_t model;      /* O_MODEL_*                                            */
    int32_t steps;      /* model time steps per subwindow                       */
    int32_t M_shared;   /* dense model: 1 = one matrix for every subwindow      */
    int32_t obs_stride; /* H_t observes s = 0, stride, 2*stride, ...            */
    int32_t obs_t0;     /* first observed time index                            */
    int32_t obs_tstride;/* observed times t = obs_t0, obs_t0 + tstride, ... <= N */
    double dt;          /* model time step                                      */
    double kappa, u;    /* advection-diffusion coefficients (grid spacing 1/n) */
    double F;           /* Lorenz-96 forcing                                    */
    double sigma_o2;    /* R_t = sigma_o2 * I                                   */
    const double *M;    /* dense propagators, N*n*n row-major (n*n if shared)   */
    const double *Bsqrt;/* first row of the symmetric circulant B^{1/2}         */
    const double *Qsqrt;/* first row of the symmetric circulant Q_t^{1/2}       */
    const double *traj; /* L96 linearisation states, (N*steps+1)*n              */
} o_problem;

/* ---- threads of the column loops (OpenMP; 1 without it) -------------- */
int o_threads(int n);

/* ---- random numbers (Philox4x32-10, Box-Muller) ---------------------- */
void o_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void o_gaussian(uint64_t seed, int64_t rows, int64_t cols, int64_t ld, double *G);
void o_philox_words(uint64_t seed, int64_t count, uint32_t *out);

/* ---- covariance rows ---------------------------------------------------- */
void o_corr_row(int32_t kind, int32_t n, double L_points, double variance, double *row);
int  o_circulant_sqrt_row(int32_t n, const double *row, double *sqrt_row, double *min_eig);
void o_cov_eigs(int32_t kind, int32_t n, double L_points, double variance, double *lam);
int  o_cov_sqrt_row(int32_t kind, int32_t n, double L_points, double variance, double *sqrt_row, double *min_eig);
void o_circulant_apply(int32_t n, const double *row, const double *x, double *y);

/* ---- models ------------------------------------------------------------- */
void o_advdiff_step(int32_t n, double kappa, double u, double dt, const double *x, double *y);
void o_advdiff_step_T(int32_t n, double kappa, double u, double dt, const double *x, double *y);
void o_advdiff_dense(int32_t n, double kappa, double u, double dt, int32_t steps, double *M);
void o_l96_tendency(int32_t n, double F, const double *x, double *f);
void o_l96_rk4(int32_t n, double F, double dt, const double *x, double *y);
void o_l96_tlm(int32_t n, double F, double dt, const double *x, const double *dx, double *dy);
void o_l96_adj(int32_t n, double F, double dt, const double *x, const double *ly, double *lx);
void o_l96_run(int32_t n, double F, double dt, int32_t nsteps, const double *x0, double *traj);

/* ---- the forcing-formulation operators (eq. 5, eq. 10) ------------------ */
int64_t o_nobs(const o_problem *p);
void o_model_apply(const o_problem *p, int32_t t, const double *x, double *y);
void o_model_apply_T(const o_problem *p, int32_t t, const double *x, double *y);
void o_Linv(const o_problem *p, int32_t K, const double *Z, int64_t ld, double *W);
void o_LinvT(const o_problem *p, int32_t K, const double *V, int64_t ld, double *S);
void o_Dsqrt(const o_problem *p, int32_t K, const double *X, int64_t ld, double *Z);
void o_obs_adjoint(const o_problem *p, int32_t K, const double *W, int64_t ld, double *V);
void o_hvp(const o_problem *p, int32_t K, const double *X, int64_t ld, double *Y);
int64_t o_hvp_count(int reset);
void o_forward_run(const o_problem *p, const double *xb, const double *eta, double *xtraj);
void o_innovation(const o_problem *p, const double *xb, const double *eta, const double *y, double *d);
void o_rhs(const o_problem *p, const double *d, const double *Dm12b, double *rhs);
double o_qcf(const o_problem *p, const double *x, const double *d, const double *Dm12b);

/* ---- small dense linear algebra ---------------------------------------- */
void o_householder_qr(int64_t m, int32_t k, const double *A, int64_t lda, double *Q, int64_t ldq, double *R);
int  o_jacobi_eig(int32_t m, const double *A, double *w, double *V);
int  o_cholesky_upper(int32_t m, const double *A, double *R);
void o_solve_right_upper(int64_t rows, int32_t m, const double *R, double *B, int64_t ldb);
int  o_jacobi_svd(int64_t rows, int32_t m, const double *A, int64_t lda, double *U, double *s, double *V);

/* ---- randomised eigensolvers (Alg. 2-5) --------------------------------- */
int o_revd(const o_problem *p, int32_t k, int32_t l, int32_t q, const double *G, double *U, double *theta);
int o_nystrom(const o_problem *p, int32_t k, int32_t l, const double *G, double *U, double *theta);
int o_ritzit(const o_problem *p, int32_t k, int32_t l, const double *G, double *U, double *theta);

/* ---- spectral LMP (eq. 15-16) and split-preconditioned CG (Alg. 1) ------ */
void o_lmp_apply(int64_t nA, int32_t k, const double *U, const double *theta, int32_t transpose,
                 const double *v, double *y);
int  o_pcg(const o_problem *p, const double *rhs, int32_t k, const double *U, const double *theta,
           double tol, int32_t maxit, int32_t force_iters, double *x, int32_t *iters,
           double *relres, double *qcf_drop, double *relres_hist);

#ifdef __cplusplus
}
#endif
#endif
