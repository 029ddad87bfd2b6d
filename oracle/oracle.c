/*
 * FP64 CPU oracle -- see oracle.h.  TEST INFRASTRUCTURE ONLY: loaded by the
 * tests, the smoke check and the benchmark's CPU-baseline leg; never by the
 * library.
 *
 * Every routine is the plain definition (or the paper's algorithm in the
 * paper's order) written out in loops.  The only parallelism is an OpenMP
 * loop over independent columns, which does not change any column's
 * arithmetic.
 *
 * Parity status (what each part is pinned to, all in tests/test_oracle_*.py):
 *   Philox4x32-10     published known-answer vectors + normality statistics
 *   correlation rows  closed forms; (C^{1/2})^2 = C; eigenvalues vs a 40-digit
 *                     DFT (mpmath) of the correlation function, tiny ones included
 *   advection-diff.   Fourier closed form of the Crank-Nicolson symbol;
 *                     residual of the cyclic tridiagonal solve
 *   Lorenz-96         fixed point x=F; RK4 order-4 convergence vs scipy;
 *                     TLM Taylor test; adjoint dot-product test
 *   L^{-1}, L^{-T}    adjoint test; L(L^{-1}x)=x with L from its definition
 *   A (eq. 10)         dense A vs an independent numpy build; symmetric;
 *                     n_A-q unit eigenvalues
 *   QR/Jacobi/Chol/SVD numpy cross-checks and identities
 *   REVD/Nystrom/ritzit subspace definitions (dense numpy), Ritz bounds,
 *                     full-sketch exactness, product counts (Table 1)
 *   LMP               C C^T = eq. 15 = eq. 14 with exact eigenvectors;
 *                     unit eigenvalues of C^T A C; k = n_A gives A^{-1}
 *   PCG               dense solve; QCF drop vs eq. 4 evaluated directly;
 *                     finite termination; eq. 12 bound
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ======================================================================
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC 2011).  Round: two 32x32->64 multiplications of
 * words 0 and 2, the high halves XORed with words 1/3 and the round key;
 * the key is bumped by the Weyl constants between rounds.
 * ====================================================================== */
void o_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t MUL0 = 0xD2511F53u, MUL1 = 0xCD9E8D57u;
    const uint32_t WEYL0 = 0x9E3779B9u, WEYL1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += WEYL0; k1 += WEYL1; }
        uint64_t p0 = (uint64_t)MUL0 * x0;
        uint64_t p1 = (uint64_t)MUL1 * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Threads of the OpenMP loops over independent columns (n > 0 sets them);
 * returns the number the next parallel loop will use. */
int o_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Raw words of the stream used for the probes: counter c = (c_lo, c_hi, 0, 0),
 * key = (seed_lo, seed_hi); out[4c .. 4c+3]. */
void o_philox_words(uint64_t seed, int64_t count, uint32_t *out)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t c = 0; c < count; ++c) {
        uint32_t ctr[4] = {(uint32_t)c, (uint32_t)((uint64_t)c >> 32), 0u, 0u};
        o_philox4x32_10(ctr, key, out + 4 * c);
    }
}

/* Two 32-bit words -> a double in (0, 1] with 53 random bits. */
static double o_uniform53(uint32_t a, uint32_t b)
{
    uint64_t m = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
    return ((double)m + 1.0) * (1.0 / 9007199254740992.0);
}

/* Gaussian probe matrix G (rows x cols, column-major, leading dimension ld):
 * element e = col*rows + row takes Box-Muller output (e & 1) of Philox
 * counter e >> 1; u1 from words (0,1), u2 from words (2,3). */
void o_gaussian(uint64_t seed, int64_t rows, int64_t cols, int64_t ld, double *G)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t j = 0; j < cols; ++j)
        for (int64_t r = 0; r < rows; ++r) {
            int64_t e = j * rows + r;
            uint64_t c = (uint64_t)e >> 1;
            uint32_t ctr[4] = {(uint32_t)c, (uint32_t)(c >> 32), 0u, 0u}, w[4];
            o_philox4x32_10(ctr, key, w);
            double u1 = o_uniform53(w[0], w[1]);
            double u2 = o_uniform53(w[2], w[3]);
            double rad = sqrt(-2.0 * log(u1));
            double ang = 2.0 * M_PI * u2;
            G[j * ld + r] = (e & 1) ? rad * sin(ang) : rad * cos(ang);
        }
}

/* ======================================================================
 * Covariances.  B = sigma_b^2 C_b and Q_t = sigma_q^2 C_q are circulant on
 * the periodic grid (Section 5).  Distance r is the periodic distance in
 * grid points.  kind 0: second-order auto-regressive (SOAR)
 * (1 + r/L) exp(-r/L); kind 1: Gaussian exp(-r^2 / (2 L^2)); kind 2: the
 * identity (a diagonal covariance variance * I).
 * ====================================================================== */
void o_corr_row(int32_t kind, int32_t n, double L, double variance, double *row)
{
    for (int32_t s = 0; s < n; ++s) {
        double r = (double)(s < n - s ? s : n - s);
        double rho;
        if (kind == 0)      rho = (1.0 + r / L) * exp(-r / L);
        else if (kind == 1) rho = exp(-r * r / (2.0 * L * L));
        else                rho = (s == 0) ? 1.0 : 0.0;
        row[s] = variance * rho;
    }
}

/* Eigenvalues of the symmetric circulant with first row `row`, by the plain
 * DFT lam_m = sum_s row[s] cos(2 pi m s / n), evaluated in long double with the
 * angle index m s reduced mod n exactly (integer arithmetic), so that
 * eigenvalues far below the largest keep their relative accuracy. */
/* pi to the precision of long double (M_PI is a double) */
static const long double PI_LD = 3.14159265358979323846264338327950288419716939937510L;

static void circ_eigs_ld(int32_t n, const long double *row, long double *lam)
{
    long double *cosv = (long double *)malloc(sizeof(long double) * n);
    for (int32_t j = 0; j < n; ++j) cosv[j] = cosl(2.0L * PI_LD * (long double)j / (long double)n);
    for (int32_t m = 0; m < n; ++m) {
        long double acc = 0.0L;
        for (int32_t s = 0; s < n; ++s) acc += row[s] * cosv[(int64_t)m * s % n];
        lam[m] = acc;
    }
    free(cosv);
}

/* First row of the symmetric square root from the eigenvalues (X13 reading:
 * negative eigenvalues, which a periodically wrapped correlation function can
 * have, are clamped to zero; every non-negative one is kept):
 * sqrt_row[s] = (1/n) sum_m sqrt(max(lam_m, 0)) cos(2 pi m s / n), in long
 * double.  Returns the number of clamped (negative) eigenvalues. */
static int circ_sqrt_from_eigs(int32_t n, const long double *lam, double *sqrt_row, double *min_eig)
{
    long double *cosv = (long double *)malloc(sizeof(long double) * n);
    long double *rt = (long double *)malloc(sizeof(long double) * n);
    for (int32_t j = 0; j < n; ++j) cosv[j] = cosl(2.0L * PI_LD * (long double)j / (long double)n);
    int clamped = 0;
    long double mn = INFINITY;
    for (int32_t m = 0; m < n; ++m) {
        if (lam[m] < mn) mn = lam[m];
        if (lam[m] < 0.0L) { rt[m] = 0.0L; ++clamped; }
        else rt[m] = sqrtl(lam[m]);
    }
    for (int32_t s = 0; s < n; ++s) {
        long double acc = 0.0L;
        for (int32_t m = 0; m < n; ++m) acc += rt[m] * cosv[(int64_t)m * s % n];
        sqrt_row[s] = (double)(acc / (long double)n);
    }
    if (min_eig) *min_eig = (double)mn;
    free(cosv); free(rt);
    return clamped;
}

/* Symmetric square root of a symmetric circulant matrix given by its first
 * row (double): eigenvalues by the long-double DFT of that row, negative ones
 * clamped to zero.  Returns the number clamped; *min_eig the smallest
 * eigenvalue before clamping. */
int o_circulant_sqrt_row(int32_t n, const double *row, double *sqrt_row, double *min_eig)
{
    long double *r = (long double *)malloc(sizeof(long double) * n);
    long double *lam = (long double *)malloc(sizeof(long double) * n);
    for (int32_t s = 0; s < n; ++s) r[s] = row[s];
    circ_eigs_ld(n, r, lam);
    int clamped = circ_sqrt_from_eigs(n, lam, sqrt_row, min_eig);
    free(r); free(lam);
    return clamped;
}

/* Eigenvalues of the covariance variance * C(kind, L) of o_corr_row, computed
 * from the correlation function itself rather than from its double row:
 *  - SOAR: the long-double DFT of the row evaluated in long double;
 *  - Gaussian: the Poisson summation formula for the periodic sum,
 *      sum_{r in Z} e^{-r^2/(2L^2)} cos(theta r)
 *        = L sqrt(2 pi) sum_{j in Z} e^{-L^2 (theta - 2 pi j)^2 / 2},
 *    a sum of positive terms (so even eigenvalues of 1e-35 keep full relative
 *    accuracy, which no DFT of rounded row values can give), minus the images
 *    that the periodic-distance row does not contain: offsets r outside
 *    (-n/2, n/2], i.e. 2 sum_{r > n/2} g(r) cos(theta r) + [n even] g(n/2)
 *    cos(theta n/2) (odd n: 2 sum_{r >= (n+1)/2});
 *  - identity: variance.
 * theta_m = 2 pi m / n; lam has n entries. */
static void cov_eigs_ld(int32_t kind, int32_t n, double L, double variance, long double *lam)
{
    if (kind == 0) {
        long double *row = (long double *)malloc(sizeof(long double) * n);
        long double Ll = L;
        for (int32_t s = 0; s < n; ++s) {
            long double r = (long double)(s < n - s ? s : n - s);
            row[s] = (long double)variance * (1.0L + r / Ll) * expl(-r / Ll);
        }
        circ_eigs_ld(n, row, lam);
        free(row);
    } else if (kind == 1) {
        const long double Ll = L, twopi = 2.0L * PI_LD;
        const int jmax = 2 + (int)(3.5 / L);
        for (int32_t m = 0; m < n; ++m) {
            long double th = twopi * (long double)m / (long double)n;
            long double P = 0.0L;
            for (int j = -jmax; j <= jmax + 1; ++j) {
                long double d = th - twopi * (long double)j;
                P += expl(-Ll * Ll * d * d / 2.0L);
            }
            P *= Ll * sqrtl(twopi);
            long double T = 0.0L;
            int32_t r0 = n / 2 + 1;                 /* first offset beyond (-n/2, n/2] */
            if (n % 2 == 0) T += expl(-(long double)(n / 2) * (n / 2) / (2.0L * Ll * Ll))
                                 * cosl(th * (long double)(n / 2));
            for (int64_t r = r0;; ++r) {
                long double e = (long double)r * (long double)r / (2.0L * Ll * Ll);
                if (e > 1000.0L) break;
                T += 2.0L * expl(-e) * cosl(th * (long double)r);
            }
            lam[m] = (long double)variance * (P - T);
        }
    } else {
        for (int32_t m = 0; m < n; ++m) lam[m] = variance;
    }
}

/* Eigenvalues of variance * C(kind, L) as doubles (cov_eigs_ld). */
void o_cov_eigs(int32_t kind, int32_t n, double L, double variance, double *lam)
{
    long double *l = (long double *)malloc(sizeof(long double) * n);
    cov_eigs_ld(kind, n, L, variance, l);
    for (int32_t m = 0; m < n; ++m) lam[m] = (double)l[m];
    free(l);
}

/* First row of (variance * C(kind, L))^{1/2}: the accurate eigenvalues of
 * cov_eigs_ld, negative ones clamped to zero (Section 5 covariances; X13
 * reading).  Returns the number clamped. */
int o_cov_sqrt_row(int32_t kind, int32_t n, double L, double variance, double *sqrt_row, double *min_eig)
{
    long double *lam = (long double *)malloc(sizeof(long double) * n);
    cov_eigs_ld(kind, n, L, variance, lam);
    int clamped = circ_sqrt_from_eigs(n, lam, sqrt_row, min_eig);
    free(lam);
    return clamped;
}

/* y = C x for the symmetric circulant C with C[s][s'] = row[(s' - s) mod n]. */
void o_circulant_apply(int32_t n, const double *row, const double *x, double *y)
{
    for (int32_t s = 0; s < n; ++s) {
        double acc = 0.0;
        for (int32_t sp = 0; sp < n; ++sp) {
            double c = row[((sp - s) % n + n) % n];
            if (c != 0.0) acc += c * x[sp];
        }
        y[s] = acc;
    }
}

/* ======================================================================
 * Periodic advection-diffusion u_t = kappa u_zz - u u_z on n points, grid
 * spacing 1/n, centred differences, Crank-Nicolson in time:
 *   (I - dt/2 K) x_new = (I + dt/2 K) x
 * K has sub-diagonal al (x_{s-1}), diagonal be, super-diagonal ga (x_{s+1}),
 * wrapped periodically.
 * ====================================================================== */
static void advdiff_coeffs(int32_t n, double kappa, double u, double *al, double *be, double *ga)
{
    double dz = 1.0 / (double)n;
    *al = kappa / (dz * dz) + u / (2.0 * dz);
    *be = -2.0 * kappa / (dz * dz);
    *ga = kappa / (dz * dz) - u / (2.0 * dz);
}

/* Solve T y = r for tridiagonal T (no corners): sub lo (row s, col s-1),
 * diagonal d[s], super up (row s, col s+1).  Thomas elimination. */
static void thomas(int32_t n, double lo, const double *d, double up, const double *r, double *y)
{
    double *cp = (double *)malloc(sizeof(double) * n);
    double *dp = (double *)malloc(sizeof(double) * n);
    cp[0] = up / d[0];
    dp[0] = r[0] / d[0];
    for (int32_t s = 1; s < n; ++s) {
        double den = d[s] - lo * cp[s - 1];
        cp[s] = up / den;
        dp[s] = (r[s] - lo * dp[s - 1]) / den;
    }
    y[n - 1] = dp[n - 1];
    for (int32_t s = n - 2; s >= 0; --s) y[s] = dp[s] - cp[s] * y[s + 1];
    free(cp); free(dp);
}

/* Solve the cyclic tridiagonal system with constant sub lo, diagonal di,
 * super up (corner A[0][n-1] = lo, A[n-1][0] = up) by Sherman-Morrison:
 * A = T + u v^T with u = (g, 0.., 0, up), v = (1, 0.., 0, lo/g). */
static void cyclic_solve(int32_t n, double lo, double di, double up, const double *r, double *x)
{
    double g = -di;
    double *d = (double *)malloc(sizeof(double) * n);
    double *uu = (double *)calloc(n, sizeof(double));
    double *y = (double *)malloc(sizeof(double) * n);
    double *z = (double *)malloc(sizeof(double) * n);
    for (int32_t s = 0; s < n; ++s) d[s] = di;
    d[0] = di - g;
    d[n - 1] = di - up * lo / g;
    uu[0] = g;
    uu[n - 1] = up;
    thomas(n, lo, d, up, r, y);
    thomas(n, lo, d, up, uu, z);
    double vy = y[0] + (lo / g) * y[n - 1];
    double vz = z[0] + (lo / g) * z[n - 1];
    double f = vy / (1.0 + vz);
    for (int32_t s = 0; s < n; ++s) x[s] = y[s] - f * z[s];
    free(d); free(uu); free(y); free(z);
}

/* One Crank-Nicolson step y = (I - a K)^{-1} (I + a K) x, a = dt/2. */
void o_advdiff_step(int32_t n, double kappa, double u, double dt, const double *x, double *y)
{
    double al, be, ga, a = 0.5 * dt;
    advdiff_coeffs(n, kappa, u, &al, &be, &ga);
    double *r = (double *)malloc(sizeof(double) * n);
    for (int32_t s = 0; s < n; ++s) {
        double xm = x[(s - 1 + n) % n], xp = x[(s + 1) % n];
        r[s] = x[s] + a * (al * xm + be * x[s] + ga * xp);
    }
    /* (I - aK): sub -a*al, diagonal 1 - a*be, super -a*ga */
    cyclic_solve(n, -a * al, 1.0 - a * be, -a * ga, r, y);
    free(r);
}

/* Transpose of one step: y = (I + a K)^T (I - a K)^{-T} x. */
void o_advdiff_step_T(int32_t n, double kappa, double u, double dt, const double *x, double *y)
{
    double al, be, ga, a = 0.5 * dt;
    advdiff_coeffs(n, kappa, u, &al, &be, &ga);
    double *z = (double *)malloc(sizeof(double) * n);
    /* (I - aK)^T has sub -a*ga and super -a*al */
    cyclic_solve(n, -a * ga, 1.0 - a * be, -a * al, x, z);
    /* (I + aK)^T: row s picks z_{s-1} with ga and z_{s+1} with al */
    for (int32_t s = 0; s < n; ++s) {
        double zm = z[(s - 1 + n) % n], zp = z[(s + 1) % n];
        y[s] = z[s] + a * (ga * zm + be * z[s] + al * zp);
    }
    free(z);
}

/* Dense propagator of `steps` Crank-Nicolson steps, built by stepping each
 * unit vector; M row-major. */
void o_advdiff_dense(int32_t n, double kappa, double u, double dt, int32_t steps, double *M)
{
#pragma omp parallel
    {
        double *a = (double *)malloc(sizeof(double) * n);
        double *b = (double *)malloc(sizeof(double) * n);
#pragma omp for schedule(static)
        for (int32_t c = 0; c < n; ++c) {
            memset(a, 0, sizeof(double) * n);
            a[c] = 1.0;
            for (int32_t k = 0; k < steps; ++k) {
                o_advdiff_step(n, kappa, u, dt, a, b);
                memcpy(a, b, sizeof(double) * n);
            }
            for (int32_t s = 0; s < n; ++s) M[(int64_t)s * n + c] = a[s];
        }
        free(a); free(b);
    }
}

/* ======================================================================
 * Lorenz-96 (Section 5.2): dX_j/dt = (X_{j+1} - X_{j-2}) X_{j-1} - X_j + F,
 * periodic; classical fourth-order Runge-Kutta.
 * ====================================================================== */
void o_l96_tendency(int32_t n, double F, const double *x, double *f)
{
    for (int32_t j = 0; j < n; ++j) {
        double xm2 = x[(j - 2 + n) % n], xm1 = x[(j - 1 + n) % n], xp1 = x[(j + 1) % n];
        f[j] = (xp1 - xm2) * xm1 - x[j] + F;
    }
}

void o_l96_rk4(int32_t n, double F, double dt, const double *x, double *y)
{
    double *k1 = malloc(sizeof(double) * n), *k2 = malloc(sizeof(double) * n);
    double *k3 = malloc(sizeof(double) * n), *k4 = malloc(sizeof(double) * n);
    double *t = malloc(sizeof(double) * n);
    o_l96_tendency(n, F, x, k1);
    for (int32_t j = 0; j < n; ++j) t[j] = x[j] + 0.5 * dt * k1[j];
    o_l96_tendency(n, F, t, k2);
    for (int32_t j = 0; j < n; ++j) t[j] = x[j] + 0.5 * dt * k2[j];
    o_l96_tendency(n, F, t, k3);
    for (int32_t j = 0; j < n; ++j) t[j] = x[j] + dt * k3[j];
    o_l96_tendency(n, F, t, k4);
    for (int32_t j = 0; j < n; ++j) y[j] = x[j] + dt / 6.0 * (k1[j] + 2.0 * k2[j] + 2.0 * k3[j] + k4[j]);
    free(k1); free(k2); free(k3); free(k4); free(t);
}

/* Jacobian of the tendency at x applied to d. */
static void l96_jac(int32_t n, const double *x, const double *d, double *o)
{
    for (int32_t j = 0; j < n; ++j) {
        int32_t jm2 = (j - 2 + n) % n, jm1 = (j - 1 + n) % n, jp1 = (j + 1) % n;
        o[j] = (d[jp1] - d[jm2]) * x[jm1] + (x[jp1] - x[jm2]) * d[jm1] - d[j];
    }
}

/* Transposed Jacobian at x applied to l. */
static void l96_jac_T(int32_t n, const double *x, const double *l, double *o)
{
    for (int32_t i = 0; i < n; ++i) {
        int32_t im2 = (i - 2 + n) % n, im1 = (i - 1 + n) % n;
        int32_t ip1 = (i + 1) % n, ip2 = (i + 2) % n;
        o[i] = x[im2] * l[im1] - x[ip1] * l[ip2] + (x[ip2] - x[im1]) * l[ip1] - l[i];
    }
}

/* The four RK4 stage states at x (recomputed from the stored state). */
static void l96_stages(int32_t n, double F, double dt, const double *x, double *s1, double *s2,
                       double *s3, double *s4)
{
    double *k = malloc(sizeof(double) * n);
    memcpy(s1, x, sizeof(double) * n);
    o_l96_tendency(n, F, s1, k);
    for (int32_t j = 0; j < n; ++j) s2[j] = x[j] + 0.5 * dt * k[j];
    o_l96_tendency(n, F, s2, k);
    for (int32_t j = 0; j < n; ++j) s3[j] = x[j] + 0.5 * dt * k[j];
    o_l96_tendency(n, F, s3, k);
    for (int32_t j = 0; j < n; ++j) s4[j] = x[j] + dt * k[j];
    free(k);
}

/* Tangent linear of one RK4 step at x (exact derivative of the discrete
 * step).  F enters only through the recomputed stage states. */
void o_l96_tlm(int32_t n, double F, double dt, const double *x, const double *dx, double *dy)
{
    double *s1 = malloc(sizeof(double) * n), *s2 = malloc(sizeof(double) * n);
    double *s3 = malloc(sizeof(double) * n), *s4 = malloc(sizeof(double) * n);
    double *d1 = malloc(sizeof(double) * n), *d2 = malloc(sizeof(double) * n);
    double *d3 = malloc(sizeof(double) * n), *d4 = malloc(sizeof(double) * n);
    double *t = malloc(sizeof(double) * n);
    l96_stages(n, F, dt, x, s1, s2, s3, s4);
    l96_jac(n, s1, dx, d1);
    for (int32_t j = 0; j < n; ++j) t[j] = dx[j] + 0.5 * dt * d1[j];
    l96_jac(n, s2, t, d2);
    for (int32_t j = 0; j < n; ++j) t[j] = dx[j] + 0.5 * dt * d2[j];
    l96_jac(n, s3, t, d3);
    for (int32_t j = 0; j < n; ++j) t[j] = dx[j] + dt * d3[j];
    l96_jac(n, s4, t, d4);
    for (int32_t j = 0; j < n; ++j) dy[j] = dx[j] + dt / 6.0 * (d1[j] + 2.0 * d2[j] + 2.0 * d3[j] + d4[j]);
    free(s1); free(s2); free(s3); free(s4); free(d1); free(d2); free(d3); free(d4); free(t);
}

/* Adjoint (transpose) of o_l96_tlm: lx = (dRK4/dx)^T ly. */
void o_l96_adj(int32_t n, double F, double dt, const double *x, const double *ly, double *lx)
{
    double *s1 = malloc(sizeof(double) * n), *s2 = malloc(sizeof(double) * n);
    double *s3 = malloc(sizeof(double) * n), *s4 = malloc(sizeof(double) * n);
    double *a1 = malloc(sizeof(double) * n), *a2 = malloc(sizeof(double) * n);
    double *a3 = malloc(sizeof(double) * n), *a4 = malloc(sizeof(double) * n);
    double *g = malloc(sizeof(double) * n);
    l96_stages(n, F, dt, x, s1, s2, s3, s4);
    for (int32_t j = 0; j < n; ++j) {
        lx[j] = ly[j];
        a1[j] = dt / 6.0 * ly[j];
        a2[j] = dt / 3.0 * ly[j];
        a3[j] = dt / 3.0 * ly[j];
        a4[j] = dt / 6.0 * ly[j];
    }
    /* d4 = J(s4) (dx + dt d3) */
    l96_jac_T(n, s4, a4, g);
    for (int32_t j = 0; j < n; ++j) { lx[j] += g[j]; a3[j] += dt * g[j]; }
    /* d3 = J(s3) (dx + dt/2 d2) */
    l96_jac_T(n, s3, a3, g);
    for (int32_t j = 0; j < n; ++j) { lx[j] += g[j]; a2[j] += 0.5 * dt * g[j]; }
    /* d2 = J(s2) (dx + dt/2 d1) */
    l96_jac_T(n, s2, a2, g);
    for (int32_t j = 0; j < n; ++j) { lx[j] += g[j]; a1[j] += 0.5 * dt * g[j]; }
    /* d1 = J(s1) dx */
    l96_jac_T(n, s1, a1, g);
    for (int32_t j = 0; j < n; ++j) lx[j] += g[j];
    free(s1); free(s2); free(s3); free(s4); free(a1); free(a2); free(a3); free(a4); free(g);
}

/* Nonlinear run: traj[0] = x0, traj[i+1] = RK4(traj[i]), i < nsteps. */
void o_l96_run(int32_t n, double F, double dt, int32_t nsteps, const double *x0, double *traj)
{
    memcpy(traj, x0, sizeof(double) * n);
    for (int32_t i = 0; i < nsteps; ++i)
        o_l96_rk4(n, F, dt, traj + (int64_t)i * n, traj + (int64_t)(i + 1) * n);
}

/* ======================================================================
 * Forcing formulation (Section 2.1-2.2).
 *   L^{-1}: block lower triangular, block (l+1, i) = M_l ... M_i (eq. 5),
 *           applied as w_0 = z_0, w_{t+1} = M_t w_t + z_{t+1}.
 *   H_t   : observes s = 0, stride, 2 stride, ... at t >= obs_t0.
 *   R_t   : sigma_o2 * I.
 *   D^{1/2}: diag(B^{1/2}, Q^{1/2}, ..., Q^{1/2}).
 *   A     = I + D^{1/2} L^{-T} H^T R^{-1} H L^{-1} D^{1/2}   (eq. 10)
 * ====================================================================== */
static int64_t g_hvp_count = 0;

int64_t o_hvp_count(int reset)
{
    int64_t c = g_hvp_count;
    if (reset) g_hvp_count = 0;
    return c;
}

static int32_t obs_per_time(const o_problem *p) { return (p->n + p->obs_stride - 1) / p->obs_stride; }

static int32_t obs_tstride(const o_problem *p) { return p->obs_tstride > 0 ? p->obs_tstride : 1; }

/* Is time index t observed? */
static int observed_time(const o_problem *p, int32_t t)
{
    return t >= p->obs_t0 && t <= p->N && (t - p->obs_t0) % obs_tstride(p) == 0;
}

int64_t o_nobs(const o_problem *p)
{
    int64_t times = 0;
    for (int32_t t = 0; t <= p->N; ++t) times += observed_time(p, t);
    return times * obs_per_time(p);
}

/* y = M_t x (the linearised model over subwindow t, t = 0..N-1). */
void o_model_apply(const o_problem *p, int32_t t, const double *x, double *y)
{
    int32_t n = p->n;
    if (p->model == O_MODEL_DENSE) {
        const double *M = p->M + (p->M_shared ? 0 : (int64_t)t * n * n);
        for (int32_t s = 0; s < n; ++s) {
            double acc = 0.0;
            for (int32_t c = 0; c < n; ++c) acc += M[(int64_t)s * n + c] * x[c];
            y[s] = acc;
        }
    } else if (p->model == O_MODEL_ADVDIFF) {
        double *a = malloc(sizeof(double) * n);
        memcpy(a, x, sizeof(double) * n);
        for (int32_t k = 0; k < p->steps; ++k) {
            o_advdiff_step(n, p->kappa, p->u, p->dt, a, y);
            memcpy(a, y, sizeof(double) * n);
        }
        free(a);
    } else {
        double *a = malloc(sizeof(double) * n);
        memcpy(a, x, sizeof(double) * n);
        for (int32_t k = 0; k < p->steps; ++k) {
            const double *xs = p->traj + ((int64_t)t * p->steps + k) * n;
            o_l96_tlm(n, p->F, p->dt, xs, a, y);
            memcpy(a, y, sizeof(double) * n);
        }
        free(a);
    }
}

/* y = M_t^T x. */
void o_model_apply_T(const o_problem *p, int32_t t, const double *x, double *y)
{
    int32_t n = p->n;
    if (p->model == O_MODEL_DENSE) {
        const double *M = p->M + (p->M_shared ? 0 : (int64_t)t * n * n);
        for (int32_t c = 0; c < n; ++c) y[c] = 0.0;
        for (int32_t s = 0; s < n; ++s) {
            double xs = x[s];
            for (int32_t c = 0; c < n; ++c) y[c] += M[(int64_t)s * n + c] * xs;
        }
    } else if (p->model == O_MODEL_ADVDIFF) {
        double *a = malloc(sizeof(double) * n);
        memcpy(a, x, sizeof(double) * n);
        for (int32_t k = 0; k < p->steps; ++k) {
            o_advdiff_step_T(n, p->kappa, p->u, p->dt, a, y);
            memcpy(a, y, sizeof(double) * n);
        }
        free(a);
    } else {
        /* M_t = T_{last} ... T_{first}; its transpose applies the step
         * adjoints in reverse order. */
        double *a = malloc(sizeof(double) * n);
        memcpy(a, x, sizeof(double) * n);
        for (int32_t k = p->steps - 1; k >= 0; --k) {
            const double *xs = p->traj + ((int64_t)t * p->steps + k) * n;
            o_l96_adj(n, p->F, p->dt, xs, a, y);
            memcpy(a, y, sizeof(double) * n);
        }
        free(a);
    }
}

/* One column of W = L^{-1} Z. */
static void linv_col(const o_problem *p, const double *z, double *w)
{
    int32_t n = p->n;
    double *tmp = malloc(sizeof(double) * n);
    memcpy(w, z, sizeof(double) * n);
    for (int32_t t = 0; t < p->N; ++t) {
        o_model_apply(p, t, w + (int64_t)t * n, tmp);
        for (int32_t s = 0; s < n; ++s) w[(int64_t)(t + 1) * n + s] = tmp[s] + z[(int64_t)(t + 1) * n + s];
    }
    free(tmp);
}

/* One column of S = L^{-T} V. */
static void linvT_col(const o_problem *p, const double *v, double *sv)
{
    int32_t n = p->n, N = p->N;
    double *tmp = malloc(sizeof(double) * n);
    memcpy(sv + (int64_t)N * n, v + (int64_t)N * n, sizeof(double) * n);
    for (int32_t t = N - 1; t >= 0; --t) {
        o_model_apply_T(p, t, sv + (int64_t)(t + 1) * n, tmp);
        for (int32_t s = 0; s < n; ++s) sv[(int64_t)t * n + s] = v[(int64_t)t * n + s] + tmp[s];
    }
    free(tmp);
}

static void dsqrt_col(const o_problem *p, const double *x, double *z)
{
    int32_t n = p->n;
    for (int32_t t = 0; t <= p->N; ++t)
        o_circulant_apply(n, t == 0 ? p->Bsqrt : p->Qsqrt, x + (int64_t)t * n, z + (int64_t)t * n);
}

/* v = H^T R^{-1} H w (zero at unobserved points and times). */
static void obs_col(const o_problem *p, const double *w, double *v)
{
    int32_t n = p->n;
    for (int32_t t = 0; t <= p->N; ++t)
        for (int32_t s = 0; s < n; ++s) {
            int64_t i = (int64_t)t * n + s;
            v[i] = (observed_time(p, t) && s % p->obs_stride == 0) ? w[i] / p->sigma_o2 : 0.0;
        }
}

void o_Linv(const o_problem *p, int32_t K, const double *Z, int64_t ld, double *W)
{
#pragma omp parallel for schedule(dynamic)
    for (int32_t j = 0; j < K; ++j) linv_col(p, Z + j * ld, W + j * ld);
}

void o_LinvT(const o_problem *p, int32_t K, const double *V, int64_t ld, double *S)
{
#pragma omp parallel for schedule(dynamic)
    for (int32_t j = 0; j < K; ++j) linvT_col(p, V + j * ld, S + j * ld);
}

void o_Dsqrt(const o_problem *p, int32_t K, const double *X, int64_t ld, double *Z)
{
#pragma omp parallel for schedule(dynamic)
    for (int32_t j = 0; j < K; ++j) dsqrt_col(p, X + j * ld, Z + j * ld);
}

void o_obs_adjoint(const o_problem *p, int32_t K, const double *W, int64_t ld, double *V)
{
    for (int32_t j = 0; j < K; ++j) obs_col(p, W + j * ld, V + j * ld);
}

/* Y = A X, column by column, following eq. 10 from right to left. */
void o_hvp(const o_problem *p, int32_t K, const double *X, int64_t ld, double *Y)
{
    int64_t nA = (int64_t)p->n * (p->N + 1);
    ++g_hvp_count;
#pragma omp parallel for schedule(dynamic)
    for (int32_t j = 0; j < K; ++j) {
        double *z = malloc(sizeof(double) * nA), *w = malloc(sizeof(double) * nA);
        const double *x = X + j * ld;
        dsqrt_col(p, x, z);      /* z = D^{1/2} x           */
        linv_col(p, z, w);       /* w = L^{-1} z            */
        obs_col(p, w, z);        /* z = H^T R^{-1} H w      */
        linvT_col(p, z, w);      /* w = L^{-T} z            */
        dsqrt_col(p, w, z);      /* z = D^{1/2} w           */
        for (int64_t i = 0; i < nA; ++i) Y[j * ld + i] = x[i] + z[i];
        free(z); free(w);
    }
}

/* State at the subwindow boundaries, x_0 = xb, x_{t+1} = M_t(x_t) + eta_{t+1}
 * (eq. 1); nonlinear RK4 for Lorenz-96, the linear propagator otherwise.
 * eta may be NULL (no forcing).  xtraj has (N+1)*n entries. */
void o_forward_run(const o_problem *p, const double *xb, const double *eta, double *xtraj)
{
    int32_t n = p->n;
    double *a = malloc(sizeof(double) * n), *b = malloc(sizeof(double) * n);
    memcpy(xtraj, xb, sizeof(double) * n);
    for (int32_t t = 0; t < p->N; ++t) {
        const double *xt = xtraj + (int64_t)t * n;
        double *xn = xtraj + (int64_t)(t + 1) * n;
        if (p->model == O_MODEL_L96) {
            memcpy(a, xt, sizeof(double) * n);
            for (int32_t k = 0; k < p->steps; ++k) {
                o_l96_rk4(n, p->F, p->dt, a, b);
                memcpy(a, b, sizeof(double) * n);
            }
            memcpy(xn, a, sizeof(double) * n);
        } else {
            o_model_apply(p, t, xt, xn);
        }
        if (eta)
            for (int32_t s = 0; s < n; ++s) xn[s] += eta[(int64_t)(t + 1) * n + s];
    }
    free(a); free(b);
}

/* d_t = y_t - H_t x_t for the observed times t = obs_t0..N (stacked). */
void o_innovation(const o_problem *p, const double *xb, const double *eta, const double *y, double *d)
{
    int32_t n = p->n, per = obs_per_time(p);
    double *xt = malloc(sizeof(double) * (int64_t)n * (p->N + 1));
    o_forward_run(p, xb, eta, xt);
    int64_t k = 0;
    for (int32_t t = p->obs_t0; t <= p->N; t += obs_tstride(p))
        for (int32_t o = 0; o < per; ++o, ++k) d[k] = y[k] - xt[(int64_t)t * n + (int64_t)o * p->obs_stride];
    free(xt);
}

/* Right-hand side of eq. 10: D^{-1/2} b + D^{1/2} L^{-T} H^T R^{-1} d.
 * Dm12b (= D^{-1/2} b) may be NULL, meaning zero (first outer loop). */
void o_rhs(const o_problem *p, const double *d, const double *Dm12b, double *rhs)
{
    int32_t n = p->n, per = obs_per_time(p);
    int64_t nA = (int64_t)n * (p->N + 1);
    double *v = calloc(nA, sizeof(double)), *s = malloc(sizeof(double) * nA);
    int64_t k = 0;
    for (int32_t t = p->obs_t0; t <= p->N; t += obs_tstride(p))
        for (int32_t o = 0; o < per; ++o, ++k) v[(int64_t)t * n + (int64_t)o * p->obs_stride] = d[k] / p->sigma_o2;
    linvT_col(p, v, s);
    dsqrt_col(p, s, rhs);
    if (Dm12b)
        for (int64_t i = 0; i < nA; ++i) rhs[i] += Dm12b[i];
    free(v); free(s);
}

/* Quadratic cost (eq. 4) in the transformed variable x = D^{-1/2} dp:
 * J = 1/2 |x - D^{-1/2} b|^2 + 1/2 sum_t |H_t w_t - d_t|^2 / sigma_o2,
 * w = L^{-1} D^{1/2} x. */
double o_qcf(const o_problem *p, const double *x, const double *d, const double *Dm12b)
{
    int32_t n = p->n, per = obs_per_time(p);
    int64_t nA = (int64_t)n * (p->N + 1);
    double *z = malloc(sizeof(double) * nA), *w = malloc(sizeof(double) * nA);
    dsqrt_col(p, x, z);
    linv_col(p, z, w);
    double jb = 0.0, jo = 0.0;
    for (int64_t i = 0; i < nA; ++i) {
        double e = x[i] - (Dm12b ? Dm12b[i] : 0.0);
        jb += e * e;
    }
    int64_t k = 0;
    for (int32_t t = p->obs_t0; t <= p->N; t += obs_tstride(p))
        for (int32_t o = 0; o < per; ++o, ++k) {
            double e = w[(int64_t)t * n + (int64_t)o * p->obs_stride] - d[k];
            jo += e * e / p->sigma_o2;
        }
    free(z); free(w);
    return 0.5 * jb + 0.5 * jo;
}

/* ======================================================================
 * Dense linear algebra (column-major).
 * ====================================================================== */

/* Thin QR by Householder reflections: A (m x k) = Q R, Q (m x k) with
 * orthonormal columns, R (k x k) upper triangular with a positive diagonal
 * (signs fixed so that the factorisation is the unique one). */
void o_householder_qr(int64_t m, int32_t k, const double *A, int64_t lda, double *Q, int64_t ldq, double *R)
{
    double *W = malloc(sizeof(double) * m * k);
    double *beta = malloc(sizeof(double) * k);
    for (int32_t j = 0; j < k; ++j) memcpy(W + j * m, A + j * lda, sizeof(double) * m);
    /* reflector j: H_j = I - beta_j v v^T, v stored in W[j..m-1, j] with v_j = 1 implied by storage */
    double *vdiag = malloc(sizeof(double) * k);
    for (int32_t j = 0; j < k; ++j) {
        double *col = W + (int64_t)j * m;
        double nrm = 0.0;
        for (int64_t i = j; i < m; ++i) nrm += col[i] * col[i];
        nrm = sqrt(nrm);
        double alpha = (col[j] >= 0.0) ? -nrm : nrm;   /* new diagonal entry */
        double v0 = col[j] - alpha;
        double vtv = v0 * v0;
        for (int64_t i = j + 1; i < m; ++i) vtv += col[i] * col[i];
        beta[j] = (vtv > 0.0) ? 2.0 / vtv : 0.0;
        vdiag[j] = v0;
        /* apply H_j to the trailing columns */
        for (int32_t c = j + 1; c < k; ++c) {
            double *cc = W + (int64_t)c * m;
            double dot = v0 * cc[j];
            for (int64_t i = j + 1; i < m; ++i) dot += col[i] * cc[i];
            double f = beta[j] * dot;
            cc[j] -= f * v0;
            for (int64_t i = j + 1; i < m; ++i) cc[i] -= f * col[i];
        }
        col[j] = alpha;
    }
    for (int32_t j = 0; j < k; ++j)
        for (int32_t i = 0; i < k; ++i) R[(int64_t)j * k + i] = (i <= j) ? W[(int64_t)j * m + i] : 0.0;
    /* Q = H_0 H_1 ... H_{k-1} [I_k; 0] */
    for (int32_t j = 0; j < k; ++j) {
        double *qc = Q + (int64_t)j * ldq;
        for (int64_t i = 0; i < m; ++i) qc[i] = 0.0;
        qc[j] = 1.0;
        for (int32_t r = k - 1; r >= 0; --r) {
            const double *col = W + (int64_t)r * m;
            double dot = vdiag[r] * qc[r];
            for (int64_t i = r + 1; i < m; ++i) dot += col[i] * qc[i];
            double f = beta[r] * dot;
            qc[r] -= f * vdiag[r];
            for (int64_t i = r + 1; i < m; ++i) qc[i] -= f * col[i];
        }
    }
    for (int32_t j = 0; j < k; ++j)
        if (R[(int64_t)j * k + j] < 0.0) {
            for (int32_t c = j; c < k; ++c) R[(int64_t)c * k + j] = -R[(int64_t)c * k + j];
            double *qc = Q + (int64_t)j * ldq;
            for (int64_t i = 0; i < m; ++i) qc[i] = -qc[i];
        }
    free(W); free(beta); free(vdiag);
}

/* Symmetric eigendecomposition by the cyclic-by-row Jacobi method (Golub &
 * Van Loan, Section 8.5): A = V diag(w) V^T, w sorted in decreasing order,
 * V column-major (column j is the eigenvector of w[j]).  Returns the number
 * of sweeps, or -1 if it did not converge. */
int o_jacobi_eig(int32_t m, const double *A, double *w, double *V)
{
    double *a = malloc(sizeof(double) * m * m);
    memcpy(a, A, sizeof(double) * m * m);
    for (int32_t j = 0; j < m; ++j)
        for (int32_t i = 0; i < m; ++i) V[(int64_t)j * m + i] = (i == j) ? 1.0 : 0.0;
    /* An off-diagonal entry is negligible once |a_pq| <= tol sqrt(|a_pp a_qq|)
     * with tol = sqrt(m) eps (relative criterion, the rounding level of the
     * m-term updates); the iteration stops after a sweep with no rotation. */
    const double tol = 2.220446049250313e-16 * sqrt((double)m);
    int sweeps = -1;
    for (int sweep = 0; sweep < 100; ++sweep) {
        int rotated = 0;
        for (int32_t p = 0; p < m - 1; ++p)
            for (int32_t q = p + 1; q < m; ++q) {
                double apq = a[(int64_t)q * m + p];
                double app = a[(int64_t)p * m + p], aqq = a[(int64_t)q * m + q];
                if (fabs(apq) <= tol * sqrt(fabs(app * aqq)) || fabs(apq) < 1e-300) continue;
                rotated = 1;
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                for (int32_t r = 0; r < m; ++r) {           /* A <- A J */
                    double arp = a[(int64_t)p * m + r], arq = a[(int64_t)q * m + r];
                    a[(int64_t)p * m + r] = c * arp - s * arq;
                    a[(int64_t)q * m + r] = s * arp + c * arq;
                }
                for (int32_t r = 0; r < m; ++r) {           /* A <- J^T A */
                    double apr = a[(int64_t)r * m + p], aqr = a[(int64_t)r * m + q];
                    a[(int64_t)r * m + p] = c * apr - s * aqr;
                    a[(int64_t)r * m + q] = s * apr + c * aqr;
                }
                for (int32_t r = 0; r < m; ++r) {           /* V <- V J */
                    double vrp = V[(int64_t)p * m + r], vrq = V[(int64_t)q * m + r];
                    V[(int64_t)p * m + r] = c * vrp - s * vrq;
                    V[(int64_t)q * m + r] = s * vrp + c * vrq;
                }
            }
        if (!rotated) { sweeps = sweep; break; }
    }
    for (int32_t i = 0; i < m; ++i) w[i] = a[(int64_t)i * m + i];
    /* selection sort into decreasing order */
    double *tmp = malloc(sizeof(double) * m);
    for (int32_t i = 0; i < m; ++i) {
        int32_t best = i;
        for (int32_t j = i + 1; j < m; ++j) if (w[j] > w[best]) best = j;
        if (best != i) {
            double t = w[i]; w[i] = w[best]; w[best] = t;
            memcpy(tmp, V + (int64_t)i * m, sizeof(double) * m);
            memcpy(V + (int64_t)i * m, V + (int64_t)best * m, sizeof(double) * m);
            memcpy(V + (int64_t)best * m, tmp, sizeof(double) * m);
        }
    }
    free(tmp); free(a);
    return sweeps;
}

/* A = R^T R with R upper triangular (column-major m x m).  Returns 0, or
 * j+1 if the j-th pivot is not positive. */
int o_cholesky_upper(int32_t m, const double *A, double *R)
{
    for (int64_t i = 0; i < (int64_t)m * m; ++i) R[i] = 0.0;
    for (int32_t j = 0; j < m; ++j) {
        double d = A[(int64_t)j * m + j];
        for (int32_t k = 0; k < j; ++k) d -= R[(int64_t)j * m + k] * R[(int64_t)j * m + k];
        if (!(d > 0.0)) return j + 1;
        double rjj = sqrt(d);
        R[(int64_t)j * m + j] = rjj;
        for (int32_t i = j + 1; i < m; ++i) {
            double v = A[(int64_t)i * m + j];
            for (int32_t k = 0; k < j; ++k) v -= R[(int64_t)j * m + k] * R[(int64_t)i * m + k];
            R[(int64_t)i * m + j] = v / rjj;
        }
    }
    return 0;
}

/* Solve X R = B for X (rows x m), R upper triangular; B is overwritten. */
void o_solve_right_upper(int64_t rows, int32_t m, const double *R, double *B, int64_t ldb)
{
    for (int32_t j = 0; j < m; ++j) {
        double *bj = B + (int64_t)j * ldb;
        for (int32_t i = 0; i < j; ++i) {
            double rij = R[(int64_t)j * m + i];
            const double *bi = B + (int64_t)i * ldb;
            for (int64_t r = 0; r < rows; ++r) bj[r] -= bi[r] * rij;
        }
        double rjj = R[(int64_t)j * m + j];
        for (int64_t r = 0; r < rows; ++r) bj[r] /= rjj;
    }
}

/* Thin SVD A = U diag(s) V^T of a tall matrix (rows >= m): Householder QR,
 * then one-sided (Hestenes) Jacobi on R.  s decreasing, U rows x m (ld =
 * rows), V m x m.  Returns the number of sweeps, or -1. */
int o_jacobi_svd(int64_t rows, int32_t m, const double *A, int64_t lda, double *U, double *s, double *V)
{
    double *Q = malloc(sizeof(double) * rows * m), *B = malloc(sizeof(double) * m * m);
    o_householder_qr(rows, m, A, lda, Q, rows, B);
    for (int32_t j = 0; j < m; ++j)
        for (int32_t i = 0; i < m; ++i) V[(int64_t)j * m + i] = (i == j) ? 1.0 : 0.0;
    const double tol = 2.220446049250313e-16 * sqrt((double)m);   /* rounding level of m-term dots */
    int sweeps = -1;
    for (int sweep = 0; sweep < 100; ++sweep) {
        int rotated = 0;
        for (int32_t p = 0; p < m - 1; ++p)
            for (int32_t q = p + 1; q < m; ++q) {
                double *bp = B + (int64_t)p * m, *bq = B + (int64_t)q * m;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int32_t r = 0; r < m; ++r) { al += bp[r] * bp[r]; be += bq[r] * bq[r]; ga += bp[r] * bq[r]; }
                if (ga == 0.0 || fabs(ga) <= tol * sqrt(al * be)) continue;
                rotated = 1;
                double zeta = (be - al) / (2.0 * ga);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
                for (int32_t r = 0; r < m; ++r) {
                    double x = bp[r], y = bq[r];
                    bp[r] = c * x - sn * y;
                    bq[r] = sn * x + c * y;
                }
                double *vp = V + (int64_t)p * m, *vq = V + (int64_t)q * m;
                for (int32_t r = 0; r < m; ++r) {
                    double x = vp[r], y = vq[r];
                    vp[r] = c * x - sn * y;
                    vq[r] = sn * x + c * y;
                }
            }
        if (!rotated) { sweeps = sweep; break; }
    }
    /* singular values = column norms of B V-rotated; left vectors B_j / s_j */
    double *Ub = malloc(sizeof(double) * m * m);
    for (int32_t j = 0; j < m; ++j) {
        double nrm = 0.0;
        for (int32_t r = 0; r < m; ++r) nrm += B[(int64_t)j * m + r] * B[(int64_t)j * m + r];
        nrm = sqrt(nrm);
        s[j] = nrm;
        for (int32_t r = 0; r < m; ++r) Ub[(int64_t)j * m + r] = nrm > 0.0 ? B[(int64_t)j * m + r] / nrm : 0.0;
    }
    /* sort decreasing */
    double *tmp = malloc(sizeof(double) * m);
    for (int32_t i = 0; i < m; ++i) {
        int32_t best = i;
        for (int32_t j = i + 1; j < m; ++j) if (s[j] > s[best]) best = j;
        if (best != i) {
            double t = s[i]; s[i] = s[best]; s[best] = t;
            memcpy(tmp, Ub + (int64_t)i * m, sizeof(double) * m);
            memcpy(Ub + (int64_t)i * m, Ub + (int64_t)best * m, sizeof(double) * m);
            memcpy(Ub + (int64_t)best * m, tmp, sizeof(double) * m);
            memcpy(tmp, V + (int64_t)i * m, sizeof(double) * m);
            memcpy(V + (int64_t)i * m, V + (int64_t)best * m, sizeof(double) * m);
            memcpy(V + (int64_t)best * m, tmp, sizeof(double) * m);
        }
    }
    /* U = Q Ub */
    for (int32_t j = 0; j < m; ++j)
        for (int64_t r = 0; r < rows; ++r) {
            double acc = 0.0;
            for (int32_t i = 0; i < m; ++i) acc += Q[(int64_t)i * rows + r] * Ub[(int64_t)j * m + i];
            U[(int64_t)j * rows + r] = acc;
        }
    free(Q); free(B); free(Ub); free(tmp);
    return sweeps;
}

/* C = A^T B for column-major A (rows x ma), B (rows x mb); C is ma x mb. */
static void gram_AtB(int64_t rows, int32_t ma, const double *A, int32_t mb, const double *B, double *C)
{
#pragma omp parallel for schedule(dynamic) collapse(2)
    for (int32_t j = 0; j < mb; ++j)
        for (int32_t i = 0; i < ma; ++i) {
            double acc = 0.0;
            const double *a = A + (int64_t)i * rows, *b = B + (int64_t)j * rows;
            for (int64_t r = 0; r < rows; ++r) acc += a[r] * b[r];
            C[(int64_t)j * ma + i] = acc;
        }
}

/* X (rows x kout) = Z (rows x m) W[:, 0:kout] */
static void mat_ZW(int64_t rows, int32_t m, const double *Z, const double *W, int32_t kout, double *X)
{
#pragma omp parallel for schedule(static)
    for (int32_t j = 0; j < kout; ++j) {
        double *x = X + (int64_t)j * rows;
        for (int64_t r = 0; r < rows; ++r) x[r] = 0.0;
        for (int32_t i = 0; i < m; ++i) {
            double wij = W[(int64_t)j * m + i];
            const double *z = Z + (int64_t)i * rows;
            for (int64_t r = 0; r < rows; ++r) x[r] += z[r] * wij;
        }
    }
}

static void symmetrize(int32_t m, double *K)
{
    for (int32_t j = 0; j < m; ++j)
        for (int32_t i = 0; i < j; ++i) {
            double v = 0.5 * (K[(int64_t)j * m + i] + K[(int64_t)i * m + j]);
            K[(int64_t)j * m + i] = v;
            K[(int64_t)i * m + j] = v;
        }
}

/* Orthonormal basis of the columns of Y (Householder QR, Q factor). */
static void orth(int64_t rows, int32_t m, const double *Y, double *Z)
{
    double *R = malloc(sizeof(double) * m * m);
    o_householder_qr(rows, m, Y, rows, Z, rows, R);
    free(R);
}

/* ======================================================================
 * Randomised eigensolvers (Section 4).
 * ====================================================================== */

/* Rayleigh-Ritz (Alg. 2) on an orthonormal basis Z, truncated to the k
 * largest Ritz values; shared by REVD. */
static int rayleigh_ritz(const o_problem *p, int32_t k, int32_t m, const double *Z, double *U, double *theta)
{
    int64_t nA = (int64_t)p->n * (p->N + 1);
    double *E = malloc(sizeof(double) * nA * m);
    double *K = malloc(sizeof(double) * m * m), *W = malloc(sizeof(double) * m * m), *w = malloc(sizeof(double) * m);
    o_hvp(p, m, Z, nA, E);                    /* A Z                      */
    gram_AtB(nA, m, Z, m, E, K);              /* K = Z^T A Z              */
    symmetrize(m, K);
    int rc = o_jacobi_eig(m, K, w, W);        /* K = W Theta W^T, sorted  */
    for (int32_t i = 0; i < k; ++i) theta[i] = w[i];
    mat_ZW(nA, m, Z, W, k, U);                /* U = Z W[:, :k]           */
    free(E); free(K); free(W); free(w);
    return rc < 0 ? -1 : 0;
}

/* REVD (Alg. 3) with q power iterations: Z = orth(A G), then q times
 * Z = orth(A Z), then Rayleigh-Ritz on Z.  q = 0 is Alg. 3 as printed. */
int o_revd(const o_problem *p, int32_t k, int32_t l, int32_t q, const double *G, double *U, double *theta)
{
    int32_t m = k + l;
    int64_t nA = (int64_t)p->n * (p->N + 1);
    double *Y = malloc(sizeof(double) * nA * m), *Z = malloc(sizeof(double) * nA * m);
    o_hvp(p, m, G, nA, Y);                    /* step 2: Y = A G          */
    orth(nA, m, Y, Z);                        /* step 3                   */
    for (int32_t it = 0; it < q; ++it) {      /* power iterations         */
        o_hvp(p, m, Z, nA, Y);
        orth(nA, m, Y, Z);
    }
    int rc = rayleigh_ritz(p, k, m, Z, U, theta);   /* steps 4-8      */
    free(Y); free(Z);
    return rc;
}

/* Randomised Nystrom (Alg. 4). */
int o_nystrom(const o_problem *p, int32_t k, int32_t l, const double *G, double *U, double *theta)
{
    int32_t m = k + l;
    int64_t nA = (int64_t)p->n * (p->N + 1);
    double *Y = malloc(sizeof(double) * nA * m), *Z = malloc(sizeof(double) * nA * m);
    double *E2 = malloc(sizeof(double) * m * m), *C = malloc(sizeof(double) * m * m);
    double *Uf = malloc(sizeof(double) * nA * m), *sg = malloc(sizeof(double) * m), *V = malloc(sizeof(double) * m * m);
    int rc = 0;
    o_hvp(p, m, G, nA, Y);                    /* step 2: Y = A G                 */
    orth(nA, m, Y, Z);                        /* step 3: Z_1                     */
    o_hvp(p, m, Z, nA, Y);                    /* step 4: E1 = A Z_1 (in Y)       */
    gram_AtB(nA, m, Z, m, Y, E2);             /*         E2 = Z_1^T E1           */
    symmetrize(m, E2);
    if (o_cholesky_upper(m, E2, C) != 0) { rc = -2; goto out; }  /* step 5: E2 = C^T C */
    o_solve_right_upper(nA, m, C, Y, nA);     /* step 6: F C = E1 -> F (in Y)    */
    if (o_jacobi_svd(nA, m, Y, nA, Uf, sg, V) < 0) rc = -1;  /* step 7: F = U S V^T */
    for (int32_t i = 0; i < k; ++i) theta[i] = sg[i] * sg[i];   /* step 9: Theta = S^2 */
    memcpy(U, Uf, sizeof(double) * nA * k);   /* step 8: first k columns         */
out:
    free(Y); free(Z); free(E2); free(C); free(Uf); free(sg); free(V);
    return rc;
}

/* REVD_ritzit (Alg. 5), single pass over A. */
int o_ritzit(const o_problem *p, int32_t k, int32_t l, const double *G, double *U, double *theta)
{
    int32_t m = k + l;
    int64_t nA = (int64_t)p->n * (p->N + 1);
    double *G3 = malloc(sizeof(double) * nA * m), *Y = malloc(sizeof(double) * nA * m);
    double *Z = malloc(sizeof(double) * nA * m), *R = malloc(sizeof(double) * m * m);
    double *K = malloc(sizeof(double) * m * m), *W = malloc(sizeof(double) * m * m), *w = malloc(sizeof(double) * m);
    orth(nA, m, G, G3);                       /* step 2: G_3 = orth(G)           */
    o_hvp(p, m, G3, nA, Y);                   /* step 3: Y_3 = A G_3             */
    o_householder_qr(nA, m, Y, nA, Z, nA, R); /* step 4: Y_3 = Z_3 R_3           */
    for (int32_t j = 0; j < m; ++j)           /* step 5: K_3 = R_3 R_3^T         */
        for (int32_t i = 0; i < m; ++i) {
            double acc = 0.0;
            for (int32_t c = 0; c < m; ++c) acc += R[(int64_t)c * m + i] * R[(int64_t)c * m + j];
            K[(int64_t)j * m + i] = acc;
        }
    int rc = o_jacobi_eig(m, K, w, W);        /* step 6: K_3 = W Theta^2 W^T     */
    for (int32_t i = 0; i < k; ++i) theta[i] = sqrt(w[i] > 0.0 ? w[i] : 0.0);  /* step 7 */
    mat_ZW(nA, m, Z, W, k, U);                /* steps 8-9: U_3 = Z_3 W_3        */
    free(G3); free(Y); free(Z); free(R); free(K); free(W); free(w);
    return rc < 0 ? -1 : 0;
}

/* ======================================================================
 * Spectral LMP factor (eq. 16): C = prod_{i=1..k} (I - (1 - theta_i^{-1/2})
 * u_i u_i^T).  C v applies the factor i = k first; C^T v applies i = 1
 * first.  A non-positive theta contributes the identity.
 * ====================================================================== */
void o_lmp_apply(int64_t nA, int32_t k, const double *U, const double *theta, int32_t transpose,
                 const double *v, double *y)
{
    memcpy(y, v, sizeof(double) * nA);
    for (int32_t step = 0; step < k; ++step) {
        int32_t i = transpose ? step : k - 1 - step;
        if (!(theta[i] > 0.0)) continue;
        double c = 1.0 - 1.0 / sqrt(theta[i]);
        const double *ui = U + (int64_t)i * nA;
        double dot = 0.0;
        for (int64_t r = 0; r < nA; ++r) dot += ui[r] * y[r];
        for (int64_t r = 0; r < nA; ++r) y[r] -= c * dot * ui[r];
    }
}

static double dotv(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Split-preconditioned CG (Alg. 1) from x_0 = 0, with the unpreconditioned
 * residual r = b - A x carried alongside rhat = C^T r for the stopping rule
 * |r| / |b| <= tol.  k = 0 means no second-level preconditioner.
 * force_iters > 0 runs exactly that many iterations.  qcf_drop[j-1] =
 * alpha_j rhat_{j-1}^T rhat_{j-1} / 2, the decrease of eq. 4 at iteration j.
 * Returns 0, -5 on breakdown (p^T A p <= 0 or not finite), -6 if maxit was
 * reached without convergence. */
int o_pcg(const o_problem *p, const double *rhs, int32_t k, const double *U, const double *theta,
          double tol, int32_t maxit, int32_t force_iters, double *x, int32_t *iters,
          double *relres, double *qcf_drop, double *relres_hist)
{
    int64_t nA = (int64_t)p->n * (p->N + 1);
    double *r = malloc(sizeof(double) * nA), *rh = malloc(sizeof(double) * nA);
    double *pv = malloc(sizeof(double) * nA), *q = malloc(sizeof(double) * nA);
    double *t = malloc(sizeof(double) * nA);
    int rc = -6;
    for (int64_t i = 0; i < nA; ++i) { x[i] = 0.0; r[i] = rhs[i]; }
    double bnorm = sqrt(dotv(nA, rhs, rhs));
    o_lmp_apply(nA, k, U, theta, 1, r, rh);          /* rhat_0 = C^T (b - A x_0) */
    o_lmp_apply(nA, k, U, theta, 0, rh, pv);         /* p_0 = C rhat_0           */
    double rho = dotv(nA, rh, rh);
    double rr = bnorm > 0.0 ? 1.0 : 0.0;
    int32_t j = 0;
    if (bnorm == 0.0) rc = 0;
    while (rc != 0 && j < maxit) {
        ++j;
        o_hvp(p, 1, pv, nA, q);                     /* A p_{j-1}                */
        double pq = dotv(nA, pv, q);
        if (!(pq > 0.0) || !isfinite(pq)) { rc = -5; --j; break; }
        double alpha = rho / pq;                     /* step 3                   */
        for (int64_t i = 0; i < nA; ++i) { x[i] += alpha * pv[i]; r[i] -= alpha * q[i]; }  /* step 4 */
        o_lmp_apply(nA, k, U, theta, 1, q, t);       /* C^T A p                  */
        for (int64_t i = 0; i < nA; ++i) rh[i] -= alpha * t[i];   /* step 5      */
        double rho_new = dotv(nA, rh, rh);
        double beta = rho_new / rho;                 /* step 6                   */
        o_lmp_apply(nA, k, U, theta, 0, rh, t);      /* C rhat_j                 */
        for (int64_t i = 0; i < nA; ++i) pv[i] = t[i] + beta * pv[i];  /* step 7 */
        if (qcf_drop) qcf_drop[j - 1] = 0.5 * alpha * rho;
        rho = rho_new;
        rr = sqrt(dotv(nA, r, r)) / bnorm;
        if (relres_hist) relres_hist[j - 1] = rr;
        if (force_iters > 0) { if (j >= force_iters) { rc = 0; break; } }
        else if (rr <= tol) { rc = 0; break; }
    }
    *iters = j;
    *relres = rr;
    free(r); free(rh); free(pv); free(q); free(t);
    return rc;
}
