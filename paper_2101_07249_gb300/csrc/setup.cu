// Problem set-up kernels: probes, covariance square roots, propagators.
#include "wc4d_internal.cuh"

// ----------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC 2011): two 32x32 multiplications per
// round on words 0 and 2, high halves XORed with words 1 and 3 and the round
// key, key bumped by the Weyl constants before rounds 2..10.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t &x0, uint32_t &x1, uint32_t &x2, uint32_t &x3,
                                              uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint32_t hi0 = __umulhi(0xD2511F53u, x0), lo0 = 0xD2511F53u * x0;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, x2), lo1 = 0xCD9E8D57u * x2;
        uint32_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
        x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
    }
}

__device__ __forceinline__ double uniform53(uint32_t a, uint32_t b)
{
    uint64_t m = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
    return ((double)m + 1.0) * (1.0 / 9007199254740992.0);
}

// One thread per counter c: elements 2c (cos branch) and 2c+1 (sin branch)
// of the column-major rows x cols block.
__global__ void k_gaussian(uint64_t seed, int64_t rows, int64_t total, int64_t ld, double *G)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * c >= total) return;
    uint32_t x0 = (uint32_t)c, x1 = (uint32_t)((uint64_t)c >> 32), x2 = 0u, x3 = 0u;
    philox4x32_10(x0, x1, x2, x3, (uint32_t)seed, (uint32_t)(seed >> 32));
    double u1 = uniform53(x0, x1), u2 = uniform53(x2, x3);
    double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    int64_t e0 = 2 * c, e1 = 2 * c + 1;
    G[(e0 / rows) * ld + (e0 % rows)] = r * cs;
    if (e1 < total) G[(e1 / rows) * ld + (e1 % rows)] = r * sn;
}

void launch_gaussian(cudaStream_t s, uint64_t seed, int64_t rows, int64_t cols, int64_t ld, double *G)
{
    int64_t total = rows * cols;
    int64_t nctr = (total + 1) / 2;
    WC4D_LAUNCH(k_gaussian<<<ceil_div(nctr, 256), 256, 0, s>>>(seed, rows, total, ld, G));
}

// ----------------------------------------------------------------------------
// Tables: tab_full[j] = e^{2 pi i j / n} (j < n) for the set-up DFTs, and the
// FFT twiddles tw[j] = e^{-2 pi i j / n} (j < n/2).
// ----------------------------------------------------------------------------
__global__ void k_twiddles(int n, double2 *tab_full, double2 *tw64, float2 *tw32)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double sn, cs;
    sincospi(2.0 * (double)j / (double)n, &sn, &cs);
    tab_full[j] = make_double2(cs, sn);
    if (j < n / 2) {
        if (tw64) tw64[j] = make_double2(cs, -sn);
        if (tw32) tw32[j] = make_float2((float)cs, (float)-sn);
    }
}

void launch_twiddles(cudaStream_t s, int n, double2 *tab_full, double2 *tw64, float2 *tw32)
{
    WC4D_LAUNCH(k_twiddles<<<ceil_div(n, 256), 256, 0, s>>>(n, tab_full, tw64, tw32));
}

// ----------------------------------------------------------------------------
// Correlation rows on the periodic grid (distance in grid points).
// ----------------------------------------------------------------------------
__global__ void k_corr_row(int n, int kind, double L, double var, double *row)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    double r = (double)min(s, n - s);
    double rho;
    if (kind == WC4D_CORR_SOAR) rho = (1.0 + r / L) * exp(-r / L);
    else if (kind == WC4D_CORR_GAUSS) rho = exp(-r * r / (2.0 * L * L));
    else rho = (s == 0) ? 1.0 : 0.0;
    row[s] = var * rho;
}

void launch_corr_row(cudaStream_t s, int n, int kind, double L, double var, double *row)
{
    WC4D_LAUNCH(k_corr_row<<<ceil_div(n, 256), 256, 0, s>>>(n, kind, L, var, row));
}

// lam[m] = sum_s row[s] cos(2 pi m s / n): eigenvalues of the symmetric circulant.
__global__ void k_circ_eig(int n, const double *row, const double2 *tab, double *lam)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    double acc = 0.0;
    for (int s = 0; s < n; ++s) acc += row[s] * tab[(int)(((int64_t)m * s) % n)].x;
    lam[m] = acc;
}

__device__ __forceinline__ int bitrev(int v, int logn) { return (int)(__brev((unsigned)v) >> (32 - logn)); }

// lam[n] = max_m lam[m] (one CTA).
__global__ void k_eig_max(int n, double *lam)
{
    __shared__ double red[1024];
    double m = -INFINITY;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, lam[i]);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) lam[n] = red[0];
}

// Eigenvalues below 1e-8 of the largest are taken as zero: there the DFT's
// rounding is comparable to the eigenvalue and its square root is noise.
__device__ __forceinline__ double kept_sqrt(double l, double lmax) { return (l >= 1e-8 * lmax) ? sqrt(l) : 0.0; }

// FFT path: spec[p] = sqrt(lam[bitrev(p)]) / n.  Direct path: first row of
// the square root, r[s] = (1/n) sum_m sqrt(lam_m) cos(2 pi m s / n).
__global__ void k_sqrt_spec(int n, int logn, const double *lam, double *spec64, float *spec32)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double v = kept_sqrt(lam[bitrev(p, logn)], lam[n]) / (double)n;
    spec64[p] = v;
    spec32[p] = (float)v;
}

__global__ void k_sqrt_row(int n, const double *lam, const double2 *tab, double *row64, float *row32)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const double lmax = lam[n];
    double acc = 0.0;
    for (int m = 0; m < n; ++m) acc += kept_sqrt(lam[m], lmax) * tab[(int)(((int64_t)m * s) % n)].x;
    acc /= (double)n;
    row64[s] = acc;
    row32[s] = (float)acc;
}

void launch_cov_sqrt(cudaStream_t s, int n, int logn, bool fft, const double *row, const double2 *tab,
                     double *lam_tmp, double *spec64, float *spec32, double *row64, float *row32)
{
    WC4D_LAUNCH(k_circ_eig<<<ceil_div(n, 128), 128, 0, s>>>(n, row, tab, lam_tmp));
    WC4D_LAUNCH(k_eig_max<<<1, 1024, 0, s>>>(n, lam_tmp));
    if (fft) WC4D_LAUNCH(k_sqrt_spec<<<ceil_div(n, 256), 256, 0, s>>>(n, logn, lam_tmp, spec64, spec32));
    else WC4D_LAUNCH(k_sqrt_row<<<ceil_div(n, 128), 128, 0, s>>>(n, lam_tmp, tab, row64, row32));
}

// ----------------------------------------------------------------------------
// Crank-Nicolson advection-diffusion propagator.  Symbol of the centred
// operator on mode e^{i th s}: k = kappa (2 cos th - 2)/dz^2 - i c sin th / dz;
// one step multiplies the mode by g = (1 + dt/2 k)/(1 - dt/2 k); the
// subwindow propagator by g^steps.  The propagator is circulant with first
// column col[s] = (1/n) sum_m Re(g_m^steps e^{2 pi i m s / n}).
// ----------------------------------------------------------------------------
__global__ void k_advdiff_symbol(int n, double kappa, double c, double dt, int steps, const double2 *tab,
                                 double2 *sym)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    double dz = 1.0 / (double)n;
    double2 e = tab[m];
    double kr = kappa * (2.0 * e.x - 2.0) / (dz * dz);
    double ki = -c * e.y / dz;
    double a = 0.5 * dt;
    // g = (1 + a k) / (1 - a k)
    double nr = 1.0 + a * kr, ni = a * ki;
    double dr = 1.0 - a * kr, di = -a * ki;
    double den = dr * dr + di * di;
    double gr = (nr * dr + ni * di) / den, gi = (ni * dr - nr * di) / den;
    double pr = 1.0, pi = 0.0;
    for (int k = 0; k < steps; ++k) {
        double tr = pr * gr - pi * gi;
        pi = pr * gi + pi * gr;
        pr = tr;
    }
    sym[m] = make_double2(pr, pi);
}

__global__ void k_inverse_dft_real(int n, const double2 *sym, const double2 *tab, double *col)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    double acc = 0.0;
    for (int m = 0; m < n; ++m) {
        double2 e = tab[(int)(((int64_t)m * s) % n)];
        double2 g = sym[m];
        acc += g.x * e.x - g.y * e.y;
    }
    col[s] = acc / (double)n;
}

void launch_advdiff_column(cudaStream_t s, int n, double kappa, double c, double dt, int steps,
                           const double2 *tab, double2 *sym_tmp, double *col)
{
    WC4D_LAUNCH(k_advdiff_symbol<<<ceil_div(n, 256), 256, 0, s>>>(n, kappa, c, dt, steps, tab, sym_tmp));
    WC4D_LAUNCH(k_inverse_dft_real<<<ceil_div(n, 128), 128, 0, s>>>(n, sym_tmp, tab, col));
}

// M[s][s'] = col[(s - s') mod n], MT[s][s'] = col[(s' - s) mod n] (row-major).
__global__ void k_expand_circulant(int n, const double *col, double *M, double *MT)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * n) return;
    int s = (int)(idx / n), sp = (int)(idx % n);
    M[idx] = col[(s - sp + n) % n];
    MT[idx] = col[(sp - s + n) % n];
}

void launch_expand_circulant(cudaStream_t s, int n, const double *col, double *M, double *MT)
{
    int64_t tot = (int64_t)n * n;
    WC4D_LAUNCH(k_expand_circulant<<<ceil_div(tot, 256), 256, 0, s>>>(n, col, M, MT));
}

__global__ void k_f64_f32(int64_t count, const double *a, float *b)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) b[i] = (float)a[i];
}

__global__ void k_f32_f64(int64_t count, const float *a, double *b)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) b[i] = (double)a[i];
}

void launch_convert_f64_f32(cudaStream_t s, int64_t count, const double *a, float *b)
{
    if (count > 0) WC4D_LAUNCH(k_f64_f32<<<ceil_div(count, 256), 256, 0, s>>>(count, a, b));
}

void launch_convert_f32_f64(cudaStream_t s, int64_t count, const float *a, double *b)
{
    if (count > 0) WC4D_LAUNCH(k_f32_f64<<<ceil_div(count, 256), 256, 0, s>>>(count, a, b));
}

// 32x32 tiled transpose of a row-major n x n matrix.
__global__ void k_transpose(int n, const double *A, double *AT)
{
    __shared__ double t[32][33];
    int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        int r = by + j, c = bx + threadIdx.x;
        if (r < n && c < n) t[j][threadIdx.x] = A[(int64_t)r * n + c];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        int r = bx + j, c = by + threadIdx.x;
        if (r < n && c < n) AT[(int64_t)r * n + c] = t[threadIdx.x][j];
    }
}

void launch_transpose_f64(cudaStream_t s, int n, const double *A, double *AT)
{
    dim3 g(ceil_div(n, 32), ceil_div(n, 32)), b(32, 8);
    WC4D_LAUNCH(k_transpose<<<g, b, 0, s>>>(n, A, AT));
}
