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

// The same probes in FP32 arithmetic for the mixed path: the same Philox
// counters and 53-bit uniforms, each rounded once to FP32 (the integer
// (m + 1) converted with one rounding, then scaled exactly by 2^-53, so u
// is the FP32 value nearest the FP64 uniform), then Box-Muller in FP32.
// Values agree with the FP64 generator to FP32 rounding of the logarithm
// and the sine/cosine, except where u1 is within a few ulp of 1 (the radius
// -2 log u1 is then tiny in both).  No FP64 arithmetic: this part's FP64
// rate is 1/64 of its FP32 rate.
__device__ __forceinline__ float uniform53_f32(uint32_t a, uint32_t b)
{
    const uint64_t m = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
    return __ull2float_rn(m + 1) * 0x1p-53f;
}

__global__ void k_gaussian_f32(uint64_t seed, int64_t rows, int64_t total, int64_t ld, float *G)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * c >= total) return;
    uint32_t x0 = (uint32_t)c, x1 = (uint32_t)((uint64_t)c >> 32), x2 = 0u, x3 = 0u;
    philox4x32_10(x0, x1, x2, x3, (uint32_t)seed, (uint32_t)(seed >> 32));
    const float u1 = uniform53_f32(x0, x1), u2 = uniform53_f32(x2, x3);
    const float r = sqrtf(-2.0f * logf(u1));
    float sn, cs;
    sincospif(2.0f * u2, &sn, &cs);
    int64_t e0 = 2 * c, e1 = 2 * c + 1;
    G[(e0 / rows) * ld + (e0 % rows)] = r * cs;
    if (e1 < total) G[(e1 / rows) * ld + (e1 % rows)] = r * sn;
}

void launch_gaussian_f32(cudaStream_t s, uint64_t seed, int64_t rows, int64_t cols, int64_t ld, float *G)
{
    int64_t total = rows * cols;
    int64_t nctr = (total + 1) / 2;
    WC4D_LAUNCH(k_gaussian_f32<<<ceil_div(nctr, 256), 256, 0, s>>>(seed, rows, total, ld, G));
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

// Per-pass twiddles of the radix-16 Stockham FFT (n a power of two >= 16):
// the passes have spans P = 1, 16, 256, ... with radix 16 while 16 P <= n,
// then one pass of radix n / P.  The pass at span P >= 16 needs
// W_n^{r k n / (P R)} for 1 <= r < R, k < P, stored at P - 16 + (r - 1) P + k
// (the passes before it, all radix 16, take 15 (16 + 256 + ... + P / 16) =
// P - 16 entries); n - 16 entries in all, the rest of the n-entry table is
// zero.
__global__ void k_pass_twiddles(int n, double2 *twp64, float2 *twp32)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double2 v = make_double2(0.0, 0.0);
    for (int P = 16; P < n;) {
        const int R = min(16, n / P);
        const int off = P - 16, cnt = (R - 1) * P;
        if (e >= off && e < off + cnt) {
            const int r = 1 + (e - off) / P, k = (e - off) % P;
            const int64_t q = (int64_t)r * k * (n / (P * R));   // < n
            double sn, cs;
            sincospi(2.0 * (double)q / (double)n, &sn, &cs);
            v = make_double2(cs, -sn);
            break;
        }
        P *= R;
    }
    twp64[e] = v;
    twp32[e] = make_float2((float)v.x, (float)v.y);
}

void launch_pass_twiddles(cudaStream_t s, int n, double2 *twp64, float2 *twp32)
{
    WC4D_LAUNCH(k_pass_twiddles<<<ceil_div(n, 256), 256, 0, s>>>(n, twp64, twp32));
}

// lam[m] = sum_s row[s] cos(2 pi m s / n): eigenvalues of the symmetric
// circulant given by an explicit first row (FP64 DFT; the angle index m s is
// reduced mod n exactly through the table).
__global__ void k_circ_eig(int n, const double *row, const double2 *tab, double *lam)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    double acc = 0.0;
    for (int s = 0; s < n; ++s) acc += row[s] * tab[(int)(((int64_t)m * s) % n)].x;
    lam[m] = acc;
}

// Eigenvalues of var * C(kind, L) in closed form, so that the smallest ones
// keep their relative accuracy (a DFT of the rounded row leaves errors of
// ~1e-16 of the largest eigenvalue, which the square root turns into
// ~1e-8 of its largest value where the spectrum is tiny).  The row holds
// offsets r in (-n/2, n/2] once each (r = n/2 only for even n); theta = 2 pi m / n.
//  SOAR, c(r) = (1 + r/L) a^r with a = e^{-1/L}: with z = a e^{i theta} and
//    h the last offset of the doubled sum (n/2 - 1 even, (n-1)/2 odd),
//    sum_{r=1..h} z^r = z (1 - z^h) / (1 - z),
//    sum_{r=1..h} r z^r = z (1 - (h+1) z^h + h z^{h+1}) / (1 - z)^2,
//    lam = 1 + 2 Re(S0 + S1 / L) [+ c(n/2) (-1)^m for even n].
//  Gaussian, g(r) = e^{-r^2/(2L^2)}: Poisson summation of the periodic sum,
//    sum_{r in Z} g(r) cos(theta r) = L sqrt(2 pi) sum_j e^{-L^2 (theta - 2 pi j)^2 / 2}
//    (positive terms), minus the images the row does not hold:
//    2 sum_{r > n/2} g(r) cos(theta r) [+ g(n/2) cos(theta n/2) for even n].
//  DIAG: var.
__global__ void k_corr_eig(int n, int kind, double L, double var, double *lam)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    double out;
    if (kind == WC4D_CORR_SOAR) {
        const int h = (n % 2 == 0) ? n / 2 - 1 : (n - 1) / 2;
        const double a = exp(-1.0 / L);
        double sn, cs;
        sincospi(2.0 * (double)m / (double)n, &sn, &cs);
        const double zr = a * cs, zi = a * sn;                        // z
        sincospi(2.0 * (double)(((int64_t)m * h) % n) / (double)n, &sn, &cs);
        const double ah = exp(-(double)h / L);
        const double hr = ah * cs, hi = ah * sn;                      // z^h
        const double h1r = hr * zr - hi * zi, h1i = hr * zi + hi * zr;  // z^{h+1}
        const double dr = 1.0 - zr, di = -zi;                         // 1 - z
        const double d2 = dr * dr + di * di;
        // S0 = z (1 - z^h) / (1 - z)
        double nr = zr - h1r, ni = zi - h1i;                          // z - z^{h+1}
        const double s0r = (nr * dr + ni * di) / d2;
        // S1 = z (1 - (h+1) z^h + h z^{h+1}) / (1 - z)^2
        double tr = 1.0 - (h + 1.0) * hr + h * h1r, ti = -(h + 1.0) * hi + h * h1i;
        nr = zr * tr - zi * ti;
        ni = zr * ti + zi * tr;
        const double q2r = dr * dr - di * di, q2i = 2.0 * dr * di;    // (1 - z)^2
        const double s1r = (nr * q2r + ni * q2i) / (d2 * d2);
        out = 1.0 + 2.0 * (s0r + s1r / L);
        if (n % 2 == 0) {
            const double hh = 0.5 * n;
            out += (1.0 + hh / L) * exp(-hh / L) * ((m & 1) ? -1.0 : 1.0);
        }
    } else if (kind == WC4D_CORR_GAUSS) {
        const double th = 2.0 * (double)m / (double)n;               // theta / pi
        const int jmax = 2 + (int)(3.5 / L);
        double P = 0.0;
        for (int j = -jmax; j <= jmax + 1; ++j) {
            const double d = M_PI * (th - 2.0 * j);
            P += exp(-0.5 * L * L * d * d);
        }
        P *= L * sqrt(2.0 * M_PI);
        double T = 0.0;
        if (n % 2 == 0) {
            const int hh = n / 2;
            T += exp(-(double)hh * hh / (2.0 * L * L)) * ((((int64_t)m * hh) % n == 0) ? 1.0 : -1.0);
        }
        for (int64_t r = n / 2 + 1;; ++r) {
            const double e = (double)r * (double)r / (2.0 * L * L);
            if (e > 745.0) break;
            T += 2.0 * exp(-e) * cospi(2.0 * (double)(((int64_t)m * r) % n) / (double)n);
        }
        out = P - T;
    } else {
        out = 1.0;
    }
    lam[m] = var * out;
}

// Negative eigenvalues (a periodically wrapped correlation function can have
// them) are clamped to zero; every non-negative one is kept.
__device__ __forceinline__ double kept_sqrt(double l) { return (l > 0.0) ? sqrt(l) : 0.0; }

// FFT path: spec[p] = sqrt(lam[p]) / n in natural frequency order (root = 1:
// the eigenvalues are those of the square root already, spec[p] = lam[p] / n).
// Direct path: first row of the square root, r[s] = (1/n) sum_m sqrt(lam_m) cos(2 pi m s / n).
__global__ void k_sqrt_spec(int n, const double *lam, double *spec64, float *spec32, int root)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double l = lam[p];
    double v = (root ? l : kept_sqrt(l)) / (double)n;
    spec64[p] = v;
    spec32[p] = (float)v;
}

__global__ void k_sqrt_row(int n, const double *lam, const double2 *tab, double *row64, float *row32)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    double acc = 0.0;
    for (int m = 0; m < n; ++m) acc += kept_sqrt(lam[m]) * tab[(int)(((int64_t)m * s) % n)].x;
    acc /= (double)n;
    row64[s] = acc;
    row32[s] = (float)acc;
}

__global__ void k_copy_row(int n, const double *row, double *row64, float *row32)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    row64[s] = row[s];
    row32[s] = (float)row[s];
}

// Square root of a circulant covariance: eigenvalues from the correlation
// function (kind >= 0; k_corr_eig) or from an explicit row (kind < 0;
// k_circ_eig), then the spectrum (FFT path) or first row (direct path).
// root_given: the explicit row is the first row of the square root itself.
void launch_cov_sqrt(cudaStream_t s, int n, int logn, bool fft, int kind, double L, double var, const double *row,
                     const double2 *tab, double *lam_tmp, double *spec64, float *spec32, double *row64, float *row32,
                     bool root_given)
{
    if (root_given && !fft) {
        WC4D_LAUNCH(k_copy_row<<<ceil_div(n, 256), 256, 0, s>>>(n, row, row64, row32));
        return;
    }
    if (kind >= 0) WC4D_LAUNCH(k_corr_eig<<<ceil_div(n, 128), 128, 0, s>>>(n, kind, L, var, lam_tmp));
    else WC4D_LAUNCH(k_circ_eig<<<ceil_div(n, 128), 128, 0, s>>>(n, row, tab, lam_tmp));
    if (fft) WC4D_LAUNCH(k_sqrt_spec<<<ceil_div(n, 256), 256, 0, s>>>(n, lam_tmp, spec64, spec32, root_given ? 1 : 0));
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
