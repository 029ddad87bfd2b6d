// Dense linear algebra of the randomised eigensolvers and the LMP / PCG
// vector kernels.  Reductions are two-stage (fixed partial layout, then a
// single-CTA sum) so that results are bitwise reproducible run to run.
#include <algorithm>
#include <climits>
#include <type_traits>

#include "wc4d_internal.cuh"

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// PCG device state: scalars and flags
enum { S_RHO = 0, S_ALPHA, S_BETA, S_BNORM, S_RELRES, S_PQ, S_RR };
enum { F_DONE = 0, F_BREAK, F_ITER };

// Sum over a CTA (blockDim.x multiple of 32, <= 1024); result valid in all threads.
__device__ double block_sum(double v)
{
    __shared__ double red[32];
    __shared__ double total;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        double x = (lane < nw) ? red[lane] : 0.0;
        x = warp_sum(x);
        if (lane == 0) total = x;
    }
    __syncthreads();
    return total;
}

// ----------------------------------------------------------------------------
// C = A^T B (FP64 accumulation) for tall column-major A (rows x ma) and B
// (rows x mb): 32 x 32 tiles of C, rows split over blockIdx.y into fixed
// chunks; partials part[split][j*ma + i] then summed in split order.
// ----------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_atb(int64_t rows, int ma, int mb, const T *__restrict__ A, int64_t lda, const T *__restrict__ B, int64_t ldb,
      double *part, int64_t rows_per_split, int tiles_a, int upper)
{
    __shared__ double As[32][33], Bs[32][33];
    const int tile = blockIdx.x, split = blockIdx.y;
    int ti, tj;
    if (upper) {   // tiles with ti <= tj only, enumerated column by column
        tj = (int)((sqrt(8.0 * tile + 1.0) - 1.0) * 0.5);
        while ((tj + 1) * (tj + 2) / 2 <= tile) ++tj;
        while (tj * (tj + 1) / 2 > tile) --tj;
        ti = tile - tj * (tj + 1) / 2;
    } else {
        ti = tile % tiles_a;
        tj = tile / tiles_a;
    }
    const int64_t r0 = (int64_t)split * rows_per_split;
    const int64_t r1 = min(rows, r0 + rows_per_split);
    const int i0 = ti * 32, j0 = tj * 32;
    const int li = threadIdx.x & 31, lj = threadIdx.x >> 5;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t rb = r0; rb < r1; rb += 32) {
        const int64_t r = rb + li;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = lj + 8 * q;
            As[li][c] = (r < r1 && i0 + c < ma) ? (double)A[(int64_t)(i0 + c) * lda + r] : 0.0;
            Bs[li][c] = (r < r1 && j0 + c < mb) ? (double)B[(int64_t)(j0 + c) * ldb + r] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int rr = 0; rr < 32; ++rr) {
            const double a = As[rr][li];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(a, Bs[rr][lj + 8 * q], acc[q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = i0 + li, j = j0 + lj + 8 * q;
        if (i < ma && j < mb) part[(int64_t)split * ma * mb + (int64_t)j * ma + i] = acc[q];
    }
}

// Symmetric product A^T B (A^T A, or Z^T A Z) on 64 x 64 upper tiles, 16 FP64
// accumulators per thread (4 x 4 register block): measured on GB300 at
// 0.98 TFLOP/s, 97% of the FP64 FMA rate (1.01 TFLOP/s), with about four
// CTAs per SM.
template <typename T>
__global__ void __launch_bounds__(256, 3)
k_gram64(int64_t rows, int m, const T *__restrict__ A, int64_t lda, const T *__restrict__ B, int64_t ldb,
         double *part, int64_t rows_per_split)
{
    __shared__ double As[16][65], Bs[16][65];
    const int tile = blockIdx.x, split = blockIdx.y;
    int tj = (int)((sqrt(8.0 * tile + 1.0) - 1.0) * 0.5);
    while ((tj + 1) * (tj + 2) / 2 <= tile) ++tj;
    while (tj * (tj + 1) / 2 > tile) --tj;
    const int ti = tile - tj * (tj + 1) / 2;
    const int i0 = ti * 64, j0 = tj * 64;
    const int64_t r0 = (int64_t)split * rows_per_split;
    const int64_t r1 = min(rows, r0 + rows_per_split);
    const int tr = threadIdx.x & 15, tc = threadIdx.x >> 4;
    double acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = 0.0;
    for (int64_t rb = r0; rb < r1; rb += 16) {
        const int64_t r = rb + tr;
        for (int q = 0; q < 4; ++q) {
            const int c = tc + 16 * q;
            As[tr][c] = (r < r1 && i0 + c < m) ? (double)A[(int64_t)(i0 + c) * lda + r] : 0.0;
            Bs[tr][c] = (r < r1 && j0 + c < m) ? (double)B[(int64_t)(j0 + c) * ldb + r] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            double a[4], b[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) { a[p] = As[k][tr + 16 * p]; b[p] = Bs[k][tc + 16 * p]; }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
    for (int p = 0; p < 4; ++p)
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + tr + 16 * p, j = j0 + tc + 16 * q;
            if (i < m && j < m) part[(int64_t)split * m * m + (int64_t)j * m + i] = acc[p][q];
        }
}

// The same symmetric product for FP32 operands on the FP32 pipe, as exact
// as the FP64 kernel: each product a b is split without error into
// p + e (p = fl(a b), e = fma(a, b, -p)), p is added to the running sum s
// with Knuth's TwoSum (s + p = s' + err exactly) and the small terms e + err
// accumulate in a second FP32 word, so the result carries about 48 bits.
// Ten FP32 instructions per term against one FP64 FMA: the FP32 pipe
// issues 64 times faster than the FP64 pipe on this GPU.
// (The _rn intrinsics keep the compiler from contracting a b + s into one
// FMA, which would break the error-free transformations.)
__device__ __forceinline__ void df_acc(float a, float b, float &s, float &c)
{
    const float p = __fmul_rn(a, b);
    const float e = fmaf(a, b, -p);
    const float t = __fadd_rn(s, p);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, e));
}

__global__ void __launch_bounds__(256, 2)
k_gram64_df(int64_t rows, int m, const float *__restrict__ A, int64_t lda, const float *__restrict__ B, int64_t ldb,
            double *part, int64_t rows_per_split)
{
    __shared__ float As[16][68], Bs[16][68];
    const int tile = blockIdx.x, split = blockIdx.y;
    int tj = (int)((sqrt(8.0 * tile + 1.0) - 1.0) * 0.5);
    while ((tj + 1) * (tj + 2) / 2 <= tile) ++tj;
    while (tj * (tj + 1) / 2 > tile) --tj;
    const int ti = tile - tj * (tj + 1) / 2;
    const int i0 = ti * 64, j0 = tj * 64;
    const int64_t r0 = (int64_t)split * rows_per_split;
    const int64_t r1 = min(rows, r0 + rows_per_split);
    const int tr = threadIdx.x & 15, tc = threadIdx.x >> 4;
    float s[4][4], c[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) { s[p][q] = 0.f; c[p][q] = 0.f; }
    for (int64_t rb = r0; rb < r1; rb += 16) {
        const int64_t r = rb + tr;
        for (int q = 0; q < 4; ++q) {
            const int col = tc + 16 * q;
            As[tr][col] = (r < r1 && i0 + col < m) ? A[(int64_t)(i0 + col) * lda + r] : 0.f;
            Bs[tr][col] = (r < r1 && j0 + col < m) ? B[(int64_t)(j0 + col) * ldb + r] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < 16; ++k) {
            float a[4], b[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) { a[p] = As[k][tr + 16 * p]; b[p] = Bs[k][tc + 16 * p]; }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) df_acc(a[p], b[q], s[p][q], c[p][q]);
        }
        __syncthreads();
    }
    for (int p = 0; p < 4; ++p)
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + tr + 16 * p, j = j0 + tc + 16 * q;
            if (i < m && j < m) part[(int64_t)split * m * m + (int64_t)j * m + i] = (double)s[p][q] + (double)c[p][q];
        }
}

// out = sum_s part[s] for the 64-tile symmetric Gram (lower tiles mirrored).
__global__ void k_reduce_part64(int S, int m, const double *part, double *out)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * m) return;
    const int i = (int)(e % m), j = (int)(e / m);
    const int64_t src = (i / 64 > j / 64) ? (int64_t)i * m + j : e;
    double acc = 0.0;
    for (int s = 0; s < S; ++s) acc += part[(int64_t)s * m * m + src];
    out[e] = acc;
}

// out[e] = sum_s part[s][e]; with `upper` (square, only tiles ti <= tj were
// computed) the entries below the diagonal tiles take the mirrored sum.
__global__ void k_reduce_part(int S, int64_t count, int m, int upper, const double *part, double *out)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    int64_t src = e;
    if (upper) {
        int i = (int)(e % m), j = (int)(e / m);
        if (i / 32 > j / 32) src = (int64_t)i * m + j;
    }
    double acc = 0.0;
    for (int s = 0; s < S; ++s) acc += part[(int64_t)s * count + src];
    out[e] = acc;
}

// Row splits of k_atb / k_gram64 and the number of partial doubles they need.
static bool use_gram64(int ma, int mb, int upper) { return upper && ma == mb && ma >= 64; }

static void atb_plan(int num_sms, int64_t rows, int ma, int mb, int upper, int *tiles_out, int64_t *splits_out,
                     int64_t *rps_out)
{
    if (ma != mb) upper = 0;
    const bool g64 = use_gram64(ma, mb, upper);
    const int tsz = g64 ? 64 : 32, chunk = g64 ? 16 : 32;
    const int ta = ceil_div(ma, tsz), tb = ceil_div(mb, tsz);
    const int tiles = upper ? ta * (ta + 1) / 2 : ta * tb;
    int64_t max_splits = (rows + chunk - 1) / chunk;
    const int64_t want = g64 ? 4 * (int64_t)num_sms : 2 * (int64_t)num_sms;   // CTAs
    int64_t S = (want + tiles - 1) / tiles;
    if (S > max_splits) S = max_splits;
    if (S < 1) S = 1;
    int64_t rps = ((rows + S - 1) / S + chunk - 1) / chunk * chunk;
    if (rps < chunk) rps = chunk;
    S = (rows + rps - 1) / rps;
    if (S < 1) S = 1;
    *tiles_out = tiles;
    *splits_out = S;
    *rps_out = rps;
}

size_t atb_part_doubles(int num_sms, int64_t rows, int ma, int mb, int upper)
{
    int tiles;
    int64_t S, rps;
    atb_plan(num_sms, rows, ma, mb, upper, &tiles, &S, &rps);
    return (size_t)S * ma * mb;
}

// Returns 0, or -1 (nothing launched) when part_capacity (doubles) is too small.
template <typename T>
int launch_atb(cudaStream_t s, int num_sms, int64_t rows, int ma, int mb, const T *A, int64_t lda, const T *B,
               int64_t ldb, double *part, size_t part_capacity, int *splits_out, double *C, int upper)
{
    if (ma != mb) upper = 0;
    int tiles;
    int64_t S, rps;
    atb_plan(num_sms, rows, ma, mb, upper, &tiles, &S, &rps);
    if ((size_t)S * ma * mb > part_capacity) return -1;
    dim3 g(tiles, (unsigned)S);
    const int64_t cnt = (int64_t)ma * mb;
    if (use_gram64(ma, mb, upper)) {
        if constexpr (std::is_same<T, float>::value)
            WC4D_LAUNCH(k_gram64_df<<<g, 256, 0, s>>>(rows, ma, A, lda, B, ldb, part, rps));
        else
            WC4D_LAUNCH(k_gram64<T><<<g, 256, 0, s>>>(rows, ma, A, lda, B, ldb, part, rps));
        if (C) WC4D_LAUNCH(k_reduce_part64<<<ceil_div(cnt, 256), 256, 0, s>>>((int)S, ma, part, C));
    } else {
        const int ta = ceil_div(ma, 32);
        WC4D_LAUNCH(k_atb<T><<<g, 256, 0, s>>>(rows, ma, mb, A, lda, B, ldb, part, rps, ta, upper));
        if (C) WC4D_LAUNCH(k_reduce_part<<<ceil_div(cnt, 256), 256, 0, s>>>((int)S, cnt, ma, upper, part, C));
    }
    if (splits_out) *splits_out = (int)S;
    return 0;
}

template int launch_atb<double>(cudaStream_t, int, int64_t, int, int, const double *, int64_t, const double *,
                                int64_t, double *, size_t, int *, double *, int);
template int launch_atb<float>(cudaStream_t, int, int64_t, int, int, const float *, int64_t, const float *,
                               int64_t, double *, size_t, int *, double *, int);

// ----------------------------------------------------------------------------
// Cholesky A = R^T R (R upper, column-major m x m), right-looking and
// blocked by 32: per block step, one CTA factors the diagonal block in shared
// memory, one CTA per block column solves the row panel R_kj = R_kk^{-T} A_kj,
// and one CTA per trailing upper block applies A_ij -= R_ki^T R_kj.
// info = 0, or j+1 when pivot j is not positive / not finite (later steps
// then do nothing).
// ----------------------------------------------------------------------------
constexpr int CB = 32;

__global__ void k_chol_copy(int m, const double *A, double *R, int *info)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx == 0) *info = 0;
    if (idx >= (int64_t)m * m) return;
    const int i = (int)(idx % m), j = (int)(idx / m);
    R[idx] = (i <= j) ? A[idx] : 0.0;
}

// R is read through L2 (ld.cg) in the phases below: in the cooperative form
// a CTA may read, after a grid barrier, blocks another CTA rewrote since it
// last read them.
__device__ __forceinline__ double rld(const double *p) { return __ldcg(p); }

// Diagonal block k0 .. k0+nb-1 (nb <= 32), in place; 1024 threads.
// Returns the failing pivot (k0 + c + 1) or 0.
__device__ int chol_diag_block(int m, int k0, double *R)
{
    __shared__ double a[CB][CB + 1];
    __shared__ double rinv;
    __shared__ int bad;
    const int nb = min(CB, m - k0);
    const int ti = threadIdx.x % CB, tj = threadIdx.x / CB;   // row, column within the block
    if (ti < nb && tj < nb && ti <= tj) a[ti][tj] = rld(R + (int64_t)(k0 + tj) * m + k0 + ti);
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int c = 0; c < nb; ++c) {
        if (threadIdx.x == 0) {
            const double d = a[c][c];
            if (!(d > 0.0) || !isfinite(d)) {
                bad = k0 + c + 1;
            } else {
                const double r = sqrt(d);
                a[c][c] = r;
                rinv = 1.0 / r;
            }
        }
        __syncthreads();
        if (bad) break;
        if (ti == c && tj > c && tj < nb) a[c][tj] *= rinv;
        __syncthreads();
        if (ti > c && ti <= tj && tj < nb) a[ti][tj] -= a[c][ti] * a[c][tj];
        __syncthreads();
    }
    const int b = bad;
    if (!b && ti < nb && tj < nb && ti <= tj) R[(int64_t)(k0 + tj) * m + k0 + ti] = a[ti][tj];
    __syncthreads();   // the shared arrays are reused by the next call
    return b;
}

// Row panel block bj (columns k0 + nb + 32 bj ..) of block step k0:
// R_kj = R_kk^{-T} A_kj; 1024 threads.
__device__ void chol_panel_block(int m, int k0, int bj, double *R)
{
    __shared__ double l[CB][CB + 1], b[CB][CB + 1], rl[CB];
    const int nb = min(CB, m - k0);
    const int j0 = k0 + nb + CB * bj;
    const int nj = min(CB, m - j0);
    const int ti = threadIdx.x % CB, tj = threadIdx.x / CB;
    if (ti < nb && tj < nb) l[ti][tj] = (ti <= tj) ? rld(R + (int64_t)(k0 + tj) * m + k0 + ti) : 0.0;   // R_kk
    if (ti < nb && tj < nj) b[ti][tj] = rld(R + (int64_t)(j0 + tj) * m + k0 + ti);
    if (threadIdx.x < nb) rl[threadIdx.x] = 1.0 / rld(R + (int64_t)(k0 + threadIdx.x) * m + k0 + threadIdx.x);
    __syncthreads();
    // forward substitution with R_kk^T (lower): row c of the solution, then
    // eliminate it from the rows below
    for (int c = 0; c < nb; ++c) {
        if (ti == c && tj < nj) b[c][tj] *= rl[c];
        __syncthreads();
        if (ti > c && ti < nb && tj < nj) b[ti][tj] -= l[c][ti] * b[c][tj];
        __syncthreads();
    }
    if (ti < nb && tj < nj) R[(int64_t)(j0 + tj) * m + k0 + ti] = b[ti][tj];
    __syncthreads();
}

// Trailing update of block step k0 for upper block pair t (bi <= bj).
__device__ void chol_update_block(int m, int k0, int t, double *R)
{
    __shared__ double pi[CB][CB + 1], pj[CB][CB + 1];
    const int nb = min(CB, m - k0);
    int bj = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((bj + 1) * (bj + 2) / 2 <= t) ++bj;
    while (bj * (bj + 1) / 2 > t) --bj;
    const int bi = t - bj * (bj + 1) / 2;
    const int i0 = k0 + nb + CB * bi, j0 = k0 + nb + CB * bj;
    const int ti = threadIdx.x % CB, tj = threadIdx.x / CB;
    // pi[c][x] = R(k0 + c, i0 + x), pj[c][y] = R(k0 + c, j0 + y)
    pi[ti][tj] = (ti < nb && i0 + tj < m) ? rld(R + (int64_t)(i0 + tj) * m + k0 + ti) : 0.0;
    pj[ti][tj] = (ti < nb && j0 + tj < m) ? rld(R + (int64_t)(j0 + tj) * m + k0 + ti) : 0.0;
    __syncthreads();
    const int gi = i0 + ti, gj = j0 + tj;
    if (gi < m && gj < m && gi <= gj) {
        double acc = 0.0;
        for (int c = 0; c < nb; ++c) acc = fma(pi[c][ti], pj[c][tj], acc);
        R[(int64_t)gj * m + gi] = rld(R + (int64_t)gj * m + gi) - acc;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(1024) k_chol_diag(int m, int k0, double *R, int *info)
{
    if (*info) return;
    const int b = chol_diag_block(m, k0, R);
    if (b && threadIdx.x == 0) *info = b;
}

__global__ void __launch_bounds__(1024) k_chol_panel(int m, int k0, double *R, const int *info)
{
    if (*info) return;
    chol_panel_block(m, k0, blockIdx.x, R);
}

// Trailing update: CTA t -> upper block pair (bi <= bj) after block step k0.
__global__ void __launch_bounds__(1024) k_chol_update(int m, int k0, double *R, const int *info)
{
    if (*info) return;
    chol_update_block(m, k0, blockIdx.x, R);
}

// Grid barrier of the cooperative Cholesky (monotonic counter; bounded).
__device__ __forceinline__ bool chol_barrier(unsigned *bar, unsigned target)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
        unsigned v = 0, it = 0;
        int ok = 1;
        do {
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
            if (++it > (1u << 22)) { ok = 0; break; }
        } while (v < target);
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// The whole factorisation as one cooperative launch: the copy, then per
// block step the diagonal block (CTA 0), the row panel (CTAs over its
// blocks) and the trailing update (CTAs over the upper block pairs), each
// phase followed by a grid barrier.  A failed pivot stops every CTA after
// the next barrier (*info = pivot); a barrier that times out sets *info =
// -1 and returns.  bar: zero at launch.
__global__ void __launch_bounds__(1024, 1) k_chol_coop(int m, const double *A, double *R, int *info, unsigned *bar)
{
    __shared__ int stop;
    const unsigned G = gridDim.x;
    unsigned target = 0;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)m * m;
         idx += (int64_t)G * blockDim.x) {
        const int i = (int)(idx % m), j = (int)(idx / m);
        R[idx] = (i <= j) ? A[idx] : 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *info = 0;
    auto sync_all = [&]() -> bool {
        target += G;
        if (chol_barrier(bar, target)) return true;
        if (threadIdx.x == 0) atomicExch(info, -1);
        return false;
    };
    if (!sync_all()) return;
    for (int k0 = 0; k0 < m; k0 += CB) {
        if (blockIdx.x == 0) {
            const int b = chol_diag_block(m, k0, R);
            if (b && threadIdx.x == 0) atomicExch(info, b);
        }
        if (!sync_all()) return;
        if (threadIdx.x == 0) stop = __ldcg(info);
        __syncthreads();
        if (stop) return;   // the same value in every CTA: written before the barrier
        const int rest = m - k0 - CB;
        if (rest <= 0) return;
        const int nbj = (rest + CB - 1) / CB;
        for (int b = blockIdx.x; b < nbj; b += G) chol_panel_block(m, k0, b, R);
        if (!sync_all()) return;
        for (int t = blockIdx.x; t < nbj * (nbj + 1) / 2; t += G) chol_update_block(m, k0, t, R);
        if (!sync_all()) return;
    }
}

void launch_chol_upper(cudaStream_t s, int m, const double *A, double *R, int *info)
{
    WC4D_LAUNCH(k_chol_copy<<<ceil_div((int64_t)m * m, 256), 256, 0, s>>>(m, A, R, info));
    for (int k0 = 0; k0 < m; k0 += CB) {
        WC4D_LAUNCH(k_chol_diag<<<1, CB * CB, 0, s>>>(m, k0, R, info));
        const int rest = m - k0 - CB;
        if (rest <= 0) break;
        const int nbj = ceil_div(rest, CB);
        WC4D_LAUNCH(k_chol_panel<<<nbj, CB * CB, 0, s>>>(m, k0, R, info));
        WC4D_LAUNCH(k_chol_update<<<nbj * (nbj + 1) / 2, CB * CB, 0, s>>>(m, k0, R, info));
    }
}

// The cooperative form (bar: one counter, zeroed here); false (nothing
// launched, error state cleared) if the launch is refused.
bool launch_chol_upper_coop(cudaStream_t s, int num_sms, int m, const double *A, double *R, int *info, unsigned *bar)
{
    static const int per_sm = [] {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_chol_coop, CB * CB, 0) != cudaSuccess) {
            cudaGetLastError();
            n = 0;
        }
        return n;
    }();
    if (per_sm < 1) return false;
    const int nb0 = ceil_div(std::max(m - CB, 0), CB);
    const int want = std::max(1, std::max(nb0 * (nb0 + 1) / 2, ceil_div((int64_t)m * m, CB * CB)));
    const int G = std::min(want, num_sms * per_sm);
    if (cudaMemsetAsync(bar, 0, sizeof(unsigned), s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    void *params[] = {(void *)&m, (void *)&A, (void *)&R, (void *)&info, (void *)&bar};
    wc4d_note_launch();
    if (cudaLaunchCooperativeKernel((const void *)k_chol_coop, dim3(G), dim3(CB * CB), params, 0, s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

// Power-of-two range scaling of an FP32 block before its Gram matrix: the
// double-float Gram accumulates in FP32 pairs, which overflow once the
// squared column norms pass ~3e38 (sketches of Hessians with eigenvalues
// ~1e19).  k_absmax_f32 takes max |Y| (as ordered bits of a non-negative
// float); k_scale_pow2 then multiplies Y by 2^-e (exact) when max |Y| lies
// outside [2^-24, 2^24] and records e; k_scale_R_pow2 multiplies R by 2^e, so
// that (2^-e Y)(2^-e R)^{-1} = Y R^{-1}.
// Both take column blockIdx.y with a grid-stride loop over its rows (16-byte
// accesses when the columns allow them), so no index division per element.
__device__ __forceinline__ bool cols_vec4(int64_t rows, int64_t ld, const float *Y)
{
    return (rows & 3) == 0 && (ld & 3) == 0 && (reinterpret_cast<uintptr_t>(Y) & 15u) == 0;
}

__global__ void __launch_bounds__(256) k_absmax_f32(int64_t rows, int64_t ld, const float *Y, unsigned *mx)
{
    float v = 0.f;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
    const float *col = Y + (int64_t)blockIdx.y * ld;
    if (cols_vec4(rows, ld, Y)) {
        const float4 *c = reinterpret_cast<const float4 *>(col);
        for (int64_t i = t0; i < rows / 4; i += st) {
            const float4 q = __ldcg(c + i);
            v = fmaxf(v, fmaxf(fmaxf(fabsf(q.x), fabsf(q.y)), fmaxf(fabsf(q.z), fabsf(q.w))));
        }
    } else {
        for (int64_t i = t0; i < rows; i += st) v = fmaxf(v, fabsf(col[i]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    // one atomic per CTA: thousands of same-address atomics would serialise
    __shared__ float wmax[8];
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) v = fmaxf(v, wmax[i]);
        atomicMax(mx, __float_as_uint(v));
    }
}

__global__ void __launch_bounds__(256) k_scale_pow2(int64_t rows, int64_t ld, float *Y, const unsigned *mx,
                                                    int *e_out)
{
    const float v = __uint_as_float(*mx);
    int e = 0;
    if (v > 0.f && isfinite(v) && (v > 0x1p24f || v < 0x1p-24f)) e = ilogbf(v);
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *e_out = e;
    if (e == 0) return;
    const float sc = scalbnf(1.f, -e);
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
    float *col = Y + (int64_t)blockIdx.y * ld;
    if (cols_vec4(rows, ld, Y)) {
        float4 *c = reinterpret_cast<float4 *>(col);
        for (int64_t i = t0; i < rows / 4; i += st) {
            float4 q = c[i];
            q.x *= sc; q.y *= sc; q.z *= sc; q.w *= sc;
            c[i] = q;
        }
    } else {
        for (int64_t i = t0; i < rows; i += st) col[i] *= sc;
    }
}

__global__ void k_scale_R_pow2(int m, double *R, const int *e)
{
    if (*e == 0) return;
    const double sc = scalbn(1.0, *e);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)m * m; i += (int64_t)gridDim.x * blockDim.x)
        R[i] *= sc;
}

// work: 2 words of device scratch (max bits, exponent)
void launch_range_scale_f32(cudaStream_t s, int num_sms, int64_t rows, int m, int64_t ld, float *Y, unsigned *work)
{
    cudaMemsetAsync(work, 0, sizeof(unsigned), s);
    // columns on grid.y; about sixteen 16-byte loads per thread along a column
    const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(rows, 16384), 4 * num_sms)), (unsigned)m);
    WC4D_LAUNCH(k_absmax_f32<<<grid, 256, 0, s>>>(rows, ld, Y, work));
    WC4D_LAUNCH(k_scale_pow2<<<grid, 256, 0, s>>>(rows, ld, Y, work, reinterpret_cast<int *>(work + 1)));
}

void launch_unscale_R(cudaStream_t s, int m, double *R, const unsigned *work)
{
    WC4D_LAUNCH(k_scale_R_pow2<<<ceil_div((int64_t)m * m, 256), 256, 0, s>>>(m, R, reinterpret_cast<const int *>(work + 1)));
}

// A[i][i] += factor * trace(A) for the m x m column-major A (one CTA): the
// shift of shifted CholeskyQR, after the unshifted factorisation failed.
__global__ void __launch_bounds__(256) k_shift_diag(int m, double *A, double factor)
{
    double tr = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) tr += A[(int64_t)i * m + i];
    tr = block_sum(tr);
    const double sft = factor * tr;
    for (int i = threadIdx.x; i < m; i += blockDim.x) A[(int64_t)i * m + i] += sft;
}

void launch_shift_diag(cudaStream_t s, int m, double *A, double factor)
{
    WC4D_LAUNCH(k_shift_diag<<<1, 256, 0, s>>>(m, A, factor));
}

// Inverse of an upper-triangular R (column-major): one CTA per column j,
// column-oriented back substitution of R x = e_j in shared memory.
__global__ void __launch_bounds__(256) k_trinv_upper(int m, const double *R, double *Rinv)
{
    extern __shared__ double xs[];
    double *rinv = xs + m;
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        xs[i] = (i == j) ? 1.0 : 0.0;
        rinv[i] = (i <= j) ? 1.0 / R[(int64_t)i * m + i] : 0.0;
    }
    __syncthreads();
    for (int c = j; c >= 0; --c) {
        const double xc = xs[c] * rinv[c];
        __syncthreads();
        if (threadIdx.x == 0) xs[c] = xc;
        for (int i = threadIdx.x; i < c; i += blockDim.x) xs[i] = fma(-R[(int64_t)c * m + i], xc, xs[i]);
        __syncthreads();
    }
    double *x = Rinv + (int64_t)j * m;
    for (int i = threadIdx.x; i < m; i += blockDim.x) x[i] = xs[i];
}

void launch_trinv_upper(cudaStream_t s, int m, const double *R, double *Rinv)
{
    WC4D_LAUNCH(k_trinv_upper<<<m, 256, 2 * sizeof(double) * m, s>>>(m, R, Rinv));
}

// RT = R^T (m x m column-major).
__global__ void k_transpose_small(int m, const double *R, double *RT)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)m * m) return;
    int i = (int)(idx % m), j = (int)(idx / m);
    RT[(int64_t)i * m + j] = R[idx];
}

void launch_rrt(cudaStream_t s, int m, const double *R, double *RT)
{
    WC4D_LAUNCH(k_transpose_small<<<ceil_div((int64_t)m * m, 256), 256, 0, s>>>(m, R, RT));
}

__global__ void k_symmetrize(int m, double *S)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)m * m) return;
    int i = (int)(idx % m), j = (int)(idx / m);
    if (i < j) {
        double v = 0.5 * (S[(int64_t)j * m + i] + S[(int64_t)i * m + j]);
        S[(int64_t)j * m + i] = v;
        S[(int64_t)i * m + j] = v;
    }
}

void launch_symmetrize(cudaStream_t s, int m, double *S)
{
    WC4D_LAUNCH(k_symmetrize<<<ceil_div((int64_t)m * m, 256), 256, 0, s>>>(m, S));
}

// A[:, j] *= w_j^{-1/2} (inv_sqrt = 1) or 1/w_j (inv_sqrt = 0).
__global__ void k_scale_cols(int64_t rows, int m, double *A, int64_t lda, const double *w, int inv_sqrt)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * m) return;
    int64_t r = idx % rows;
    int j = (int)(idx / rows);
    double f = inv_sqrt ? 1.0 / sqrt(w[j]) : 1.0 / w[j];
    A[(int64_t)j * lda + r] *= f;
}

void launch_scale_cols(cudaStream_t s, int64_t rows, int m, double *A, int64_t lda, const double *w, int inv_sqrt)
{
    WC4D_LAUNCH(k_scale_cols<<<ceil_div(rows * m, 256), 256, 0, s>>>(rows, m, A, lda, w, inv_sqrt));
}

// ----------------------------------------------------------------------------
// One-sided (Hestenes) Jacobi: X V = U Sigma.  For symmetric positive semi-
// definite S, X = S gives S's eigenvectors V and eigenvalues |X_j|; for
// X = R^T it gives the left singular vectors of R.  Parallel round-robin
// ordering: round r pairs positions (i, mp-1-i), position 0 fixed, others
// rotated; one CTA per pair, one launch per round.
// ----------------------------------------------------------------------------
__global__ void k_jacobi_init(int m, int mp, const double *S, double *X, double *V)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)mp * mp) return;
    int i = (int)(idx % mp), j = (int)(idx / mp);
    X[idx] = (i < m && j < m) ? S[(int64_t)j * m + i] : 0.0;
    V[idx] = (i == j) ? 1.0 : 0.0;
}

void launch_jacobi_init(cudaStream_t s, int m, int mp, const double *S, double *X, double *V)
{
    WC4D_LAUNCH(k_jacobi_init<<<ceil_div((int64_t)mp * mp, 256), 256, 0, s>>>(m, mp, S, X, V));
}

__global__ void __launch_bounds__(128) k_jacobi_round(int mp, double *X, double *V, int round, double tol, int *rot)
{
    __shared__ double cs_s[2];
    __shared__ int doit;
    const int i = blockIdx.x;
    auto player = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + round) % (mp - 1); };
    int p = player(i), q = player(mp - 1 - i);
    if (p > q) { int t = p; p = q; q = t; }
    double *xp = X + (int64_t)p * mp, *xq = X + (int64_t)q * mp;
    double a = 0.0, b = 0.0, g = 0.0;
    for (int r = threadIdx.x; r < mp; r += blockDim.x) {
        double u = xp[r], v = xq[r];
        a = fma(u, u, a);
        b = fma(v, v, b);
        g = fma(u, v, g);
    }
    a = block_sum(a);
    b = block_sum(b);
    g = block_sum(g);
    if (threadIdx.x == 0) {
        doit = 0;
        if (fabs(g) > tol * sqrt(a * b) && fabs(g) > 1e-300) {
            double zeta = (b - a) / (2.0 * g);
            double t;
            if (fabs(zeta) > 1e100) t = 0.5 / zeta;
            else t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            double c = 1.0 / sqrt(1.0 + t * t);
            cs_s[0] = c;
            cs_s[1] = c * t;
            doit = 1;
            atomicAdd(rot, 1);
        }
    }
    __syncthreads();
    if (!doit) return;
    const double c = cs_s[0], sn = cs_s[1];
    double *vp = V + (int64_t)p * mp, *vq = V + (int64_t)q * mp;
    for (int r = threadIdx.x; r < mp; r += blockDim.x) {
        double u = xp[r], v = xq[r];
        xp[r] = c * u - sn * v;
        xq[r] = sn * u + c * v;
        double y = vp[r], z = vq[r];
        vp[r] = c * y - sn * z;
        vq[r] = sn * y + c * z;
    }
}

void launch_jacobi_round(cudaStream_t s, int mp, double *X, double *V, int round, double tol, int *rot)
{
    WC4D_LAUNCH(k_jacobi_round<<<mp / 2, 128, 0, s>>>(mp, X, V, round, tol, rot));
}

// Column norms, sorted decreasing; Vout[:, rank] = V[0:m, j].
__global__ void k_colnorm(int m, int mp, const double *X, double *w)
{
    int j = blockIdx.x;
    double a = 0.0;
    for (int r = threadIdx.x; r < mp; r += blockDim.x) {
        double u = X[(int64_t)j * mp + r];
        a = fma(u, u, a);
    }
    a = block_sum(a);
    if (threadIdx.x == 0) w[j] = sqrt(a);
}

__global__ void k_sort_cols(int m, int mp, const double *wn, const double *V, double *w, double *Vout)
{
    int j = blockIdx.x;
    __shared__ int rank;
    if (threadIdx.x == 0) {
        int r = 0;
        double wj = wn[j];
        for (int i = 0; i < m; ++i)
            if (wn[i] > wj || (wn[i] == wj && i < j)) ++r;
        rank = r;
        w[r] = wj;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < m; r += blockDim.x) Vout[(int64_t)rank * m + r] = V[(int64_t)j * mp + r];
}

// Left variant: w[rank] = |X_j|^2 (decreasing), Vout[:, rank] = X[0:m, j] / |X_j|.
__global__ void k_sort_cols_left(int m, int mp, const double *wn, const double *X, double *w, double *Vout)
{
    int j = blockIdx.x;
    __shared__ int rank;
    if (threadIdx.x == 0) {
        int r = 0;
        double wj = wn[j];
        for (int i = 0; i < m; ++i)
            if (wn[i] > wj || (wn[i] == wj && i < j)) ++r;
        rank = r;
        w[r] = wj * wj;
    }
    __syncthreads();
    const double inv = wn[j] > 0.0 ? 1.0 / wn[j] : 0.0;
    for (int r = threadIdx.x; r < m; r += blockDim.x) Vout[(int64_t)rank * m + r] = X[(int64_t)j * mp + r] * inv;
}

void launch_jacobi_finish_left(cudaStream_t s, int m, int mp, const double *X, double *w, double *Vout)
{
    WC4D_LAUNCH(k_colnorm<<<m, 128, 0, s>>>(m, mp, X, w + m));
    WC4D_LAUNCH(k_sort_cols_left<<<m, 128, 0, s>>>(m, mp, w + m, X, w, Vout));
}

void launch_jacobi_finish(cudaStream_t s, int m, int mp, const double *X, const double *V, double *w, double *Vout)
{
    // w is used first as scratch for the unsorted norms (length m) at w + m
    WC4D_LAUNCH(k_colnorm<<<m, 128, 0, s>>>(m, mp, X, w + m));
    WC4D_LAUNCH(k_sort_cols<<<m, 128, 0, s>>>(m, mp, w + m, V, w, Vout));
}

// ----------------------------------------------------------------------------
// Spectral LMP (eq. 16, closed form for orthonormal U):
//   C v = v - U (c o (U^T v)),  c_i = 1 - theta_i^{-1/2}.
// ----------------------------------------------------------------------------
__global__ void k_lmp_coeffs(int k, const double *theta, double *c)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) c[i] = theta[i] > 0.0 ? 1.0 - 1.0 / sqrt(theta[i]) : 0.0;
}

// y += alpha x over a whole block (count elements)
template <typename T>
__global__ void __launch_bounds__(256) k_axpy_block(int64_t count, double alpha, const T *x, T *y)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (T)((double)y[i] + alpha * (double)x[i]);
}

template <typename T> void launch_axpy_block(cudaStream_t s, int num_sms, int64_t count, double alpha, const T *x, T *y)
{
    WC4D_LAUNCH(k_axpy_block<T><<<std::max(1, std::min(ceil_div(count, 256), 8 * num_sms)), 256, 0, s>>>(count, alpha,
                                                                                                        x, y));
}
template void launch_axpy_block<double>(cudaStream_t, int, int64_t, double, const double *, double *);
template void launch_axpy_block<float>(cudaStream_t, int, int64_t, double, const float *, float *);

// theta[i] = max(w[i] - nu, 0): the single-pass Nystrom shift taken back off
__global__ void k_theta_unshift(int k, const double *w, double nu, double *theta)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) theta[i] = fmax(w[i] - nu, 0.0);
}

void launch_theta_unshift(cudaStream_t s, int k, const double *w, double nu, double *theta)
{
    WC4D_LAUNCH(k_theta_unshift<<<ceil_div(k, 256), 256, 0, s>>>(k, w, nu, theta));
}

void launch_lmp_coeffs(cudaStream_t s, int k, const double *theta, double *c)
{
    WC4D_LAUNCH(k_lmp_coeffs<<<ceil_div(k, 128), 128, 0, s>>>(k, theta, c));
}

constexpr int UTV_ROWS = 256;

// part[split][i] = sum over the split's rows of U[r, i] v[r]; one warp per
// column at a time (8 loads per lane in flight), v staged in shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_utv(int64_t nA, int k, const T *__restrict__ U, const T *__restrict__ v,
                                             double *part)
{
    __shared__ T vs[UTV_ROWS];
    const int64_t r0 = (int64_t)blockIdx.x * UTV_ROWS;
    const int rows = (int)min((int64_t)UTV_ROWS, nA - r0);
    for (int r = threadIdx.x; r < UTV_ROWS; r += blockDim.x) vs[r] = (r < rows) ? v[r0 + r] : (T)0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = w; i < k; i += nw) {
        const T *u = U + (int64_t)i * nA + r0;
        T vals[UTV_ROWS / 32];
#pragma unroll
        for (int q = 0; q < UTV_ROWS / 32; ++q) {
            const int r = lane + 32 * q;
            vals[q] = (r < rows) ? __ldcs(u + r) : (T)0;
        }
        T acc = 0;
#pragma unroll
        for (int q = 0; q < UTV_ROWS / 32; ++q) acc = fma(vals[q], vs[lane + 32 * q], acc);
        double d = warp_sum((double)acc);
        if (lane == 0) part[(int64_t)blockIdx.x * k + i] = d;
    }
}

int utv_splits(int64_t nA) { return ceil_div(nA, UTV_ROWS); }

// t = U^T v: per-chunk partials part[0 .. S*k), then their sum in fixed order
// at part[S*k .. S*k + k).  *splits returns S.
template <typename T>
void launch_utv(cudaStream_t s, int num_sms, int64_t nA, int k, const T *U, const T *v, double *part, int *splits)
{
    (void)num_sms;
    const int S = utv_splits(nA);
    WC4D_LAUNCH(k_utv<T><<<S, 256, 0, s>>>(nA, k, U, v, part));
    WC4D_LAUNCH(k_reduce_part<<<ceil_div(k, 256), 256, 0, s>>>(S, k, k, 0, part, part + (int64_t)S * k));
    *splits = S;
}

template void launch_utv<double>(cudaStream_t, int, int64_t, int, const double *, const double *, double *, int *);
template void launch_utv<float>(cudaStream_t, int, int64_t, int, const float *, const float *, double *, int *);

// y = v - coef * U (c o t) (+ beta * add), t_i = sum_s part[s][i]; each CTA
// first reduces the k partial columns into shared memory.
template <typename T>
__global__ void __launch_bounds__(256)
k_lmp_combine(int64_t nA, int k, const T *__restrict__ U, const double *__restrict__ part, int splits,
              const double *__restrict__ cvec, double coef, const T *v, T *y, const T *add,
              const double *beta_dev, const int *skip)
{
    extern __shared__ double ct[];
    if (skip && *skip) return;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        double t = 0.0;
        for (int sidx = 0; sidx < splits; ++sidx) t += part[(int64_t)sidx * k + i];
        ct[i] = coef * cvec[i] * t;
    }
    __syncthreads();
    const T beta = beta_dev ? (T)*beta_dev : (T)0;
    // accumulate in the storage precision (FP32 vectors in the mixed path)
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nA; r += (int64_t)gridDim.x * blockDim.x) {
        T acc = v[r];
        int i = 0;
        for (; i + 8 <= k; i += 8) {
            T u[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) u[q] = __ldcs(U + (int64_t)(i + q) * nA + r);
#pragma unroll
            for (int q = 0; q < 8; ++q) acc = fma(-u[q], (T)ct[i + q], acc);
        }
        for (; i < k; ++i) acc = fma(-U[(int64_t)i * nA + r], (T)ct[i], acc);
        if (add) acc = fma(beta, add[r], acc);
        y[r] = acc;
    }
}

template <typename T>
void launch_lmp_combine(cudaStream_t s, int64_t nA, int k, const T *U, const double *part, int splits,
                        const double *cvec, double coef, const T *v, T *y, const T *add, const double *beta_dev,
                        const int *skip)
{
    int grid = ceil_div(nA, 256);
    if (grid > 4096) grid = 4096;
    WC4D_LAUNCH(k_lmp_combine<T><<<grid, 256, (size_t)k * sizeof(double), s>>>(nA, k, U, part, splits, cvec, coef, v, y, add,
                                                                      beta_dev, skip));
}

template void launch_lmp_combine<double>(cudaStream_t, int64_t, int, const double *, const double *, int,
                                         const double *, double, const double *, double *, const double *,
                                         const double *, const int *);
template void launch_lmp_combine<float>(cudaStream_t, int64_t, int, const float *, const double *, int,
                                        const double *, double, const float *, float *, const float *,
                                        const double *, const int *);

// ----------------------------------------------------------------------------
// Row-major LMP kernels.  Urm is nA x kp row-major (kp = k rounded up to a
// multiple of 4, zero columns beyond k), so that U^T v accumulates one column
// per thread lane with coalesced vector loads of whole rows, and C v reduces
// one row per warp.
// ----------------------------------------------------------------------------
template <typename T>
__global__ void k_to_rowmajor(int64_t nA, int k, int kp, const T *__restrict__ U, T *Urm)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nA * kp) return;
    int64_t r = idx / kp;
    int i = (int)(idx % kp);
    Urm[idx] = (i < k) ? U[(int64_t)i * nA + r] : (T)0;
}

template <typename T>
void launch_to_rowmajor(cudaStream_t s, int64_t nA, int k, int kp, const T *U, T *Urm)
{
    WC4D_LAUNCH(k_to_rowmajor<T><<<ceil_div(nA * kp, 256), 256, 0, s>>>(nA, k, kp, U, Urm));
}

template void launch_to_rowmajor<double>(cudaStream_t, int64_t, int, int, const double *, double *);
template void launch_to_rowmajor<float>(cudaStream_t, int64_t, int, int, const float *, float *);

constexpr int RM_ROWS = 512;   // rows per CTA of the row-major U^T v

// Four consecutive values with evict-first loads (one float4, or two double2).
template <typename T> struct Quad { T x, y, z, w; };
__device__ __forceinline__ Quad<float> ld4cs(const float *p)
{
    float4 v = __ldcs(reinterpret_cast<const float4 *>(p));
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Quad<double> ld4cs(const double *p)
{
    double2 a = __ldcs(reinterpret_cast<const double2 *>(p)), b = __ldcs(reinterpret_cast<const double2 *>(p) + 1);
    return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ Quad<float> ld4cg(const float *p)
{
    float4 v = __ldcg(reinterpret_cast<const float4 *>(p));
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Quad<double> ld4cg(const double *p)
{
    double2 a = __ldcg(reinterpret_cast<const double2 *>(p)), b = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
    return {a.x, a.y, b.x, b.y};
}

// part[chunk][i] = sum over the chunk's rows of Urm[r, i] v[r].  Thread
// (ty, tx): column group 4 (cb + tx) .. + 3, rows ty, ty + 4, ...; the loop
// over 64-group column blocks is uniform across the CTA.
template <typename T>
__global__ void __launch_bounds__(256) k_utv_rm(int64_t nA, int kp, const T *__restrict__ Urm,
                                                const T *__restrict__ v, double *part)
{
    __shared__ T vs[RM_ROWS];
    __shared__ double acc4[4][256];
    const int64_t r0 = (int64_t)blockIdx.x * RM_ROWS;
    const int rows = (int)min((int64_t)RM_ROWS, nA - r0);
    for (int r = threadIdx.x; r < RM_ROWS; r += blockDim.x) vs[r] = (r < rows) ? v[r0 + r] : (T)0;
    __syncthreads();
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
    const int kq = kp / 4;
    for (int cb = 0; cb < kq; cb += 64) {
        const int cg = cb + tx;
        T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        if (cg < kq) {
            const T *base = Urm + r0 * kp + 4 * cg;
            int r = ty;
            for (; r + 12 < rows; r += 16) {
                Quad<T> u0 = ld4cs(base + (int64_t)r * kp), u1 = ld4cs(base + (int64_t)(r + 4) * kp);
                Quad<T> u2 = ld4cs(base + (int64_t)(r + 8) * kp), u3 = ld4cs(base + (int64_t)(r + 12) * kp);
                T x0 = vs[r], x1 = vs[r + 4], x2 = vs[r + 8], x3 = vs[r + 12];
                a0 = fma(u0.x, x0, a0); a1 = fma(u0.y, x0, a1); a2 = fma(u0.z, x0, a2); a3 = fma(u0.w, x0, a3);
                a0 = fma(u1.x, x1, a0); a1 = fma(u1.y, x1, a1); a2 = fma(u1.z, x1, a2); a3 = fma(u1.w, x1, a3);
                a0 = fma(u2.x, x2, a0); a1 = fma(u2.y, x2, a1); a2 = fma(u2.z, x2, a2); a3 = fma(u2.w, x2, a3);
                a0 = fma(u3.x, x3, a0); a1 = fma(u3.y, x3, a1); a2 = fma(u3.z, x3, a2); a3 = fma(u3.w, x3, a3);
            }
            for (; r < rows; r += 4) {
                Quad<T> u = ld4cs(base + (int64_t)r * kp);
                T x = vs[r];
                a0 = fma(u.x, x, a0); a1 = fma(u.y, x, a1); a2 = fma(u.z, x, a2); a3 = fma(u.w, x, a3);
            }
        }
        acc4[ty][4 * tx + 0] = (double)a0;
        acc4[ty][4 * tx + 1] = (double)a1;
        acc4[ty][4 * tx + 2] = (double)a2;
        acc4[ty][4 * tx + 3] = (double)a3;
        __syncthreads();
        if (ty == 0 && cg < kq) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = 4 * tx + q;
                part[(int64_t)blockIdx.x * kp + 4 * cg + q] = acc4[0][j] + acc4[1][j] + acc4[2][j] + acc4[3][j];
            }
        }
        __syncthreads();
    }
}

int utv_rm_splits(int64_t nA) { return ceil_div(nA, RM_ROWS); }

// t = U^T v into part[S*kp .. S*kp + kp) (partials first).
template <typename T>
void launch_utv_rm(cudaStream_t s, int64_t nA, int kp, const T *Urm, const T *v, double *part, int *splits)
{
    const int S = utv_rm_splits(nA);
    WC4D_LAUNCH(k_utv_rm<T><<<S, 256, 0, s>>>(nA, kp, Urm, v, part));
    WC4D_LAUNCH(k_reduce_part<<<ceil_div(kp, 256), 256, 0, s>>>(S, kp, kp, 0, part, part + (int64_t)S * kp));
    *splits = S;
}

template void launch_utv_rm<double>(cudaStream_t, int64_t, int, const double *, const double *, double *, int *);
template void launch_utv_rm<float>(cudaStream_t, int64_t, int, const float *, const float *, double *, int *);

// y[r] = v[r] - sum_i Urm[r, i] c_i t_i; one warp per row, lanes over the
// kp/4 vector groups of the row.
template <typename T>
__global__ void __launch_bounds__(256) k_lmp_combine_rm(int64_t nA, int k, int kp, const T *__restrict__ Urm,
                                                        const double *__restrict__ t, const double *__restrict__ cvec,
                                                        const T *v, T *y, const int *skip)
{
    extern __shared__ double ctd[];
    if (skip && *skip) return;
    T *ct = reinterpret_cast<T *>(ctd);
    for (int i = threadIdx.x; i < kp; i += blockDim.x) ct[i] = (i < k) ? (T)(cvec[i] * t[i]) : (T)0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int kq = kp / 4;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < nA; r += warps) {
        const T *row = Urm + r * kp;
        T acc = 0;
        for (int g = lane; g < kq; g += 32) {
            Quad<T> u = ld4cs(row + 4 * g);
            acc = fma(u.x, ct[4 * g], acc);
            acc = fma(u.y, ct[4 * g + 1], acc);
            acc = fma(u.z, ct[4 * g + 2], acc);
            acc = fma(u.w, ct[4 * g + 3], acc);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) y[r] = v[r] - acc;
    }
}

template <typename T>
void launch_lmp_combine_rm(cudaStream_t s, int num_sms, int64_t nA, int k, int kp, const T *Urm, const double *t,
                           const double *cvec, const T *v, T *y, const int *skip)
{
    int grid = std::min<int64_t>((int64_t)num_sms * 8, ceil_div(nA, 8));
    WC4D_LAUNCH(k_lmp_combine_rm<T><<<grid, 256, (size_t)kp * sizeof(double), s>>>(nA, k, kp, Urm, t, cvec, v, y,
                                                                                      skip));
}

template void launch_lmp_combine_rm<double>(cudaStream_t, int, int64_t, int, int, const double *, const double *,
                                            const double *, const double *, double *, const int *);
template void launch_lmp_combine_rm<float>(cudaStream_t, int, int64_t, int, int, const float *, const double *,
                                           const double *, const float *, float *, const int *);

// ----------------------------------------------------------------------------
// One split-preconditioned CG iteration (Alg. 1 with the spectral LMP of
// eq. 15) after q = A p, with two passes over the row-major Ritz vectors
// instead of two LMP applications of two passes each:
//   pass A : s = U^T q, e = U^T rhat, p^T q;
//   coef   : alpha = rho / p^T q, w1 = alpha c o s,
//            w2 = c o (e - alpha (1 - c) o s)   [= c o U^T rhat_new when
//            U^T U = I; e is recomputed from rhat every iteration, so the
//            identity enters one step only];
//   pass B : rhat <- rhat - alpha C q = rhat - alpha q + U w1,
//            t = C rhat = rhat - U w2, x += alpha p, r -= alpha q, with the
//            partial sums of |rhat|^2 and |r|^2 for the beta kernel.
// ----------------------------------------------------------------------------
constexpr int PA_ROWS = 512;   // rows per CTA of pass A (at most)
constexpr double LMP_L2_KEEP = 64.0 * 1024 * 1024;   // Ritz-vector bytes the first pass leaves in L2

int lmp_pass_a_splits(int64_t nA, int num_sms)
{
    const int s = ceil_div(nA, PA_ROWS);
    return ceil_div(s, num_sms) * num_sms;   // a whole number of CTAs per SM
}

template <typename T>
__global__ void __launch_bounds__(256, 4) k_lmp_pass_a(int64_t nA, int kp, int64_t rows_per, const T *__restrict__ Urm,
                                                    const T *__restrict__ q, const T *__restrict__ rh,
                                                    const T *__restrict__ p, double *part, int keep_from)
{
    __shared__ T qs[PA_ROWS], es[PA_ROWS];
    __shared__ double acc[4][2][256];
    const int64_t r0 = (int64_t)blockIdx.x * rows_per;
    const int rows = (int)max((int64_t)0, min(rows_per, nA - r0));
    double pq = 0.0;
    for (int r = threadIdx.x; r < PA_ROWS; r += blockDim.x) {
        T qv = 0, ev = 0;
        if (r < rows) {
            qv = q[r0 + r];
            ev = rh[r0 + r];
            pq = fma((double)p[r0 + r], (double)qv, pq);
        }
        qs[r] = qv;
        es[r] = ev;
    }
    pq = block_sum(pq);   // synchronises: qs, es are visible
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
    const int kq = kp / 4;
    for (int cb = 0; cb < kq; cb += 64) {
        const int cg = cb + tx;
        T a0 = 0, a1 = 0, a2 = 0, a3 = 0, b0 = 0, b1 = 0, b2 = 0, b3 = 0;
        if (cg < kq) {
            const T *base = Urm + r0 * kp + 4 * cg;
            int r = ty;
            for (; r + 12 < rows; r += 16) {   // four rows of loads in flight per thread
                Quad<T> u[4];
                // rows from keep_from on stay in L2 for the second pass,
                // which reads each CTA's rows from the end backwards
                if (r >= keep_from) {
#pragma unroll
                    for (int h = 0; h < 4; ++h) u[h] = ld4cg(base + (int64_t)(r + 4 * h) * kp);
                } else {
#pragma unroll
                    for (int h = 0; h < 4; ++h) u[h] = ld4cs(base + (int64_t)(r + 4 * h) * kp);
                }
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const T x = qs[r + 4 * h], y = es[r + 4 * h];
                    a0 = fma(u[h].x, x, a0); a1 = fma(u[h].y, x, a1); a2 = fma(u[h].z, x, a2); a3 = fma(u[h].w, x, a3);
                    b0 = fma(u[h].x, y, b0); b1 = fma(u[h].y, y, b1); b2 = fma(u[h].z, y, b2); b3 = fma(u[h].w, y, b3);
                }
            }
            for (; r < rows; r += 4) {
                Quad<T> u = ld4cg(base + (int64_t)r * kp);
                const T x = qs[r], y = es[r];
                a0 = fma(u.x, x, a0); a1 = fma(u.y, x, a1); a2 = fma(u.z, x, a2); a3 = fma(u.w, x, a3);
                b0 = fma(u.x, y, b0); b1 = fma(u.y, y, b1); b2 = fma(u.z, y, b2); b3 = fma(u.w, y, b3);
            }
        }
        acc[ty][0][4 * tx + 0] = (double)a0; acc[ty][0][4 * tx + 1] = (double)a1;
        acc[ty][0][4 * tx + 2] = (double)a2; acc[ty][0][4 * tx + 3] = (double)a3;
        acc[ty][1][4 * tx + 0] = (double)b0; acc[ty][1][4 * tx + 1] = (double)b1;
        acc[ty][1][4 * tx + 2] = (double)b2; acc[ty][1][4 * tx + 3] = (double)b3;
        __syncthreads();
        if (ty < 2 && cg < kq) {   // ty 0 writes s, ty 1 writes e
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = 4 * tx + j;
                part[((int64_t)ty * kp + 4 * cg + j) * gridDim.x + blockIdx.x] =
                    acc[0][ty][c] + acc[1][ty][c] + acc[2][ty][c] + acc[3][ty][c];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[2 * (int64_t)kp * gridDim.x + blockIdx.x] = pq;
}

// Sums the pass-A partials (column c of the transposed layout: part[c S + b];
// c < kp: s, kp <= c < 2 kp: e, c = 2 kp: p^T q), one warp per sum in a fixed
// order, into sums[]; the last CTA to finish (counter *done, reset by it)
// forms alpha, w1, w2 and publishes alpha (and the breakdown flag).
__global__ void __launch_bounds__(256) k_lmp_coef(int S, int k, int kp, const double *part, const double *cvec,
                                                  double *scal, int *flags, double *sums, double *w,
                                                  unsigned *done)
{
    __shared__ int last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * 8 + warp;
    if (c <= 2 * kp) {
        const double *src = part + (int64_t)c * S;
        double a0 = 0.0, a1 = 0.0;
        int s = lane;
        for (; s + 32 < S; s += 64) {
            a0 += src[s];
            a1 += src[s + 32];
        }
        if (s < S) a0 += src[s];
        double a = warp_sum(a0 + a1);
        if (lane == 0) sums[c] = a;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(done, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    const double pq = __ldcg(sums + 2 * kp);
    const bool fin = flags[0] != 0;
    const bool bad = !fin && (!(pq > 0.0) || !isfinite(pq));
    const double alpha = (!fin && !bad) ? scal[0] / pq : 0.0;   // scal[0] = rho
    for (int i = threadIdx.x; i < kp; i += blockDim.x) {
        const double cc = (i < k) ? cvec[i] : 0.0;
        const double si = __ldcg(sums + i), ei = __ldcg(sums + kp + i);
        w[i] = alpha * cc * si;
        w[kp + i] = cc * (ei - alpha * (1.0 - cc) * si);
    }
    if (threadIdx.x == 0) {
        scal[5] = pq;
        scal[1] = alpha;
        if (bad) { flags[1] = 1; flags[0] = 1; }
        *done = 0u;
    }
}

// Four consecutive values of a 16-byte aligned shared-memory array.
__device__ __forceinline__ Quad<float> ld4s(const float *p)
{
    const float4 v = *reinterpret_cast<const float4 *>(p);
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Quad<double> ld4s(const double *p)
{
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    return {a.x, a.y, b.x, b.y};
}

// Pass B reads the column-major copy of U (ld nA) like a GEMV y = U w: a CTA
// owns PB_ROWS consecutive rows; thread (g, ch) = (threadIdx.x % 32,
// threadIdx.x / 32) accumulates rows 4g .. 4g+3 of the CTA (one 16-byte load
// per column: a warp reads 512 contiguous bytes of a column) over the ch-th
// eighth of the k columns, eight columns of loads in flight; the eight
// partial sums of a row are added in shared memory and one thread per row
// finishes it.
constexpr int PB_ROWS = 128;
constexpr int PB_CHUNKS = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_lmp_pass_b(int64_t nA, int k, int kp, const T *__restrict__ U,
                                                    const double *__restrict__ w, const double *__restrict__ scal,
                                                    const T *__restrict__ q, const T *__restrict__ p, T *rh, T *t,
                                                    T *x, T *r, double *part, double *scal_rw, int *flags,
                                                    unsigned *done, double tol, double *qcf_drop)
{
    extern __shared__ __align__(16) double wsm[];
    __shared__ int last;
    T *w1 = reinterpret_cast<T *>(wsm), *w2 = w1 + kp;
    T (*red)[PB_CHUNKS][PB_ROWS] = reinterpret_cast<T (*)[PB_CHUNKS][PB_ROWS]>(w2 + kp);
    for (int i = threadIdx.x; i < kp; i += blockDim.x) {
        w1[i] = (T)w[i];
        w2[i] = (T)w[kp + i];
    }
    __syncthreads();
    const int g = threadIdx.x & 31, ch = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * PB_ROWS;
    const int64_t row0 = base + 4 * g;
    const int cpc = (k + PB_CHUNKS - 1) / PB_CHUNKS;
    const int i0 = min(k, ch * cpc), i1 = min(k, i0 + cpc);
    T a1[4] = {0, 0, 0, 0}, a2[4] = {0, 0, 0, 0};
    if (row0 + 3 < nA && (nA & 3) == 0) {
        const T *col = U + row0;
        for (int i = i0; i < i1; i += 8) {
            Quad<T> v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                v[u] = (i + u < i1) ? ld4cs(col + (int64_t)(i + u) * nA) : Quad<T>{0, 0, 0, 0};
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int ii = min(i + u, kp - 1);   // v[u] is zero past i1
                const T c1 = w1[ii], c2 = w2[ii];
                a1[0] = fma(v[u].x, c1, a1[0]); a1[1] = fma(v[u].y, c1, a1[1]);
                a1[2] = fma(v[u].z, c1, a1[2]); a1[3] = fma(v[u].w, c1, a1[3]);
                a2[0] = fma(v[u].x, c2, a2[0]); a2[1] = fma(v[u].y, c2, a2[1]);
                a2[2] = fma(v[u].z, c2, a2[2]); a2[3] = fma(v[u].w, c2, a2[3]);
            }
        }
    } else {   // ragged tail (or nA not a multiple of 4): one row at a time
        for (int j = 0; j < 4; ++j) {
            const int64_t row = row0 + j;
            if (row >= nA) break;
            for (int i = i0; i < i1; ++i) {
                const T v = U[(int64_t)i * nA + row];
                a1[j] = fma(v, w1[i], a1[j]);
                a2[j] = fma(v, w2[i], a2[j]);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        red[0][ch][4 * g + j] = a1[j];
        red[1][ch][4 * g + j] = a2[j];
    }
    __syncthreads();
    const double alpha = scal[1];
    double srh = 0.0, sr = 0.0;
    if (threadIdx.x < PB_ROWS) {
        const int rr = threadIdx.x;
        const int64_t row = base + rr;
        if (row < nA) {
            T d1 = 0, d2 = 0;
#pragma unroll
            for (int c = 0; c < PB_CHUNKS; ++c) {
                d1 += red[0][c][rr];
                d2 += red[1][c][rr];
            }
            const double qv = (double)q[row];
            const double rhn = (double)rh[row] - alpha * qv + (double)d1;
            rh[row] = (T)rhn;
            t[row] = (T)(rhn - (double)d2);
            x[row] = (T)((double)x[row] + alpha * (double)p[row]);
            const double rn = (double)r[row] - alpha * qv;
            r[row] = (T)rn;
            srh = rhn * rhn;
            sr = rn * rn;
        }
    }
    srh = block_sum(srh);
    sr = block_sum(sr);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = srh;
        part[gridDim.x + blockIdx.x] = sr;
        __threadfence();
        last = (atomicAdd(done, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    // the last CTA: beta, rho, relative residual, QCF decrease and the done
    // flag from all partial sums (fixed order), as the CG beta step
    __threadfence();
    double t1 = 0.0, t2 = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        t1 += __ldcg(part + i);
        t2 += __ldcg(part + gridDim.x + i);
    }
    const double rho_new = block_sum(t1);
    const double rr = block_sum(t2);
    if (threadIdx.x == 0) {
        *done = 0u;
        if (flags[F_DONE]) {
            scal_rw[S_BETA] = 0.0;
            return;
        }
        const double rho = scal_rw[S_RHO];
        scal_rw[S_BETA] = rho_new / rho;
        if (qcf_drop) qcf_drop[flags[F_ITER]] = 0.5 * scal_rw[S_ALPHA] * rho;   // iterations done so far
        scal_rw[S_RHO] = rho_new;
        scal_rw[S_RR] = rr;
        const double rel = sqrt(rr) / scal_rw[S_BNORM];
        scal_rw[S_RELRES] = rel;
        flags[F_ITER] += 1;
        if (!isfinite(rel)) { flags[F_BREAK] = 2; flags[F_DONE] = 1; }
        else if (tol > 0.0 && rel <= tol) flags[F_DONE] = 1;
    }
}

// Second pass over the ROW-MAJOR Ritz vectors with the first pass's split
// (CTA b: rows [b R, b R + R), R <= PA_ROWS), walked from the end of the
// range backwards so that the rows the first pass read last -- still in L2 --
// come first.  Each warp takes groups of RW consecutive rows on its own (no
// CTA barrier until the range is done): lane l holds column quads l and
// l + 32 of w1 and w2 and loads the same quads of the RW rows (2 RW loads in
// flight per lane); the V = 2 RW row dot products are then summed over the
// warp by a halving butterfly (V - 1 + log2(32 / V) shuffles instead of
// 5 V).  Then the CTA updates its rows with
// coalesced accesses, as the column-major pass does, and the last CTA takes
// the CG beta step.
template <int V, typename T> __device__ __forceinline__ void butterfly_sums(T (&v)[V], int lane)
{
    // V values per lane (V a power of two, 2 <= V <= 32); step o = 16, 8, ...
    // sends half of the remaining values to lane l ^ o and adds the half it
    // receives, so after log2(V) steps v[0] of lane l holds value
    // l / (32 / V), summed over the lanes that share those high lane bits
#pragma unroll
    for (int h = V / 2, o = 16; h >= 1; h /= 2, o /= 2) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const T send = up ? v[i] : v[i + h];
            const T keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_lmp_pass_b_rm(int64_t nA, int kp, int64_t rows_per, const T *__restrict__ U,
                                                       const double *__restrict__ w, const double *__restrict__ scal,
                                                       const T *__restrict__ q, const T *__restrict__ p, T *rh, T *t,
                                                       T *x, T *r, double *part, double *scal_rw, int *flags,
                                                       unsigned *done, double tol, double *qcf_drop)
{
    constexpr int RW = sizeof(T) == 4 ? 8 : 4;   // rows per warp step (2 RW sums <= 16)
    constexpr int V = 2 * RW;                    // sums per step: product 0 rows 0..RW-1, product 1 rows 0..RW-1
    constexpr int NB = 32 / V;                   // lanes beyond the butterfly's reach: after log2(V) halvings
    static_assert(V == 8 || V == 16, "butterfly width");
    __shared__ T dsum[2][PA_ROWS];
    __shared__ int last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kq = kp / 4;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per;
    const int rows = (int)max((int64_t)0, min(rows_per, nA - r0));
    const bool h0 = lane < kq, h1 = lane + 32 < kq;
    const Quad<T> z{0, 0, 0, 0};
    Quad<T> w1a = z, w1b = z, w2a = z, w2b = z;
    if (h0) {
        w1a = {(T)w[4 * lane], (T)w[4 * lane + 1], (T)w[4 * lane + 2], (T)w[4 * lane + 3]};
        w2a = {(T)w[kp + 4 * lane], (T)w[kp + 4 * lane + 1], (T)w[kp + 4 * lane + 2], (T)w[kp + 4 * lane + 3]};
    }
    if (h1) {
        const int c = 4 * (lane + 32);
        w1b = {(T)w[c], (T)w[c + 1], (T)w[c + 2], (T)w[c + 3]};
        w2b = {(T)w[kp + c], (T)w[kp + c + 1], (T)w[kp + c + 2], (T)w[kp + c + 3]};
    }
    const int ngroups = (rows + RW - 1) / RW;
    for (int gi = warp; gi < ngroups; gi += 8) {
        const int hi = rows - RW * gi;   // rows hi - RW .. hi - 1 (those >= 0)
        Quad<T> ua[RW], ub[RW];
#pragma unroll
        for (int h = 0; h < RW; ++h) {
            const int rl = hi - 1 - h;
            const T *row = U + (r0 + max(rl, 0)) * kp;
            ua[h] = (rl >= 0 && h0) ? ld4cs(row + 4 * lane) : z;
            ub[h] = (rl >= 0 && h1) ? ld4cs(row + 4 * (lane + 32)) : z;
        }
        T v[V];
#pragma unroll
        for (int h = 0; h < RW; ++h) {
            T a = ua[h].x * w1a.x, b = ua[h].x * w2a.x;
            a = fma(ua[h].y, w1a.y, a); b = fma(ua[h].y, w2a.y, b);
            a = fma(ua[h].z, w1a.z, a); b = fma(ua[h].z, w2a.z, b);
            a = fma(ua[h].w, w1a.w, a); b = fma(ua[h].w, w2a.w, b);
            a = fma(ub[h].x, w1b.x, a); b = fma(ub[h].x, w2b.x, b);
            a = fma(ub[h].y, w1b.y, a); b = fma(ub[h].y, w2b.y, b);
            a = fma(ub[h].z, w1b.z, a); b = fma(ub[h].z, w2b.z, b);
            a = fma(ub[h].w, w1b.w, a); b = fma(ub[h].w, w2b.w, b);
            v[h] = a;
            v[RW + h] = b;
        }
        butterfly_sums<V>(v, lane);
        // after log2(V) halvings over lane bits 4, 3, ...: value index from
        // those bits, most significant first; the remaining low lane bits
        // hold partial sums of the same value
#pragma unroll
        for (int o = NB / 2; o >= 1; o /= 2) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
        if ((lane & (NB - 1)) == 0) {
            const int idx = lane / NB;   // 0 .. V-1
            const int which = idx / RW, h = idx % RW;
            const int rl = hi - 1 - h;
            if (rl >= 0) dsum[which][rl] = v[0];
        }
    }
    __syncthreads();
    const double alpha = scal[1];
    double srh = 0.0, sr = 0.0;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
        const int64_t row = r0 + i;
        const double qv = (double)q[row];
        const double rhn = (double)rh[row] - alpha * qv + (double)dsum[0][i];
        rh[row] = (T)rhn;
        t[row] = (T)(rhn - (double)dsum[1][i]);
        x[row] = (T)((double)x[row] + alpha * (double)p[row]);
        const double rn = (double)r[row] - alpha * qv;
        r[row] = (T)rn;
        srh += rhn * rhn;
        sr += rn * rn;
    }
    srh = block_sum(srh);
    sr = block_sum(sr);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = srh;
        part[gridDim.x + blockIdx.x] = sr;
        __threadfence();
        last = (atomicAdd(done, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    // the last CTA: beta, rho, relative residual, QCF decrease and the done
    // flag from all partial sums (fixed order), as the CG beta step
    __threadfence();
    double t1 = 0.0, t2 = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        t1 += __ldcg(part + i);
        t2 += __ldcg(part + gridDim.x + i);
    }
    const double rho_new = block_sum(t1);
    const double rr = block_sum(t2);
    if (threadIdx.x == 0) {
        *done = 0u;
        if (flags[F_DONE]) {
            scal_rw[S_BETA] = 0.0;
            return;
        }
        const double rho = scal_rw[S_RHO];
        scal_rw[S_BETA] = rho_new / rho;
        if (qcf_drop) qcf_drop[flags[F_ITER]] = 0.5 * scal_rw[S_ALPHA] * rho;   // iterations done so far
        scal_rw[S_RHO] = rho_new;
        scal_rw[S_RR] = rr;
        const double rel = sqrt(rr) / scal_rw[S_BNORM];
        scal_rw[S_RELRES] = rel;
        flags[F_ITER] += 1;
        if (!isfinite(rel)) { flags[F_BREAK] = 2; flags[F_DONE] = 1; }
        else if (tol > 0.0 && rel <= tol) flags[F_DONE] = 1;
    }
}

int lmp_pass_b_grid(int64_t nA) { return ceil_div(nA, PB_ROWS); }

template <typename T>
void launch_lmp_fused(cudaStream_t s, int num_sms, int64_t nA, int k, int kp, const T *Urm, const T *Ucm,
                      const double *cvec, const T *q, const T *p, T *rh, T *t, T *x, T *r, double *scal, int *flags,
                      double *partA, double *w, double *partB, unsigned *done, double tol, double *qcf_drop)
{
    const int S = lmp_pass_a_splits(nA, num_sms);
    const int64_t rows_per = (nA + S - 1) / S;
    // Row-major second pass (kp / 4 <= 64): the first pass leaves the last
    // part of every CTA's rows in L2 -- at most LMP_L2_KEEP bytes in all --
    // and the second pass reads those first.
    const bool rm = kp / 4 <= 64;
    const double ubytes = (double)nA * kp * sizeof(T);
    const double keep = rm ? std::min(1.0, LMP_L2_KEEP / ubytes) : 0.0;
    const int keep_from = (int)((double)rows_per * (1.0 - keep));
    WC4D_LAUNCH(k_lmp_pass_a<T><<<S, 256, 0, s>>>(nA, kp, rows_per, Urm, q, rh, p, partA, rm ? keep_from : INT_MAX));
    double *sums = w + 2 * kp;
    WC4D_LAUNCH(k_lmp_coef<<<ceil_div(2 * kp + 1, 8), 256, 0, s>>>(S, k, kp, partA, cvec, scal, flags, sums, w, done));
    if (rm) {
        WC4D_LAUNCH(k_lmp_pass_b_rm<T><<<S, 256, 0, s>>>(nA, kp, rows_per, Urm, w, scal, q, p, rh, t, x, r, partB, scal,
                                                         flags, done + 1, tol, qcf_drop));
        return;
    }
    const int G = lmp_pass_b_grid(nA);
    const size_t smem = (2 * (size_t)kp + 2 * PB_CHUNKS * PB_ROWS) * sizeof(T);
    WC4D_LAUNCH(k_lmp_pass_b<T><<<G, 256, smem, s>>>(nA, k, kp, Ucm, w, scal, q, p, rh, t, x, r, partB, scal, flags,
                                                     done + 1, tol, qcf_drop));
}

template void launch_lmp_fused<double>(cudaStream_t, int, int64_t, int, int, const double *, const double *,
                                       const double *, const double *, const double *, double *, double *, double *,
                                       double *, double *, int *, double *, double *, double *, unsigned *, double,
                                       double *);
template void launch_lmp_fused<float>(cudaStream_t, int, int64_t, int, int, const float *, const float *,
                                      const double *, const float *, const float *, float *, float *, float *,
                                      float *, double *, int *, double *, double *, double *, unsigned *, double,
                                      double *);

// ----------------------------------------------------------------------------
// PCG (Alg. 1) vector and scalar kernels.  Scalars live in device memory:
// scal[0] rho = rhat^T rhat, [1] alpha, [2] beta, [3] |b|, [4] |r|/|b|,
// [5] p^T A p, [6] |r|^2; flags[0] done, [1] breakdown, [2] iterations.
// ----------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(256) k_dot_partial(int64_t n, const T *a, const T *b, double *part)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc = fma((double)a[i], (double)b[i], acc);
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

template <typename T>
void launch_dot_partial(cudaStream_t s, int grid, int64_t n, const T *a, const T *b, double *part)
{
    WC4D_LAUNCH(k_dot_partial<T><<<grid, 256, 0, s>>>(n, a, b, part));
}

template void launch_dot_partial<double>(cudaStream_t, int, int64_t, const double *, const double *, double *);
template void launch_dot_partial<float>(cudaStream_t, int, int64_t, const float *, const float *, double *);

__device__ double sum_part(int grid, const double *part)
{
    double a = 0.0;
    for (int i = threadIdx.x; i < grid; i += blockDim.x) a += part[i];
    return block_sum(a);
}

__global__ void k_pcg_init(int grid, const double *part_b, const double *part_rh, double *scal, int *flags)
{
    double bb = sum_part(grid, part_b);
    double rho = sum_part(grid, part_rh);
    if (threadIdx.x == 0) {
        // a non-finite right-hand side (or preconditioned residual) is a
        // breakdown before the first iteration, not a zero right-hand side
        const bool bad = !isfinite(bb) || !isfinite(rho);
        scal[S_RHO] = rho;
        scal[S_BNORM] = sqrt(bb);
        scal[S_RELRES] = bb > 0.0 ? 1.0 : 0.0;
        scal[S_ALPHA] = 0.0;
        scal[S_BETA] = 0.0;
        flags[F_DONE] = (bb > 0.0 && !bad) ? 0 : 1;
        flags[F_BREAK] = bad ? 2 : 0;
        flags[F_ITER] = 0;
    }
}

void launch_pcg_init(cudaStream_t s, int grid, const double *part_b, const double *part_rh, double *scal, int *flags)
{
    WC4D_LAUNCH(k_pcg_init<<<1, 256, 0, s>>>(grid, part_b, part_rh, scal, flags));
}

__global__ void k_pcg_alpha(int grid, const double *part, double *scal, int *flags)
{
    double pq = sum_part(grid, part);
    if (threadIdx.x == 0) {
        scal[S_PQ] = pq;
        if (flags[F_DONE]) {
            scal[S_ALPHA] = 0.0;
        } else if (!(pq > 0.0) || !isfinite(pq)) {
            flags[F_BREAK] = 1;
            flags[F_DONE] = 1;
            scal[S_ALPHA] = 0.0;
        } else {
            scal[S_ALPHA] = scal[S_RHO] / pq;
        }
    }
}

void launch_pcg_alpha(cudaStream_t s, int grid, const double *part, double *scal, int *flags)
{
    WC4D_LAUNCH(k_pcg_alpha<<<1, 256, 0, s>>>(grid, part, scal, flags));
}

// x += alpha p; r -= alpha q; partial |r|^2
template <typename T>
__global__ void __launch_bounds__(256) k_pcg_xr(int64_t n, const double *scal, T *x, T *r, const T *p, const T *q,
                                                double *part)
{
    const double alpha = scal[S_ALPHA];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = (T)((double)x[i] + alpha * (double)p[i]);
        double ri = (double)r[i] - alpha * (double)q[i];
        r[i] = (T)ri;
        acc = fma(ri, ri, acc);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

template <typename T>
void launch_pcg_xr(cudaStream_t s, int grid, int64_t n, const double *scal, T *x, T *r, const T *p, const T *q,
                   double *part)
{
    WC4D_LAUNCH(k_pcg_xr<T><<<grid, 256, 0, s>>>(n, scal, x, r, p, q, part));
}

// rhat -= alpha t; partial rhat^T rhat
template <typename T>
__global__ void __launch_bounds__(256) k_pcg_rh(int64_t n, const double *scal, T *rh, const T *t, double *part)
{
    const double alpha = scal[S_ALPHA];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = (double)rh[i] - alpha * (double)t[i];
        rh[i] = (T)v;
        acc = fma(v, v, acc);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

template <typename T>
void launch_pcg_rh(cudaStream_t s, int grid, int64_t n, const double *scal, T *rh, const T *t, double *part)
{
    WC4D_LAUNCH(k_pcg_rh<T><<<grid, 256, 0, s>>>(n, scal, rh, t, part));
}

__global__ void k_pcg_beta(int grid, const double *part_rh, const double *part_r, double *scal, int *flags,
                           double tol, double *qcf_drop)
{
    double rho_new = sum_part(grid, part_rh);
    double rr = sum_part(grid, part_r);
    if (threadIdx.x == 0) {
        if (flags[F_DONE]) {
            scal[S_BETA] = 0.0;
            return;
        }
        double rho = scal[S_RHO];
        scal[S_BETA] = rho_new / rho;
        if (qcf_drop) qcf_drop[flags[F_ITER]] = 0.5 * scal[S_ALPHA] * rho;   // iterations done so far
        scal[S_RHO] = rho_new;
        scal[S_RR] = rr;
        double rel = sqrt(rr) / scal[S_BNORM];
        scal[S_RELRES] = rel;
        flags[F_ITER] += 1;
        if (!isfinite(rel)) { flags[F_BREAK] = 2; flags[F_DONE] = 1; }
        else if (tol > 0.0 && rel <= tol) flags[F_DONE] = 1;
    }
}

void launch_pcg_beta(cudaStream_t s, int grid, const double *part_rh, const double *part_r, double *scal,
                     int *flags, double tol, double *qcf_drop)
{
    WC4D_LAUNCH(k_pcg_beta<<<1, 256, 0, s>>>(grid, part_rh, part_r, scal, flags, tol, qcf_drop));
}

// After a reliable update: rho and |r|^2 from the replaced residual; the
// iteration goes on (the done flag is cleared unless CG broke down).
__global__ void k_pcg_restart(int grid, const double *part_rh, const double *part_r, double *scal, int *flags)
{
    double rho = sum_part(grid, part_rh);
    double rr = sum_part(grid, part_r);
    if (threadIdx.x == 0) {
        scal[S_RHO] = rho;
        scal[S_RR] = rr;
        scal[S_RELRES] = sqrt(rr) / scal[S_BNORM];
        if (!flags[F_BREAK]) flags[F_DONE] = 0;
    }
}

void launch_pcg_restart(cudaStream_t s, int grid, const double *part_rh, const double *part_r, double *scal,
                        int *flags)
{
    WC4D_LAUNCH(k_pcg_restart<<<1, 256, 0, s>>>(grid, part_rh, part_r, scal, flags));
}

// Lanczos vectors from CG (Section 3.3).  k_lanczos_first: F[:, 0] = b / |b|.
// k_lanczos_record, after the beta step of iteration j (flags[F_ITER] = j + 1
// iterations done): F[:, j + 1] = (-1)^(j+1) r / |r| (|r|^2 = scal[S_RR]; the
// sign makes consecutive columns Lanczos vectors, whose tridiagonal has
// positive off-diagonals) and ab[2 j], ab[2 j + 1] = alpha_j, beta_j.
// cap: columns of F.
__global__ void __launch_bounds__(256) k_lanczos_first(int64_t n, const double *b, const double *scal, double *F)
{
    const double s = 1.0 / scal[S_BNORM];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        F[i] = s * b[i];
}

__global__ void __launch_bounds__(256) k_lanczos_record(int64_t n, const double *r, const double *scal,
                                                        const int *flags, double *F, double *ab, int cap)
{
    const int col = flags[F_ITER];
    if (col < 1 || col >= cap) return;
    const double s = ((col & 1) ? -1.0 : 1.0) / sqrt(scal[S_RR]);
    double *f = F + (int64_t)col * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        f[i] = s * r[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ab[2 * (col - 1)] = scal[S_ALPHA];
        ab[2 * (col - 1) + 1] = scal[S_BETA];
    }
}

void launch_lanczos_first(cudaStream_t s, int grid, int64_t n, const double *b, const double *scal, double *F)
{
    WC4D_LAUNCH(k_lanczos_first<<<grid, 256, 0, s>>>(n, b, scal, F));
}

void launch_lanczos_record(cudaStream_t s, int grid, int64_t n, const double *r, const double *scal, const int *flags,
                           double *F, double *ab, int cap)
{
    WC4D_LAUNCH(k_lanczos_record<<<grid, 256, 0, s>>>(n, r, scal, flags, F, ab, cap));
}

// p = t + beta p
template <typename T>
__global__ void __launch_bounds__(256) k_pcg_p(int64_t n, const double *scal, T *p, const T *t)
{
    const double beta = scal[S_BETA];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (T)((double)t[i] + beta * (double)p[i]);
}

template <typename T>
void launch_pcg_p(cudaStream_t s, int grid, int64_t n, const double *scal, T *p, const T *t)
{
    WC4D_LAUNCH(k_pcg_p<T><<<grid, 256, 0, s>>>(n, scal, p, t));
}

template void launch_pcg_xr<double>(cudaStream_t, int, int64_t, const double *, double *, double *, const double *,
                                    const double *, double *);
template void launch_pcg_xr<float>(cudaStream_t, int, int64_t, const double *, float *, float *, const float *,
                                   const float *, double *);
template void launch_pcg_rh<double>(cudaStream_t, int, int64_t, const double *, double *, const double *, double *);
template void launch_pcg_rh<float>(cudaStream_t, int, int64_t, const double *, float *, const float *, double *);
template void launch_pcg_p<double>(cudaStream_t, int, int64_t, const double *, double *, const double *);
template void launch_pcg_p<float>(cudaStream_t, int, int64_t, const double *, float *, const float *);

template <typename T>
__global__ void k_copy(int64_t n, const T *a, T *b)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

template <typename T>
void launch_copy(cudaStream_t s, int64_t n, const T *a, T *b)
{
    if (n > 0) WC4D_LAUNCH(k_copy<T><<<ceil_div(n, 256), 256, 0, s>>>(n, a, b));
}

template void launch_copy<double>(cudaStream_t, int64_t, const double *, double *);
template void launch_copy<float>(cudaStream_t, int64_t, const float *, float *);

// y = alpha x + beta y
template <typename T>
__global__ void k_axpby(int64_t n, double alpha, const T *x, double beta, T *y)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = (T)(alpha * (double)x[i] + beta * (double)y[i]);
}

template <typename T>
void launch_axpby(cudaStream_t s, int64_t n, double alpha, const T *x, double beta, T *y)
{
    if (n > 0) WC4D_LAUNCH(k_axpby<T><<<ceil_div(n, 256), 256, 0, s>>>(n, alpha, x, beta, y));
}

template void launch_axpby<double>(cudaStream_t, int64_t, double, const double *, double, double *);
template void launch_axpby<float>(cudaStream_t, int64_t, double, const float *, double, float *);

__global__ void k_sub_f64(int64_t n, const double *a, const double *b, double *out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] - b[i];
}

void launch_sub_f64(cudaStream_t s, int64_t n, const double *a, const double *b, double *out)
{
    if (n > 0) WC4D_LAUNCH(k_sub_f64<<<ceil_div(n, 256), 256, 0, s>>>(n, a, b, out));
}

__global__ void k_add_f32_to_f64(int64_t n, const float *a, double *b)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] += (double)a[i];
}

void launch_add_f32_to_f64(cudaStream_t s, int64_t n, const float *a, double *b)
{
    if (n > 0) WC4D_LAUNCH(k_add_f32_to_f64<<<ceil_div(n, 256), 256, 0, s>>>(n, a, b));
}
