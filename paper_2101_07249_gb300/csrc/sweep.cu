// Kernels of the Hessian product (eq. 10): D^{1/2} (circulant, FFT or
// direct), the tangent-linear / adjoint sweeps as SIMT GEMM / GEMV over the
// dense propagators, and the observation term H^T R^{-1} H.
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include <algorithm>

#include "wc4d_internal.cuh"
#include "bulk.cuh"

template <typename T> struct Cplx;
template <> struct Cplx<double> { using t = double2; };
template <> struct Cplx<float> { using t = float2; };

template <typename CT> __device__ __forceinline__ CT cadd(CT a, CT b) { a.x += b.x; a.y += b.y; return a; }
template <typename CT> __device__ __forceinline__ CT csub(CT a, CT b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename CT> __device__ __forceinline__ CT cmul(CT a, CT b)
{
    CT r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename CT> __device__ __forceinline__ CT cmulconj(CT a, CT b)   // a * conj(b)
{
    CT r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.y * b.x - a.x * b.y;
    return r;
}

// Shared-memory index of FFT element i: one complex pad after every 16, so
// that the power-of-two strides of the butterfly layers spread over the banks.
__device__ __forceinline__ int fpad(int i) { return i + (i >> 4); }

// ----------------------------------------------------------------------------
// D^{1/2} on two real vectors at once: z = x_a + i x_b, radix-2 decimation-
// in-frequency FFT (natural in, bit-reversed out) in shared memory, scale by
// the real sqrt spectrum (stored bit-reversed, already divided by n), then
// a decimation-in-time inverse FFT (bit-reversed in, natural out).  The
// circulant is real and symmetric, so Re / Im of the result are D^{1/2} x_a
// and D^{1/2} x_b.  Vectors of block 0 use B's spectrum and pair among
// themselves; vectors of blocks 1..N use Q's.
// ----------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(512)
k_circ_fft(int n, int logn, int N, int K, const T *__restrict__ X, int64_t ldx, T *Y, int64_t ldy,
           const T *addX, int64_t ld_add, const T *__restrict__ specB, const T *__restrict__ specQ,
           const typename Cplx<T>::t *__restrict__ tw, int nBpairs)
{
    using CT = typename Cplx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CT *buf = reinterpret_cast<CT *>(smem_raw);
    const int tid = threadIdx.x, nt = blockDim.x;
    int pair = blockIdx.x;
    const T *spec;
    int64_t ja, ta, jb = 0, tb = 0;
    bool hasb;
    if (pair < nBpairs) {
        int64_t va = 2 * (int64_t)pair, vb = va + 1;
        spec = specB;
        ja = va; ta = 0;
        hasb = vb < K;
        if (hasb) { jb = vb; tb = 0; }
    } else {
        int64_t p = pair - nBpairs;
        int64_t va = 2 * p, vb = va + 1, cnt = (int64_t)K * N;
        spec = specQ;
        ja = va / N; ta = 1 + va % N;
        hasb = vb < cnt;
        if (hasb) { jb = vb / N; tb = 1 + vb % N; }
    }
    const T *xa = X + ja * ldx + ta * n;
    const T *xb = X + jb * ldx + tb * n;
    const int half = n >> 1;
    CT *tws = buf + n + (n >> 4);   // twiddles W_n^k, k < n/2, staged once
    // the global loads of each loop are unrolled so that they are all in flight at once
#pragma unroll 8
    for (int k = tid; k < half; k += nt) tws[k] = tw[k];
#pragma unroll 8
    for (int s = tid; s < n; s += nt) {
        CT v;
        v.x = xa[s];
        v.y = hasb ? xb[s] : (T)0;
        buf[fpad(s)] = v;
    }
    __syncthreads();
    const int quarter = n >> 2;
    // forward DIF, two radix-2 spans (h, h/2) per pass: each group of four
    // points {j, j+h/2, j+h, j+3h/2} is closed under both butterfly layers
    int lh = logn - 1;
    for (; lh >= 1; lh -= 2) {
        const int h = 1 << lh, hh = h >> 1;
        const int s1 = half >> lh, s2 = n >> lh;   // W_{2h}^k = tws[k s1], W_h^k = tws[k s2]
        for (int b = tid; b < quarter; b += nt) {
            const int pos = b & (hh - 1);
            const int j = ((b >> (lh - 1)) << (lh + 1)) + pos;
            const CT e0 = buf[fpad(j)], e1 = buf[fpad(j + hh)], e2 = buf[fpad(j + h)], e3 = buf[fpad(j + h + hh)];
            const CT a0 = cadd(e0, e2), a2 = cmul(csub(e0, e2), tws[pos * s1]);
            const CT a1 = cadd(e1, e3), a3 = cmul(csub(e1, e3), tws[(pos + hh) * s1]);
            const CT w = tws[pos * s2];
            buf[fpad(j)] = cadd(a0, a1);
            buf[fpad(j + hh)] = cmul(csub(a0, a1), w);
            buf[fpad(j + h)] = cadd(a2, a3);
            buf[fpad(j + h + hh)] = cmul(csub(a2, a3), w);
        }
        __syncthreads();
    }
    if (lh == 0) {   // odd log2 n: the last span-1 layer alone
        for (int b = tid; b < half; b += nt) {
            const int j = 2 * b;
            const CT a = buf[fpad(j)], c = buf[fpad(j + 1)];
            buf[fpad(j)] = cadd(a, c);
            buf[fpad(j + 1)] = csub(a, c);
        }
        __syncthreads();
    }
#pragma unroll 8
    for (int p = tid; p < n; p += nt) {
        T w = spec[__brev((unsigned)p) >> (32 - logn)];   // the DIF output is in bit-reversed order
        CT v = buf[fpad(p)];
        v.x *= w; v.y *= w;
        buf[fpad(p)] = v;
    }
    __syncthreads();
    // inverse DIT, spans (h, 2h) per pass on groups {j, j+h, j+2h, j+3h}
    lh = 0;
    for (; lh + 1 < logn; lh += 2) {
        const int h = 1 << lh;
        const int s1 = half >> lh, s2 = half >> (lh + 1);   // W_{2h}^k = tws[k s1], W_{4h}^k = tws[k s2]
        for (int b = tid; b < quarter; b += nt) {
            const int pos = b & (h - 1);
            const int j = ((b >> lh) << (lh + 2)) + pos;
            const CT e0 = buf[fpad(j)], e1 = cmulconj(buf[fpad(j + h)], tws[pos * s1]);
            const CT e2 = buf[fpad(j + 2 * h)], e3 = cmulconj(buf[fpad(j + 3 * h)], tws[pos * s1]);
            const CT a0 = cadd(e0, e1), a1 = csub(e0, e1), a2 = cadd(e2, e3), a3 = csub(e2, e3);
            const CT c2 = cmulconj(a2, tws[pos * s2]), c3 = cmulconj(a3, tws[(pos + h) * s2]);
            buf[fpad(j)] = cadd(a0, c2);
            buf[fpad(j + 2 * h)] = csub(a0, c2);
            buf[fpad(j + h)] = cadd(a1, c3);
            buf[fpad(j + 3 * h)] = csub(a1, c3);
        }
        __syncthreads();
    }
    if (lh == logn - 1) {   // odd log2 n: the last span-n/2 layer alone
        for (int b = tid; b < half; b += nt) {
            const CT a = buf[fpad(b)], c = cmulconj(buf[fpad(b + half)], tws[b]);
            buf[fpad(b)] = cadd(a, c);
            buf[fpad(b + half)] = csub(a, c);
        }
        __syncthreads();
    }
    T *ya = Y + ja * ldy + ta * n;
    T *yb = Y + jb * ldy + tb * n;
    const T *aa = addX ? addX + ja * ld_add + ta * n : nullptr;
    const T *ab = addX ? addX + jb * ld_add + tb * n : nullptr;
#pragma unroll 8
    for (int s = tid; s < n; s += nt) {
        CT v = buf[fpad(s)];
        ya[s] = v.x + (aa ? aa[s] : (T)0);
        if (hasb) yb[s] = v.y + (ab ? ab[s] : (T)0);
    }
}

// ----------------------------------------------------------------------------
// D^{1/2} for 512 <= n <= 8192 (a power of two) with a Stockham auto-sort
// FFT: n / 16 threads, each holding 16 complex values in registers per pass;
// passes of radix 16 and one final pass of radix n / 16^P in {2, 4, 8} (n =
// 4096: three radix-16 passes), one shared-memory exchange per pass instead
// of one per radix-4 pair of layers.  Pass (radix R, span p): butterfly j
// reads buf[j + r n / R] (r < R), scales value r by W_n^{r (j mod p) n / (p R)},
// applies the R-point DFT and writes buf[(j / p) p R + j mod p + r p]; after
// the last pass buf holds the transform in natural order.  The inverse uses
// the same forward passes: y = conj(FFT(conj(s Z))) with the real spectrum s
// (already divided by n), so the result's real part is D^{1/2} x_a and minus
// its imaginary part D^{1/2} x_b.
// ----------------------------------------------------------------------------
template <typename CT> __device__ __forceinline__ CT cmuls(CT a, double c, double s)   // a * (c + i s)
{
    CT r;
    r.x = a.x * (decltype(a.x))c - a.y * (decltype(a.x))s;
    r.y = a.x * (decltype(a.x))s + a.y * (decltype(a.x))c;
    return r;
}
template <typename CT> __device__ __forceinline__ CT cmul_mi(CT a)   // a * (-i)
{
    CT r;
    r.x = a.y;
    r.y = -a.x;
    return r;
}

// in-place forward DFTs of size 2, 4, 8, 16 on v[0 .. R) (W_R = e^{-2 pi i / R})
template <typename CT> __device__ __forceinline__ void dft2(CT &a, CT &b)
{
    const CT t = a;
    a = cadd(t, b);
    b = csub(t, b);
}
template <typename CT> __device__ __forceinline__ void dft4(CT *v)
{
    const CT a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    const CT b0 = cadd(v[1], v[3]), b1 = cmul_mi(csub(v[1], v[3]));
    v[0] = cadd(a0, b0);
    v[2] = csub(a0, b0);
    v[1] = cadd(a1, b1);
    v[3] = csub(a1, b1);
}
template <typename CT> __device__ __forceinline__ void dft8(CT *v)
{
    CT e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    dft4(e);
    dft4(o);
    constexpr double h = 0.70710678118654752440;   // cos(pi / 4)
    o[1] = cmuls(o[1], h, -h);
    o[2] = cmul_mi(o[2]);
    o[3] = cmuls(o[3], -h, -h);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = cadd(e[k], o[k]);
        v[k + 4] = csub(e[k], o[k]);
    }
}
template <typename CT> __device__ __forceinline__ void dft16(CT *v)
{
    CT e[8], o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        e[k] = v[2 * k];
        o[k] = v[2 * k + 1];
    }
    dft8(e);
    dft8(o);
    constexpr double c1 = 0.92387953251128675613, s1 = 0.38268343236508977173;   // cos, sin(pi / 8)
    constexpr double h = 0.70710678118654752440;
    o[1] = cmuls(o[1], c1, -s1);
    o[2] = cmuls(o[2], h, -h);
    o[3] = cmuls(o[3], s1, -c1);
    o[4] = cmul_mi(o[4]);
    o[5] = cmuls(o[5], -s1, -c1);
    o[6] = cmuls(o[6], -h, -h);
    o[7] = cmuls(o[7], -c1, -s1);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        v[k] = cadd(e[k], o[k]);
        v[k + 8] = csub(e[k], o[k]);
    }
}
template <int R, typename CT> __device__ __forceinline__ void dftR(CT *v)
{
    if constexpr (R == 2) dft2(v[0], v[1]);
    else if constexpr (R == 4) dft4(v);
    else if constexpr (R == 8) dft8(v);
    else dft16(v);
}

// one Stockham pass of radix R at span P of an NN-point transform; NN / 16
// threads, 16 / R butterflies per thread (everything but the thread index is
// a compile-time constant).  The twiddles W_NN^{r k NN / (P R)} of the pass
// come from its own slice of the per-pass table (built by
// launch_pass_twiddles): entry P - 16 + (r - 1) P + k, so that neighbouring
// threads (neighbouring k) read neighbouring entries through L1 instead of
// the strided, bank-conflicted reads of a shared W^q table.
template <int R, int NN, int P, typename CT>
__device__ __forceinline__ void stockham_pass(CT *buf, const CT *__restrict__ twp, int tid)
{
    constexpr int B = 16 / R, T = NN / R, NT = NN / 16;
    CT v[B][R];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = tid + b * NT, k = j & (P - 1);
        CT w[R];
        if constexpr (P > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) w[r] = __ldg(twp + (P - 16) + (r - 1) * P + k);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            CT x = buf[fpad(j + r * T)];
            if constexpr (P > 1) {
                if (r > 0) x = cmul(x, w[r]);
            }
            v[b][r] = x;
        }
        dftR<R>(v[b]);
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = tid + b * NT, k = j & (P - 1);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) buf[fpad(base + r * P)] = v[b][r];
    }
    __syncthreads();
}

template <typename CT, int NN, int P> __device__ __forceinline__ void stockham_passes(CT *buf, const CT *twp, int tid)
{
    if constexpr (P * 16 <= NN) {
        stockham_pass<16, NN, P>(buf, twp, tid);
        stockham_passes<CT, NN, P * 16>(buf, twp, tid);
    } else if constexpr (NN / P > 1) {
        stockham_pass<NN / P, NN, P>(buf, twp, tid);
    }
}

// the whole forward transform, not inlined: the kernel calls it twice and one
// copy of the unrolled passes keeps the instruction footprint small
template <typename CT, int NN> __device__ __noinline__ void stockham_fft(CT *buf, const CT *twp, int tid)
{
    stockham_passes<CT, NN, 1>(buf, twp, tid);
}

template <typename T, int LOGN>
__global__ void __launch_bounds__((1 << LOGN) / 16)
k_circ_stockham(int N, int K, const T *__restrict__ X, int64_t ldx, T *Y, int64_t ldy, const T *addX, int64_t ld_add,
                const T *__restrict__ specB, const T *__restrict__ specQ, const typename Cplx<T>::t *__restrict__ twp,
                int nBpairs)
{
    using CT = typename Cplx<T>::t;
    constexpr int n = 1 << LOGN, nt = n / 16;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CT *buf = reinterpret_cast<CT *>(smem_raw);
    const int tid = threadIdx.x;
    int pair = blockIdx.x;
    const T *spec;
    int64_t ja, ta, jb = 0, tb = 0;
    bool hasb;
    if (pair < nBpairs) {
        int64_t va = 2 * (int64_t)pair, vb = va + 1;
        spec = specB;
        ja = va; ta = 0;
        hasb = vb < K;
        if (hasb) { jb = vb; tb = 0; }
    } else {
        int64_t p = pair - nBpairs;
        int64_t va = 2 * p, vb = va + 1, cnt = (int64_t)K * N;
        spec = specQ;
        ja = va / N; ta = 1 + va % N;
        hasb = vb < cnt;
        if (hasb) { jb = vb / N; tb = 1 + vb % N; }
    }
    const T *xa = X + ja * ldx + ta * n;
    const T *xb = X + jb * ldx + tb * n;
#pragma unroll
    for (int s = tid; s < n; s += nt) {
        CT v;
        v.x = xa[s];
        v.y = hasb ? xb[s] : (T)0;
        buf[fpad(s)] = v;
    }
    __syncthreads();
    stockham_fft<CT, n>(buf, twp, tid);
    // scale by the real spectrum (natural order, like the self-sorting
    // transform's output) and conjugate
#pragma unroll
    for (int q = tid; q < n; q += nt) {
        const T w = spec[q];
        CT v = buf[fpad(q)];
        v.x *= w;
        v.y *= -w;
        buf[fpad(q)] = v;
    }
    __syncthreads();
    stockham_fft<CT, n>(buf, twp, tid);
    T *ya = Y + ja * ldy + ta * n;
    T *yb = Y + jb * ldy + tb * n;
    const T *aa = addX ? addX + ja * ld_add + ta * n : nullptr;
    const T *ab = addX ? addX + jb * ld_add + tb * n : nullptr;
    // the added vectors are read into registers before any store: Y may
    // alias them as far as the compiler knows, which would otherwise
    // serialise one global load latency per value
    T ra[16], rb[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int s = tid + i * nt;
        ra[i] = aa ? aa[s] : (T)0;
        rb[i] = (hasb && ab) ? ab[s] : (T)0;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int s = tid + i * nt;
        const CT v = buf[fpad(s)];
        ya[s] = v.x + ra[i];
        if (hasb) yb[s] = -v.y + rb[i];
    }
}

template <typename T, int LOGN>
static void launch_stockham(cudaStream_t s, int grid, size_t smem, int N, int K, const T *X, int64_t ldx, T *Y,
                            int64_t ldy, const T *addX, int64_t ld_add, const T *specB, const T *specQ,
                            const void *twp, int nB)
{
    // once per instantiation (smem is fixed by T and LOGN); a function-local
    // static is initialised once even when host threads launch concurrently
    static const bool attr = [smem] {
        return cudaFuncSetAttribute(k_circ_stockham<T, LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem) == cudaSuccess;
    }();
    (void)attr;
    WC4D_LAUNCH(k_circ_stockham<T, LOGN><<<grid, (1 << LOGN) / 16, smem, s>>>(
        N, K, X, ldx, Y, ldy, addX, ld_add, specB, specQ, (const typename Cplx<T>::t *)twp, nB));
}

// Direct symmetric circulant product for any n: y_s = sum_r row[r] x[(s+r) mod n].
template <typename T>
__global__ void __launch_bounds__(256)
k_circ_direct(int n, int N, int K, const T *__restrict__ X, int64_t ldx, T *Y, int64_t ldy, const T *addX,
              int64_t ld_add, const T *__restrict__ rowB, const T *__restrict__ rowQ, int skip)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *xs = reinterpret_cast<T *>(smem_raw);
    T *rs = xs + n;
    int64_t v = blockIdx.x;
    int64_t j = v / (N + 1), t = v % (N + 1);
    if (skip & (t == 0 ? 1 : 2)) return;   // block handled elsewhere (dense square root)
    const T *row = (t == 0) ? rowB : rowQ;
    const T *x = X + j * ldx + t * n;
    for (int s = threadIdx.x; s < n; s += blockDim.x) { xs[s] = x[s]; rs[s] = row[s]; }
    __syncthreads();
    T *y = Y + j * ldy + t * n;
    const T *a = addX ? addX + j * ld_add + t * n : nullptr;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        T acc = 0;
        int idx = s;
        for (int r = 0; r < n; ++r) {
            acc += rs[r] * xs[idx];
            idx = (idx + 1 == n) ? 0 : idx + 1;
        }
        y[s] = acc + (a ? a[s] : (T)0);
    }
}

// Y = sd X (+ addX) on time blocks t0 .. t1-1 of K columns: a covariance
// block that is a multiple of the identity needs no transform.
template <typename T>
__global__ void k_diag_blocks(int n, int t0, int t1, int K, const T *__restrict__ X, int64_t ldx, T *Y, int64_t ldy,
                              const T *addX, int64_t ld_add, T sd)
{
    const int64_t per = (int64_t)(t1 - t0) * n, tot = per * K;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / per, r = (int64_t)t0 * n + e % per;
        const T v = sd * X[j * ldx + r];
        Y[j * ldy + r] = addX ? v + addX[j * ld_add + r] : v;
    }
}

template <typename T>
static void launch_diag_blocks(cudaStream_t s, const wc4d_ctx *c, int t0, int t1, int K, const T *X, int64_t ldx,
                               T *Y, int64_t ldy, const T *addX, int64_t ld_add, double sd)
{
    const int64_t tot = (int64_t)(t1 - t0) * c->prob.n * K;
    const int grid = (int)std::min<int64_t>((tot + 255) / 256, 8 * (int64_t)c->num_sms);
    WC4D_LAUNCH(k_diag_blocks<T><<<grid, 256, 0, s>>>(c->prob.n, t0, t1, K, X, ldx, Y, ldy, addX, ld_add, (T)sd));
}

template <typename T>
void launch_circulant(cudaStream_t s, const wc4d_ctx *c, int K, const T *X, int64_t ldx, T *Y, int64_t ldy,
                      const T *addX, int64_t ld_add, bool fft, const T *specB, const T *specQ, const T *rowB,
                      const T *rowQ, const void *tw, int skip)
{
    const int n = c->prob.n, N = c->prob.N;
    // the FFT path transforms only the non-diagonal covariance blocks
    // (Lorenz-96: Q = 0.05 I needs no transform for its N blocks); blocks in
    // `skip` are left to the caller
    const double sdB = (skip & 1) ? -2.0 : c->cov_sd[0], sdQ = (skip & 2) ? -2.0 : c->cov_sd[1];
    const bool doneB = (skip & 1) || sdB >= 0.0, doneQ = (skip & 2) || sdQ >= 0.0;
    if (fft && (doneB || doneQ)) {
        if (sdB >= 0.0) launch_diag_blocks<T>(s, c, 0, 1, K, X, ldx, Y, ldy, addX, ld_add, sdB);
        if (sdQ >= 0.0) launch_diag_blocks<T>(s, c, 1, N + 1, K, X, ldx, Y, ldy, addX, ld_add, sdQ);
        if (doneB && doneQ) return;
    }
    if (fft) {
        size_t smem = (size_t)(n + n / 16 + n / 2) * sizeof(typename Cplx<T>::t);
        static const bool attr = [] {
            return cudaFuncSetAttribute(k_circ_fft<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)((WC4D_FFT_MAX_N + WC4D_FFT_MAX_N / 16 + WC4D_FFT_MAX_N / 2) *
                                              sizeof(typename Cplx<T>::t))) == cudaSuccess;
        }();
        (void)attr;
        int nB = (K + 1) / 2;
        int64_t nQ = ((int64_t)K * N + 1) / 2;
        int grid = (int)(nB + nQ);
        if (doneQ) grid = nB;                      // block 0 only (pairs < nB are B's)
        else if (doneB) { grid = (int)nQ; nB = 0; }  // Q blocks only
        const void *twp = sizeof(T) == 8 ? c->twp64.p : c->twp32.p;   // per-pass twiddles (n >= 512)
        const size_t smem_s = (size_t)(n + n / 16) * sizeof(typename Cplx<T>::t);
        switch (c->logn) {   // n / 16 threads, 16 values each
        case 9: launch_stockham<T, 9>(s, grid, smem_s, N, K, X, ldx, Y, ldy, addX, ld_add, specB, specQ, twp, nB); return;
        case 10: launch_stockham<T, 10>(s, grid, smem_s, N, K, X, ldx, Y, ldy, addX, ld_add, specB, specQ, twp, nB); return;
        case 11: launch_stockham<T, 11>(s, grid, smem_s, N, K, X, ldx, Y, ldy, addX, ld_add, specB, specQ, twp, nB); return;
        case 12: launch_stockham<T, 12>(s, grid, smem_s, N, K, X, ldx, Y, ldy, addX, ld_add, specB, specQ, twp, nB); return;
        case 13: launch_stockham<T, 13>(s, grid, smem_s, N, K, X, ldx, Y, ldy, addX, ld_add, specB, specQ, twp, nB); return;
        default: break;
        }
        WC4D_LAUNCH(k_circ_fft<T><<<grid, 512, smem, s>>>(n, c->logn, N, K, X, ldx, Y, ldy, addX, ld_add, specB, specQ,
                                              (const typename Cplx<T>::t *)tw, nB));
    } else {
        size_t smem = 2 * (size_t)n * sizeof(T);
        static const bool attr = [] {
            return cudaFuncSetAttribute(k_circ_direct<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)(2 * WC4D_FFT_MAX_N * sizeof(T))) == cudaSuccess;
        }();
        (void)attr;
        int64_t grid = (int64_t)K * (N + 1);
        WC4D_LAUNCH(k_circ_direct<T><<<(unsigned)grid, 256, smem, s>>>(n, N, K, X, ldx, Y, ldy, addX, ld_add, rowB, rowQ,
                                                                       skip));
    }
}

template void launch_circulant<double>(cudaStream_t, const wc4d_ctx *, int, const double *, int64_t, double *,
                                       int64_t, const double *, int64_t, bool, const double *, const double *,
                                       const double *, const double *, const void *, int);
template void launch_circulant<float>(cudaStream_t, const wc4d_ctx *, int, const float *, int64_t, float *,
                                      int64_t, const float *, int64_t, bool, const float *, const float *,
                                      const float *, const float *, const void *, int);

// ----------------------------------------------------------------------------
// SIMT GEMM: C(i,j) = epi(sum_k A(i,k) B(k,j)); A(i,k) = A[i*sam + k*sak],
// B(k,j) = B[k + j*ldb] (column-major, k contiguous), C column-major.
// BM x BN tile per CTA, BK-deep k slices staged in shared memory, TM x TN
// outputs per thread (rows strided by BM/TM so that a warp stores
// consecutive rows of the column-major C).
// ----------------------------------------------------------------------------
template <typename Acc>
__device__ __forceinline__ Acc apply_epi(const Epi &e, Acc acc, int i, const Acc *old)
{
    if (e.mode == 1) {
        Acc o = (i % e.obs_stride == 0) ? (Acc)e.obs_scale * (*old) : (Acc)0;
        return acc + o;
    }
    Acc r = (Acc)e.alpha * acc;
    if (e.beta != 0.0) r += (Acc)e.beta * (*old);
    return r;
}

template <typename T, typename Acc, int BM, int BN, int BK, int TM, int TN, bool A_KCONTIG>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_gemm_simt(int Mrows, int Ncols, int Kdim, const T *__restrict__ A, int64_t sam, int64_t sak,
            const T *__restrict__ B, int64_t ldb, T *C, int64_t ldc, Epi e)
{
    constexpr int RT = BM / TM, CTt = BN / TN, NT = RT * CTt;
    __shared__ Acc As[BK][BM + 1];
    __shared__ Acc Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tr = tid % RT, tc = tid / RT;
    const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
    Acc acc[TM][TN];
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int q = 0; q < TN; ++q) acc[r][q] = (Acc)0;

    for (int k0 = 0; k0 < Kdim; k0 += BK) {
        for (int l = tid; l < BM * BK; l += NT) {
            int i, kk;
            if (A_KCONTIG) { kk = l % BK; i = l / BK; }
            else { i = l % BM; kk = l / BM; }
            int64_t gi = m0 + i;
            int gk = k0 + kk;
            As[kk][i] = (gi < Mrows && gk < Kdim) ? (Acc)A[gi * sam + (int64_t)gk * sak] : (Acc)0;
        }
        for (int l = tid; l < BN * BK; l += NT) {
            int kk = l % BK, j = l / BK;
            int64_t gj = n0 + j;
            int gk = k0 + kk;
            Bs[kk][j] = (gj < Ncols && gk < Kdim) ? (Acc)B[gk + gj * ldb] : (Acc)0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            Acc a[TM], b[TN];
#pragma unroll
            for (int r = 0; r < TM; ++r) a[r] = As[kk][tr + r * RT];
#pragma unroll
            for (int q = 0; q < TN; ++q) b[q] = Bs[kk][tc + q * CTt];
#pragma unroll
            for (int r = 0; r < TM; ++r)
#pragma unroll
                for (int q = 0; q < TN; ++q) acc[r][q] = fma(a[r], b[q], acc[r][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int q = 0; q < TN; ++q) {
            int64_t i = m0 + tr + r * RT, j = n0 + tc + q * CTt;
            if (i < Mrows && j < Ncols) {
                T *dst = C + i + j * ldc;
                Acc old = (e.mode == 1 || e.beta != 0.0) ? (Acc)(*dst) : (Acc)0;
                *dst = (T)apply_epi<Acc>(e, acc[r][q], (int)i, &old);
            }
        }
}

// y = epi(M x) for the row-major n x n M.  Each warp owns RPW consecutive
// rows; every lane keeps UNR vector loads per row in flight (the kernel is
// bound by HBM latency x bytes in flight), M is read with evict-first
// streaming loads so that x stays in L1 for all warps of the SM.  Small CTAs
// (2 warps) spread the rows evenly over the 152 SMs.
template <typename T, typename Acc, int RPW, int UNR>
__global__ void __launch_bounds__(64)
k_gemv_rows(int n, const T *__restrict__ M, const T *__restrict__ x, T *y, Epi e)
{
    using V = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
    constexpr int VEC = sizeof(V) / sizeof(T);
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int row0 = warp * RPW;
    if (row0 >= n) return;
    const int nv = n / VEC;
    const V *x4 = reinterpret_cast<const V *>(x);
    const V *r4[RPW];
#pragma unroll
    for (int r = 0; r < RPW; ++r) r4[r] = reinterpret_cast<const V *>(M + (int64_t)min(row0 + r, n - 1) * n);
    Acc acc[RPW];
#pragma unroll
    for (int r = 0; r < RPW; ++r) acc[r] = 0;
    for (int c0 = lane; c0 < nv; c0 += 32 * UNR) {
        V a[RPW][UNR], b[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const int idx = c0 + 32 * u;
            if (idx < nv) {
                b[u] = __ldg(x4 + idx);
#pragma unroll
                for (int r = 0; r < RPW; ++r) a[r][u] = __ldcs(r4[r] + idx);
            }
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            if (c0 + 32 * u < nv) {
                const T *bf = reinterpret_cast<const T *>(&b[u]);
#pragma unroll
                for (int r = 0; r < RPW; ++r) {
                    const T *af = reinterpret_cast<const T *>(&a[r][u]);
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[r] = fma((Acc)af[v], (Acc)bf[v], acc[r]);
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    }
    if (lane < RPW && row0 + lane < n) {
        Acc mine = acc[0];
#pragma unroll
        for (int r = 1; r < RPW; ++r)
            if (lane == r) mine = acc[r];
        const int row = row0 + lane;
        Acc old = (e.mode == 1 || e.beta != 0.0) ? (Acc)y[row] : (Acc)0;
        y[row] = (T)apply_epi<Acc>(e, mine, row, &old);
    }
}

// Scalar fallback for n not a multiple of the vector width or unaligned operands.
template <typename T, typename Acc>
__global__ void __launch_bounds__(256)
k_gemv_scalar(int n, const T *__restrict__ M, const T *__restrict__ x, T *y, Epi e)
{
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const T *row = M + (int64_t)warp * n;
    Acc acc = 0;
    for (int c = lane; c < n; c += 32) acc = fma((Acc)row[c], (Acc)__ldg(x + c), acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        Acc old = (e.mode == 1 || e.beta != 0.0) ? (Acc)y[warp] : (Acc)0;
        y[warp] = (T)apply_epi<Acc>(e, acc, warp, &old);
    }
}

template <typename T>
static bool aligned16(const T *p) { return ((uintptr_t)p & 15u) == 0; }

// ----------------------------------------------------------------------------
// Persistent one-column sweep (the PCG matvec): all N subwindow GEMVs of
// L^{-1} (mode 0) or of L^{-T} with the observation term (mode 1) in one
// cooperative launch.  CTA b owns a fixed slice of rows of every M_t; after
// its rows of step t are written it waits at a bounded grid barrier.
// Vectors written by other SMs are read
// through L2 (ld.global.cg), never through the non-coherent L1.  (Measured on
// GB300, n = 4096 FP32: 13.7 us per subwindow with this barrier; prefetching
// the next propagator into L2 or registers made it slower.)
// ----------------------------------------------------------------------------
struct SweepArgs {
    int n, N;
    int64_t mstride;      // elements between consecutive subwindow propagators (0: shared)
    int mode;             // 0 forward, 1 adjoint with observations
    double obs_inv;       // 1 / sigma_o^2
    int obs_stride, t0, ts;
    int rows_per_cta;     // multiple of 2
    int pf;               // staged form: stages prefetched into L2 ahead of the ring
    unsigned *bar;        // N zeroed arrival counters, one per step barrier
    int *err;
    unsigned wait_limit;  // polls of a barrier before it gives up (0: fail unless already complete)
};

// Grid barrier of step t: every CTA adds one to its own counter cnt[t]
// (release) and waits until it reads nblocks (acquire).  Counters are zeroed
// before each launch, so no reset or generation word is needed.  Bounded: after
// `limit` unsuccessful polls it records the error and returns false (limit 0:
// fail unless the barrier is already complete at the first poll).
__device__ __forceinline__ bool step_barrier(unsigned *cnt, int t, unsigned nblocks, int *err, unsigned limit)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(cnt + t) : "memory");
        unsigned v = 0, it = 0;
        int ok = 1;
        for (;;) {
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(cnt + t) : "memory");
            if (v >= nblocks) break;
            if (it++ >= limit) { ok = 0; atomicExch(err, 1); break; }
        }
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// Loads of a propagator row.  A propagator shared by every subwindow (the
// time-invariant case) is read N times per sweep and is loaded with the
// default L2 policy (ld.global.cg) so that it may stay resident between
// subwindows; otherwise each M_t is read once per sweep and streams with
// evict-first loads.
template <bool KEEP, typename V> __device__ __forceinline__ V ld_row(const V *p) { return KEEP ? __ldcg(p) : __ldcs(p); }

template <typename T, typename Acc, bool KEEP>
__global__ void __launch_bounds__(512)
k_gemv_sweep(const T *__restrict__ M0, T *W, SweepArgs a)
{
    using V = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
    constexpr int VEC = sizeof(V) / sizeof(T), UNR = sizeof(T) == 4 ? 8 : 4;   // 128 B of each row in flight per lane (FP32)
    const int n = a.n, nv = n / VEC;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int rbeg = blockIdx.x * a.rows_per_cta;
    const int rend = min(n, rbeg + a.rows_per_cta);
    for (int step = 0; step < a.N; ++step) {
        const int t = (a.mode == 0) ? step : a.N - 1 - step;
        const T *M = M0 + (int64_t)t * a.mstride;
        const T *x = W + (int64_t)((a.mode == 0) ? t : t + 1) * n;       // source block
        T *y = W + (int64_t)((a.mode == 0) ? t + 1 : t) * n;             // target block
        const V *x4 = reinterpret_cast<const V *>(x);
        double scale = 0.0;
        if (a.mode == 1 && t >= a.t0 && (t - a.t0) % a.ts == 0) scale = a.obs_inv;
        for (int r0 = rbeg + 2 * warp; r0 < rend; r0 += 2 * nwarps) {
            const V *ra = reinterpret_cast<const V *>(M + (int64_t)r0 * n);
            const V *rb = reinterpret_cast<const V *>(M + (int64_t)min(r0 + 1, n - 1) * n);
            Acc acc0 = 0, acc1 = 0;
            for (int c0 = lane; c0 < nv; c0 += 32 * UNR) {
                V av[UNR], bv[UNR], xv[UNR];
#pragma unroll
                for (int u = 0; u < UNR; ++u) {
                    const int idx = c0 + 32 * u;
                    if (idx < nv) {
                        xv[u] = __ldcg(x4 + idx);
                        av[u] = ld_row<KEEP>(ra + idx);
                        bv[u] = ld_row<KEEP>(rb + idx);
                    }
                }
#pragma unroll
                for (int u = 0; u < UNR; ++u) {
                    if (c0 + 32 * u < nv) {
                        const T *xf = reinterpret_cast<const T *>(&xv[u]);
                        const T *af = reinterpret_cast<const T *>(&av[u]);
                        const T *bf = reinterpret_cast<const T *>(&bv[u]);
#pragma unroll
                        for (int q = 0; q < VEC; ++q) {
                            acc0 = fma((Acc)af[q], (Acc)xf[q], acc0);
                            acc1 = fma((Acc)bf[q], (Acc)xf[q], acc1);
                        }
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                acc0 += __shfl_xor_sync(0xffffffffu, acc0, o);
                acc1 += __shfl_xor_sync(0xffffffffu, acc1, o);
            }
            if (lane < 2 && r0 + lane < rend) {
                const int row = r0 + lane;
                const Acc sum = lane ? acc1 : acc0;
                const Acc old = (Acc)__ldcg(y + row);
                Acc out;
                if (a.mode == 0) out = old + sum;
                else out = sum + ((row % a.obs_stride == 0) ? (Acc)scale * old : (Acc)0);
                y[row] = (T)out;
            }
        }
        if (step + 1 < a.N && !step_barrier(a.bar, step, gridDim.x, a.err, a.wait_limit)) return;
    }
}

// ----------------------------------------------------------------------------
// Staged form of the persistent FP32 sweep for n a multiple of 2048 (n =
// 2048, 4096, 8192): the same work split (CTA b owns rows [b R, b R + R) of
// every M_t), with the propagator rows brought into a ring of shared memory
// by a producer warp through bulk asynchronous copies (one cp.async.bulk per
// row, completion counted on a "full" mbarrier per slot).  Sixteen consumer
// warps each own a fixed set of J = n / 2048 float4 column slots of every
// row (slot j of thread i: columns 4 (i + 512 j) .. + 3), so the x values they
// need sit in registers for a whole subwindow; after reading a stage they
// arrive on the slot's "empty" mbarrier and the producer refills it.  The
// producer is not part of the grid barrier: it runs SW_NS stages ahead across
// subwindow boundaries (the rows of M_{t+1} do not depend on x), so the copy
// engine keeps streaming while the consumers wait for x_{t+1}; once the ring
// is full it prefetches a few further rows into L2, so that HBM does not
// idle during the grid barrier either.  Row sums: warp shuffle, then the 16
// warp partials in a fixed order.  All waits are bounded; after a
// grid-barrier timeout the consumers keep draining the ring (without further
// barriers) so that no copy is in flight when the CTA exits.  Measured on
// GB300 (n = 4096, N = 40, 2.7 GB of propagators): 411 us per sweep with an
// L2 look-ahead of 2 to 8 rows (447 us without, 434 us at 16 rows, 734 us at
// 32) against 491 us for per-thread cp.async staging and 533 us for the
// register-staged k_gemv_sweep.
// ----------------------------------------------------------------------------
constexpr int SW_THREADS = 512;                       // consumer threads
constexpr int SW_RING = 192 * 1024;                   // bytes of shared memory in the ring
constexpr int SW_RMAX = 64;                           // rows per CTA
constexpr int SW_PF = 4;                              // default L2 look-ahead, stages

template <int J> struct SwShape {
    static constexpr int G = J == 1 ? 2 : 1;                          // rows per stage
    static constexpr int NS = SW_RING / (G * J * SW_THREADS * 16);    // stages in the ring
};

// barrier of the 512 consumer threads only (the producer warp is not in it)
__device__ __forceinline__ void sw_cbar() { asm volatile("bar.sync 1, 512;" ::: "memory"); }

// step_barrier for the consumer threads
__device__ __forceinline__ bool sw_step_barrier(unsigned *cnt, int t, unsigned nblocks, int *err)
{
    __shared__ int ok_c;
    sw_cbar();
    if (threadIdx.x == 0) {
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(cnt + t) : "memory");
        unsigned v = 0, it = 0;
        int ok = 1;
        do {
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(cnt + t) : "memory");
            if (++it > (1u << 22)) { ok = 0; atomicExch(err, 1); break; }
        } while (v < nblocks);
        ok_c = ok;
    }
    sw_cbar();
    return ok_c != 0;
}

__device__ __forceinline__ float dot_acc(float4 m, float4 x, float acc)
{
    acc = fmaf(m.x, x.x, acc);
    acc = fmaf(m.y, x.y, acc);
    acc = fmaf(m.z, x.z, acc);
    return fmaf(m.w, x.w, acc);
}

template <int J>
__global__ void __launch_bounds__(SW_THREADS + 32, 1) k_gemv_sweep_staged(const float *__restrict__ M0, float *W,
                                                                          SweepArgs a)
{
    constexpr int G = SwShape<J>::G, NS = SwShape<J>::NS;
    extern __shared__ __align__(128) unsigned char sw_smem[];
    __shared__ __align__(8) unsigned long long mbar[2 * NS];   // full[NS] | empty[NS]
    __shared__ float part[SW_RMAX][SW_THREADS / 32];
    const float4 *ring = reinterpret_cast<const float4 *>(sw_smem);   // [NS][G][n / 4]
    const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(sw_smem);
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);
    const int n = a.n, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rbeg = blockIdx.x * a.rows_per_cta;
    const int R = max(0, min(n, rbeg + a.rows_per_cta) - rbeg);
    const int S = (R + G - 1) / G;   // stages per subwindow
    const int total = a.N * S;
    const unsigned rowb = (unsigned)n * 4u;
    // bulk copies need 16-byte aligned addresses and sizes: the condition is
    // the same in every CTA, so a failed check exits the whole grid
    if ((ring_s & 15u) != 0u || (reinterpret_cast<uintptr_t>(M0) & 15u) != 0u ||
        (reinterpret_cast<uintptr_t>(W) & 15u) != 0u || (rowb & 15u) != 0u) {
        if (blockIdx.x == 0 && tid == 0) atomicExch(a.err, 2);
        return;
    }
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            sw_mb_init(mb + 8 * i, 1);
            sw_mb_init(mb + 8 * (NS + i), SW_THREADS / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == SW_THREADS / 32) {   // producer warp: one thread issues
        if (lane == 0) {
            // rows of stage kk: M_t rows [rbeg + s0, rbeg + s0 + rows)
            auto stage_rows = [&](int kk, int &rows) -> const float * {
                const int step = kk / S, s0 = (kk % S) * G;
                rows = min(G, R - s0);
                const int t = (a.mode == 0) ? step : a.N - 1 - step;
                return M0 + (int64_t)t * a.mstride + (int64_t)(rbeg + s0) * n;
            };
            // L2 look-ahead: stage k + pf is prefetched when stage k is
            // copied, so HBM keeps streaming while the ring is full (during
            // the grid barrier and the read of x_{t+1}); stages the ring
            // takes straight away need none
            for (int kk = NS; kk < min(a.pf, total); ++kk) {
                int pr;
                const float *P = stage_rows(kk, pr);
                sw_prefetch_l2(P, rowb * (unsigned)pr);
            }
            for (int k = 0; k < total; ++k) {
                const int slot = k % NS;
                if (a.pf > 0 && k + a.pf < total && k + a.pf >= NS) {
                    int pr;
                    const float *P = stage_rows(k + a.pf, pr);
                    sw_prefetch_l2(P, rowb * (unsigned)pr);
                }
                if (k >= NS && !sw_mb_wait(mb + 8 * (NS + slot), ((k / NS) - 1) & 1)) {
                    atomicExch(a.err, 3);
                    break;
                }
                int rows;
                const float *M = stage_rows(k, rows);
                sw_mb_expect(mb + 8 * slot, rowb * (unsigned)rows);
                for (int g = 0; g < rows; ++g)
                    sw_bulk_g2s(ring_s + (uint32_t)(slot * G + g) * rowb, M + (int64_t)g * n, rowb, mb + 8 * slot);
            }
        }
        return;
    }

    const int nv = n / 4;
    int k = 0;
    bool bad = false;    // a grid barrier timed out
    bool dead = false;   // a ring wait of this thread timed out
    for (int step = 0; step < a.N; ++step) {
        const int t = (a.mode == 0) ? step : a.N - 1 - step;
        const float4 *x4 = reinterpret_cast<const float4 *>(W + (int64_t)((a.mode == 0) ? t : t + 1) * n);
        float *y = W + (int64_t)((a.mode == 0) ? t + 1 : t) * n;
        float4 xr[J];
#pragma unroll
        for (int j = 0; j < J; ++j) xr[j] = __ldcg(x4 + tid + SW_THREADS * j);
        for (int s = 0; s < S; ++s, ++k) {
            const int slot = k % NS;
            // after a timed-out wait the thread stops waiting but follows the
            // same path on the stale slot, so that every lane reaches every
            // __syncwarp and CTA barrier; the copies still in flight are
            // waited for (bounded) before the CTA exits
            if (!dead && !sw_mb_wait(mb + 8 * slot, (k / NS) & 1)) {
                dead = true;
                atomicExch(a.err, 4);
            }
            float v[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                float acc = 0.f;
                if (s * G + g < R) {
#pragma unroll
                    for (int j = 0; j < J; ++j)
                        acc = dot_acc(ring[(slot * G + g) * nv + tid + SW_THREADS * j], xr[j], acc);
                }
                v[g] = acc;
            }
            __syncwarp();
            if (lane == 0) sw_mb_arrive(mb + 8 * (NS + slot));   // the slot may be refilled
#pragma unroll
            for (int g = 0; g < G; ++g) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v[g] += __shfl_xor_sync(0xffffffffu, v[g], o);
                if (lane == 0 && s * G + g < R) part[s * G + g][warp] = v[g];
            }
        }
        sw_cbar();
        if (tid < R) {
            float sum = 0.f;
#pragma unroll
            for (int i = 0; i < SW_THREADS / 32; ++i) sum += part[tid][i];
            const int row = rbeg + tid;
            const float old = __ldcg(y + row);
            float out;
            if (a.mode == 0) {
                out = old + sum;
            } else {
                const bool obs = (t >= a.t0 && (t - a.t0) % a.ts == 0 && row % a.obs_stride == 0);
                out = sum + (obs ? (float)a.obs_inv * old : 0.f);
            }
            y[row] = out;
        }
        if (step + 1 < a.N) {
            if (!bad) bad = !sw_step_barrier(a.bar, step, gridDim.x, a.err);
            else sw_cbar();   // keep draining the ring after a barrier timeout
        }
    }
    if (dead) {   // copies may still be in flight into the ring: wait (bounded) for the last one of every slot
        for (int kk = max(0, total - NS); kk < total; ++kk) sw_mb_wait(mb + 8 * (kk % NS), (kk / NS) & 1);
    }
}

template <int J>
static bool launch_sweep_staged(cudaStream_t s, int num_sms, const float *M0, float *W, SweepArgs &args)
{
    const void *fn = (const void *)k_gemv_sweep_staged<J>;
    const int smem = SwShape<J>::NS * SwShape<J>::G * J * SW_THREADS * 16;
    static const bool st = [fn, smem] {
        int per_sm = 0;
        const bool ok = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess &&
                        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, SW_THREADS + 32, smem) ==
                            cudaSuccess &&
                        per_sm >= 1;
        cudaGetLastError();
        return ok;
    }();
    if (!st) return false;
    const int n = args.n;
    const int rpc = ceil_div(n, num_sms);
    if (rpc > SW_RMAX) return false;
    args.rows_per_cta = rpc;
    static const int pf = [] {
        const char *e = getenv("WC4D_SWEEP_PF");
        return e ? std::max(0, atoi(e)) : SW_PF;
    }();
    args.pf = pf;
    const int grid = ceil_div(n, rpc);
    void *params[] = {(void *)&M0, (void *)&W, (void *)&args};
    wc4d_note_launch();
    if (cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(SW_THREADS + 32), params, smem, s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

// Launch configuration of the persistent sweep (one CTA of 512 threads per
// SM, co-resident by cooperative launch).  Returns false if it cannot be used.
template <typename T>
bool launch_gemv_sweep(cudaStream_t s, int num_sms, int n, int N, const T *M0, int64_t mstride, T *W, int mode,
                       double obs_inv, int obs_stride, int t0, int ts, unsigned *bar, int *err, unsigned wait_limit)
{
    constexpr int VEC = sizeof(T) == 8 ? 2 : 4;
    if (n % VEC != 0 || !aligned16(M0) || !aligned16(W) || ((int64_t)n * sizeof(T)) % 16 != 0) return false;
    using Acc = T;
    const bool keep = (mstride == 0 && N > 1);
    const void *fn = keep ? (const void *)k_gemv_sweep<T, Acc, true> : (const void *)k_gemv_sweep<T, Acc, false>;
    static const int mb = [num_sms] {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gemv_sweep<T, Acc, false>, 512, 0);
        int per_sm_keep = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_keep, k_gemv_sweep<T, Acc, true>, 512, 0);
        return std::min(per_sm, per_sm_keep) * num_sms;
    }();
    int grid = std::min(num_sms, mb);
    if (grid < 1) return false;
    SweepArgs args;
    args.n = n;
    args.N = N;
    args.pf = 0;
    args.mstride = mstride;
    args.mode = mode;
    args.obs_inv = obs_inv;
    args.obs_stride = obs_stride;
    args.t0 = t0;
    args.ts = ts > 0 ? ts : 1;
    args.bar = bar;
    args.err = err;
    args.wait_limit = wait_limit;
    {
        // FP32 only: the FP64 sweep is bound by the FP64 pipe, where the
        // per-row shuffle reductions of the staged form cost more than the
        // barrier time it hides
        if constexpr (sizeof(T) == 4) {
            const int slots = n / (SW_THREADS * VEC);   // J
            if (n % (SW_THREADS * VEC) == 0) {
                if (slots == 1 && launch_sweep_staged<1>(s, num_sms, M0, W, args)) return true;
                if (slots == 2 && launch_sweep_staged<2>(s, num_sms, M0, W, args)) return true;
                if (slots == 4 && launch_sweep_staged<4>(s, num_sms, M0, W, args)) return true;
            }
        }
    }
    int rpc = (n + grid - 1) / grid;
    rpc = (rpc + 1) / 2 * 2;
    grid = (n + rpc - 1) / rpc;
    args.rows_per_cta = rpc;
    args.bar = bar;
    args.err = err;
    void *params[] = {(void *)&M0, (void *)&W, (void *)&args};
    wc4d_note_launch();
    if (cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(512), params, 0, s) !=
        cudaSuccess) {
        cudaGetLastError();   // fall back to one launch per subwindow
        return false;
    }
    return true;
}

template bool launch_gemv_sweep<double>(cudaStream_t, int, int, int, const double *, int64_t, double *, int, double,
                                        int, int, int, unsigned *, int *, unsigned);
template bool launch_gemv_sweep<float>(cudaStream_t, int, int, int, const float *, int64_t, float *, int, double,
                                       int, int, int, unsigned *, int *, unsigned);

// ----------------------------------------------------------------------------
// Double-float form of the staged sweep, for the FP64 product of the mixed
// CG's true residual.  Each FP64 propagator entry is held as its FP32
// rounding Mh (the mixed path's FP32 copy) plus the FP32 rounding of the
// remainder Ml = M - Mh (48 bits in all, 8 bytes per entry as in FP64), and
// the vector as hi / lo floats; every term (Mh + Ml)(xh + xl) is summed as
// Mh xh exactly (TwoProduct by FMA) plus Mh xl + Ml xh into a double-float
// accumulator (TwoSum), so the FP32 pipe does the work of the FP64 pipe,
// which runs at 1/64 of its rate on this GPU, and the sweep is bound by
// HBM again.  Same work split, ring and grid barriers as the FP32 staged
// sweep; a stage carries G rows of Mh and G rows of Ml.  The row finaliser
// writes the FP64 result and its hi / lo split (Wh, Wl), which the next
// subwindow reads; the first subwindow splits its FP64 input itself.
// ----------------------------------------------------------------------------
template <int J> struct SwShapeDf {
    static constexpr int G = J == 1 ? 2 : 1;                              // rows per stage
    static constexpr int NS = SW_RING / (2 * G * J * SW_THREADS * 16);    // stages in the ring
};

__device__ __forceinline__ void df_two_sum(float &s, float &c, float p)
{
    const float t = __fadd_rn(s, p), bp = __fsub_rn(t, s);
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp)));
    s = t;
}

// s + c += (a + al)(b + bl), dropping al bl
__device__ __forceinline__ void df_term(float a, float al, float b, float bl, float &s, float &c)
{
    const float p = __fmul_rn(a, b);
    const float e = fmaf(a, b, -p);   // a b = p + e exactly
    df_two_sum(s, c, p);
    c = __fadd_rn(c, fmaf(a, bl, fmaf(al, b, e)));
}

__device__ __forceinline__ void df_split(double x, float &h, float &l)
{
    h = __double2float_rn(x);
    l = __double2float_rn(x - (double)h);
}

template <int J>
__global__ void __launch_bounds__(SW_THREADS + 32, 1)
k_gemv_sweep_df(const float *__restrict__ Mh0, const float *__restrict__ Ml0, double *W, float *Wh, float *Wl,
                SweepArgs a)
{
    constexpr int G = SwShapeDf<J>::G, NS = SwShapeDf<J>::NS;
    extern __shared__ __align__(128) unsigned char sw_smem[];
    __shared__ __align__(8) unsigned long long mbar[2 * NS];   // full[NS] | empty[NS]
    __shared__ float part_s[SW_RMAX][SW_THREADS / 32], part_c[SW_RMAX][SW_THREADS / 32];
    const float4 *ring = reinterpret_cast<const float4 *>(sw_smem);   // [NS][2][G][n / 4]: hi rows, then lo rows
    const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(sw_smem);
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);
    const int n = a.n, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rbeg = blockIdx.x * a.rows_per_cta;
    const int R = max(0, min(n, rbeg + a.rows_per_cta) - rbeg);
    const int S = (R + G - 1) / G;   // stages per subwindow
    const int total = a.N * S;
    const unsigned rowb = (unsigned)n * 4u;
    if ((ring_s & 15u) != 0u || (reinterpret_cast<uintptr_t>(Mh0) & 15u) != 0u ||
        (reinterpret_cast<uintptr_t>(Ml0) & 15u) != 0u || (reinterpret_cast<uintptr_t>(Wh) & 15u) != 0u ||
        (reinterpret_cast<uintptr_t>(Wl) & 15u) != 0u || (reinterpret_cast<uintptr_t>(W) & 15u) != 0u ||
        (rowb & 15u) != 0u) {
        if (blockIdx.x == 0 && tid == 0) atomicExch(a.err, 2);
        return;
    }
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            sw_mb_init(mb + 8 * i, 1);
            sw_mb_init(mb + 8 * (NS + i), SW_THREADS / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == SW_THREADS / 32) {   // producer warp: one thread issues
        if (lane == 0) {
            for (int k = 0; k < total; ++k) {
                const int slot = k % NS;
                if (k >= NS && !sw_mb_wait(mb + 8 * (NS + slot), ((k / NS) - 1) & 1)) {
                    atomicExch(a.err, 3);
                    break;
                }
                const int step = k / S, s0 = (k % S) * G;
                const int rows = min(G, R - s0);
                const int t = (a.mode == 0) ? step : a.N - 1 - step;
                const int64_t off = (int64_t)t * a.mstride + (int64_t)(rbeg + s0) * n;
                sw_mb_expect(mb + 8 * slot, 2u * rowb * (unsigned)rows);
                for (int g = 0; g < rows; ++g) {
                    sw_bulk_g2s(ring_s + (uint32_t)((slot * 2 + 0) * G + g) * rowb, Mh0 + off + (int64_t)g * n, rowb,
                                mb + 8 * slot);
                    sw_bulk_g2s(ring_s + (uint32_t)((slot * 2 + 1) * G + g) * rowb, Ml0 + off + (int64_t)g * n, rowb,
                                mb + 8 * slot);
                }
            }
        }
        return;
    }

    const int nv = n / 4;
    int k = 0;
    bool bad = false, dead = false;
    for (int step = 0; step < a.N; ++step) {
        const int t = (a.mode == 0) ? step : a.N - 1 - step;
        const int64_t xoff = (int64_t)((a.mode == 0) ? t : t + 1) * n;
        const int64_t yoff = (int64_t)((a.mode == 0) ? t + 1 : t) * n;
        float4 xh[J], xl[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int64_t e = xoff + 4 * (int64_t)(tid + SW_THREADS * j);
            if (step == 0) {   // the input block: split here
                const double2 u = __ldcg(reinterpret_cast<const double2 *>(W + e));
                const double2 v = __ldcg(reinterpret_cast<const double2 *>(W + e + 2));
                df_split(u.x, xh[j].x, xl[j].x);
                df_split(u.y, xh[j].y, xl[j].y);
                df_split(v.x, xh[j].z, xl[j].z);
                df_split(v.y, xh[j].w, xl[j].w);
            } else {           // written by the previous subwindow's finaliser
                xh[j] = __ldcg(reinterpret_cast<const float4 *>(Wh + e));
                xl[j] = __ldcg(reinterpret_cast<const float4 *>(Wl + e));
            }
        }
        for (int s = 0; s < S; ++s, ++k) {
            const int slot = k % NS;
            // after a timed-out wait the thread stops waiting but follows the
            // same path on the stale slot (every lane reaches every barrier)
            if (!dead && !sw_mb_wait(mb + 8 * slot, (k / NS) & 1)) {
                dead = true;
                atomicExch(a.err, 4);
            }
            float vs[G], vc[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                float sum = 0.f, cor = 0.f;
                if (s * G + g < R) {
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        const float4 mh = ring[((slot * 2 + 0) * G + g) * nv + tid + SW_THREADS * j];
                        const float4 ml = ring[((slot * 2 + 1) * G + g) * nv + tid + SW_THREADS * j];
                        df_term(mh.x, ml.x, xh[j].x, xl[j].x, sum, cor);
                        df_term(mh.y, ml.y, xh[j].y, xl[j].y, sum, cor);
                        df_term(mh.z, ml.z, xh[j].z, xl[j].z, sum, cor);
                        df_term(mh.w, ml.w, xh[j].w, xl[j].w, sum, cor);
                    }
                }
                vs[g] = sum;
                vc[g] = cor;
            }
            __syncwarp();
            if (lane == 0) sw_mb_arrive(mb + 8 * (NS + slot));   // the slot may be refilled
#pragma unroll
            for (int g = 0; g < G; ++g) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float s2 = __shfl_xor_sync(0xffffffffu, vs[g], o);
                    const float c2 = __shfl_xor_sync(0xffffffffu, vc[g], o);
                    vc[g] = __fadd_rn(vc[g], c2);
                    df_two_sum(vs[g], vc[g], s2);
                }
                if (lane == 0 && s * G + g < R) {
                    part_s[s * G + g][warp] = vs[g];
                    part_c[s * G + g][warp] = vc[g];
                }
            }
        }
        sw_cbar();
        if (tid < R) {
            float sum = 0.f, cor = 0.f;
#pragma unroll
            for (int i = 0; i < SW_THREADS / 32; ++i) {
                cor = __fadd_rn(cor, part_c[tid][i]);
                df_two_sum(sum, cor, part_s[tid][i]);
            }
            const int row = rbeg + tid;
            const double tot = (double)sum + (double)cor;
            const double old = __ldcg(W + yoff + row);
            double out;
            if (a.mode == 0) {
                out = old + tot;
            } else {
                const bool obs = (t >= a.t0 && (t - a.t0) % a.ts == 0 && row % a.obs_stride == 0);
                out = tot + (obs ? a.obs_inv * old : 0.0);
            }
            W[yoff + row] = out;
            float h, l;
            df_split(out, h, l);
            Wh[yoff + row] = h;
            Wl[yoff + row] = l;
        }
        if (step + 1 < a.N) {
            if (!bad) bad = !sw_step_barrier(a.bar, step, gridDim.x, a.err);
            else sw_cbar();
        }
    }
    if (dead) {   // copies may still be in flight into the ring: wait (bounded) for the last one of every slot
        for (int kk = max(0, total - NS); kk < total; ++kk) sw_mb_wait(mb + 8 * (kk % NS), (kk / NS) & 1);
    }
}

template <int J>
static bool launch_sweep_df(cudaStream_t s, int num_sms, const float *Mh0, const float *Ml0, double *W, float *Wh,
                            float *Wl, SweepArgs &args)
{
    const void *fn = (const void *)k_gemv_sweep_df<J>;
    const int smem = SwShapeDf<J>::NS * 2 * SwShapeDf<J>::G * J * SW_THREADS * 16;
    static const bool st = [fn, smem] {
        int per_sm = 0;
        const bool ok = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess &&
                        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, SW_THREADS + 32, smem) ==
                            cudaSuccess &&
                        per_sm >= 1;
        cudaGetLastError();
        return ok;
    }();
    if (!st) return false;
    const int rpc = ceil_div(args.n, num_sms);
    if (rpc > SW_RMAX) return false;
    args.rows_per_cta = rpc;
    args.pf = 0;
    const int grid = ceil_div(args.n, rpc);
    void *params[] = {(void *)&Mh0, (void *)&Ml0, (void *)&W, (void *)&Wh, (void *)&Wl, (void *)&args};
    wc4d_note_launch();
    if (cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(SW_THREADS + 32), params, smem, s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

// The double-float persistent sweep over FP64 vectors W (ld n per time
// block): n a multiple of 2048 (J = n / 2048 = 1, 2 or 4), Mh0 / Ml0 the
// FP32 propagators and remainders, Wh / Wl FP32 scratch of W's size.
// Returns false (nothing launched) when it does not apply.
bool launch_gemv_sweep_df(cudaStream_t s, int num_sms, int n, int N, const float *Mh0, const float *Ml0,
                          int64_t mstride, double *W, float *Wh, float *Wl, int mode, double obs_inv, int obs_stride,
                          int t0, int ts, unsigned *bar, int *err, unsigned wait_limit)
{
    if (n % (SW_THREADS * 4) != 0) return false;
    SweepArgs args;
    args.n = n;
    args.N = N;
    args.pf = 0;
    args.mstride = mstride;
    args.mode = mode;
    args.obs_inv = obs_inv;
    args.obs_stride = obs_stride;
    args.t0 = t0;
    args.ts = ts > 0 ? ts : 1;
    args.bar = bar;
    args.err = err;
    args.wait_limit = wait_limit;
    const int slots = n / (SW_THREADS * 4);
    if (slots == 1) return launch_sweep_df<1>(s, num_sms, Mh0, Ml0, W, Wh, Wl, args);
    if (slots == 2) return launch_sweep_df<2>(s, num_sms, Mh0, Ml0, W, Wh, Wl, args);
    if (slots == 4) return launch_sweep_df<4>(s, num_sms, Mh0, Ml0, W, Wh, Wl, args);
    return false;
}

template <typename T>
void launch_sweep_gemm(cudaStream_t s, int n, int K, const T *M, const T *B, int64_t ldb, T *C, int64_t ldc,
                       const Epi &e)
{
    using Acc = T;
    if (K == 1) {
        constexpr int VEC = sizeof(T) == 8 ? 2 : 4;
        constexpr int RPW = 2, UNR = 4;
        if (n % VEC == 0 && aligned16(M) && aligned16(B)) {
            const int warps = ceil_div(n, RPW);
            WC4D_LAUNCH(k_gemv_rows<T, Acc, RPW, UNR><<<ceil_div(warps, 2), 64, 0, s>>>(n, M, B, C, e));
        } else {
            WC4D_LAUNCH(k_gemv_scalar<T, Acc><<<ceil_div((int64_t)n * 32, 256), 256, 0, s>>>(n, M, B, C, e));
        }
        return;
    }
    launch_gemm<T>(s, n, K, n, M, n, 1, B, ldb, C, ldc, e);
}

// ----------------------------------------------------------------------------
// Autotuned tile shape of the SIMT GEMM when A is K-contiguous (the
// propagator products of the sweeps, M row-major times a block of columns).
// On the first call for a shape (rows, columns, reduction) every candidate
// tile is timed -- three launches each with CUDA events on the caller's
// stream, writing a scratch C so that the real output is untouched -- and the
// fastest is kept in a process-wide table; later calls launch it directly.
// Candidates trade reuse per thread (larger TM x TN) against the number of
// CTAs (small n and few columns leave most SMs idle with 64 x 64 tiles).
// Tuning is skipped (heuristic tile) while the stream is being captured into
// a graph or when autotuning is off.
// ----------------------------------------------------------------------------
namespace {
struct TuneKey {
    int kind, a, b, c;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(kind, a, b, c) < std::tie(o.kind, o.a, o.b, o.c);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;
std::atomic<int> g_autotune{1};

// KC: A is K-contiguous (A(i, k) = A[i sam + k]); otherwise row-contiguous
// (A(i, k) = A[i + k sak], the tall-skinny products Y R^{-1}, Z W).
template <typename T, bool KC, int BM, int BN, int BK, int TM, int TN>
void gemm_variant(cudaStream_t s, int Mrows, int Ncols, int Kdim, const T *A, int64_t sa, const T *B, int64_t ldb,
                  T *C, int64_t ldc, const Epi &e)
{
    dim3 g(ceil_div(Mrows, BM), ceil_div(Ncols, BN));
    WC4D_LAUNCH(k_gemm_simt<T, T, BM, BN, BK, TM, TN, KC><<<g, (BM / TM) * (BN / TN), 0, s>>>(
        Mrows, Ncols, Kdim, A, KC ? sa : 1, KC ? 1 : sa, B, ldb, C, ldc, e));
}

constexpr int GEMM_CANDIDATES = 5;
template <typename T, bool KC>
void gemm_candidate(int v, cudaStream_t s, int Mrows, int Ncols, int Kdim, const T *A, int64_t sa, const T *B,
                    int64_t ldb, T *C, int64_t ldc, const Epi &e)
{
    switch (v) {
    case 0: gemm_variant<T, KC, 64, 64, 16, 4, 4>(s, Mrows, Ncols, Kdim, A, sa, B, ldb, C, ldc, e); break;
    case 1: gemm_variant<T, KC, 128, 64, 16, 8, 4>(s, Mrows, Ncols, Kdim, A, sa, B, ldb, C, ldc, e); break;
    case 2: gemm_variant<T, KC, 64, 32, 16, 4, 2>(s, Mrows, Ncols, Kdim, A, sa, B, ldb, C, ldc, e); break;
    case 3: gemm_variant<T, KC, 32, 32, 16, 2, 2>(s, Mrows, Ncols, Kdim, A, sa, B, ldb, C, ldc, e); break;
    default: gemm_variant<T, KC, 128, 128, 8, 8, 8>(s, Mrows, Ncols, Kdim, A, sa, B, ldb, C, ldc, e); break;
    }
}

template <typename T, bool KC>
int tune_gemm(cudaStream_t s, int Mrows, int Ncols, int Kdim, const T *A, int64_t sa, const T *B, int64_t ldb)
{
    const TuneKey key{(sizeof(T) == 8 ? 1 : 0) + (KC ? 0 : 2), Mrows, Ncols, Kdim};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) return it->second;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (!g_autotune.load() || cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return -1;
    T *scratch = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int best = -1;
    if (cudaMallocAsync(&scratch, sizeof(T) * (size_t)Mrows * Ncols, s) == cudaSuccess &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        const Epi plain{0, 1.0, 0.0, 0.0, 1};
        float best_ms = 0.f;
        for (int v = 0; v < GEMM_CANDIDATES; ++v) {
            gemm_candidate<T, KC>(v, s, Mrows, Ncols, Kdim, A, sa, B, ldb, scratch, Mrows, plain);   // warm
            cudaEventRecord(e0, s);
            for (int r = 0; r < 3; ++r)
                gemm_candidate<T, KC>(v, s, Mrows, Ncols, Kdim, A, sa, B, ldb, scratch, Mrows, plain);
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                best = -1;
                break;
            }
            if (best < 0 || ms < best_ms) {
                best = v;
                best_ms = ms;
            }
        }
    }
    if (scratch) cudaFreeAsync(scratch, s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaGetLastError();
    if (best >= 0) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune.emplace(key, best);
    }
    return best;
}
}  // namespace

extern "C" void wc4d_set_autotune(int32_t enable) { g_autotune.store(enable != 0); }

extern "C" int32_t wc4d_autotune_choice(int32_t fp64, int32_t rows, int32_t cols, int32_t kdim)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(TuneKey{(fp64 & 1) + (fp64 & 2), rows, cols, kdim});
    return it == g_tune.end() ? -1 : it->second;
}

template <typename T>
void launch_gemm(cudaStream_t s, int Mrows, int Ncols, int Kdim, const T *A, int64_t sam, int64_t sak,
                 const T *B, int64_t ldb, T *C, int64_t ldc, const Epi &e)
{
    using Acc = T;
    if (Mrows <= 0 || Ncols <= 0) return;
    const bool kc = (sak == 1);
    if (kc && Ncols > 16 && Kdim >= 256) {   // sweep products: tuned tile
        const int v = tune_gemm<T, true>(s, Mrows, Ncols, Kdim, A, sam, B, ldb);
        gemm_candidate<T, true>(v < 0 ? 0 : v, s, Mrows, Ncols, Kdim, A, sam, B, ldb, C, ldc, e);
        return;
    }
    if (!kc && sam == 1 && Ncols > 16 && Mrows >= 16384) {   // tall-skinny block products: tuned tile
        const int v = tune_gemm<T, false>(s, Mrows, Ncols, Kdim, A, sak, B, ldb);
        gemm_candidate<T, false>(v < 0 ? 0 : v, s, Mrows, Ncols, Kdim, A, sak, B, ldb, C, ldc, e);
        return;
    }
    if (Ncols <= 16) {
        dim3 g(ceil_div(Mrows, 64), ceil_div(Ncols, 16));
        if (kc) WC4D_LAUNCH(k_gemm_simt<T, Acc, 64, 16, 16, 4, 4, true><<<g, 64, 0, s>>>(Mrows, Ncols, Kdim, A, sam, sak, B, ldb, C, ldc, e));
        else WC4D_LAUNCH(k_gemm_simt<T, Acc, 64, 16, 16, 4, 4, false><<<g, 64, 0, s>>>(Mrows, Ncols, Kdim, A, sam, sak, B, ldb, C, ldc, e));
    } else {
        dim3 g(ceil_div(Mrows, 64), ceil_div(Ncols, 64));
        if (kc) WC4D_LAUNCH(k_gemm_simt<T, Acc, 64, 64, 16, 4, 4, true><<<g, 256, 0, s>>>(Mrows, Ncols, Kdim, A, sam, sak, B, ldb, C, ldc, e));
        else WC4D_LAUNCH(k_gemm_simt<T, Acc, 64, 64, 16, 4, 4, false><<<g, 256, 0, s>>>(Mrows, Ncols, Kdim, A, sam, sak, B, ldb, C, ldc, e));
    }
}

template void launch_sweep_gemm<double>(cudaStream_t, int, int, const double *, const double *, int64_t, double *,
                                        int64_t, const Epi &);
template void launch_sweep_gemm<float>(cudaStream_t, int, int, const float *, const float *, int64_t, float *,
                                       int64_t, const Epi &);
template void launch_gemm<double>(cudaStream_t, int, int, int, const double *, int64_t, int64_t, const double *,
                                  int64_t, double *, int64_t, const Epi &);
template void launch_gemm<float>(cudaStream_t, int, int, int, const float *, int64_t, int64_t, const float *,
                                 int64_t, float *, int64_t, const Epi &);

// W(t block) <- H^T R^{-1} H W for one time block: keep observed points
// (s % stride == 0) scaled by `scale`, zero the rest.
template <typename T>
__global__ void k_obs_block(int n, int K, T *W, int64_t ld, double scale, int stride)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * K) return;
    int s = (int)(idx % n);
    int64_t j = idx / n;
    T *w = W + j * ld + s;
    *w = (s % stride == 0) ? (T)(scale * (double)(*w)) : (T)0;
}

template <typename T>
void launch_obs_block(cudaStream_t s, int n, int K, T *W, int64_t ld, double scale, int stride)
{
    int64_t tot = (int64_t)n * K;
    WC4D_LAUNCH(k_obs_block<T><<<ceil_div(tot, 256), 256, 0, s>>>(n, K, W, ld, scale, stride));
}

template void launch_obs_block<double>(cudaStream_t, int, int, double *, int64_t, double, int);
template void launch_obs_block<float>(cudaStream_t, int, int, float *, int64_t, double, int);
