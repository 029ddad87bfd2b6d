// One-sided (Hestenes) Jacobi for the small eigenproblems of the sketch (the
// EVD of K_1 in Alg. 3, of F^T F in Alg. 4, the SVD of R_3 in Alg. 5) with
// m <= 256, as ONE persistent cooperative launch instead of one launch per
// round plus a host synchronisation per sweep.
//
// CTA b rotates column pair b of the round-robin ordering (P/2 CTAs, one
// per SM, P = m rounded up to a multiple of 2, zero padded), one row per
// thread, in FP64.  The FP64 pipe of this GPU retires about 1.6 FMA per
// clock per SM, so the rotations are spread over as many SMs as there are
// pairs rather than packed into a few.  X and the accumulated rotations V
// are double-buffered in global memory (L2-resident): round r reads buffer
// r % 2 and writes every column, rotated or not, to the other, then a grid
// barrier (release/acquire on one counter, bounded spin) ends the round.
// Reads bypass L1 (the columns were written by other SMs).  Sweeps repeat
// until one makes no rotation, or max_sweeps.  Zero padding columns never
// rotate.
#include <cooperative_groups.h>

#include "wc4d_internal.cuh"

namespace {

constexpr int JQ_MAXP = 256;
constexpr int JQ_THREADS = 256;   // one row per thread
constexpr unsigned JQ_SPIN = 1u << 22;

// Arrive on the grid barrier and wait until `target` arrivals; false (and
// *err = 1) when the bounded wait gives up.
__device__ __forceinline__ bool jq_barrier(unsigned *bar, unsigned target, int *err)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
        unsigned v = 0, it = 0;
        int ok = 1;
        do {
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
            if (++it > JQ_SPIN) { ok = 0; atomicExch(err, 1); break; }
        } while (v < target);
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

template <typename T> struct JqArgs {
    int m, P;
    const double *X0;   // m x m, column-major, ld m (scaled by *x0_scale when not null)
    T *XV;              // four P x P buffers X_a, V_a, X_b, V_b; the result ends in X_a, V_a
    double tol;
    int max_sweeps;
    int *rot;           // max_sweeps rotation counters (zeroed here)
    unsigned *bar;      // barrier counter (zero at launch)
    int *err;           // 1 after a barrier timeout
    int *status;        // sweeps used, or -1 when not converged
    int want_v;         // 0: V is neither accumulated nor written
    double stop2;       // > 0: early stop threshold on the largest g^2 / (a b) of a sweep
    unsigned long long *maxm;   // max_sweeps largest g^2 / (a b) (double bits, zeroed here)
    const double *x0_scale;     // optional scale of X0 (an exact power of two)
};

// T = double: the FP64 solve.  T = float: the FP32 pre-rotation phase (the
// products, sums and rotations in FP32; V accumulated in FP32).
template <typename T>
__global__ void __launch_bounds__(JQ_THREADS, 1) k_jacobi_coop(JqArgs<T> a)
{
    __shared__ T prod[2][3][JQ_THREADS];      // double-buffered by round parity
    __shared__ double red[2][3];
    __shared__ T cs[2][2];
    __shared__ int doit_s[2], conv_s;
    const int P = a.P, pair = blockIdx.x, r = threadIdx.x;
    const unsigned G = gridDim.x;
    const int64_t PP = (int64_t)P * P;
    T *Xc = a.XV, *Vc = a.XV + PP, *Xn = a.XV + 2 * PP, *Vn = a.XV + 3 * PP;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool wv = a.want_v != 0;
    const double sc0 = a.x0_scale ? *a.x0_scale : 1.0;
    for (int k = 0; k < 2; ++k) {   // this CTA initialises columns 2 pair, 2 pair + 1
        const int j = 2 * pair + k;
        if (r < P) {
            Xc[(int64_t)j * P + r] = (r < a.m && j < a.m) ? (T)(sc0 * a.X0[(int64_t)j * a.m + r]) : (T)0;
            if (wv) Vc[(int64_t)j * P + r] = (r == j) ? (T)1 : (T)0;
        }
    }
    if (pair == 0)
        for (int s = r; s < a.max_sweeps; s += blockDim.x) {
            a.rot[s] = 0;
            a.maxm[s] = 0ull;
        }
    unsigned target = G;
    if (!jq_barrier(a.bar, target, a.err)) return;

    int sweeps = 0;
    bool converged = false;
    for (; sweeps < a.max_sweeps && !converged; ++sweeps) {
        int nrot = 0;       // rotations and largest rotation measure of this CTA in this sweep (thread 0)
        double mmax = 0.0;
        for (int round = 0; round < P - 1; ++round) {
            const int pos_b = P - 1 - pair;
            const int ja = pair == 0 ? 0 : 1 + (pair - 1 + round) % (P - 1);
            const int jb = 1 + (pos_b - 1 + round) % (P - 1);
            const int p = min(ja, jb), q = max(ja, jb);
            T u = 0, w = 0, y = 0, z = 0;
            if (r < P) {
                u = __ldcg(Xc + (int64_t)p * P + r);
                w = __ldcg(Xc + (int64_t)q * P + r);
                if (wv) {
                    y = __ldcg(Vc + (int64_t)p * P + r);
                    z = __ldcg(Vc + (int64_t)q * P + r);
                }
            }
            // The FP64 pipe retires about 1.6 operations per clock per SM, so
            // the three sums are not reduced by a butterfly over all 256
            // threads (15 FP64 additions each): the products go to shared
            // memory and warp v (v < 3) adds the 256 values of sum v (8
            // per lane, then 5 shuffle levels), a third of the FP64 work.
            const int par = round & 1;
            prod[par][0][r] = u * u;
            prod[par][1][r] = w * w;
            prod[par][2][r] = u * w;
            __syncthreads();
            if (warp < 3) {
                T acc = 0;
#pragma unroll
                for (int i = lane; i < JQ_THREADS; i += 32) acc += prod[par][warp][i];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) red[par][warp] = (double)acc;
            }
            __syncthreads();
            // thread 0 alone forms the rotation (256 redundant copies of this
            // scalar FP64 work would cost more than the broadcast)
            if (threadIdx.x == 0) {
                const double aa = red[par][0], bb = red[par][1], g = red[par][2];
                int doit = 0;
                // |g| > tol sqrt(a b), squared: no FP64 square root or division
                if (g * g > a.tol * a.tol * (aa * bb) && fabs(g) > 1e-300) {
                    // The tangent only needs FP32 accuracy (the rotation then
                    // leaves |g| ~1e-7 of its value instead of 0, and the next
                    // sweep removes it); c = (1 + t^2)^{-1/2} is completed to
                    // FP64 by two Newton steps so that c^2 + s^2 = 1 holds to
                    // rounding and the column norms are preserved.
                    // zeta = (b - a) / (2 g), both scaled by 2^-e into FP32 range
                    const double d = bb - aa, g2 = 2.0 * g;
                    const int e = ilogb(g2);
                    const float zeta = (float)scalbn(d, -e) / (float)scalbn(g2, -e);
                    double tn;
                    if (isfinite(zeta) && fabsf(zeta) < 1e18f)
                        tn = (double)(copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f))));
                    else
                        tn = g2 / (2.0 * d);   // |zeta| huge: t = 1 / (2 zeta)
                    const double h = fma(tn, tn, 1.0);
                    double c = (double)rsqrtf((float)h);
                    c = c * fma(-0.5 * h, c * c, 1.5);
                    if (sizeof(T) == 8) c = c * fma(-0.5 * h, c * c, 1.5);
                    cs[par][0] = (T)c;
                    cs[par][1] = (T)(c * tn);
                    doit = 1;
                    ++nrot;
                    if (a.stop2 > 0.0) mmax = fmax(mmax, (g * g) / (aa * bb));
                }
                doit_s[par] = doit;
            }
            __syncthreads();
            const bool doit = doit_s[par] != 0;
            const T c = cs[par][0], sn = cs[par][1];
            if (r < P) {
                if (doit) {
                    Xn[(int64_t)p * P + r] = c * u - sn * w;
                    Xn[(int64_t)q * P + r] = sn * u + c * w;
                    if (wv) {
                        Vn[(int64_t)p * P + r] = c * y - sn * z;
                        Vn[(int64_t)q * P + r] = sn * y + c * z;
                    }
                } else {
                    Xn[(int64_t)p * P + r] = u;
                    Xn[(int64_t)q * P + r] = w;
                    if (wv) {
                        Vn[(int64_t)p * P + r] = y;
                        Vn[(int64_t)q * P + r] = z;
                    }
                }
            }
            if (round == P - 2 && threadIdx.x == 0) {   // this CTA's counts, before the sweep's last barrier
                if (nrot) atomicAdd(a.rot + sweeps, nrot);
                if (a.stop2 > 0.0 && mmax > 0.0)   // non-negative doubles order as their bit patterns
                    atomicMax(a.maxm + sweeps, (unsigned long long)__double_as_longlong(mmax));
            }
            target += G;
            if (!jq_barrier(a.bar, target, a.err)) return;
            T *t0 = Xc, *t1 = Vc;
            Xc = Xn; Vc = Vn; Xn = t0; Vn = t1;
        }
        if (threadIdx.x == 0)
            conv_s = (__ldcg(a.rot + sweeps) == 0) ||
                     (a.stop2 > 0.0 && __longlong_as_double((long long)__ldcg(a.maxm + sweeps)) <= a.stop2);
        __syncthreads();
        converged = conv_s != 0;
    }
    if (Xc != a.XV) {   // the result sits in the b buffers: move this CTA's two columns
        for (int k = 0; k < 2; ++k) {
            const int64_t j = 2 * pair + k;
            if (r < P) {
                a.XV[j * P + r] = __ldcg(Xc + j * P + r);
                if (wv) a.XV[PP + j * P + r] = __ldcg(Vc + j * P + r);
            }
        }
    }
    if (pair == 0 && threadIdx.x == 0) *a.status = converged ? sweeps : -1;
}

__global__ void k_add_diag(int m, double *A, int lda, double v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) A[(int64_t)i * lda + i] += v;
}

// max |X0| -> the power of two 2^-e that brings it to [1, 2) (for the FP32
// phase: squared column norms and their products stay in range)
__global__ void k_x0_scale(int64_t count, const double *X0, double *scale)
{
    __shared__ double red[32];
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x) v = fmax(v, fabs(X0[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) mx = fmax(mx, red[i]);
        *scale = (mx > 0.0 && isfinite(mx)) ? scalbn(1.0, -ilogb(mx)) : 1.0;
    }
}

}  // namespace

int jacobi_coop_size(int m) { return (m >= 2 && m <= JQ_MAXP) ? m + (m & 1) : 0; }

size_t jacobi_coop_doubles(int m)
{
    const size_t P = (size_t)jacobi_coop_size(m);
    return 4 * P * P;
}

template <typename T>
static bool launch_coop(cudaStream_t s, int m, const double *X0, T *XV, double tol, int max_sweeps, int *rot,
                        unsigned *bar, int *err, int *status, bool want_v, double stop2, unsigned long long *maxm,
                        const double *x0_scale)
{
    const int P = jacobi_coop_size(m);
    if (P == 0) return false;
    if (cudaMemsetAsync(bar, 0, sizeof(unsigned), s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    JqArgs<T> args{m, P, X0, XV, tol, max_sweeps, rot, bar, err, status, want_v ? 1 : 0, stop2, maxm, x0_scale};
    void *params[] = {&args};
    wc4d_note_launch();
    if (cudaLaunchCooperativeKernel((const void *)k_jacobi_coop<T>, dim3(P / 2), dim3(JQ_THREADS), params, 0, s) !=
        cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

// Returns false (nothing runs, error state cleared) when the cooperative
// launch is refused.  XV: jacobi_coop_doubles(m) doubles; the result is
// X = XV[0, P^2), V = XV[P^2, 2 P^2).  rot: max_sweeps ints; bar: one
// counter, zeroed here; err: set to 1 if a grid barrier times out.  With
// want_v false only X is produced.  stop2 > 0 enables the early stop (maxm:
// max_sweeps 64-bit words).
bool launch_jacobi_coop(cudaStream_t s, int m, const double *X0, double *XV, double tol, int max_sweeps, int *rot,
                        unsigned *bar, int *err, int *status, bool want_v, double stop2, unsigned long long *maxm)
{
    return launch_coop<double>(s, m, X0, XV, tol, max_sweeps, rot, bar, err, status, want_v, stop2, maxm, nullptr);
}

// FP32 pre-rotation: one-sided Jacobi in FP32 on 2^-e X0 (2^-e from max |X0|,
// computed into *scale_work) accumulating V (FP32) until a sweep's largest
// rotation has |cos| <= sqrt(stop2) or makes none at tol.  XV32: 4 P^2 floats,
// V = XV32[P^2, 2 P^2) on return.  Same counters as launch_jacobi_coop.
bool launch_jacobi_coop_f32(cudaStream_t s, int m, const double *X0, float *XV32, double tol, int max_sweeps,
                            int *rot, unsigned *bar, int *err, int *status, double stop2, unsigned long long *maxm,
                            double *scale_work)
{
    if (jacobi_coop_size(m) == 0) return false;
    WC4D_LAUNCH(k_x0_scale<<<1, 256, 0, s>>>((int64_t)m * m, X0, scale_work));
    return launch_coop<float>(s, m, X0, XV32, tol, max_sweeps, rot, bar, err, status, true, stop2, maxm, scale_work);
}

// C (m x m) = alpha A^T B + beta C or alpha A B + beta C for small column-major
// FP64 matrices with leading dimensions lda, ldb, ldc: 16 x 16 output tiles, one
// CTA each, so that an m = 256 product spreads over 256 SMs' worth of CTAs
// (the FP64 pipe retires ~1.6 FMA per clock per SM).
__global__ void __launch_bounds__(256) k_small_gemm64(int m, const double *A, int lda, int transA, const double *B,
                                                      int ldb, double *C, int ldc, double alpha, double beta)
{
    __shared__ double As[16][17], Bs[16][17];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i = blockIdx.x * 16 + tx, j = blockIdx.y * 16 + ty;
    double acc = 0.0;
    for (int k0 = 0; k0 < m; k0 += 16) {
        // As[kk][ii] = op(A)(blockIdx.x*16 + ii, k0 + kk)
        const int ii = tx, kk = ty;
        const int gi = blockIdx.x * 16 + ii, gk = k0 + kk;
        double av = 0.0;
        if (gi < m && gk < m) av = transA ? A[(int64_t)gi * lda + gk] : A[(int64_t)gk * lda + gi];
        As[kk][ii] = av;
        const int gj = blockIdx.y * 16 + ty, gk2 = k0 + tx;
        Bs[ty][tx] = (gj < m && gk2 < m) ? B[(int64_t)gj * ldb + gk2] : 0.0;   // Bs[j][k]
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) acc = fma(As[k][tx], Bs[ty][k], acc);
        __syncthreads();
    }
    if (i < m && j < m) {
        double *dst = C + (int64_t)j * ldc + i;
        *dst = alpha * acc + (beta != 0.0 ? beta * (*dst) : 0.0);
    }
}

void launch_small_gemm64(cudaStream_t s, int m, const double *A, int lda, bool transA, const double *B, int ldb,
                         double *C, int ldc, double alpha, double beta)
{
    dim3 g(ceil_div(m, 16), ceil_div(m, 16));
    WC4D_LAUNCH(k_small_gemm64<<<g, 256, 0, s>>>(m, A, lda, transA ? 1 : 0, B, ldb, C, ldc, alpha, beta));
}

// V (m x m, ld ldv) <- V (3 I - V^T V) / 2, twice: an FP32-accurate orthogonal
// V becomes orthogonal to FP64 rounding (Newton-Schulz; the error e -> ~ e^2).
// tmp: 2 m^2 doubles.
void launch_orthogonalise_ns(cudaStream_t s, int m, double *V, int ldv, double *tmp)
{
    double *G = tmp, *W = tmp + (size_t)m * m;
    // step 1: W = V (3 I - V^T V) / 2
    launch_small_gemm64(s, m, V, ldv, true, V, ldv, G, m, -0.5, 0.0);
    WC4D_LAUNCH(k_add_diag<<<ceil_div(m, 256), 256, 0, s>>>(m, G, m, 1.5));
    launch_small_gemm64(s, m, V, ldv, false, G, m, W, m, 1.0, 0.0);
    // step 2: V = W (3 I - W^T W) / 2
    launch_small_gemm64(s, m, W, m, true, W, m, G, m, -0.5, 0.0);
    WC4D_LAUNCH(k_add_diag<<<ceil_div(m, 256), 256, 0, s>>>(m, G, m, 1.5));
    launch_small_gemm64(s, m, W, m, false, G, m, V, ldv, 1.0, 0.0);
}

// ----------------------------------------------------------------------------
// FP32 pre-rotation on one thread-block cluster of 16 CTAs (distributed
// shared memory) instead of the whole GPU: in FP32 the rotations are cheap,
// and what limits the cooperative kernel's rounds is the grid barrier and the
// L2 round trip of the columns.  Pair b of the round-robin ordering (warp
// b % 8 of CTA b / 8) keeps its two columns -- and their V columns -- in its
// own CTA's shared memory, so a round reads nothing remote: the warp rotates
// its pair and writes the two results straight into the slots they occupy in
// the next round (the ordering shifts the columns one position: the first
// column of pair b moves to pair b - 1, the second to pair b + 1, with the
// turn-arounds at both ends), a remote store only across a CTA boundary.
// Double-buffered slots and one cluster barrier per round; a whole sweep
// brings every column back to its starting slot.
// Sweeps stop when a sweep's largest rotation has cos^2 <= stop2, makes no
// rotation at tol, or after max_sweeps.  Output: V (P x P, FP32).
// ----------------------------------------------------------------------------
namespace {
namespace cgx = cooperative_groups;
constexpr int JC_CL = 16;
constexpr int JC_THREADS = 256;   // 8 warps: one pair each

__global__ void __launch_bounds__(JC_THREADS, 1)
k_jacobi_cluster_f32(int m, int P, const double *__restrict__ X0, const double *x0_scale, float *Vout, float tol,
                     float stop2, int max_sweeps, int *status)
{
    cgx::cluster_group cl = cgx::this_cluster();
    const int rank = (int)cl.block_rank();
    // [buffer][x or v][local pair][top or bottom][row]
    extern __shared__ __align__(16) float jcs[];
    auto slot = [&](float *base, int buf, int xv, int lp, int tb) { return base + ((((buf * 2 + xv) * 8 + lp) * 2 + tb) * P); };
    __shared__ int rot_s, conv_s;
    __shared__ unsigned maxm_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int npairs = P / 2, b = rank * 8 + warp;
    const float sc = (float)*x0_scale;
    if (b < npairs) {   // round 0: pair b holds columns b and P - 1 - b
        const int cols[2] = {b, P - 1 - b};
        for (int tb = 0; tb < 2; ++tb) {
            const int j = cols[tb];
            float *xs = slot(jcs, 0, 0, warp, tb), *vs = slot(jcs, 0, 1, warp, tb);
            for (int r = lane; r < P; r += 32) {
                xs[r] = (j < m && r < m) ? sc * (float)X0[(int64_t)j * m + r] : 0.f;
                vs[r] = (r == j) ? 1.f : 0.f;
            }
        }
    }
    if (tid == 0) { rot_s = 0; maxm_s = 0u; conv_s = 0; }
    cl.sync();
    // destinations of this pair's two columns for the next round
    int dt_pair, dt_tb, db_pair, db_tb;
    if (b == 0) { dt_pair = 0; dt_tb = 0; }
    else if (b == 1) { dt_pair = 0; dt_tb = 1; }
    else { dt_pair = b - 1; dt_tb = 0; }
    if (b == npairs - 1) { db_pair = b; db_tb = 0; }
    else { db_pair = b + 1; db_tb = 1; }
    if (b == 0 && npairs == 1) { dt_pair = 0; dt_tb = 0; db_pair = 0; db_tb = 1; }
    int buf = 0, sweeps = 0;
    bool converged = false;
    for (; sweeps < max_sweeps && !converged; ++sweeps) {
        for (int round = 0; round < P - 1; ++round) {
            if (b < npairs) {
                const float *xp = slot(jcs, buf, 0, warp, 0), *xq = slot(jcs, buf, 0, warp, 1);
                const float *vp = slot(jcs, buf, 1, warp, 0), *vq = slot(jcs, buf, 1, warp, 1);
                float u[8], v[8], y[8], z[8];
                float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int r = lane + 32 * i;
                    u[i] = r < P ? xp[r] : 0.f;
                    v[i] = r < P ? xq[r] : 0.f;
                    y[i] = r < P ? vp[r] : 0.f;
                    z[i] = r < P ? vq[r] : 0.f;
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    s0 = fmaf(u[i], u[i], s0);
                    s1 = fmaf(v[i], v[i], s1);
                    s2 = fmaf(u[i], v[i], s2);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
                    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
                }
                float c = 1.f, sn = 0.f;
                if ((s2 * s2 > tol * tol * (s0 * s1)) && fabsf(s2) > 1e-30f) {   // the same in every lane
                    const float zeta = (s1 - s0) / (2.f * s2);
                    const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
                    c = rsqrtf(fmaf(t, t, 1.f));
                    sn = c * t;
                    if (lane == 0) {
                        atomicAdd(&rot_s, 1);
                        atomicMax(&maxm_s, __float_as_uint((s2 * s2) / (s0 * s1)));
                    }
                }
                const int nb = buf ^ 1;
                float *tx = cl.map_shared_rank(slot(jcs, nb, 0, dt_pair & 7, dt_tb), dt_pair >> 3);
                float *tv = cl.map_shared_rank(slot(jcs, nb, 1, dt_pair & 7, dt_tb), dt_pair >> 3);
                float *bx = cl.map_shared_rank(slot(jcs, nb, 0, db_pair & 7, db_tb), db_pair >> 3);
                float *bv = cl.map_shared_rank(slot(jcs, nb, 1, db_pair & 7, db_tb), db_pair >> 3);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int r = lane + 32 * i;
                    if (r < P) {
                        tx[r] = c * u[i] - sn * v[i];
                        bx[r] = sn * u[i] + c * v[i];
                        tv[r] = c * y[i] - sn * z[i];
                        bv[r] = sn * y[i] + c * z[i];
                    }
                }
            }
            cl.sync();
            buf ^= 1;
        }
        // sweep end: CTA 0 combines the counts of all CTAs
        if (rank == 0 && tid == 0) {
            int rot = 0;
            unsigned mx = 0u;
            for (int cta = 0; cta < JC_CL; ++cta) {
                rot += *cl.map_shared_rank(&rot_s, cta);
                mx = max(mx, *cl.map_shared_rank(&maxm_s, cta));
            }
            conv_s = (rot == 0 || __uint_as_float(mx) <= stop2) ? 1 : 0;
        }
        cl.sync();
        converged = *cl.map_shared_rank(&conv_s, 0) != 0;
        cl.sync();   // every CTA has read the decision (and CTA 0 all counts) before they are reset
        if (tid == 0) { rot_s = 0; maxm_s = 0u; }
        cl.sync();
    }
    // after each whole sweep (P - 1 rounds) every column is back in the slot
    // it started in, so V is written in column order -- which matters: the
    // caller uses the leading m x m block of V, and for odd m column P - 1 is
    // the zero padding column
    if (b < npairs)
        for (int tb = 0; tb < 2; ++tb) {
            const float *vs = slot(jcs, buf, 1, warp, tb);
            const int j = tb == 0 ? b : P - 1 - b;
            for (int r = lane; r < P; r += 32) Vout[(int64_t)j * P + r] = vs[r];
        }
    if (rank == 0 && tid == 0) *status = converged ? sweeps : -1;
}
}  // namespace

bool launch_jacobi_cluster_f32(cudaStream_t s, int m, const double *X0, float *Vout, double tol, int max_sweeps,
                               int *status, double stop2, double *scale_work)
{
    const int P = jacobi_coop_size(m);
    if (P == 0 || P > JC_CL * 16) return false;
    const size_t smem = sizeof(float) * 2 * 2 * 8 * 2 * (size_t)P;   // [buf][x|v][pair][top|bottom][P]
    // once (a function-local static is initialised once even when host
    // threads launch concurrently): attributes, then whether one 16-CTA
    // cluster with 64 KB of shared memory per CTA can be scheduled
    static const bool ok = [] {
        const int smem_max = (int)(sizeof(float) * 2 * 2 * 8 * 2 * 256);   // 64 KB: above the default 48 KB
        bool r = cudaFuncSetAttribute(k_jacobi_cluster_f32, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                     cudaSuccess &&
                 cudaFuncSetAttribute(k_jacobi_cluster_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max) ==
                     cudaSuccess;
        cudaLaunchConfig_t q = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = JC_CL;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        q.gridDim = dim3(JC_CL);
        q.blockDim = dim3(JC_THREADS);
        q.dynamicSmemBytes = smem_max;
        q.attrs = at;
        q.numAttrs = 1;
        int clusters = 0;
        if (r && (cudaOccupancyMaxActiveClusters(&clusters, k_jacobi_cluster_f32, &q) != cudaSuccess || clusters < 1))
            r = false;
        cudaGetLastError();
        return r;
    }();
    if (!ok) return false;
    WC4D_LAUNCH(k_x0_scale<<<1, 256, 0, s>>>((int64_t)m * m, X0, scale_work));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = JC_CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(JC_CL);
    cfg.blockDim = dim3(JC_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    wc4d_note_launch();
    if (cudaLaunchKernelEx(&cfg, k_jacobi_cluster_f32, m, P, X0, (const double *)scale_work, Vout, (float)tol,
                           (float)stop2, max_sweeps, status) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}
