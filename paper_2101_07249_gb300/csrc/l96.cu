// Lorenz-96 (Section 5.2): nonlinear RK4 run, and the exact tangent-linear
// and adjoint of the RK4 step applied as stencil sweeps to probe blocks.
//
// dX_j/dt = (X_{j+1} - X_{j-2}) X_{j-1} - X_j + F (periodic).  Jacobian at x:
//   (J d)_j   = (d_{j+1} - d_{j-2}) x_{j-1} + (x_{j+1} - x_{j-2}) d_{j-1} - d_j
//   (J^T a)_i = x_{i-2} a_{i-1} - x_{i+1} a_{i+2} + (x_{i+2} - x_{i-1}) a_{i+1} - a_i
// The RK4 stage states s1 = x, s2 = x + h/2 k1, s3 = x + h/2 k2, s4 = x + h k3
// of every step are stored once by the nonlinear run and shared by all
// probe columns (an L2-resident read-only table).
#include <cooperative_groups.h>

#include "wc4d_internal.cuh"

namespace cg = cooperative_groups;

constexpr int L96_THREADS = 512;
constexpr int L96_PPT = WC4D_FFT_MAX_N / L96_THREADS;   // points per thread (n <= 8192)

__device__ __forceinline__ int wrap(int j, int n) { return j < 0 ? j + n : (j >= n ? j - n : j); }

template <typename T>
__device__ __forceinline__ T jac(const T *__restrict__ x, const T *d, int j, int n)
{
    const int jm2 = wrap(j - 2, n), jm1 = wrap(j - 1, n), jp1 = wrap(j + 1, n);
    return (d[jp1] - d[jm2]) * __ldg(x + jm1) + (__ldg(x + jp1) - __ldg(x + jm2)) * d[jm1] - d[j];
}

template <typename T>
__device__ __forceinline__ T jacT(const T *__restrict__ x, const T *a, int i, int n)
{
    const int im2 = wrap(i - 2, n), im1 = wrap(i - 1, n), ip1 = wrap(i + 1, n), ip2 = wrap(i + 2, n);
    return __ldg(x + im2) * a[im1] - __ldg(x + ip1) * a[ip2] + (__ldg(x + ip2) - __ldg(x + im1)) * a[ip1] - a[i];
}

// Forward sweep L^{-1} on one column per CTA: W_{t+1} = M_t W_t + W_{t+1},
// M_t = `steps` tangent-linear RK4 steps.
template <typename T>
__global__ void __launch_bounds__(L96_THREADS)
k_l96_tlm(int n, int N, int steps, T h, const T *__restrict__ stages, T *W, int64_t ld)
{
    extern __shared__ __align__(16) unsigned char sm[];
    T *dl = reinterpret_cast<T *>(sm);
    T *ta = dl + n, *tb = ta + n;
    T *w = W + (int64_t)blockIdx.x * ld;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int j = tid; j < n; j += nt) dl[j] = w[j];
    __syncthreads();
    T acc[L96_PPT];
    const T h2 = h * (T)0.5, h6 = h / (T)6;
    for (int t = 0; t < N; ++t) {
        for (int k = 0; k < steps; ++k) {
            const int64_t g = (int64_t)t * steps + k;
            const T *s1 = stages + (4 * g + 0) * n, *s2 = stages + (4 * g + 1) * n;
            const T *s3 = stages + (4 * g + 2) * n, *s4 = stages + (4 * g + 3) * n;
#pragma unroll
            for (int r = 0; r < L96_PPT; ++r) {
                int j = tid + r * nt;
                if (j < n) { T d = jac(s1, dl, j, n); acc[r] = d; ta[j] = dl[j] + h2 * d; }
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < L96_PPT; ++r) {
                int j = tid + r * nt;
                if (j < n) { T d = jac(s2, ta, j, n); acc[r] += (T)2 * d; tb[j] = dl[j] + h2 * d; }
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < L96_PPT; ++r) {
                int j = tid + r * nt;
                if (j < n) { T d = jac(s3, tb, j, n); acc[r] += (T)2 * d; ta[j] = dl[j] + h * d; }
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < L96_PPT; ++r) {
                int j = tid + r * nt;
                if (j < n) { T d = jac(s4, ta, j, n); acc[r] += d; dl[j] = dl[j] + h6 * acc[r]; }
            }
            __syncthreads();
        }
        T *wn = w + (int64_t)(t + 1) * n;
        for (int j = tid; j < n; j += nt) {
            T v = dl[j] + wn[j];
            dl[j] = v;
            wn[j] = v;
        }
        __syncthreads();
    }
}

// Adjoint sweep L^{-T} on one column per CTA.  obs_mode 1:
// W_N = obs(W_N), W_t = obs_t(W_t) + M_t^T W_{t+1}; obs_mode 0: plain
// W_t = W_t + M_t^T W_{t+1}.  obs(v)[s] = obs_scale v[s] at observed times
// and points, zero elsewhere.
template <typename T>
__global__ void __launch_bounds__(L96_THREADS)
k_l96_adj(int n, int N, int steps, T h, const T *__restrict__ stages, T *W, int64_t ld, int obs_mode, T obs_scale,
          int obs_stride, int t0, int ts)
{
    extern __shared__ __align__(16) unsigned char sm[];
    T *lam = reinterpret_cast<T *>(sm);
    T *aa = lam + n, *ab = aa + n;
    T *w = W + (int64_t)blockIdx.x * ld;
    const int tid = threadIdx.x, nt = blockDim.x;
    auto obs_at = [&](int t) { return t >= t0 && (t - t0) % ts == 0; };
    {
        T *wN = w + (int64_t)N * n;
        const bool ob = obs_at(N);
        for (int j = tid; j < n; j += nt) {
            T v = wN[j];
            if (obs_mode == 1) v = (ob && j % obs_stride == 0) ? obs_scale * v : (T)0;
            lam[j] = v;
            wN[j] = v;
        }
    }
    __syncthreads();
    T acc[L96_PPT];
    const T h2 = h * (T)0.5, h3 = h / (T)3, h6 = h / (T)6;
    for (int t = N - 1; t >= 0; --t) {
        for (int k = steps - 1; k >= 0; --k) {
            const int64_t g = (int64_t)t * steps + k;
            const T *s1 = stages + (4 * g + 0) * n, *s2 = stages + (4 * g + 1) * n;
            const T *s3 = stages + (4 * g + 2) * n, *s4 = stages + (4 * g + 3) * n;
            for (int j = tid; j < n; j += nt) aa[j] = h6 * lam[j];            // a4
            __syncthreads();
#pragma unroll
            for (int r = 0; r < L96_PPT; ++r) {
                int j = tid + r * nt;
                if (j < n) { T g4 = jacT(s4, aa, j, n); acc[r] = lam[j] + g4; ab[j] = h3 * lam[j] + h * g4; }
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < L96_PPT; ++r) {
                int j = tid + r * nt;
                if (j < n) { T g3 = jacT(s3, ab, j, n); acc[r] += g3; aa[j] = h3 * lam[j] + h2 * g3; }
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < L96_PPT; ++r) {
                int j = tid + r * nt;
                if (j < n) { T g2 = jacT(s2, aa, j, n); acc[r] += g2; ab[j] = h6 * lam[j] + h2 * g2; }
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < L96_PPT; ++r) {
                int j = tid + r * nt;
                if (j < n) { T g1 = jacT(s1, ab, j, n); lam[j] = acc[r] + g1; }
            }
            __syncthreads();
        }
        T *wt = w + (int64_t)t * n;
        const bool ob = obs_at(t);
        for (int j = tid; j < n; j += nt) {
            T v = wt[j];
            if (obs_mode == 1) v = (ob && j % obs_stride == 0) ? obs_scale * v : (T)0;
            v += lam[j];
            lam[j] = v;
            wt[j] = v;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Few columns (the PCG matvec): one column per 8-CTA thread-block cluster.
// CTA r of the cluster owns points r P .. r P + P - 1 (P = n / 8, one point
// per thread); the stencils' neighbours beyond the slice are read from the
// adjacent CTAs' shared memory (distributed shared memory), and a cluster
// barrier separates the RK4 stages, as __syncthreads does in the one-CTA
// kernels above.
// ---------------------------------------------------------------------------
constexpr int L96_CL = 8;

// v at global point j of a vector distributed over the cluster (slices of P)
template <typename T>
__device__ __forceinline__ T cl_get(cg::cluster_group &cl, T *slice, int j, int P, int rank)
{
    const int owner = j / P, li = j - owner * P;
    if (owner == rank) return slice[li];
    return *cl.map_shared_rank(slice + li, owner);
}

template <typename T>
__device__ __forceinline__ T jac_cl(cg::cluster_group &cl, const T *__restrict__ x, T *d, int j, int n, int P, int rank,
                                    T dj)
{
    const int jm2 = wrap(j - 2, n), jm1 = wrap(j - 1, n), jp1 = wrap(j + 1, n);
    return (cl_get(cl, d, jp1, P, rank) - cl_get(cl, d, jm2, P, rank)) * __ldg(x + jm1) +
           (__ldg(x + jp1) - __ldg(x + jm2)) * cl_get(cl, d, jm1, P, rank) - dj;
}

template <typename T>
__device__ __forceinline__ T jacT_cl(cg::cluster_group &cl, const T *__restrict__ x, T *a, int i, int n, int P,
                                     int rank, T ai)
{
    const int im2 = wrap(i - 2, n), im1 = wrap(i - 1, n), ip1 = wrap(i + 1, n), ip2 = wrap(i + 2, n);
    return __ldg(x + im2) * cl_get(cl, a, im1, P, rank) - __ldg(x + ip1) * cl_get(cl, a, ip2, P, rank) +
           (__ldg(x + ip2) - __ldg(x + im1)) * cl_get(cl, a, ip1, P, rank) - ai;
}

template <typename T>
__global__ void __cluster_dims__(L96_CL, 1, 1) __launch_bounds__(1024, 1)
k_l96_tlm_cl(int n, int N, int steps, T h, const T *__restrict__ stages, T *W, int64_t ld)
{
    extern __shared__ __align__(16) unsigned char sm[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), P = n / L96_CL, tid = threadIdx.x;
    T *dl = reinterpret_cast<T *>(sm), *ta = dl + P, *tb = ta + P;
    T *w = W + (int64_t)(blockIdx.x / L96_CL) * ld;
    const bool act = tid < P;
    const int j = rank * P + tid;
    if (act) dl[tid] = w[j];
    cl.sync();
    const T h2 = h * (T)0.5, h6 = h / (T)6;
    for (int t = 0; t < N; ++t) {
        for (int k = 0; k < steps; ++k) {
            const int64_t g = (int64_t)t * steps + k;
            const T *s1 = stages + (4 * g + 0) * n, *s2 = stages + (4 * g + 1) * n;
            const T *s3 = stages + (4 * g + 2) * n, *s4 = stages + (4 * g + 3) * n;
            T acc = 0;
            if (act) { const T d = jac_cl(cl, s1, dl, j, n, P, rank, dl[tid]); acc = d; ta[tid] = dl[tid] + h2 * d; }
            cl.sync();
            if (act) { const T d = jac_cl(cl, s2, ta, j, n, P, rank, ta[tid]); acc += (T)2 * d; tb[tid] = dl[tid] + h2 * d; }
            cl.sync();
            if (act) { const T d = jac_cl(cl, s3, tb, j, n, P, rank, tb[tid]); acc += (T)2 * d; ta[tid] = dl[tid] + h * d; }
            cl.sync();
            if (act) { const T d = jac_cl(cl, s4, ta, j, n, P, rank, ta[tid]); acc += d; dl[tid] = dl[tid] + h6 * acc; }
            cl.sync();
        }
        if (act) {
            T *wn = w + (int64_t)(t + 1) * n;
            const T v = dl[tid] + wn[j];
            dl[tid] = v;
            wn[j] = v;
        }
        cl.sync();
    }
}

template <typename T>
__global__ void __cluster_dims__(L96_CL, 1, 1) __launch_bounds__(1024, 1)
k_l96_adj_cl(int n, int N, int steps, T h, const T *__restrict__ stages, T *W, int64_t ld, int obs_mode, T obs_scale,
             int obs_stride, int t0, int ts)
{
    extern __shared__ __align__(16) unsigned char sm[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), P = n / L96_CL, tid = threadIdx.x;
    T *lam = reinterpret_cast<T *>(sm), *aa = lam + P, *ab = aa + P;
    T *w = W + (int64_t)(blockIdx.x / L96_CL) * ld;
    const bool act = tid < P;
    const int j = rank * P + tid;
    auto obs_at = [&](int t) { return t >= t0 && (t - t0) % ts == 0; };
    if (act) {
        T *wN = w + (int64_t)N * n;
        T v = wN[j];
        if (obs_mode == 1) v = (obs_at(N) && j % obs_stride == 0) ? obs_scale * v : (T)0;
        lam[tid] = v;
        wN[j] = v;
    }
    cl.sync();
    const T h2 = h * (T)0.5, h3 = h / (T)3, h6 = h / (T)6;
    for (int t = N - 1; t >= 0; --t) {
        for (int k = steps - 1; k >= 0; --k) {
            const int64_t g = (int64_t)t * steps + k;
            const T *s1 = stages + (4 * g + 0) * n, *s2 = stages + (4 * g + 1) * n;
            const T *s3 = stages + (4 * g + 2) * n, *s4 = stages + (4 * g + 3) * n;
            T acc = 0;
            if (act) aa[tid] = h6 * lam[tid];                                   // a4
            cl.sync();
            if (act) { const T g4 = jacT_cl(cl, s4, aa, j, n, P, rank, aa[tid]); acc = lam[tid] + g4; ab[tid] = h3 * lam[tid] + h * g4; }
            cl.sync();
            if (act) { const T g3 = jacT_cl(cl, s3, ab, j, n, P, rank, ab[tid]); acc += g3; aa[tid] = h3 * lam[tid] + h2 * g3; }
            cl.sync();
            if (act) { const T g2 = jacT_cl(cl, s2, aa, j, n, P, rank, aa[tid]); acc += g2; ab[tid] = h6 * lam[tid] + h2 * g2; }
            cl.sync();
            if (act) { const T g1 = jacT_cl(cl, s1, ab, j, n, P, rank, ab[tid]); lam[tid] = acc + g1; }
            cl.sync();
        }
        if (act) {
            T *wt = w + (int64_t)t * n;
            T v = wt[j];
            if (obs_mode == 1) v = (obs_at(t) && j % obs_stride == 0) ? obs_scale * v : (T)0;
            v += lam[tid];
            lam[tid] = v;
            wt[j] = v;
        }
        cl.sync();
    }
}

// ---------------------------------------------------------------------------
// Register-blocked FP32 sweeps (n = P nt, nt a multiple of 32 and <= 1024; P
// = 8 points per thread): thread tau owns
// the contiguous run of points P tau .. P tau + P - 1 of C probe columns.
// The running stage input u and the RK4 accumulator live in registers; the
// step's base state (d for the tangent-linear sweep, lambda for the adjoint)
// is thread-private and kept in shared memory as float4 quads laid out
// [c][p/4][tau] (consecutive lanes, consecutive 16-byte words: one
// conflict-free 128-bit access per quad).  The stage state x of the
// trajectory is staged in shared memory, double-buffered: each thread copies
// its slice of the next stage's x with cp.async while the current stage
// computes, so the L2 latency is off the critical path, and x serves all C
// columns.  The stencils' halos of u and x come from the neighbouring lanes by
// warp shuffles and, at warp boundaries, from a small double-buffered edge
// table (u) or the staged x; one __syncthreads per RK4 stage orders it all.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
                 "l"(gmem_src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Stage this thread's P points of the stage state x into xb.
template <int P>
__device__ __forceinline__ void stage_x_async(float *xb, const float *__restrict__ x, int j0)
{
#pragma unroll
    for (int q = 0; q < P / 4; ++q) cp_async16(xb + j0 + 4 * q, x + j0 + 4 * q);
    cp_async_commit();
}

// x at points j0 - 2 .. j0 + P + 1 from the staged vector xs (v[q] = x[j0 - 2 + q]).
template <int P>
__device__ __forceinline__ void read_xwin(float (&v)[P + 4], const float *xs, int j0, int n, int lane)
{
#pragma unroll
    for (int q = 0; q < P / 4; ++q) {
        const float4 a = *reinterpret_cast<const float4 *>(xs + j0 + 4 * q);
        v[2 + 4 * q] = a.x; v[3 + 4 * q] = a.y; v[4 + 4 * q] = a.z; v[5 + 4 * q] = a.w;
    }
    const float l0 = __shfl_up_sync(0xffffffffu, v[P], 1), l1 = __shfl_up_sync(0xffffffffu, v[P + 1], 1);
    const float r0 = __shfl_down_sync(0xffffffffu, v[2], 1), r1 = __shfl_down_sync(0xffffffffu, v[3], 1);
    v[0] = (lane == 0) ? xs[wrap(j0 - 2, n)] : l0;
    v[1] = (lane == 0) ? xs[wrap(j0 - 1, n)] : l1;
    v[P + 2] = (lane == 31) ? xs[wrap(j0 + P, n)] : r0;
    v[P + 3] = (lane == 31) ? xs[wrap(j0 + P + 1, n)] : r1;
}

__device__ __forceinline__ float shfl_up1(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shfl_dn1(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// Shared memory of the register-blocked sweeps: [C][P/4][nt] float4 base
// state, two staged stage states of n floats, [2][C][nw][3] warp edges.
template <int C, int P>
static size_t rb_smem(int n)
{
    return sizeof(float) * ((size_t)C * n + 2 * (size_t)n + (size_t)2 * C * (n / P / 32) * 3);
}

// Per-CTA state of the register-blocked sweeps, shared by the stage bodies.
struct RbCta {
    int n, nt, tid, lane, wid, nw, j0;
    float4 *base;   // [C][P/4][nt] thread-private base state (d or lambda)
    float *xbuf;    // [2][n] staged stage states
    float *edge;    // [2][C][nw][3] warp edges of the stage input
};

template <int C, int P>
__device__ __forceinline__ void load_base(const RbCta &r, int c, float (&d)[P])
{
#pragma unroll
    for (int q = 0; q < P / 4; ++q) {
        const float4 v = r.base[(size_t)(c * (P / 4) + q) * r.nt + r.tid];
        d[4 * q] = v.x; d[4 * q + 1] = v.y; d[4 * q + 2] = v.z; d[4 * q + 3] = v.w;
    }
}

template <int C, int P>
__device__ __forceinline__ void store_base(const RbCta &r, int c, const float (&d)[P])
{
#pragma unroll
    for (int q = 0; q < P / 4; ++q)
        r.base[(size_t)(c * (P / 4) + q) * r.nt + r.tid] = make_float4(d[4 * q], d[4 * q + 1], d[4 * q + 2], d[4 * q + 3]);
}

// Halo exchange of the stage input u at the start of a stage (buffer `par`):
// TLM needs u at j0 - 2, j0 - 1 (left) and j0 + P (right); the adjoint at
// j0 - 1 (left) and j0 + P, j0 + P + 1 (right).  Lanes get them from their
// neighbours by shuffles; warp edges go through the edge table, read after
// the stage's __syncthreads (done by the caller between the two halves).
template <int C, int P, bool ADJ>
__device__ __forceinline__ void halo_publish(const RbCta &r, const float (&u)[C][P], int par, float (&HL)[C][2],
                                             float (&HR)[C][2])
{
    float *eb = r.edge + (size_t)par * C * r.nw * 3;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        if (!ADJ) {
            HL[c][0] = shfl_up1(u[c][P - 2]);      // u_{j0-2}
            HL[c][1] = shfl_up1(u[c][P - 1]);      // u_{j0-1}
            HR[c][0] = shfl_dn1(u[c][0]);          // u_{j0+P}
            if (r.lane == 31) { eb[(c * r.nw + r.wid) * 3 + 0] = u[c][P - 2]; eb[(c * r.nw + r.wid) * 3 + 1] = u[c][P - 1]; }
            if (r.lane == 0) eb[(c * r.nw + r.wid) * 3 + 2] = u[c][0];
        } else {
            HL[c][1] = shfl_up1(u[c][P - 1]);      // a_{j0-1}
            HR[c][0] = shfl_dn1(u[c][0]);          // a_{j0+P}
            HR[c][1] = shfl_dn1(u[c][1]);          // a_{j0+P+1}
            if (r.lane == 31) eb[(c * r.nw + r.wid) * 3 + 0] = u[c][P - 1];
            if (r.lane == 0) { eb[(c * r.nw + r.wid) * 3 + 1] = u[c][0]; eb[(c * r.nw + r.wid) * 3 + 2] = u[c][1]; }
        }
    }
}

template <int C, bool ADJ>
__device__ __forceinline__ void halo_collect(const RbCta &r, int par, float (&HL)[C][2], float (&HR)[C][2])
{
    const float *eb = r.edge + (size_t)par * C * r.nw * 3;
    const int wp = (r.wid == 0) ? r.nw - 1 : r.wid - 1, wn = (r.wid == r.nw - 1) ? 0 : r.wid + 1;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        if (!ADJ) {
            if (r.lane == 0) { HL[c][0] = eb[(c * r.nw + wp) * 3 + 0]; HL[c][1] = eb[(c * r.nw + wp) * 3 + 1]; }
            if (r.lane == 31) HR[c][0] = eb[(c * r.nw + wn) * 3 + 2];
        } else {
            if (r.lane == 0) HL[c][1] = eb[(c * r.nw + wp) * 3 + 0];
            if (r.lane == 31) { HR[c][0] = eb[(c * r.nw + wn) * 3 + 1]; HR[c][1] = eb[(c * r.nw + wn) * 3 + 2]; }
        }
    }
}

// One RK4 stage I (0..3) of the tangent-linear step: k = J(s_I) u,
// acc (+)= w_I k, next input u = d + c_I k (I < 3) or d = d + h/6 (acc + k).
template <int C, int P, int I>
__device__ __forceinline__ void tlm_stage(const RbCta &r, float (&u)[C][P], float (&acc)[C][P],
                                          const float *__restrict__ stages, int g, int G, int &sidx, float h)
{
    cp_async_wait_all();
    float HL[C][2], HR[C][2];
    halo_publish<C, P, false>(r, u, sidx & 1, HL, HR);
    __syncthreads();
    {   // stage the next stage state into the other buffer
        const int gn = (I < 3) ? g : g + 1, in = (I < 3) ? I + 1 : 0;
        if (gn < G) stage_x_async<P>(r.xbuf + (size_t)((sidx + 1) & 1) * r.n, stages + (int64_t)(4 * gn + in) * r.n, r.j0);
    }
    halo_collect<C, false>(r, sidx & 1, HL, HR);
    float xv[P + 4];
    read_xwin<P>(xv, r.xbuf + (size_t)(sidx & 1) * r.n, r.j0, r.n, r.lane);
    const float cf = (I == 2) ? h : 0.5f * h;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        float d[P];
        load_base<C, P>(r, c, d);
        float um2 = HL[c][0], um1 = HL[c][1];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const float up1 = (p + 1 < P) ? u[c][p + 1] : HR[c][0];
            const float cur = u[c][p];
            // (J u)_j = (u_{j+1} - u_{j-2}) x_{j-1} + (x_{j+1} - x_{j-2}) u_{j-1} - u_j
            const float kk = fmaf(up1 - um2, xv[p + 1], fmaf(xv[p + 3] - xv[p], um1, -cur));
            um2 = um1;
            um1 = cur;
            if (I == 0) {
                acc[c][p] = kk;
                u[c][p] = fmaf(cf, kk, d[p]);
            } else if (I < 3) {
                acc[c][p] = fmaf(2.f, kk, acc[c][p]);
                u[c][p] = fmaf(cf, kk, d[p]);
            } else {
                u[c][p] = fmaf(h * (1.f / 6.f), acc[c][p] + kk, d[p]);
            }
        }
        if (I == 3) store_base<C, P>(r, c, u[c]);
    }
    ++sidx;
}

// One RK4 stage I (3..0) of the adjoint step (stage state s_I): g = J(s_I)^T a;
// I = 3: acc = lam + g, a = h/3 lam + h g; I = 2: acc += g, a = h/3 lam + h/2 g;
// I = 1: acc += g, a = h/6 lam + h/2 g; I = 0: lam = acc + g.
template <int C, int P, int I>
__device__ __forceinline__ void adj_stage(const RbCta &r, float (&u)[C][P], float (&acc)[C][P],
                                          const float *__restrict__ stages, int g, int &sidx, float h)
{
    cp_async_wait_all();
    float HL[C][2], HR[C][2];
    halo_publish<C, P, true>(r, u, sidx & 1, HL, HR);
    __syncthreads();
    {   // stage the next stage state (backwards) into the other buffer
        const int gn = (I > 0) ? g : g - 1, in = (I > 0) ? I - 1 : 3;
        if (gn >= 0) stage_x_async<P>(r.xbuf + (size_t)((sidx + 1) & 1) * r.n, stages + (int64_t)(4 * gn + in) * r.n, r.j0);
    }
    halo_collect<C, true>(r, sidx & 1, HL, HR);
    float xv[P + 4];
    read_xwin<P>(xv, r.xbuf + (size_t)(sidx & 1) * r.n, r.j0, r.n, r.lane);
#pragma unroll
    for (int c = 0; c < C; ++c) {
        float lam[P];
        load_base<C, P>(r, c, lam);
        float am1 = HL[c][1];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const float ap1 = (p + 1 < P) ? u[c][p + 1] : HR[c][0];
            const float ap2 = (p + 2 < P) ? u[c][p + 2] : ((p + 2 == P) ? HR[c][0] : HR[c][1]);
            const float cur = u[c][p];
            // (J^T a)_i = x_{i-2} a_{i-1} - x_{i+1} a_{i+2} + (x_{i+2} - x_{i-1}) a_{i+1} - a_i
            const float gg = fmaf(xv[p], am1, fmaf(-xv[p + 3], ap2, fmaf(xv[p + 4] - xv[p + 1], ap1, -cur)));
            am1 = cur;
            if (I == 3) {
                acc[c][p] = lam[p] + gg;
                u[c][p] = fmaf(h * (1.f / 3.f), lam[p], h * gg);
            } else if (I == 2) {
                acc[c][p] += gg;
                u[c][p] = fmaf(h * (1.f / 3.f), lam[p], 0.5f * h * gg);
            } else if (I == 1) {
                acc[c][p] += gg;
                u[c][p] = fmaf(h * (1.f / 6.f), lam[p], 0.5f * h * gg);
            } else {
                lam[p] = acc[c][p] + gg;
            }
        }
        if (I == 0) store_base<C, P>(r, c, lam);
    }
    ++sidx;
}

// Forward sweep L^{-1} (w_{t+1} += M_t w_t) for columns blockIdx.x*C .. +C-1 (< K).
template <int C, int P>
__global__ void __launch_bounds__(P == 16 ? 512 : 1024, 1)
k_l96_tlm_rb(int n, int N, int steps, float h, const float *__restrict__ stages, float *W, int64_t ld, int K)
{
    extern __shared__ __align__(16) unsigned char sm[];
    RbCta r;
    r.n = n; r.nt = blockDim.x; r.tid = threadIdx.x; r.lane = r.tid & 31; r.wid = r.tid >> 5; r.nw = r.nt >> 5;
    r.j0 = r.tid * P;
    r.base = reinterpret_cast<float4 *>(sm);
    r.xbuf = reinterpret_cast<float *>(sm) + (size_t)C * n;
    r.edge = r.xbuf + 2 * (size_t)n;
    const int G = N * steps;
    stage_x_async<P>(r.xbuf, stages, r.j0);                  // stage (g = 0, I = 0)
    float u[C][P], acc[C][P];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const int col = blockIdx.x * C + c;
        const float *w = W + (int64_t)min(col, K - 1) * ld;
#pragma unroll
        for (int p = 0; p < P; ++p) u[c][p] = (col < K) ? w[r.j0 + p] : 0.f;
        store_base<C, P>(r, c, u[c]);
    }
    int sidx = 0;
    for (int t = 0; t < N; ++t) {
        for (int k = 0; k < steps; ++k) {
            const int g = t * steps + k;
            tlm_stage<C, P, 0>(r, u, acc, stages, g, G, sidx, h);
            tlm_stage<C, P, 1>(r, u, acc, stages, g, G, sidx, h);
            tlm_stage<C, P, 2>(r, u, acc, stages, g, G, sidx, h);
            tlm_stage<C, P, 3>(r, u, acc, stages, g, G, sidx, h);
        }
        // subwindow boundary: w_{t+1} += d, d = w_{t+1}
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int col = blockIdx.x * C + c;
            if (col >= K) continue;
            float *wn = W + (int64_t)col * ld + (int64_t)(t + 1) * n;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float v = u[c][p] + wn[r.j0 + p];
                wn[r.j0 + p] = v;
                u[c][p] = v;
            }
            store_base<C, P>(r, c, u[c]);
        }
    }
    cp_async_wait_all();
}

// Adjoint sweep L^{-T} for columns blockIdx.x*C .. +C-1 (< K); obs_mode as
// k_l96_adj.
template <int C, int P>
__global__ void __launch_bounds__(P == 16 ? 512 : 1024, 1)
k_l96_adj_rb(int n, int N, int steps, float h, const float *__restrict__ stages, float *W, int64_t ld, int K,
             int obs_mode, float obs_scale, int obs_stride, int t0, int ts)
{
    extern __shared__ __align__(16) unsigned char sm[];
    RbCta r;
    r.n = n; r.nt = blockDim.x; r.tid = threadIdx.x; r.lane = r.tid & 31; r.wid = r.tid >> 5; r.nw = r.nt >> 5;
    r.j0 = r.tid * P;
    r.base = reinterpret_cast<float4 *>(sm);
    r.xbuf = reinterpret_cast<float *>(sm) + (size_t)C * n;
    r.edge = r.xbuf + 2 * (size_t)n;
    const int G = N * steps;
    stage_x_async<P>(r.xbuf, stages + (int64_t)(4 * (G - 1) + 3) * n, r.j0);   // stage (g = G - 1, I = 3)
    auto obs_at = [&](int t) { return t >= t0 && (t - t0) % ts == 0; };
    float u[C][P], acc[C][P];
    {
        const bool ob = obs_at(N);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int col = blockIdx.x * C + c;
            float *wN = W + (int64_t)min(col, K - 1) * ld + (int64_t)N * n;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                float v = (col < K) ? wN[r.j0 + p] : 0.f;
                if (obs_mode == 1) v = (ob && (r.j0 + p) % obs_stride == 0) ? obs_scale * v : 0.f;
                if (col < K) wN[r.j0 + p] = v;
                u[c][p] = v;
            }
            store_base<C, P>(r, c, u[c]);
        }
    }
    int sidx = 0;
    for (int t = N - 1; t >= 0; --t) {
        for (int k = steps - 1; k >= 0; --k) {
            const int g = t * steps + k;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                float lam[P];
                load_base<C, P>(r, c, lam);
#pragma unroll
                for (int p = 0; p < P; ++p) u[c][p] = (h * (1.f / 6.f)) * lam[p];
            }
            adj_stage<C, P, 3>(r, u, acc, stages, g, sidx, h);
            adj_stage<C, P, 2>(r, u, acc, stages, g, sidx, h);
            adj_stage<C, P, 1>(r, u, acc, stages, g, sidx, h);
            adj_stage<C, P, 0>(r, u, acc, stages, g, sidx, h);
        }
        // subwindow boundary: lam = obs(w_t) + lam, w_t = lam
        const bool ob = obs_at(t);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int col = blockIdx.x * C + c;
            if (col >= K) continue;
            float lam[P];
            load_base<C, P>(r, c, lam);
            float *wt = W + (int64_t)col * ld + (int64_t)t * n;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                float v = wt[r.j0 + p];
                if (obs_mode == 1) v = (ob && (r.j0 + p) % obs_stride == 0) ? obs_scale * v : 0.f;
                lam[p] += v;
                wt[r.j0 + p] = lam[p];
            }
            store_base<C, P>(r, c, lam);
        }
    }
    cp_async_wait_all();
}

// Register-blocked form: FP32, n = 8 nt with nt a multiple of 32 and at most
// 1024 (0: not applicable).  Sixteen points per thread on half the threads
// measured slower at n = 8192 (6.1 against 5.6 ms for a 256-column product).
template <typename T> static int rb_points(int n)
{
    if (sizeof(T) != 4) return 0;
    if (n % 256 == 0 && n / 8 <= 1024) return 8;
    return 0;
}
// Columns per CTA: two for blocks (the staged stage states then serve both),
// one for few columns, where the CTAs are the parallelism.
static int rb_cols(int K) { return K >= 64 ? 2 : 1; }

static bool use_cluster(int n, int K) { return K <= 32 && n % L96_CL == 0 && n / L96_CL >= 2 && n / L96_CL <= 1024; }

template <int C, int P>
static void launch_tlm_rb(cudaStream_t s, int n, int N, int steps, double dt, const float *stages, int K, float *W,
                          int64_t ld)
{
    static const bool attr = [] {
        return cudaFuncSetAttribute(k_l96_tlm_rb<C, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)rb_smem<C, P>(WC4D_FFT_MAX_N)) == cudaSuccess;
    }();   // once, thread-safe
    (void)attr;
    WC4D_LAUNCH(k_l96_tlm_rb<C, P><<<ceil_div(K, C), n / P, rb_smem<C, P>(n), s>>>(n, N, steps, (float)dt, stages, W,
                                                                                  ld, K));
}

template <typename T>
void launch_l96_tlm_sweep(cudaStream_t s, int n, int N, int steps, double dt, const T *stages, int K, T *W,
                          int64_t ld)
{
    if constexpr (sizeof(T) == 4) {
        const int P = rb_points<T>(n);
        if (P == 8) {
            if (rb_cols(K) == 2) launch_tlm_rb<2, 8>(s, n, N, steps, dt, stages, K, W, ld);
            else launch_tlm_rb<1, 8>(s, n, N, steps, dt, stages, K, W, ld);
            return;
        }
    }
    static const bool attr = [] {
        return cudaFuncSetAttribute(k_l96_tlm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(3 * WC4D_FFT_MAX_N * sizeof(T))) == cudaSuccess;
    }();   // once, thread-safe
    (void)attr;
    if (use_cluster(n, K)) {
        WC4D_LAUNCH(k_l96_tlm_cl<T><<<K * L96_CL, 1024, 3 * (size_t)(n / L96_CL) * sizeof(T), s>>>(n, N, steps, (T)dt,
                                                                                                 stages, W, ld));
        return;
    }
    WC4D_LAUNCH(k_l96_tlm<T><<<K, L96_THREADS, 3 * (size_t)n * sizeof(T), s>>>(n, N, steps, (T)dt, stages, W, ld));
}

template <int C, int P>
static void launch_adj_rb(cudaStream_t s, int n, int N, int steps, double dt, const float *stages, int K, float *W,
                          int64_t ld, int obs_mode, double obs_scale, int obs_stride, int obs_t0, int obs_tstride)
{
    static const bool attr = [] {
        return cudaFuncSetAttribute(k_l96_adj_rb<C, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)rb_smem<C, P>(WC4D_FFT_MAX_N)) == cudaSuccess;
    }();   // once, thread-safe
    (void)attr;
    WC4D_LAUNCH(k_l96_adj_rb<C, P><<<ceil_div(K, C), n / P, rb_smem<C, P>(n), s>>>(
        n, N, steps, (float)dt, stages, W, ld, K, obs_mode, (float)obs_scale, obs_stride, obs_t0,
        obs_tstride > 0 ? obs_tstride : 1));
}

template <typename T>
void launch_l96_adj_sweep(cudaStream_t s, int n, int N, int steps, double dt, const T *stages, int K, T *W,
                          int64_t ld, int obs_mode, double obs_scale, int obs_stride, int obs_t0, int obs_tstride)
{
    if constexpr (sizeof(T) == 4) {
        const int P = rb_points<T>(n);
#define WC4D_ADJ_RB(CC, PP)                                                                                      \
    launch_adj_rb<CC, PP>(s, n, N, steps, dt, stages, K, W, ld, obs_mode, obs_scale, obs_stride, obs_t0, obs_tstride)
        if (P == 8) {
            if (rb_cols(K) == 2) WC4D_ADJ_RB(2, 8);
            else WC4D_ADJ_RB(1, 8);
            return;
        }
#undef WC4D_ADJ_RB
    }
    static const bool attr = [] {
        return cudaFuncSetAttribute(k_l96_adj<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(3 * WC4D_FFT_MAX_N * sizeof(T))) == cudaSuccess;
    }();   // once, thread-safe
    (void)attr;
    if (use_cluster(n, K)) {
        WC4D_LAUNCH(k_l96_adj_cl<T><<<K * L96_CL, 1024, 3 * (size_t)(n / L96_CL) * sizeof(T), s>>>(
            n, N, steps, (T)dt, stages, W, ld, obs_mode, (T)obs_scale, obs_stride, obs_t0,
            obs_tstride > 0 ? obs_tstride : 1));
        return;
    }
    WC4D_LAUNCH(k_l96_adj<T><<<K, L96_THREADS, 3 * (size_t)n * sizeof(T), s>>>(n, N, steps, (T)dt, stages, W, ld, obs_mode,
                                                                     (T)obs_scale, obs_stride, obs_t0,
                                                                     obs_tstride > 0 ? obs_tstride : 1));
}

template void launch_l96_tlm_sweep<double>(cudaStream_t, int, int, int, double, const double *, int, double *,
                                           int64_t);
template void launch_l96_tlm_sweep<float>(cudaStream_t, int, int, int, double, const float *, int, float *, int64_t);
template void launch_l96_adj_sweep<double>(cudaStream_t, int, int, int, double, const double *, int, double *,
                                           int64_t, int, double, int, int, int);
template void launch_l96_adj_sweep<float>(cudaStream_t, int, int, int, double, const float *, int, float *, int64_t,
                                          int, double, int, int, int);

// Nonlinear RK4 run in FP64 on one CTA: traj[g+1] = RK4(traj[g]) for
// g < nsteps, storing the stage states of every step; with eta (forcing,
// (N+1) x n, block t added at the end of subwindow t-1, eq. 1) the state
// after every `steps` steps receives eta_t.
__device__ __forceinline__ double l96f(const double *y, int j, int n, double F)
{
    return (y[wrap(j + 1, n)] - y[wrap(j - 2, n)]) * y[wrap(j - 1, n)] - y[j] + F;
}

__global__ void __launch_bounds__(1024) k_l96_run(int n, int nsteps, double F, double h, double *traj, double *stages,
                                                 const double *eta, int steps)
{
    extern __shared__ __align__(16) unsigned char sm[];
    double *x = reinterpret_cast<double *>(sm);
    double *st = x + n;
    const int tid = threadIdx.x, nt = blockDim.x;
    constexpr int R = WC4D_FFT_MAX_N / 1024;
    double acc[R], d[R];
    for (int j = tid; j < n; j += nt) x[j] = traj[j];
    __syncthreads();
    for (int g = 0; g < nsteps; ++g) {
        double *sg = stages + (int64_t)4 * g * n;
        const double cf[3] = {0.5 * h, 0.5 * h, h};
        const double wgt[4] = {1.0, 2.0, 2.0, 1.0};
        for (int j = tid; j < n; j += nt) sg[j] = x[j];
        // stage 1 from x, stages 2-4 from st
        for (int stage = 0; stage < 4; ++stage) {
            const double *src = (stage == 0) ? x : st;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                int j = tid + r * nt;
                if (j < n) {
                    d[r] = l96f(src, j, n, F);
                    acc[r] = (stage == 0 ? 0.0 : acc[r]) + wgt[stage] * d[r];
                }
            }
            __syncthreads();
            if (stage < 3) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    int j = tid + r * nt;
                    if (j < n) {
                        double v = x[j] + cf[stage] * d[r];
                        st[j] = v;
                        sg[(int64_t)(stage + 1) * n + j] = v;
                    }
                }
            } else {
#pragma unroll
                const bool forced = eta && (g + 1) % steps == 0;
                const double *eg = forced ? eta + (int64_t)((g + 1) / steps) * n : nullptr;
                for (int r = 0; r < R; ++r) {
                    int j = tid + r * nt;
                    if (j < n) {
                        double v = x[j] + h / 6.0 * acc[r];
                        if (forced) v += eg[j];
                        x[j] = v;
                        traj[(int64_t)(g + 1) * n + j] = v;
                    }
                }
            }
            __syncthreads();
        }
    }
}

void launch_l96_run(cudaStream_t s, int n, int nsteps, double F, double dt, double *traj, double *stages,
                    const double *eta, int steps)
{
    static const bool attr = [] {
        return cudaFuncSetAttribute(k_l96_run, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(2 * WC4D_FFT_MAX_N * sizeof(double))) == cudaSuccess;
    }();   // once, thread-safe
    (void)attr;
    WC4D_LAUNCH(k_l96_run<<<1, 1024, 2 * (size_t)n * sizeof(double), s>>>(n, nsteps, F, dt, traj, stages, eta,
                                                                           steps));
}

// Stage states of every RK4 step from a given trajectory (states x_g, g <
// nsteps): s1 = x_g, s2 = x_g + h/2 f(s1), s3 = x_g + h/2 f(s2), s4 = x_g + h
// f(s3), the convention of k_l96_run; one CTA per step, two n-vectors of
// shared memory.
__global__ void __launch_bounds__(1024) k_l96_stages(int n, double F, double h, const double *traj, double *stages)
{
    extern __shared__ __align__(16) unsigned char sm[];
    double *x = reinterpret_cast<double *>(sm);
    double *st = x + n;
    const int64_t g = blockIdx.x;
    const double *xg = traj + g * n;
    double *sg = stages + 4 * g * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        x[j] = xg[j];
        st[j] = xg[j];
        sg[j] = xg[j];
    }
    __syncthreads();
    const double cf[3] = {0.5 * h, 0.5 * h, h};
    for (int i = 0; i < 3; ++i) {
        double d[WC4D_FFT_MAX_N / 1024];
#pragma unroll
        for (int r = 0; r < WC4D_FFT_MAX_N / 1024; ++r) {
            const int j = threadIdx.x + r * blockDim.x;
            if (j < n) d[r] = l96f(st, j, n, F);
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < WC4D_FFT_MAX_N / 1024; ++r) {
            const int j = threadIdx.x + r * blockDim.x;
            if (j < n) {
                const double v = x[j] + cf[i] * d[r];
                st[j] = v;
                sg[(int64_t)(i + 1) * n + j] = v;
            }
        }
        __syncthreads();
    }
}

void launch_l96_stages(cudaStream_t s, int n, int nsteps, double F, double dt, const double *traj, double *stages)
{
    static const bool attr = [] {
        return cudaFuncSetAttribute(k_l96_stages, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(2 * WC4D_FFT_MAX_N * sizeof(double))) == cudaSuccess;
    }();   // once, thread-safe
    (void)attr;
    WC4D_LAUNCH(k_l96_stages<<<nsteps, 1024, 2 * (size_t)n * sizeof(double), s>>>(n, F, dt, traj, stages));
}

