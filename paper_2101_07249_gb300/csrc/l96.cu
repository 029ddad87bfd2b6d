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
#include "bulk.cuh"

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
// Register-blocked FP32 sweeps (n = 8 nt, nt a multiple of 32 and at most
// 1024): thread tau owns points 8 tau .. 8 tau + 7 of C probe columns (C = 2
// for blocks, where each staged stage state then serves both columns; 1 for
// few columns, where the CTAs are the parallelism).
//  * The running stage input u and the RK4 accumulator live in registers.
//    The step's base state (d for the tangent-linear sweep, lambda for the
//    adjoint) is thread-private in shared memory, point-major and
//    column-minor: quad s of thread tau holds entries 4s .. 4s + 3 of its
//    flattened (point, column) run, at float4 slot s nt + tau (one
//    conflict-free 128-bit access per quad).
//  * The trajectory's stage states, shared by all probe columns, stream
//    through a ring of RB_NB shared-memory buffers: after a stage's barrier
//    one thread issues a single bulk asynchronous copy of the stage state
//    RB_NB - 1 stages ahead into the buffer the previous stage read,
//    completing on that buffer's mbarrier.  (Copying the state with one
//    16-byte cp.async per thread instead loaded the memory pipeline so much
//    that the sweep ran 1.4x slower.)
//  * The stencils' halos of u come from the neighbours' edge values,
//    published to shared memory (double-buffered by stage parity) before the
//    stage's barrier; the halos of x are read from the neighbours' points of
//    the staged state.
//  * One __syncthreads per RK4 stage.  The tangent-linear stage 0 takes d
//    from u itself (they are equal there); the adjoint's per-step start
//    a = h/6 lambda is folded into its stage 0.
//  * Every wait on a copy is bounded (the context's wait limit).  If one
//    gives up, the stage's barrier tells every thread, the sweep stops,
//    thread 0 waits (bounded) for the copies still in flight, sets the error
//    word and the CTA returns.
// ---------------------------------------------------------------------------
constexpr int RB_P = 8;    // points per thread
constexpr int RB_NB = 3;   // staged stage states: prefetch distance 2

// Shared memory (floats): base [C n], ring [RB_NB][n], edges A [2][nt][2C]
// and B [2][nt][C]; then RB_NB mbarriers.
template <int C>
static size_t rb_smem(int n)
{
    const int nt = n / RB_P;
    return sizeof(float) * ((size_t)C * n + (size_t)RB_NB * n + (size_t)6 * nt * C) + 8 * RB_NB;
}

// Per-CTA layout (constant through the sweep; kept apart from the ring
// bookkeeping so that it stays in registers with its pointer known to be
// shared memory).
struct RbCta {
    float *sm;      // dynamic shared memory
    int n, nt, tau;
    int tm1, tp1;   // neighbouring threads (periodic)
    int ring0;      // offset (floats) of ring buffer 0
    int ea0, eb0;   // offsets (floats) of edges A and B
    uint32_t mb0;   // shared address of the ring's first mbarrier
    unsigned limit; // polls of a ring wait before it gives up
};

// Parity of the next completion of each ring buffer.  It changes the same
// way in every thread (after each stage's wait, whatever the wait's outcome),
// so it stays warp-uniform.
struct RbRing {
    unsigned ph = 0;
};

template <int C>
__device__ __forceinline__ RbCta rb_setup(float *sm, int n, unsigned limit)
{
    RbCta L;
    L.sm = sm;
    L.n = n;
    L.nt = blockDim.x;
    L.tau = threadIdx.x;
    L.tm1 = L.tau == 0 ? L.nt - 1 : L.tau - 1;
    L.tp1 = L.tau == L.nt - 1 ? 0 : L.tau + 1;
    L.ring0 = C * n;
    L.ea0 = (C + RB_NB) * n;
    L.eb0 = L.ea0 + 4 * L.nt * C;
    L.mb0 = (uint32_t)__cvta_generic_to_shared(sm + L.eb0 + 2 * L.nt * C);
    L.limit = limit;
    return L;
}

// Thread 0: start the copy of the stage state at src (none if null) into
// ring buffer b.  The buffer was last read before the barrier the caller has
// passed; the proxy fence orders those generic-proxy reads before the
// asynchronous write.
__device__ __forceinline__ void rb_fetch(const RbCta &L, int b, const float *__restrict__ src)
{
    if (src && L.tau == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        sw_mb_expect(L.mb0 + 8 * b, (unsigned)L.n * 4u);
        sw_bulk_g2s((uint32_t)__cvta_generic_to_shared(L.sm + L.ring0 + b * L.n), src, (unsigned)L.n * 4u, L.mb0 + 8 * b);
    }
}

// Wait (at most L.limit further polls; none with a limit of 0, which makes
// every wait give up at once) for the copy into ring buffer b, then advance
// the buffer's parity.
__device__ __forceinline__ bool rb_wait(const RbCta &L, RbRing &R, int b)
{
    const uint32_t a = L.mb0 + 8 * b;
    const unsigned par = (R.ph >> b) & 1u;
    R.ph ^= 1u << b;
    if (L.limit == 0) return false;
    for (unsigned it = 0;; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(a), "r"(par)
                     : "memory");
        if (done) return true;
        if (it >= L.limit) return false;
    }
}

// x_{8 tau - 2 + q}, q = 0 .. 11, from ring buffer b.  ROT: the four
// 16-byte units 2 tau - 1 .. 2 tau + 2 (left neighbour's upper half, own two
// halves, right neighbour's lower half) as four 128-bit loads, lanes with bit
// 2 set taking them rotated by one, so that the eight lanes of a
// quarter-warp hit 32 distinct banks in every load (16 wavefronts a warp,
// against 32 for the two own loads at a 32-byte stride and the two 64-bit
// halo loads); the selects that undo the rotation cost registers, so the
// two-column sweeps keep the plain form.
template <bool ROT>
__device__ __forceinline__ void rb_read_x(const RbCta &L, int b, float (&X)[RB_P + 4])
{
    const float *xs = L.sm + L.ring0 + b * L.n;
    if constexpr (ROT) {
        const float4 *u4 = reinterpret_cast<const float4 *>(xs);
        const bool r = (L.tau >> 2) & 1;
        const int um = 2 * L.tm1 + 1, u0 = 2 * L.tau, u1 = u0 + 1, u2 = 2 * L.tp1;
        const float4 v0 = u4[r ? u0 : um], v1 = u4[r ? u1 : u0], v2 = u4[r ? u2 : u1], v3 = u4[r ? um : u2];
        const float4 lh = r ? v3 : v0, a = r ? v0 : v1, c = r ? v1 : v2, rh = r ? v2 : v3;
        X[0] = lh.z; X[1] = lh.w;
        X[2] = a.x; X[3] = a.y; X[4] = a.z; X[5] = a.w;
        X[6] = c.x; X[7] = c.y; X[8] = c.z; X[9] = c.w;
        X[10] = rh.x; X[11] = rh.y;
    } else {
        const float2 lh = *reinterpret_cast<const float2 *>(xs + RB_P * L.tm1 + RB_P - 2);
        const float4 a = *reinterpret_cast<const float4 *>(xs + RB_P * L.tau);
        const float4 c = *reinterpret_cast<const float4 *>(xs + RB_P * L.tau + 4);
        const float2 rh = *reinterpret_cast<const float2 *>(xs + RB_P * L.tp1);
        X[0] = lh.x; X[1] = lh.y;
        X[2] = a.x; X[3] = a.y; X[4] = a.z; X[5] = a.w;
        X[6] = c.x; X[7] = c.y; X[8] = c.z; X[9] = c.w;
        X[10] = rh.x; X[11] = rh.y;
    }
}

// Base-state quad s of this thread.
__device__ __forceinline__ float4 &rb_base(const RbCta &L, int s)
{
    return reinterpret_cast<float4 *>(L.sm)[s * L.nt + L.tau];
}

template <int C>
__device__ __forceinline__ void rb_store_base(const RbCta &L, const float (&v)[RB_P][C])
{
#pragma unroll
    for (int s = 0; s < RB_P * C / 4; ++s) {
        const int f = 4 * s;
        rb_base(L, s) = make_float4(v[f / C][f % C], v[(f + 1) / C][(f + 1) % C], v[(f + 2) / C][(f + 2) % C],
                                    v[(f + 3) / C][(f + 3) % C]);
    }
}

// Publish two points' values (points p0, p0 + 1, all columns) to edge A and
// one point's (p1) to edge B, in edge buffer e.
template <int C>
__device__ __forceinline__ void rb_publish(const RbCta &L, int e, const float (&u)[RB_P][C], int p0, int p1)
{
    float *ea = L.sm + L.ea0 + (e * L.nt + L.tau) * 2 * C;
    float *eb = L.sm + L.eb0 + (e * L.nt + L.tau) * C;
    if constexpr (C == 2) {
        *reinterpret_cast<float4 *>(ea) = make_float4(u[p0][0], u[p0][1], u[p0 + 1][0], u[p0 + 1][1]);
        *reinterpret_cast<float2 *>(eb) = make_float2(u[p1][0], u[p1][1]);
    } else {
        *reinterpret_cast<float2 *>(ea) = make_float2(u[p0][0], u[p0 + 1][0]);
        eb[0] = u[p1][0];
    }
}

template <int C>
__device__ __forceinline__ void rb_edge_a(const RbCta &L, int e, int who, float (&e0)[C], float (&e1)[C])
{
    const float *ea = L.sm + L.ea0 + (e * L.nt + who) * 2 * C;
    if constexpr (C == 2) {
        const float4 v = *reinterpret_cast<const float4 *>(ea);
        e0[0] = v.x; e0[1] = v.y; e1[0] = v.z; e1[1] = v.w;
    } else {
        const float2 v = *reinterpret_cast<const float2 *>(ea);
        e0[0] = v.x; e1[0] = v.y;
    }
}

template <int C>
__device__ __forceinline__ void rb_edge_b(const RbCta &L, int e, int who, float (&v)[C])
{
    const float *eb = L.sm + L.eb0 + (e * L.nt + who) * C;
    if constexpr (C == 2) {
        const float2 q = *reinterpret_cast<const float2 *>(eb);
        v[0] = q.x; v[1] = q.y;
    } else {
        v[0] = eb[0];
    }
}

// Start of an RK4 stage: wait for this stage's state in ring buffer xb,
// publish the edges of u, pass the stage's barrier (false: a wait gave up
// somewhere in the CTA), then start the copy of `next` (null: none) into the
// buffer the previous stage read.
template <int C>
__device__ __forceinline__ bool rb_stage_begin(const RbCta &L, RbRing &R, int xb, int e, const float (&u)[RB_P][C],
                                               int p0, int p1, const float *__restrict__ next)
{
    const bool ok = rb_wait(L, R, xb);
    rb_publish<C>(L, e, u, p0, p1);
    if (__syncthreads_or(!ok)) return false;
    rb_fetch(L, xb == 0 ? RB_NB - 1 : xb - 1, next);
    return true;
}

// One tangent-linear RK4 stage I on ring buffer xb (advanced on return):
// k = J(s_I) u, acc (+)= w_I k, next input u = d + c_I k (I < 3) or
// d = d + h/6 (acc + k).
template <int C, int I>
__device__ __forceinline__ bool rb_tlm_stage(const RbCta &L, RbRing &R, int &xb, const float *__restrict__ next,
                                             float (&u)[RB_P][C], float (&acc)[RB_P][C], float h)
{
    constexpr int P = RB_P, e = I & 1;
    if (!rb_stage_begin<C>(L, R, xb, e, u, P - 2, 0, next)) return false;
    // Points run from the last down, so only the old u_{j+1} has to be
    // carried (u_{j-1}, u_{j-2} are still the stage input when j is reached).
    float lm2[C], lm1[C], up1[C];
    rb_edge_b<C>(L, e, L.tp1, up1);                        // u_{8 tau + 8}
    rb_edge_a<C>(L, e, L.tm1, lm2, lm1);                   // u_{8 tau - 2}, u_{8 tau - 1}
    float X[P + 4];
    rb_read_x<C == 1>(L, xb, X);
    const float cf = (I == 2) ? h : 0.5f * h;
    float dq[4];
#pragma unroll
    for (int p = P - 1; p >= 0; --p) {
        if (I > 0 && ((p + 1) * C) % 4 == 0) {
            const float4 q = rb_base(L, ((p + 1) * C - 4) / 4);
            dq[0] = q.x; dq[1] = q.y; dq[2] = q.z; dq[3] = q.w;
        }
        const float xa = X[p + 1], xd = X[p + 3] - X[p];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float um2 = (p >= 2) ? u[p - 2][c] : (p == 1 ? lm1[c] : lm2[c]);
            const float um1 = (p >= 1) ? u[p - 1][c] : lm1[c];
            const float cur = u[p][c];
            // (J u)_j = (u_{j+1} - u_{j-2}) x_{j-1} + (x_{j+1} - x_{j-2}) u_{j-1} - u_j
            const float kk = fmaf(up1[c] - um2, xa, fmaf(xd, um1, -cur));
            up1[c] = cur;
            if (I == 0) {
                acc[p][c] = kk;
                u[p][c] = fmaf(cf, kk, cur);                // d = u at stage 0
            } else if (I < 3) {
                acc[p][c] = fmaf(2.f, kk, acc[p][c]);
                u[p][c] = fmaf(cf, kk, dq[(p * C + c) % 4]);
            } else {
                u[p][c] = fmaf(h * (1.f / 6.f), acc[p][c] + kk, dq[(p * C + c) % 4]);
            }
        }
    }
    if (I == 3) rb_store_base<C>(L, u);
    xb = (xb == RB_NB - 1) ? 0 : xb + 1;
    return true;
}

// One adjoint RK4 stage I (3 .. 0) on ring buffer xb: g = J(s_I)^T a;
// I = 3: acc = lam + g, a = h/3 lam + h g; I = 2: acc += g, a = h/3 lam + h/2 g;
// I = 1: acc += g, a = h/6 lam + h/2 g; I = 0: lam = acc + g, a = h/6 lam
// (the next step's first input).
template <int C, int I>
__device__ __forceinline__ bool rb_adj_stage(const RbCta &L, RbRing &R, int &xb, const float *__restrict__ next,
                                             float (&u)[RB_P][C], float (&acc)[RB_P][C], float h)
{
    constexpr int P = RB_P, e = I & 1;
    if (!rb_stage_begin<C>(L, R, xb, e, u, 0, P - 1, next)) return false;
    float am1[C], apa[C], apb[C];
    rb_edge_b<C>(L, e, L.tm1, am1);                        // a_{8 tau - 1}
    rb_edge_a<C>(L, e, L.tp1, apa, apb);                   // a_{8 tau + 8}, a_{8 tau + 9}
    float X[P + 4];
    rb_read_x<C == 1>(L, xb, X);
    float dq[4], lq[4];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (I > 0 && (p * C) % 4 == 0) {
            const float4 q = rb_base(L, p * C / 4);
            dq[0] = q.x; dq[1] = q.y; dq[2] = q.z; dq[3] = q.w;
        }
        const float xm2 = X[p], xp1 = X[p + 3], xd = X[p + 4] - X[p + 1];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float ap1 = (p + 1 < P) ? u[p + 1][c] : apa[c];
            const float ap2 = (p + 2 < P) ? u[p + 2][c] : ((p + 2 == P) ? apa[c] : apb[c]);
            const float cur = u[p][c];
            // (J^T a)_i = x_{i-2} a_{i-1} - x_{i+1} a_{i+2} + (x_{i+2} - x_{i-1}) a_{i+1} - a_i
            const float gg = fmaf(xm2, am1[c], fmaf(-xp1, ap2, fmaf(xd, ap1, -cur)));
            am1[c] = cur;
            if (I == 3) {
                const float lam = dq[(p * C + c) % 4];
                acc[p][c] = lam + gg;
                u[p][c] = fmaf(h * (1.f / 3.f), lam, h * gg);
            } else if (I == 2) {
                acc[p][c] += gg;
                u[p][c] = fmaf(h * (1.f / 3.f), dq[(p * C + c) % 4], 0.5f * h * gg);
            } else if (I == 1) {
                acc[p][c] += gg;
                u[p][c] = fmaf(h * (1.f / 6.f), dq[(p * C + c) % 4], 0.5f * h * gg);
            } else {
                const float lam = acc[p][c] + gg;
                lq[(p * C + c) % 4] = lam;
                u[p][c] = (h * (1.f / 6.f)) * lam;
            }
        }
        if (I == 0 && ((p + 1) * C) % 4 == 0) rb_base(L, ((p + 1) * C - 4) / 4) = make_float4(lq[0], lq[1], lq[2], lq[3]);
    }
    xb = (xb == RB_NB - 1) ? 0 : xb + 1;
    return true;
}

// Set up the ring: thread 0 initialises its mbarriers and starts the copies
// of the first RB_NB - 1 stage states (stage indices first, first + dir, ...).
__device__ __forceinline__ void rb_ring_start(const RbCta &L, const float *__restrict__ stages, int S, int first,
                                              int dir)
{
    if (L.tau == 0) {
        for (int b = 0; b < RB_NB; ++b) sw_mb_init(L.mb0 + 8 * b, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    for (int d = 0; d < RB_NB - 1; ++d) {
        const int si = first + dir * d;
        rb_fetch(L, d, (si >= 0 && si < S) ? stages + (int64_t)si * L.n : nullptr);
    }
}

// After the wait on ring buffer xb gave up somewhere in the CTA (before the
// stage's copy was started): thread 0 waits (bounded) for the copies that
// may still be in flight -- the one into xb and the one into the next buffer,
// started one stage earlier unless this was the sweep's last stage -- and
// records the failure.
__device__ __forceinline__ void rb_abort(const RbCta &L, const RbRing &R, int xb, bool last, int *err)
{
    if (L.tau != 0) return;
    const int nb = xb == RB_NB - 1 ? 0 : xb + 1;
    sw_mb_wait(L.mb0 + 8 * xb, ((R.ph >> xb) & 1u) ^ 1u);
    if (!last) sw_mb_wait(L.mb0 + 8 * nb, (R.ph >> nb) & 1u);
    if (err) atomicExch(err, 1);
}

// A thread's eight points of one column of W: two 16-byte accesses when W
// and its leading dimension allow (vec), else eight 4-byte ones.
__device__ __forceinline__ void rb_load8(const float *w, bool vec, float (&v)[RB_P])
{
    if (vec) {
        const float4 a = *reinterpret_cast<const float4 *>(w), b = *reinterpret_cast<const float4 *>(w + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int p = 0; p < RB_P; ++p) v[p] = w[p];
    }
}
__device__ __forceinline__ void rb_store8(float *w, bool vec, const float (&v)[RB_P])
{
    if (vec) {
        *reinterpret_cast<float4 *>(w) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4 *>(w + 4) = make_float4(v[4], v[5], v[6], v[7]);
    } else {
#pragma unroll
        for (int p = 0; p < RB_P; ++p) w[p] = v[p];
    }
}
// Bit p set when grid point j0 + p is observed (every obs_stride-th point).
__device__ __forceinline__ unsigned rb_obs_mask(int j0, int obs_stride)
{
    unsigned m = 0;
    int r = j0 % obs_stride;
#pragma unroll
    for (int p = 0; p < RB_P; ++p) {
        if (r == 0) m |= 1u << p;
        r = (r + 1 == obs_stride) ? 0 : r + 1;
    }
    return m;
}

// Forward sweep L^{-1} (w_{t+1} += M_t w_t) for columns blockIdx.x*C .. +C-1 (< K).
template <int C>
__global__ void __launch_bounds__(1024, 1)
k_l96_tlm_rb(int n, int N, int steps, float h, const float *__restrict__ stages, float *W, int64_t ld, int K,
             int vec, int *err, unsigned limit)
{
    constexpr int P = RB_P, D = RB_NB - 1;
    extern __shared__ __align__(16) float rsm[];
    const RbCta L = rb_setup<C>(rsm, n, limit);
    RbRing R;
    const int j0 = L.tau * P;
    const int S = 4 * N * steps;                           // stage states, used in order 0 .. S - 1
    rb_ring_start(L, stages, S, 0, 1);
    float u[P][C], acc[P][C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const int col = blockIdx.x * C + c;
        float v[P];
        rb_load8(W + (int64_t)min(col, K - 1) * ld + j0, vec, v);
#pragma unroll
        for (int p = 0; p < P; ++p) u[p][c] = (col < K) ? v[p] : 0.f;
    }
    rb_store_base<C>(L, u);
    int q = 0, xb = 0;                                     // stages begun; ring buffer of the next
    bool good = true;
    for (int t = 0; t < N && good; ++t) {
        for (int k = 0; k < steps; ++k) {
            const int s = q;                                // stage state 4 (t steps + k)
            const float *x = stages + (int64_t)s * n;
            if (!(good = rb_tlm_stage<C, 0>(L, R, xb, s + D < S ? x + D * n : nullptr, u, acc, h))) break;
            ++q;
            if (!(good = rb_tlm_stage<C, 1>(L, R, xb, s + 1 + D < S ? x + (1 + D) * n : nullptr, u, acc, h))) break;
            ++q;
            if (!(good = rb_tlm_stage<C, 2>(L, R, xb, s + 2 + D < S ? x + (2 + D) * n : nullptr, u, acc, h))) break;
            ++q;
            if (!(good = rb_tlm_stage<C, 3>(L, R, xb, s + 3 + D < S ? x + (3 + D) * n : nullptr, u, acc, h))) break;
            ++q;
        }
        if (!good) break;
        // subwindow boundary: w_{t+1} += d, d = w_{t+1}
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int col = blockIdx.x * C + c;
            if (col >= K) continue;
            float *wn = W + (int64_t)col * ld + (int64_t)(t + 1) * n + j0;
            float v[P];
            rb_load8(wn, vec, v);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                v[p] = u[p][c] + v[p];
                u[p][c] = v[p];
            }
            rb_store8(wn, vec, v);
        }
        rb_store_base<C>(L, u);
    }
    if (!good) rb_abort(L, R, xb, q == S - 1, err);   // q: the stage whose wait gave up
}

// Adjoint sweep L^{-T} for columns blockIdx.x*C .. +C-1 (< K); obs_mode as
// k_l96_adj.
template <int C>
__global__ void __launch_bounds__(1024, 1)
k_l96_adj_rb(int n, int N, int steps, float h, const float *__restrict__ stages, float *W, int64_t ld, int K,
             int obs_mode, float obs_scale, int obs_stride, int t0, int ts, int vec, int *err, unsigned limit)
{
    constexpr int P = RB_P, D = RB_NB - 1;
    extern __shared__ __align__(16) float rsm[];
    const RbCta L = rb_setup<C>(rsm, n, limit);
    RbRing R;
    const int j0 = L.tau * P;
    const int S = 4 * N * steps;                           // stage states, used in order S - 1 .. 0
    rb_ring_start(L, stages, S, S - 1, -1);
    auto obs_at = [&](int t) { return t >= t0 && (t - t0) % ts == 0; };
    float u[P][C], acc[P][C];
    {
        const bool ob = obs_at(N);
        const unsigned om = obs_mode == 1 ? rb_obs_mask(j0, obs_stride) : 0u;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int col = blockIdx.x * C + c;
            float *wN = W + (int64_t)min(col, K - 1) * ld + (int64_t)N * n + j0;
            float v[P];
            rb_load8(wN, vec, v);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                if (col >= K) v[p] = 0.f;
                if (obs_mode == 1) v[p] = (ob && ((om >> p) & 1u)) ? obs_scale * v[p] : 0.f;
                u[p][c] = v[p];
            }
            if (col < K) rb_store8(wN, vec, v);
        }
        rb_store_base<C>(L, u);
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
            for (int c = 0; c < C; ++c) u[p][c] = (h * (1.f / 6.f)) * u[p][c];
    }
    int q = 0, xb = 0;                                     // stages begun; ring buffer of the next
    bool good = true;
    for (int t = N - 1; t >= 0 && good; --t) {
        for (int k = steps - 1; k >= 0; --k) {
            const int s = S - 1 - q;                        // stage state 4 (t steps + k) + 3
            const float *x = stages + (int64_t)s * n;
            if (!(good = rb_adj_stage<C, 3>(L, R, xb, s - D >= 0 ? x - D * n : nullptr, u, acc, h))) break;
            ++q;
            if (!(good = rb_adj_stage<C, 2>(L, R, xb, s - 1 - D >= 0 ? x - (1 + D) * n : nullptr, u, acc, h))) break;
            ++q;
            if (!(good = rb_adj_stage<C, 1>(L, R, xb, s - 2 - D >= 0 ? x - (2 + D) * n : nullptr, u, acc, h))) break;
            ++q;
            if (!(good = rb_adj_stage<C, 0>(L, R, xb, s - 3 - D >= 0 ? x - (3 + D) * n : nullptr, u, acc, h))) break;
            ++q;
        }
        if (!good) break;
        // subwindow boundary: lam = obs(w_t) + lam, w_t = lam, a = h/6 lam
        const bool ob = obs_at(t);
        const unsigned om = obs_mode == 1 ? rb_obs_mask(j0, obs_stride) : 0u;
        float lam[P][C];
#pragma unroll
        for (int q = 0; q < P * C / 4; ++q) {
            const float4 v = rb_base(L, q);
            const int f = 4 * q;
            lam[f / C][f % C] = v.x; lam[(f + 1) / C][(f + 1) % C] = v.y;
            lam[(f + 2) / C][(f + 2) % C] = v.z; lam[(f + 3) / C][(f + 3) % C] = v.w;
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int col = blockIdx.x * C + c;
            if (col >= K) continue;
            float *wt = W + (int64_t)col * ld + (int64_t)t * n + j0;
            float v[P];
            rb_load8(wt, vec, v);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                if (obs_mode == 1) v[p] = (ob && ((om >> p) & 1u)) ? obs_scale * v[p] : 0.f;
                lam[p][c] += v[p];
                v[p] = lam[p][c];
            }
            rb_store8(wt, vec, v);
        }
        rb_store_base<C>(L, lam);
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
            for (int c = 0; c < C; ++c) u[p][c] = (h * (1.f / 6.f)) * lam[p][c];
    }
    if (!good) rb_abort(L, R, xb, q == S - 1, err);   // q: the stage whose wait gave up
}

// Register-blocked form: FP32 and n = 8 nt with nt a multiple of 32 and at
// most 1024.
template <typename T> static bool rb_applies(int n)
{
    return sizeof(T) == 4 && n % 256 == 0 && n / RB_P <= 1024;
}
// Columns per CTA: two for blocks, one for few columns.
static int rb_cols(int K) { return K >= 64 ? 2 : 1; }

static bool use_cluster(int n, int K) { return K <= 32 && n % L96_CL == 0 && n / L96_CL >= 2 && n / L96_CL <= 1024; }

template <int C>
static void launch_tlm_rb(cudaStream_t s, int n, int N, int steps, double dt, const float *stages, int K, float *W,
                          int64_t ld, int *err, unsigned limit)
{
    static const bool attr = [] {
        return cudaFuncSetAttribute(k_l96_tlm_rb<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)rb_smem<C>(WC4D_FFT_MAX_N)) == cudaSuccess;
    }();   // once, thread-safe
    (void)attr;
    const int vec = (reinterpret_cast<uintptr_t>(W) % 16 == 0 && ld % 4 == 0) ? 1 : 0;
    WC4D_LAUNCH(k_l96_tlm_rb<C><<<ceil_div(K, C), n / RB_P, rb_smem<C>(n), s>>>(n, N, steps, (float)dt, stages, W, ld,
                                                                                K, vec, err, limit));
}

template <int C>
static void launch_adj_rb(cudaStream_t s, int n, int N, int steps, double dt, const float *stages, int K, float *W,
                          int64_t ld, int obs_mode, double obs_scale, int obs_stride, int obs_t0, int obs_tstride,
                          int *err, unsigned limit)
{
    static const bool attr = [] {
        return cudaFuncSetAttribute(k_l96_adj_rb<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)rb_smem<C>(WC4D_FFT_MAX_N)) == cudaSuccess;
    }();   // once, thread-safe
    (void)attr;
    const int vec = (reinterpret_cast<uintptr_t>(W) % 16 == 0 && ld % 4 == 0) ? 1 : 0;
    WC4D_LAUNCH(k_l96_adj_rb<C><<<ceil_div(K, C), n / RB_P, rb_smem<C>(n), s>>>(
        n, N, steps, (float)dt, stages, W, ld, K, obs_mode, (float)obs_scale, obs_stride, obs_t0,
        obs_tstride > 0 ? obs_tstride : 1, vec, err, limit));
}

template <typename T>
void launch_l96_tlm_sweep(cudaStream_t s, int n, int N, int steps, double dt, const T *stages, int K, T *W,
                          int64_t ld, int *err, unsigned wait_limit)
{
    if constexpr (sizeof(T) == 4) {
        if (rb_applies<T>(n)) {
            if (rb_cols(K) == 2) launch_tlm_rb<2>(s, n, N, steps, dt, stages, K, W, ld, err, wait_limit);
            else launch_tlm_rb<1>(s, n, N, steps, dt, stages, K, W, ld, err, wait_limit);
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

template <typename T>
void launch_l96_adj_sweep(cudaStream_t s, int n, int N, int steps, double dt, const T *stages, int K, T *W,
                          int64_t ld, int obs_mode, double obs_scale, int obs_stride, int obs_t0, int obs_tstride,
                          int *err, unsigned wait_limit)
{
    if constexpr (sizeof(T) == 4) {
        if (rb_applies<T>(n)) {
            if (rb_cols(K) == 2)
                launch_adj_rb<2>(s, n, N, steps, dt, stages, K, W, ld, obs_mode, obs_scale, obs_stride, obs_t0,
                                 obs_tstride, err, wait_limit);
            else
                launch_adj_rb<1>(s, n, N, steps, dt, stages, K, W, ld, obs_mode, obs_scale, obs_stride, obs_t0,
                                 obs_tstride, err, wait_limit);
            return;
        }
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
                                           int64_t, int *, unsigned);
template void launch_l96_tlm_sweep<float>(cudaStream_t, int, int, int, double, const float *, int, float *, int64_t,
                                          int *, unsigned);
template void launch_l96_adj_sweep<double>(cudaStream_t, int, int, int, double, const double *, int, double *,
                                           int64_t, int, double, int, int, int, int *, unsigned);
template void launch_l96_adj_sweep<float>(cudaStream_t, int, int, int, double, const float *, int, float *, int64_t,
                                          int, double, int, int, int, int *, unsigned);

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
                const bool forced = eta && (g + 1) % steps == 0;
                const double *eg = forced ? eta + (int64_t)((g + 1) / steps) * n : nullptr;
#pragma unroll
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

