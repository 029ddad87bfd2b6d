// Allocation-free spectral-LMP application, y = C v with
// C = I - U diag(1 - theta^{-1/2}) U^T.
//
// Some callers cannot allocate device memory at the point where they need
// the preconditioner: data-assimilation systems that reserve their whole
// device memory budget up front (a pool that owns all of it) and forbid
// allocations afterwards, code that must not pay the device-wide
// synchronisation a cudaMalloc/cudaFree can cause in the middle of a solve,
// and callers that hold no library context at all.  This entry point takes
// only the caller's inputs and output and keeps its scratch (the weighted
// coefficients c_i (U^T v)_i and the partial dot products U^T v) in one
// file-scope device array of fixed size, which every GPU that loads the
// library holds until the process exits.  It creates no context and calls no
// allocating routine.
#include <algorithm>
#include <mutex>

#include "wc4d_internal.cuh"

namespace {

constexpr int kMaxK = 1024;                    // largest number of Ritz pairs
constexpr int kMaxSplits = 128;                // row chunks of U^T v
constexpr int kScratchDoubles = kMaxK + kMaxSplits * kMaxK;   // 1 MiB + 8 KiB

// The shared scratch: [0, kMaxK) the weighted coefficients c_i t_i, then
// kMaxSplits x k partial sums of t = U^T v.  Every call writes what it later
// reads, so nothing has to start at zero; calls that overlap on the GPU race
// on it.
static __device__ __align__(256) double g_lmp_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked
// up with cudaGetSymbolAddress once per device (the first call on a device)
// and cached; a cudaDeviceReset after that first call is not supported (the
// cached address would be stale).
wc4d_status scratch_on_current_device(double **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return WC4D_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_lmp_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return WC4D_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_addr[dev];
    return WC4D_OK;
}

__device__ double warp_sum_static(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// part[s*k + i] = sum over the rows of chunk s of U[r, i] v[r]; one warp per
// column at a time.
__global__ void __launch_bounds__(256) k_static_utv(int64_t nA, int k, int64_t rows_per, const double *__restrict__ U,
                                                    const double *__restrict__ v, double *part)
{
    const int64_t r0 = (int64_t)blockIdx.x * rows_per;
    const int64_t r1 = min(nA, r0 + rows_per);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = w; i < k; i += nw) {
        const double *u = U + (int64_t)i * nA;
        double acc = 0.0;
        for (int64_t r = r0 + lane; r < r1; r += 32) acc = fma(u[r], __ldg(v + r), acc);
        acc = warp_sum_static(acc);
        if (lane == 0) part[(int64_t)blockIdx.x * k + i] = acc;
    }
}

// ct[i] = c_i t_i with c_i = 1 - theta_i^{-1/2} (0 for theta_i <= 0, the
// identity factor) and t_i = sum_s part[s*k + i]: the split sums reduced once.
__global__ void k_static_weights(int k, int splits, const double *__restrict__ theta,
                                 const double *__restrict__ part, double *ct)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k) return;
    double t = 0.0;
    for (int s = 0; s < splits; ++s) t += part[(int64_t)s * k + i];
    const double th = theta[i];
    ct[i] = (th > 0.0 ? 1.0 - 1.0 / sqrt(th) : 0.0) * t;
}

// y = v - U ct
__global__ void __launch_bounds__(256) k_static_combine(int64_t nA, int k, const double *__restrict__ U,
                                                        const double *__restrict__ ct_g, const double *v, double *y)
{
    __shared__ double ct[kMaxK];
    for (int i = threadIdx.x; i < k; i += blockDim.x) ct[i] = ct_g[i];
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nA; r += (int64_t)gridDim.x * blockDim.x) {
        double acc = v[r];
        for (int i = 0; i < k; ++i) acc = fma(-U[(int64_t)i * nA + r], ct[i], acc);
        y[r] = acc;
    }
}

}  // namespace

extern "C" wc4d_status wc4d_lmp_apply_static(const double *U, const double *theta, int32_t k, int64_t nA,
                                             const double *v, double *y, void *cuda_stream)
{
    if (!U || !theta || !v || !y || nA < 1 || k < 1) return WC4D_EINVAL;
    if (k > kMaxK) return WC4D_EINVAL;                 // more Ritz pairs than the scratch holds
    if (v == y) return WC4D_EINVAL;                    // in place is not supported
    double *scratch = nullptr;
    wc4d_status st = scratch_on_current_device(&scratch);
    if (st != WC4D_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int splits = (int)std::min<int64_t>(kMaxSplits, (nA + 1023) / 1024);
    if (splits < 1) splits = 1;
    const int64_t rows_per = (nA + splits - 1) / splits;
    double *ct = scratch, *part = scratch + kMaxK;
    WC4D_LAUNCH(k_static_utv<<<splits, 256, 0, s>>>(nA, k, rows_per, U, v, part));
    WC4D_LAUNCH(k_static_weights<<<(k + 127) / 128, 128, 0, s>>>(k, splits, theta, part, ct));
    int grid = (int)std::min<int64_t>(4096, (nA + 255) / 256);
    WC4D_LAUNCH(k_static_combine<<<grid, 256, 0, s>>>(nA, k, U, ct, v, y));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? WC4D_OK : WC4D_ECUDA;
}
