// Learned sketch proposal (no counterpart in the paper; its output always
// passes through the randomised range finder of Alg. 3).  A fixed 4-layer 1D
// convolutional encoder over the periodic Lorenz-96 grid maps the
// linearisation trajectory and the observation mask to m start columns of
// the control space:
//   input  channels: x_t / F (t = 0..N, states at the subwindow boundaries),
//                    then the observation mask of every time t (0 / 1);
//   layer 0: 2(N+1) -> 64, width 5, ReLU;  layers 1, 2: 64 -> 64, width 5,
//   ReLU;  layer 3: 64 -> m (N+1), width 1;
//   output channel c = j (N+1) + t  ->  column j, time block t.
// Weights are BF16, products and sums FP32.  Parameters: one packed BF16
// array W0 | W1 | W2 | W3 (each [out][in][width]) and one FP32 array
// b0 | b1 | b2 | b3.
#include <cuda_bf16.h>

#include "wc4d_internal.cuh"

namespace {

template <typename T> T *P(DevBuf &b) { return reinterpret_cast<T *>(b.p); }
template <typename T> const T *P(const DevBuf &b) { return reinterpret_cast<const T *>(b.p); }

constexpr int LS_HID = 64;
constexpr int LS_W = 5;

__global__ void k_ls_features(int n, int N, int steps, double F, const double *__restrict__ traj, int obs_stride,
                              int t0, int ts, float *feat)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int C = 2 * (N + 1);
    if (idx >= (int64_t)C * n) return;
    const int c = (int)(idx / n), s = (int)(idx % n);
    float v;
    if (c <= N) {
        v = (float)(traj[(int64_t)c * steps * n + s] / F);
    } else {
        const int t = c - (N + 1);
        v = (t >= t0 && (t - t0) % ts == 0 && s % obs_stride == 0) ? 1.f : 0.f;
    }
    feat[idx] = v;
}

// y[co][s] = b[co] + sum_{ci, k} W[co][ci][k] x[ci][(s + k - width/2) mod n]
__global__ void __launch_bounds__(256) k_ls_conv(int n, int cin, int cout, int width, const float *__restrict__ x,
                                                 const __nv_bfloat16 *__restrict__ W, const float *__restrict__ b,
                                                 float *y, int relu)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int co = blockIdx.y;
    if (s >= n) return;
    const __nv_bfloat16 *w = W + (int64_t)co * cin * width;
    const int h = width / 2;
    float acc = b[co];
    for (int ci = 0; ci < cin; ++ci) {
        const float *xc = x + (int64_t)ci * n;
        for (int k = 0; k < width; ++k) {
            int j = s + k - h;
            j = j < 0 ? j + n : (j >= n ? j - n : j);
            acc = fmaf(__bfloat162float(w[ci * width + k]), xc[j], acc);
        }
    }
    if (relu) acc = fmaxf(acc, 0.f);
    y[(int64_t)co * n + s] = acc;
}

// S[j ld + t n + s] = y[(j (N+1) + t) n + s]
__global__ void k_ls_scatter(int n, int N, int m, const float *__restrict__ y, double *S, int64_t ld)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nA = (int64_t)n * (N + 1);
    if (idx >= nA * m) return;
    const int j = (int)(idx / nA);
    const int64_t r = idx % nA;
    S[(int64_t)j * ld + r] = (double)y[idx];
}

}  // namespace

extern "C" wc4d_status wc4d_learned_probes(wc4d_ctx *c, const uint16_t *w_bf16, const float *bias, int32_t m,
                                           double *S, int64_t ld)
{
    if (!c || !w_bf16 || !bias || !S || m < 1 || ld < c->nA) return WC4D_EINVAL;
    if (c->prob.model != WC4D_MODEL_L96) return set_err(c, WC4D_EINVAL, "learned probes: Lorenz-96 windows only");
    if (!c->have_traj) return set_err(c, WC4D_ESTATE, "learned probes: no trajectory (call wc4d_set_background_obs)");
    const int n = c->prob.n, N = c->prob.N;
    const int C0 = 2 * (N + 1), Cm = m * (N + 1);
    const size_t f0 = (size_t)C0 * n, fh = (size_t)LS_HID * n, fo = (size_t)Cm * n;
    WC4D_TRY(ensure(c, c->learn_buf, sizeof(float) * (f0 + 2 * fh + fo)));
    float *feat = P<float>(c->learn_buf), *ha = feat + f0, *hb = ha + fh, *out = hb + fh;
    const __nv_bfloat16 *W = reinterpret_cast<const __nv_bfloat16 *>(w_bf16);
    const size_t w0 = (size_t)LS_HID * C0 * LS_W, w1 = (size_t)LS_HID * LS_HID * LS_W;
    const int ts = c->prob.obs_tstride > 0 ? c->prob.obs_tstride : 1;
    WC4D_LAUNCH(k_ls_features<<<ceil_div((int64_t)f0, 256), 256, 0, c->stream>>>(
        n, N, c->prob.steps, c->prob.F, P<double>(c->traj64), c->prob.obs_stride, c->prob.obs_t0, ts, feat));
    const dim3 blk(256);
    WC4D_LAUNCH(k_ls_conv<<<dim3(ceil_div(n, 256), LS_HID), blk, 0, c->stream>>>(n, C0, LS_HID, LS_W, feat, W, bias,
                                                                                  ha, 1));
    WC4D_LAUNCH(k_ls_conv<<<dim3(ceil_div(n, 256), LS_HID), blk, 0, c->stream>>>(n, LS_HID, LS_HID, LS_W, ha, W + w0,
                                                                                  bias + LS_HID, hb, 1));
    WC4D_LAUNCH(k_ls_conv<<<dim3(ceil_div(n, 256), LS_HID), blk, 0, c->stream>>>(n, LS_HID, LS_HID, LS_W, hb,
                                                                                  W + w0 + w1, bias + 2 * LS_HID, ha,
                                                                                  1));
    WC4D_LAUNCH(k_ls_conv<<<dim3(ceil_div(n, 256), Cm), blk, 0, c->stream>>>(n, LS_HID, Cm, 1, ha, W + w0 + 2 * w1,
                                                                             bias + 3 * LS_HID, out, 0));
    const int64_t tot = (int64_t)c->nA * m;
    WC4D_LAUNCH(k_ls_scatter<<<ceil_div(tot, 256), 256, 0, c->stream>>>(n, N, m, out, S, ld));
    return check_launch(c, "learned probes");
}
