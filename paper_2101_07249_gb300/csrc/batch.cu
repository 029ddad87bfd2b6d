// Batched inner loops of independent problems (many windows of different
// sizes solved together).  Each instance keeps its own context and CUDA
// stream; a pool of host threads drives the instances' inner loops (sketch,
// LMP, PCG: control flow that waits on the device between steps), so the
// kernels of different instances overlap on the GPU and the small,
// latency-bound windows fill the SMs together.  Grid-synchronised kernels
// are replaced by their per-launch forms while a context runs in a batch:
// a cooperative launch needs every CTA resident at once.  The CG iterations
// run as one graph launch each (the host reading the flags in between), not
// as the device-side loop graph: with 64 uneven windows on 16 threads the
// per-iteration launches interleave better across the streams (GB300: 8.3 s
// against 10.3 s for the loop graph and 9.1 s eager).
#include <atomic>
#include <thread>
#include <vector>

#include "wc4d_internal.cuh"

extern "C" wc4d_status wc4d_inner_loop(wc4d_ctx *c, int32_t method, int32_t k, int32_t l, int32_t q, uint64_t seed,
                                       double tol, int32_t maxit, int32_t precision, double *x, int32_t *iters,
                                       double *relres);

extern "C" wc4d_status wc4d_batch_inner_loop(wc4d_ctx *const *ctxs, int32_t count, int32_t method, const int32_t *k,
                                             const int32_t *l, int32_t q_power, const uint64_t *seeds, double tol,
                                             int32_t maxit, int32_t precision, double *const *x, int32_t *iters,
                                             double *relres, int32_t *status, int32_t workers)
{
    if (!ctxs || count < 0 || !k || !l || !seeds || !x || !iters || !relres || !status) return WC4D_EINVAL;
    for (int i = 0; i < count; ++i) {
        if (!ctxs[i] || !x[i]) return WC4D_EINVAL;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i] || ctxs[j]->stream == ctxs[i]->stream) {   // one context, one stream each
                const char *what = ctxs[j] == ctxs[i] ? "context" : "stream";
                const char *fmt = "batch: instance %d shares its %s with instance %d (each instance needs its own "
                                  "context and stream; wc4d_stream_create makes one)";
                set_err(ctxs[j], WC4D_EINVAL, fmt, i, what, j);   // the message on both contexts
                return set_err(ctxs[i], WC4D_EINVAL, fmt, i, what, j);
            }
    }
    if (count == 0) return WC4D_OK;
    const int nw = std::max(1, std::min<int>(workers > 0 ? workers : 16, count));
    std::atomic<int> next{0};
    auto worker = [&]() {
        for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1)) {
            wc4d_ctx *c = ctxs[i];
            cudaSetDevice(c->device);
            const bool coop = c->allow_coop, loop = c->use_loop_graph;
            c->allow_coop = false;
            c->use_loop_graph = false;
            status[i] = wc4d_inner_loop(c, method, k[i], l[i], q_power, seeds[i], tol, maxit, precision, x[i],
                                        iters + i, relres + i);
            c->allow_coop = coop;
            c->use_loop_graph = loop;
        }
    };
    std::vector<std::thread> pool;
    for (int t = 0; t < nw; ++t) pool.emplace_back(worker);
    for (auto &t : pool) t.join();
    for (int i = 0; i < count; ++i)
        if (status[i] != WC4D_OK) return (wc4d_status)status[i];
    return WC4D_OK;
}

extern "C" wc4d_status wc4d_stream_create(void **stream)
{
    if (!stream) return WC4D_EINVAL;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return WC4D_ECUDA;
    }
    *stream = st;
    return WC4D_OK;
}

extern "C" wc4d_status wc4d_stream_destroy(void *stream)
{
    if (!stream) return WC4D_EINVAL;
    return cudaStreamDestroy((cudaStream_t)stream) == cudaSuccess ? WC4D_OK : WC4D_ECUDA;
}
