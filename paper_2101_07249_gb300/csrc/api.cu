// C-ABI entry points of libwc4d: set-up, the Hessian product, the
// randomised eigensolvers, the spectral LMP and PCG.  Every numerical step
// runs in the kernels of setup.cu / sweep.cu / linalg.cu / tc_gemm.cu /
// l96.cu; this file only sequences them on the context's stream.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>

#include "wc4d_internal.cuh"

// ============================================================================
// helpers
// ============================================================================
wc4d_status set_err(wc4d_ctx *c, wc4d_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

void free_buf(DevBuf &b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

wc4d_status ensure(wc4d_ctx *c, DevBuf &b, size_t bytes)
{
    if (b.p && b.bytes >= bytes) return WC4D_OK;
    if (b.p) {
        cudaStreamSynchronize(c->stream);
        free_buf(b);
    }
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return set_err(c, WC4D_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    b.bytes = bytes;
    return WC4D_OK;
}

static wc4d_status ensure_host(wc4d_ctx *c, DevBuf &b, size_t bytes)
{
    if (b.p && b.bytes >= bytes) return WC4D_OK;
    if (b.p) {
        cudaStreamSynchronize(c->stream);
        cudaFreeHost(b.p);
        b.p = nullptr;
    }
    cudaError_t e = cudaMallocHost(&b.p, bytes < 64 ? 64 : bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return set_err(c, WC4D_ENOMEM, "cudaMallocHost failed: %s", cudaGetErrorString(e));
    }
    b.bytes = bytes;
    return WC4D_OK;
}

wc4d_status check_launch(wc4d_ctx *c, const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(c, WC4D_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return WC4D_OK;
}

static std::atomic<int64_t> g_launches{0};
static thread_local int64_t tl_launches = 0;   // launches issued by this host thread (graph capture counts)
void wc4d_note_launch()
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    ++tl_launches;
}

// ----------------------------------------------------------------------------
// One CG iteration body (the Hessian product, the LMP step and the p update,
// or the unpreconditioned vector kernels) as a CUDA graph.  The first
// iteration of a solve runs eagerly (every workspace then exists and every
// one-time function attribute is set); the second is captured on the
// context's stream (thread-local capture mode, so other host threads driving
// other contexts are unaffected), instantiated and launched; the rest of the
// solve replays it, one graph launch instead of ~10 (or, when the sweeps run
// per subwindow, 2 N + 10) kernel launches per iteration.  The body's
// arguments are fixed for the whole solve (the QCF slot comes from the
// device iteration counter).  Anything the capture cannot take -- a
// cooperative launch on a driver that refuses it, an allocation -- makes the
// capture fail; the iteration then runs eagerly and the solve stays eager.
// Not used while kernel-class profiling is on (its events are host-driven).
// ----------------------------------------------------------------------------
struct IterGraph {
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;    // kernels per replay
    int64_t hvps = 0;        // products with A per replay
    bool failed = false;
    IterGraph() = default;
    IterGraph(const IterGraph &) = delete;
    IterGraph &operator=(const IterGraph &) = delete;
    ~IterGraph()
    {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

// The stream the iteration bodies are captured on.  The legacy and
// per-thread default streams cannot be captured, and the caller's stream is
// often one of them, so capture runs on a private non-blocking stream of the
// context (nullptr if it cannot be created); capture executes nothing, and
// the instantiated graph is launched on c->stream.
static cudaStream_t capture_stream(wc4d_ctx *c)
{
    if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        c->cap_stream = nullptr;
    }
    return c->cap_stream;
}

// c->stream points at the capture stream while a body is captured (every
// launch of the body reads c->stream), and back at the caller's stream after.
struct CaptureStreamScope {
    wc4d_ctx *c;
    cudaStream_t user;
    CaptureStreamScope(wc4d_ctx *ctx, cudaStream_t cs) : c(ctx), user(ctx->stream) { c->stream = cs; }
    ~CaptureStreamScope() { c->stream = user; }
};

template <typename F> static wc4d_status run_iteration(wc4d_ctx *c, IterGraph &g, int it, F body)
{
    if (g.exec) {
        if (cudaGraphLaunch(g.exec, c->stream) != cudaSuccess) return check_launch(c, "CG iteration graph");
        g_launches.fetch_add(g.launches, std::memory_order_relaxed);
        tl_launches += g.launches;
        c->hvp_count += g.hvps;
        return WC4D_OK;
    }
    if (it == 0 || g.failed || c->prof_on || !c->use_graphs) return body();
    cudaStream_t cs = capture_stream(c);
    const int64_t l0 = tl_launches, h0 = c->hvp_count;
    if (!cs || cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        g.failed = true;
        return body();
    }
    wc4d_status st;
    cudaGraph_t graph = nullptr;
    cudaError_t ec;
    {
        CaptureStreamScope scope(c, cs);
        st = body();
        ec = cudaStreamEndCapture(cs, &graph);
    }
    const int64_t nl = tl_launches - l0, nh = c->hvp_count - h0;
    // the captured kernels have not run: take them off the counters
    g_launches.fetch_sub(nl, std::memory_order_relaxed);
    tl_launches -= nl;
    c->hvp_count = h0;
    if (st != WC4D_OK || ec != cudaSuccess || !graph ||
        cudaGraphInstantiate(&g.exec, graph, 0) != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        g.exec = nullptr;
        cudaGetLastError();
        g.failed = true;
        c->err.clear();
        return body();   // run this iteration eagerly, and the rest of the solve too
    }
    cudaGraphDestroy(graph);
    g.launches = nl;
    g.hvps = nh;
    return run_iteration(c, g, it, body);   // first replay
}

ProfScope::ProfScope(wc4d_ctx *ctx, int pid) : c(ctx), id(pid), slot(-1)
{
    if (!c || !c->prof_on) return;
    if (c->ev_used + 2 > c->ev_pool.size()) {
        for (int i = 0; i < 256; ++i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return; }
            c->ev_pool.push_back(e);
        }
    }
    slot = (int)c->prof_log.size();
    ProfEntry pe{id, c->ev_pool[c->ev_used], c->ev_pool[c->ev_used + 1]};
    c->ev_used += 2;
    c->prof_log.push_back(pe);
    cudaEventRecord(pe.e0, c->stream);
}

ProfScope::~ProfScope()
{
    if (slot >= 0) cudaEventRecord(c->prof_log[slot].e1, c->stream);
}

static wc4d_status sync(wc4d_ctx *c, const char *what)
{
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return set_err(c, WC4D_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return WC4D_OK;
}

template <typename T> static T *P(DevBuf &b) { return reinterpret_cast<T *>(b.p); }

// ----------------------------------------------------------------------------
// The CG loop on the device: a CUDA graph whose single node is a conditional
// WHILE node; its body is one iteration (the same launches as IterGraph's)
// followed by k_cg_continue, which sets the node's condition from the device
// flags.  One graph launch then runs iterations until CG converges or breaks
// down, the iteration limit is reached, or -- for the mixed path's reliable
// updates -- the recurrence residual falls below the update threshold
// (scal[8]); only then does the host look at the flags, so no host round trip
// separates the iterations.  The decisions are those the host loop takes
// after every iteration, so the iterates are bitwise those of the eager
// launches.  A guard counter (counter word 14, set by the host before each
// launch) bounds the loop whatever the flags say.  Built after the first
// eager iteration of a solve; if the driver refuses any part of it, the
// solve continues with IterGraph (one graph launch per iteration).
// ----------------------------------------------------------------------------
__global__ void k_cg_continue(cudaGraphConditionalHandle h, const int *flags, const double *scal, int it_end,
                              int use_thresh, int *guard)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int g = guard[0] - 1;
    guard[0] = g;
    bool go = flags[0] == 0 && flags[1] == 0 && flags[2] < it_end && g > 0;
    if (use_thresh && !(scal[4] >= scal[8])) go = false;   // a reliable update is due (or the residual is NaN)
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

struct LoopGraph {
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;    // kernels per iteration (the decision kernel included)
    int64_t hvps = 0;        // products with A per iteration
    bool failed = false;
    LoopGraph() = default;
    LoopGraph(const LoopGraph &) = delete;
    LoopGraph &operator=(const LoopGraph &) = delete;
    ~LoopGraph()
    {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

// Builds the loop graph around `body` (false: not available; the caller
// keeps iterating one iteration at a time).
template <typename F>
static bool build_loop(wc4d_ctx *c, LoopGraph &L, F body, int it_end, bool use_thresh)
{
    if (L.exec) return true;
    if (L.failed || c->prof_on || !c->use_graphs || !c->use_loop_graph) return false;
    // the first call that fails names the reason in c->loop_note
    const char *step = nullptr;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t r, const char *what) {
        if (!step && r != cudaSuccess) {
            step = what;
            e = r;
        }
        return !step;
    };
    cudaGraph_t outer = nullptr;
    chk(cudaGraphCreate(&outer, 0), "cudaGraphCreate");
    cudaGraphConditionalHandle h{};
    if (!step) chk(cudaGraphConditionalHandleCreate(&h, outer, 1, cudaGraphCondAssignDefault),
                   "cudaGraphConditionalHandleCreate");
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (!step) chk(cudaGraphAddNode(&node, outer, nullptr, nullptr, 0, &np), "cudaGraphAddNode (conditional)");
    const int64_t l0 = tl_launches, h0 = c->hvp_count;
    cudaStream_t cs = step ? nullptr : capture_stream(c);
    if (!step && !cs) {
        step = "cudaStreamCreateWithFlags (capture stream)";
        e = cudaErrorUnknown;
    }
    if (!step) {
        cudaGraph_t bodyg = np.conditional.phGraph_out[0];
        if (chk(cudaStreamBeginCaptureToGraph(cs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                "cudaStreamBeginCaptureToGraph")) {
            CaptureStreamScope scope(c, cs);
            const wc4d_status st = body();
            WC4D_LAUNCH(k_cg_continue<<<1, 32, 0, cs>>>(h, P<int>(c->counter) + 4, P<double>(c->scal), it_end,
                                                      use_thresh ? 1 : 0, P<int>(c->counter) + 14));
            const cudaError_t el = cudaGetLastError();
            cudaGraph_t got = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(cs, &got);
            if (st != WC4D_OK && !step) {
                step = "capture of the iteration body";
                e = el != cudaSuccess ? el : cudaErrorUnknown;
            }
            chk(el, "capture of the decision kernel");
            chk(ec, "cudaStreamEndCapture");
        }
    }
    const int64_t nl = tl_launches - l0, nh = c->hvp_count - h0;
    g_launches.fetch_sub(nl, std::memory_order_relaxed);   // captured, not run
    tl_launches -= nl;
    c->hvp_count = h0;
    if (!step) chk(cudaGraphInstantiate(&L.exec, outer, 0), "cudaGraphInstantiate");
    if (outer) cudaGraphDestroy(outer);
    if (step) {
        if (L.exec) cudaGraphExecDestroy(L.exec);
        L.exec = nullptr;
        cudaGetLastError();
        c->err.clear();
        c->loop_note = std::string(step) + ": " + cudaGetErrorString(e);
        L.failed = true;
        return false;
    }
    L.launches = nl;
    L.hvps = nh;
    return true;
}

// Runs the loop graph for at most `max_iters` iterations; *done_iters receives
// the device iteration counter afterwards (flags and residual are read into
// the pinned slots hflags[0..2], hrel).
static wc4d_status run_loop(wc4d_ctx *c, LoopGraph &L, int max_iters, int it_before, int *hflags, double *hrel,
                            int *iters_after)
{
    int *hguard = reinterpret_cast<int *>(P<char>(c->pinned) + 128);
    *hguard = max_iters;   // at most max_iters iterations whatever the flags say
    WC4D_CUDA(c, cudaMemcpyAsync(P<int>(c->counter) + 14, hguard, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    if (cudaGraphLaunch(L.exec, c->stream) != cudaSuccess) return check_launch(c, "CG loop graph");
    WC4D_CUDA(c, cudaMemcpyAsync(hflags, P<int>(c->counter) + 4, sizeof(int) * 3, cudaMemcpyDeviceToHost, c->stream));
    WC4D_CUDA(c, cudaMemcpyAsync(hrel, P<double>(c->scal) + 4, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    WC4D_TRY(sync(c, "CG loop"));
    const int ran = hflags[2] - it_before;
    g_launches.fetch_add(L.launches * ran, std::memory_order_relaxed);
    tl_launches += L.launches * ran;
    c->hvp_count += L.hvps * ran;
    *iters_after = hflags[2];
    return WC4D_OK;
}


static bool observed_time(const wc4d_problem &p, int t)
{
    int ts = p.obs_tstride > 0 ? p.obs_tstride : 1;
    return t >= p.obs_t0 && t <= p.N && (t - p.obs_t0) % ts == 0;
}

static double obs_scale(const wc4d_ctx *c, int t)
{
    return observed_time(c->prob, t) ? 1.0 / c->prob.sigma_o2 : 0.0;
}

static int64_t mblk(const wc4d_ctx *c, int t) { return (c->nM == 1 ? 0 : (int64_t)t) * c->prob.n * c->prob.n; }

// ============================================================================
// small kernels used only by the orchestration
// ============================================================================
// d[k] = y[k] - x[t*n + s], observation k = i*per + o at t = t0 + i*ts, s = o*stride
__global__ void k_innovation(int64_t nobs, int per, int t0, int ts, int stride, int n, const double *y,
                             const double *x, double *d)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nobs) return;
    int64_t i = k / per;
    int o = (int)(k % per);
    int64_t t = t0 + i * ts;
    d[k] = y[k] - x[t * n + (int64_t)o * stride];
}

// v[t*n + s] = d[k] * scale (v zeroed beforehand)
__global__ void k_scatter_obs(int64_t nobs, int per, int t0, int ts, int stride, int n, const double *d,
                              double scale, double *v)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nobs) return;
    int64_t i = k / per;
    int o = (int)(k % per);
    int64_t t = t0 + i * ts;
    v[t * n + (int64_t)o * stride] = d[k] * scale;
}

// x[i] = (double) a[i] for float vectors
__global__ void k_f64_from_f32_scaled(int64_t n, const float *a, double *b)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}

// theta_out[i] = w[i] (eigenvalues) or w[i]^2 handled on the host side
// (k values only).

// ============================================================================
// creation / destruction
// ============================================================================
extern "C" wc4d_status wc4d_create(wc4d_ctx **out, const wc4d_problem *prob, void *stream)
{
    if (!out || !prob) return WC4D_EINVAL;
    *out = nullptr;
    const wc4d_problem &p = *prob;
    if (p.n < 2 || p.n > WC4D_FFT_MAX_N || p.N < 1 || !(p.sigma_o2 > 0.0) || p.obs_stride < 1 || p.obs_t0 < 0 ||
        p.obs_tstride < 0 || (p.model != WC4D_MODEL_DENSE && p.model != WC4D_MODEL_L96))
        return WC4D_EINVAL;
    if (p.model == WC4D_MODEL_L96 && (p.steps < 1 || !(p.dt > 0.0) || p.n < 4)) return WC4D_EINVAL;
    wc4d_ctx *c = new wc4d_ctx();
    c->prob = p;
    if (c->prob.obs_tstride == 0) c->prob.obs_tstride = 1;
    c->stream = (cudaStream_t)stream;
    cudaGetDevice(&c->device);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (c->num_sms <= 0) c->num_sms = 1;
    c->nA = (int64_t)p.n * (p.N + 1);
    c->obs_per_time = (p.n + p.obs_stride - 1) / p.obs_stride;
    for (int t = 0; t <= p.N; ++t)
        if (observed_time(c->prob, t)) c->obs_times.push_back(t);
    c->nobs = (int64_t)c->obs_times.size() * c->obs_per_time;
    c->fft = (p.n >= 4) && ((p.n & (p.n - 1)) == 0) && p.n <= WC4D_FFT_MAX_N;
    c->logn = 0;
    while ((1 << c->logn) < p.n) ++c->logn;
    c->nM = (p.model == WC4D_MODEL_DENSE) ? (p.M_shared ? 1 : p.N) : 0;
    wc4d_status s = WC4D_OK;
    if ((s = ensure(c, c->cosn, sizeof(double2) * p.n)) != WC4D_OK ||
        (s = ensure(c, c->tw64, sizeof(double2) * (p.n / 2 + 1))) != WC4D_OK ||
        (s = ensure(c, c->tw32, sizeof(float2) * (p.n / 2 + 1))) != WC4D_OK ||
        (s = ensure(c, c->twp64, sizeof(double2) * p.n)) != WC4D_OK ||
        (s = ensure(c, c->twp32, sizeof(float2) * p.n)) != WC4D_OK ||
        (s = ensure(c, c->scal, sizeof(double) * 32)) != WC4D_OK ||
        (s = ensure(c, c->counter, sizeof(int) * 16)) != WC4D_OK ||
        (s = ensure_host(c, c->pinned, 4096)) != WC4D_OK) {
        wc4d_destroy(c);
        return s;
    }
    // counters that kernels expect at zero (the LMP coefficient kernel's
    // arrival counter is counter[8])
    if (cudaMemsetAsync(c->counter.p, 0, sizeof(int) * 16, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        wc4d_destroy(c);
        return WC4D_ECUDA;
    }
    launch_twiddles(c->stream, p.n, P<double2>(c->cosn), P<double2>(c->tw64), P<float2>(c->tw32));
    if (c->fft) launch_pass_twiddles(c->stream, p.n, P<double2>(c->twp64), P<float2>(c->twp32));
    if ((s = check_launch(c, "twiddles")) != WC4D_OK || (s = sync(c, "create")) != WC4D_OK) {
        wc4d_destroy(c);
        return s;
    }
    *out = c;
    return WC4D_OK;
}

extern "C" void wc4d_destroy(wc4d_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    DevBuf *bufs[] = {&c->M64, &c->MT64, &c->M32, &c->MT32, &c->traj64, &c->stage64, &c->stage32, &c->spec64[0], &c->spec64[1],
                      &c->spec32[0], &c->spec32[1], &c->row64[0], &c->row64[1], &c->row32[0], &c->row32[1],
                      &c->tw64, &c->tw32, &c->twp64, &c->twp32, &c->cosn, &c->d, &c->rhs, &c->Dm12b, &c->work64, &c->work32,
                      &c->blkA, &c->blkB, &c->blkC, &c->blkD, &c->small0, &c->small1, &c->small2, &c->small3,
                      &c->part, &c->scal, &c->counter, &c->U64, &c->U32, &c->theta64, &c->c64, &c->c32,
                      &c->tc_part, &c->tc_err, &c->oz_slices, &c->oz_work, &c->chol_bar, &c->tall_ys, &c->tall_ws, &c->Mlo, &c->MTlo, &c->df_vec, &c->Urm64, &c->Urm32, &c->sweep_bar, &c->Mtf, &c->MTtf, &c->tc_round,
                      &c->lin, &c->ydev, &c->sk_k, &c->sk_w, &c->sk_r, &c->evd_r, &c->qcf, &c->learn_buf,
                      &c->lz_F, &c->lz_ab, &c->lz_h, &c->jq32};
    for (DevBuf *b : bufs) free_buf(*b);
    for (int i = 0; i < 8; ++i) { free_buf(c->pcg64[i]); free_buf(c->pcg32[i]); }
    if (c->pinned.p) cudaFreeHost(c->pinned.p);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

extern "C" const char *wc4d_last_error(const wc4d_ctx *c) { return c ? c->err.c_str() : "null context"; }

extern "C" wc4d_status wc4d_set_stream(wc4d_ctx *c, void *stream)
{
    if (!c) return WC4D_EINVAL;
    c->stream = (cudaStream_t)stream;
    return WC4D_OK;
}

extern "C" int64_t wc4d_nobs(const wc4d_ctx *c) { return c ? c->nobs : -1; }
extern "C" int64_t wc4d_control_dim(const wc4d_ctx *c) { return c ? c->nA : -1; }
extern "C" wc4d_status wc4d_get_problem(const wc4d_ctx *c, wc4d_problem *out)
{
    if (!c || !out) return WC4D_EINVAL;
    *out = c->prob;
    return WC4D_OK;
}
extern "C" int32_t wc4d_ritz_count(const wc4d_ctx *c) { return c ? c->kU : -1; }

extern "C" int64_t wc4d_launch_count(int32_t reset)
{
    return reset ? g_launches.exchange(0) : g_launches.load();
}

extern "C" wc4d_status wc4d_profile(wc4d_ctx *c, int32_t enable)
{
    if (!c) return WC4D_EINVAL;
    WC4D_TRY(sync(c, "profile"));
    c->prof_log.clear();
    c->ev_used = 0;
    c->prof_on = enable != 0;
    return WC4D_OK;
}

extern "C" wc4d_status wc4d_profile_read(wc4d_ctx *c, int32_t cls, double *total_ms, int64_t *launch_groups)
{
    if (!c || cls < 0 || cls >= PROF_N) return WC4D_EINVAL;
    WC4D_TRY(sync(c, "profile_read"));
    double ms = 0.0;
    int64_t cnt = 0;
    for (const ProfEntry &e : c->prof_log) {
        if (e.id != cls) continue;
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, e.e0, e.e1) == cudaSuccess) { ms += t; ++cnt; }
        else cudaGetLastError();
    }
    if (total_ms) *total_ms = ms;
    if (launch_groups) *launch_groups = cnt;
    return WC4D_OK;
}

extern "C" int32_t wc4d_jacobi_sweeps(const wc4d_ctx *c) { return c ? c->jacobi_sweeps : -1; }
extern "C" int32_t wc4d_jacobi_sweeps_fp32(const wc4d_ctx *c) { return c ? c->jacobi_sweeps32 : -1; }
extern "C" int32_t wc4d_jacobi_fp32_kernel(const wc4d_ctx *c) { return c ? c->jacobi_kernel32 : -1; }

extern "C" wc4d_status wc4d_set_reliable_delta(wc4d_ctx *c, double delta)
{
    if (!c || !(delta > 0.0 && delta <= 1.0)) return WC4D_EINVAL;
    c->reliable_delta = delta;
    return WC4D_OK;
}

extern "C" wc4d_status wc4d_set_wait_limit(wc4d_ctx *c, int64_t polls)
{
    if (!c || polls > (int64_t)UINT32_MAX) return WC4D_EINVAL;
    c->wait_limit = polls < 0 ? (1u << 22) : (unsigned)polls;
    return WC4D_OK;
}

extern "C" wc4d_status wc4d_set_gram_path(wc4d_ctx *c, int32_t tensor_cores)
{
    if (!c) return WC4D_EINVAL;
    c->gram_tc = tensor_cores != 0;
    return WC4D_OK;
}

extern "C" int32_t wc4d_iteration_mode(const wc4d_ctx *c, char *note, int32_t note_len)
{
    if (!c) return -1;
    if (note && note_len > 0) {
        const size_t m = std::min<size_t>(c->loop_note.size(), (size_t)note_len - 1);
        std::memcpy(note, c->loop_note.data(), m);
        note[m] = '\0';
    }
    return c->iter_mode;
}

extern "C" wc4d_status wc4d_set_graphs(wc4d_ctx *c, int32_t enable)
{
    if (!c) return WC4D_EINVAL;
    if (enable < 0 || enable > 2) return WC4D_EINVAL;
    c->use_graphs = enable != 0;
    c->use_loop_graph = enable == 1;
    return WC4D_OK;
}

extern "C" int64_t wc4d_hvp_count(wc4d_ctx *c, int32_t reset)
{
    if (!c) return -1;
    int64_t v = c->hvp_count;
    if (reset) c->hvp_count = 0;
    return v;
}

// ============================================================================
// set-up
// ============================================================================
static wc4d_status alloc_M(wc4d_ctx *c)
{
    size_t bytes = sizeof(double) * (size_t)c->nM * c->prob.n * c->prob.n;
    WC4D_TRY(ensure(c, c->M64, bytes));
    WC4D_TRY(ensure(c, c->MT64, bytes));
    return WC4D_OK;
}

// replicate block 0 of M64 / MT64 into every subwindow block
static wc4d_status replicate_M(wc4d_ctx *c)
{
    size_t nn = (size_t)c->prob.n * c->prob.n;
    for (int t = 1; t < c->nM; ++t) {
        WC4D_CUDA(c, cudaMemcpyAsync(P<double>(c->M64) + t * nn, P<double>(c->M64), nn * sizeof(double),
                                     cudaMemcpyDeviceToDevice, c->stream));
        WC4D_CUDA(c, cudaMemcpyAsync(P<double>(c->MT64) + t * nn, P<double>(c->MT64), nn * sizeof(double),
                                     cudaMemcpyDeviceToDevice, c->stream));
    }
    return WC4D_OK;
}

extern "C" wc4d_status wc4d_set_propagator(wc4d_ctx *c, int32_t t, const double *M)
{
    if (!c || !M) return WC4D_EINVAL;
    if (c->prob.model != WC4D_MODEL_DENSE) return set_err(c, WC4D_EINVAL, "set_propagator: model is not dense");
    if (t < -1 || t >= c->nM) return set_err(c, WC4D_EINVAL, "set_propagator: t=%d out of range", t);
    WC4D_TRY(alloc_M(c));
    const int n = c->prob.n;
    size_t nn = (size_t)n * n;
    int tt = (t < 0) ? 0 : t;
    WC4D_CUDA(c, cudaMemcpyAsync(P<double>(c->M64) + tt * nn, M, nn * sizeof(double), cudaMemcpyDeviceToDevice,
                                 c->stream));
    launch_transpose_f64(c->stream, n, P<double>(c->M64) + tt * nn, P<double>(c->MT64) + tt * nn);
    WC4D_TRY(check_launch(c, "transpose"));
    if (t < 0) WC4D_TRY(replicate_M(c));
    if (t < 0 || c->nM == 1) c->have_M = true;
    else c->have_M = true;  // caller is responsible for setting every subwindow
    c->have_M32 = false;
    c->have_Mtf = false;
    c->have_Mlo = false;
    return WC4D_OK;
}

extern "C" wc4d_status wc4d_build_advdiff_propagator(wc4d_ctx *c, double kappa, double vel, double dt, int32_t steps)
{
    if (!c || steps < 1 || !(dt > 0.0)) return WC4D_EINVAL;
    if (c->prob.model != WC4D_MODEL_DENSE) return set_err(c, WC4D_EINVAL, "build_advdiff: model is not dense");
    WC4D_TRY(alloc_M(c));
    const int n = c->prob.n;
    WC4D_TRY(ensure(c, c->small0, sizeof(double2) * n));
    WC4D_TRY(ensure(c, c->small1, sizeof(double) * n));
    launch_advdiff_column(c->stream, n, kappa, vel, dt, steps, P<double2>(c->cosn), P<double2>(c->small0),
                          P<double>(c->small1));
    launch_expand_circulant(c->stream, n, P<double>(c->small1), P<double>(c->M64), P<double>(c->MT64));
    WC4D_TRY(check_launch(c, "build_advdiff"));
    WC4D_TRY(replicate_M(c));
    c->have_M = true;
    c->have_M32 = false;
    c->have_Mtf = false;
    c->have_Mlo = false;
    return sync(c, "build_advdiff");
}

static wc4d_status ensure_M32(wc4d_ctx *c)
{
    if (c->have_M32) return WC4D_OK;
    size_t cnt = (size_t)c->nM * c->prob.n * c->prob.n;
    WC4D_TRY(ensure(c, c->M32, cnt * sizeof(float)));
    WC4D_TRY(ensure(c, c->MT32, cnt * sizeof(float)));
    launch_convert_f64_f32(c->stream, (int64_t)cnt, P<double>(c->M64), P<float>(c->M32));
    launch_convert_f64_f32(c->stream, (int64_t)cnt, P<double>(c->MT64), P<float>(c->MT32));
    WC4D_TRY(check_launch(c, "convert M"));
    c->have_M32 = true;
    return WC4D_OK;
}

// FP32 remainders of the FP64 propagators (M - M32, M^T - MT32) for the
// double-float sweeps of the mixed CG's true residual.
__global__ void k_f32_remainder(int64_t cnt, const double *__restrict__ A, const float *__restrict__ Ah, float *Al)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        Al[i] = __double2float_rn(A[i] - (double)Ah[i]);
}

static wc4d_status ensure_Mlo(wc4d_ctx *c)
{
    if (c->have_Mlo) return WC4D_OK;
    WC4D_TRY(ensure_M32(c));
    const size_t cnt = (size_t)c->nM * c->prob.n * c->prob.n;
    WC4D_TRY(ensure(c, c->Mlo, cnt * sizeof(float)));
    WC4D_TRY(ensure(c, c->MTlo, cnt * sizeof(float)));
    const int grid = 8 * c->num_sms;
    WC4D_LAUNCH(k_f32_remainder<<<grid, 256, 0, c->stream>>>((int64_t)cnt, P<double>(c->M64), P<float>(c->M32),
                                                             P<float>(c->Mlo)));
    WC4D_LAUNCH(k_f32_remainder<<<grid, 256, 0, c->stream>>>((int64_t)cnt, P<double>(c->MT64), P<float>(c->MT32),
                                                             P<float>(c->MTlo)));
    WC4D_TRY(check_launch(c, "propagator remainders"));
    c->have_Mlo = true;
    return WC4D_OK;
}

// kind >= 0: eigenvalues of variance * C(kind, L) in closed form; kind < 0:
// from the explicit first row row_dev.
static wc4d_status cov_sqrt_setup(wc4d_ctx *c, int block, int kind, double L, double variance, const double *row_dev,
                                  bool root_given = false)
{
    const int n = c->prob.n;
    WC4D_TRY(ensure(c, c->small2, sizeof(double) * (n + 1)));
    if (c->fft) {
        WC4D_TRY(ensure(c, c->spec64[block], sizeof(double) * n));
        WC4D_TRY(ensure(c, c->spec32[block], sizeof(float) * n));
    } else {
        WC4D_TRY(ensure(c, c->row64[block], sizeof(double) * n));
        WC4D_TRY(ensure(c, c->row32[block], sizeof(float) * n));
    }
    launch_cov_sqrt(c->stream, n, c->logn, c->fft, kind, L, variance, row_dev, P<double2>(c->cosn),
                    P<double>(c->small2), P<double>(c->spec64[block]), P<float>(c->spec32[block]),
                    P<double>(c->row64[block]), P<float>(c->row32[block]), root_given);
    WC4D_TRY(check_launch(c, "cov_sqrt"));
    c->have_cov[block] = true;
    return sync(c, "cov_sqrt");
}

extern "C" wc4d_status wc4d_set_covariance(wc4d_ctx *c, int32_t block, int32_t corr, double variance, double L)
{
    if (!c || block < 0 || block > 1 || corr < 0 || corr > 2 || !(variance >= 0.0)) return WC4D_EINVAL;
    if (corr != WC4D_CORR_DIAG && !(L > 0.0 && L < 1e300)) return WC4D_EINVAL;
    c->cov_sd[block] = (corr == WC4D_CORR_DIAG) ? std::sqrt(variance) : -1.0;
    c->cov_dense[block] = false;
    return cov_sqrt_setup(c, block, corr, L, variance, nullptr);
}

extern "C" wc4d_status wc4d_set_covariance_row(wc4d_ctx *c, int32_t block, const double *row_host)
{
    if (!c || block < 0 || block > 1 || !row_host) return WC4D_EINVAL;
    c->cov_sd[block] = -1.0;
    c->cov_dense[block] = false;
    WC4D_TRY(ensure(c, c->small3, sizeof(double) * c->prob.n));
    WC4D_CUDA(c, cudaMemcpyAsync(c->small3.p, row_host, sizeof(double) * c->prob.n, cudaMemcpyHostToDevice,
                                 c->stream));
    return cov_sqrt_setup(c, block, -1, 0.0, 1.0, P<double>(c->small3));
}

extern "C" wc4d_status wc4d_set_cov_sqrt(wc4d_ctx *c, int32_t block, int32_t kind, const double *data)
{
    if (!c || block < 0 || block > 1 || !data) return WC4D_EINVAL;
    const int n = c->prob.n;
    if (kind == 0) {                                   // first row of the circulant square root (host)
        c->cov_sd[block] = -1.0;
        c->cov_dense[block] = false;
        WC4D_TRY(ensure(c, c->small3, sizeof(double) * n));
        WC4D_CUDA(c, cudaMemcpyAsync(c->small3.p, data, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
        return cov_sqrt_setup(c, block, -1, 0.0, 1.0, P<double>(c->small3), true);
    }
    if (kind == 1) {                                   // dense n x n square root (device, row-major)
        const size_t nn = (size_t)n * n;
        WC4D_TRY(ensure(c, c->dense64[block], sizeof(double) * nn));
        WC4D_TRY(ensure(c, c->dense32[block], sizeof(float) * nn));
        WC4D_CUDA(c, cudaMemcpyAsync(c->dense64[block].p, data, sizeof(double) * nn, cudaMemcpyDeviceToDevice,
                                     c->stream));
        launch_convert_f64_f32(c->stream, (int64_t)nn, P<double>(c->dense64[block]), P<float>(c->dense32[block]));
        WC4D_TRY(check_launch(c, "dense square root"));
        c->cov_sd[block] = -1.0;
        c->cov_dense[block] = true;
        c->have_cov[block] = true;
        return sync(c, "dense square root");
    }
    if (kind == 2) {                                   // scalar: the block is sigma^2 I (host, one value sigma)
        const double sd = data[0];
        if (!(sd >= 0.0) || !std::isfinite(sd)) return WC4D_EINVAL;
        WC4D_TRY(wc4d_set_covariance(c, block, WC4D_CORR_DIAG, sd * sd, 1.0));
        c->cov_sd[block] = sd;
        return WC4D_OK;
    }
    return WC4D_EINVAL;
}

static wc4d_status require_operator(wc4d_ctx *c)
{
    if (!c->have_cov[0] || !c->have_cov[1]) return set_err(c, WC4D_ESTATE, "covariances B and Q are not set");
    if (c->prob.model == WC4D_MODEL_DENSE && !c->have_M) return set_err(c, WC4D_ESTATE, "propagator not set");
    if (c->prob.model == WC4D_MODEL_L96 && !c->have_traj)
        return set_err(c, WC4D_ESTATE, "Lorenz-96 trajectory not set (call wc4d_set_background_obs)");
    return WC4D_OK;
}

// ============================================================================
// The Hessian product Y = A X (eq. 10)
// ============================================================================
template <typename T> struct Ops;
template <> struct Ops<double> {
    static const double *M(wc4d_ctx *c, int t) { return P<double>(c->M64) + mblk(c, t); }
    static const double *MT(wc4d_ctx *c, int t) { return P<double>(c->MT64) + mblk(c, t); }
    static const double *spec(wc4d_ctx *c, int b) { return P<double>(c->spec64[b]); }
    static const double *row(wc4d_ctx *c, int b) { return P<double>(c->row64[b]); }
    static const void *tw(wc4d_ctx *c) { return c->tw64.p; }
    static const double *stages(wc4d_ctx *c) { return P<double>(c->stage64); }
    static DevBuf &work(wc4d_ctx *c) { return c->work64; }
};
template <> struct Ops<float> {
    static const float *M(wc4d_ctx *c, int t) { return P<float>(c->M32) + mblk(c, t); }
    static const float *MT(wc4d_ctx *c, int t) { return P<float>(c->MT32) + mblk(c, t); }
    static const float *spec(wc4d_ctx *c, int b) { return P<float>(c->spec32[b]); }
    static const float *row(wc4d_ctx *c, int b) { return P<float>(c->row32[b]); }
    static const void *tw(wc4d_ctx *c) { return c->tw32.p; }
    static const float *stages(wc4d_ctx *c) { return P<float>(c->stage32); }
    static DevBuf &work(wc4d_ctx *c) { return c->work32; }
};

// Dense-model sweeps on tensor cores (tc_gemm.cu); returns false when the
// shape is not supported so the SIMT path is taken.
bool tc_sweep_supported(const wc4d_ctx *c, int K);
int tc_read_error(wc4d_ctx *c);
bool oz_gram_supported(const wc4d_ctx *c, int64_t rows, int m);
size_t oz_gram_part_doubles(const wc4d_ctx *c, int64_t rows, int m);
int64_t oz_rows_pad(int64_t rows);
bool launch_oz_gram(wc4d_ctx *c, int64_t rows, int m, const float *A, int64_t lda, const float *B, int64_t ldb,
                    uint16_t *slices, int *work, double *part, size_t part_cap, double *C, int *err);

// Symmetric Gram-type product G = A^T B (m x m, FP64; upper tiles computed
// and mirrored): FP32 blocks go to the tensor-core sliced product when the
// shape allows it (m a multiple of 128, at least 512 rows) and the context
// has not switched it off, otherwise (and for FP64 blocks) to the FP32- or
// FP64-pipe kernels.  Returns 0, or -1 when the partial buffer is too small.
template <typename T>
static int gram_sym(wc4d_ctx *c, int64_t rows, int m, const T *A, int64_t lda, const T *B, int64_t ldb, double *G,
                    int *S)
{
    if constexpr (sizeof(T) == 4) {
        if (c->gram_tc && oz_gram_supported(c, rows, m)) {
            const size_t per = (size_t)6 * m * (size_t)oz_rows_pad(rows);
            const size_t sl = per * ((A == B && lda == ldb) ? 1 : 2);
            if (ensure(c, c->oz_slices, sizeof(uint16_t) * sl) == WC4D_OK &&
                ensure(c, c->oz_work, sizeof(int) * 4 * (size_t)m) == WC4D_OK &&
                ensure(c, c->part, sizeof(double) * oz_gram_part_doubles(c, rows, m)) == WC4D_OK &&
                ensure(c, c->tc_err, sizeof(int)) == WC4D_OK) {
                bool zero_ok = true;
                if (!c->tc_err_zeroed) {
                    zero_ok = cudaMemsetAsync(c->tc_err.p, 0, sizeof(int), c->stream) == cudaSuccess;
                    c->tc_err_zeroed = zero_ok;
                }
                if (zero_ok &&
                    launch_oz_gram(c, rows, m, A, lda, B, ldb, P<uint16_t>(c->oz_slices), P<int>(c->oz_work),
                                   P<double>(c->part), c->part.bytes / 8, G, P<int>(c->tc_err))) {
                    if (S) *S = 1;
                    c->tc_err_pending = true;
                    return 0;
                }
                cudaGetLastError();
            }
        }
    }
    return launch_atb<T>(c->stream, c->num_sms, rows, m, m, A, lda, B, ldb, P<double>(c->part), c->part.bytes / 8, S,
                         G, 1);
}

bool tall_tc_supported(const wc4d_ctx *c, int64_t rows, int N, int Kd);
int64_t tall_rows_pad(int64_t rows);
bool launch_tall_tc(wc4d_ctx *c, int64_t rows, int N, int Kd, const float *Y, int64_t ldy, const double *W, int ldw,
                    float *C, int64_t ldc, float *YS, float *WS, int *err);

// C = Y W for a tall FP32 block Y (rows x Kd, ldy) and an FP64 factor W
// (Kd x N, ldw) on the tensor cores in 3xTF32 when the shape allows it and
// the context has not switched the tensor-core linear algebra off; false:
// nothing launched, the caller takes the SIMT product.  Used for Y R^{-1}
// of CholeskyQR only: its second pass restores the orthogonality the
// ~2^-21 products lose, while the Ritz vectors of the LMP need FP32
// accuracy.
static bool tall_product_tc(wc4d_ctx *c, int64_t rows, int N, int Kd, const float *Y, int64_t ldy, const double *W,
                            int ldw, float *C, int64_t ldc)
{
    if (!c->gram_tc || !tall_tc_supported(c, rows, N, Kd)) return false;
    const size_t ys = (size_t)2 * tall_rows_pad(rows) * Kd, ws = (size_t)2 * N * Kd;
    if (ensure(c, c->tall_ys, sizeof(float) * ys) != WC4D_OK || ensure(c, c->tall_ws, sizeof(float) * ws) != WC4D_OK ||
        ensure(c, c->tc_err, sizeof(int)) != WC4D_OK)
        return false;
    if (!c->tc_err_zeroed) {
        if (cudaMemsetAsync(c->tc_err.p, 0, sizeof(int), c->stream) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        c->tc_err_zeroed = true;
    }
    if (!launch_tall_tc(c, rows, N, Kd, Y, ldy, W, ldw, C, ldc, P<float>(c->tall_ys), P<float>(c->tall_ws),
                        P<int>(c->tc_err))) {
        cudaGetLastError();
        return false;
    }
    c->tc_err_pending = true;
    return true;
}

// Cholesky A = R^T R into R (info in counter word 0: 0, the failing pivot,
// or -1 when a grid barrier of the cooperative form timed out): one
// cooperative launch when the context may use them, else one launch per
// phase of every block step.
static void chol_upper(wc4d_ctx *c, int m, const double *A, double *R)
{
    int *info = P<int>(c->counter);
    if (c->allow_coop && ensure(c, c->chol_bar, sizeof(unsigned)) == WC4D_OK &&
        launch_chol_upper_coop(c->stream, c->num_sms, m, A, R, info, P<unsigned>(c->chol_bar)))
        return;
    launch_chol_upper(c->stream, m, A, R, info);
}
bool tc_sweep_forward(wc4d_ctx *c, int K, float *W, int64_t ld);
bool tc_sweep_adjoint(wc4d_ctx *c, int K, float *W, int64_t ld);

template <typename T> static const T *dense_sqrt(wc4d_ctx *c, int b);
template <> const double *dense_sqrt<double>(wc4d_ctx *c, int b) { return P<double>(c->dense64[b]); }
template <> const float *dense_sqrt<float>(wc4d_ctx *c, int b) { return P<float>(c->dense32[b]); }

// Y = D^{1/2} X (+ addX): circulant blocks by FFT or direct products,
// diagonal blocks by scaling, dense square roots (wc4d_set_cov_sqrt kind 1)
// by one n x n by n x K product per time block.
template <typename T>
static wc4d_status apply_circ(wc4d_ctx *c, int K, const T *X, int64_t ldx, T *Y, int64_t ldy, const T *addX,
                              int64_t ld_add)
{
    ProfScope ps(c, PROF_CIRC);
    const int skip = (c->cov_dense[0] ? 1 : 0) | (c->cov_dense[1] ? 2 : 0);
    if (skip != 3)
        launch_circulant<T>(c->stream, c, K, X, ldx, Y, ldy, addX, ld_add, c->fft, Ops<T>::spec(c, 0),
                            Ops<T>::spec(c, 1), Ops<T>::row(c, 0), Ops<T>::row(c, 1), Ops<T>::tw(c), skip);
    if (skip) {
        const int n = c->prob.n;
        for (int t = 0; t <= c->prob.N; ++t) {
            const int b = (t == 0) ? 0 : 1;
            if (!c->cov_dense[b]) continue;
            T *y = Y + (int64_t)t * n;
            if (addX)
                WC4D_CUDA(c, cudaMemcpy2DAsync(y, sizeof(T) * ldy, addX + (int64_t)t * n, sizeof(T) * ld_add,
                                               sizeof(T) * n, K, cudaMemcpyDeviceToDevice, c->stream));
            Epi e{0, 1.0, addX ? 1.0 : 0.0, 0.0, 1};
            launch_gemm<T>(c->stream, n, K, n, dense_sqrt<T>(c, b), n, 1, X + (int64_t)t * n, ldx, y, ldy, e);
        }
    }
    return check_launch(c, "circulant");
}

// One-column dense sweeps as one persistent launch; false = not applicable.
template <typename T>
static bool persistent_sweep(wc4d_ctx *c, T *W, int mode)
{
    if (c->prob.model != WC4D_MODEL_DENSE || !c->allow_coop || getenv("WC4D_NO_PERSISTENT")) return false;
    const int N = c->prob.N;
    // layout: [0] error flag (kept until read), [1 .. N] step counters
    if (ensure(c, c->sweep_bar, (size_t)(N + 1) * sizeof(unsigned)) != WC4D_OK) return false;
    unsigned *bar = P<unsigned>(c->sweep_bar);
    if (!c->sweep_bar_zeroed) {
        if (cudaMemsetAsync(bar, 0, sizeof(unsigned), c->stream) != cudaSuccess) return false;
        c->sweep_bar_zeroed = true;
    }
    if (cudaMemsetAsync(bar + 1, 0, (size_t)N * sizeof(unsigned), c->stream) != cudaSuccess) return false;
    const int n = c->prob.n;
    const int64_t mstride = (c->nM == 1) ? 0 : (int64_t)n * n;
    if constexpr (sizeof(T) == 8) {
        // the mixed CG's true residual: double-float on the FP32 pipe
        if (c->sweep_df && ensure_Mlo(c) == WC4D_OK &&
            ensure(c, c->df_vec, sizeof(float) * 2 * (size_t)c->nA) == WC4D_OK) {
            const float *Mh = P<float>(mode == 0 ? c->M32 : c->MT32), *Ml = P<float>(mode == 0 ? c->Mlo : c->MTlo);
            float *Wh = P<float>(c->df_vec), *Wl = Wh + c->nA;
            if (launch_gemv_sweep_df(c->stream, c->num_sms, n, c->prob.N, Mh, Ml, mstride, (double *)W, Wh, Wl, mode,
                                     1.0 / c->prob.sigma_o2, c->prob.obs_stride, c->prob.obs_t0,
                                     c->prob.obs_tstride, bar + 1, reinterpret_cast<int *>(bar), c->wait_limit))
                return true;
        }
    }
    const T *M0 = (mode == 0) ? Ops<T>::M(c, 0) : Ops<T>::MT(c, 0);
    return launch_gemv_sweep<T>(c->stream, c->num_sms, n, c->prob.N, M0, mstride, W, mode, 1.0 / c->prob.sigma_o2,
                                c->prob.obs_stride, c->prob.obs_t0, c->prob.obs_tstride,
                                bar + 1, reinterpret_cast<int *>(bar), c->wait_limit);
}

// Timeout flag of the persistent sweeps (cleared on read).
static int sweep_error(wc4d_ctx *c)
{
    if (!c->sweep_bar.p || !c->sweep_bar_zeroed) return 0;
    int h = 0;
    cudaMemcpyAsync(&h, P<unsigned>(c->sweep_bar), sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    if (h) cudaMemsetAsync(P<unsigned>(c->sweep_bar), 0, sizeof(int), c->stream);
    return h;
}

// Error word of the kernels whose waits on asynchronous copies are bounded
// (the tensor-core kernels, the FP32 Lorenz-96 sweeps): allocated and zeroed
// once per context (the first iteration of a solve runs eagerly, so this
// never happens inside a graph capture); null if that fails, and the kernels
// then record nothing.
static int *wait_err_word(wc4d_ctx *c)
{
    if (ensure(c, c->tc_err, sizeof(int)) != WC4D_OK) return nullptr;
    if (!c->tc_err_zeroed) {
        if (cudaMemsetAsync(c->tc_err.p, 0, sizeof(int), c->stream) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        c->tc_err_zeroed = true;
    }
    return P<int>(c->tc_err);
}

// WC4D_ETIMEOUT if a kernel with bounded copy waits ran since the error word
// was last read and one of its waits gave up (reading synchronises).
static wc4d_status pending_wait_error(wc4d_ctx *c)
{
    if (!c->tc_err_pending) return WC4D_OK;
    c->tc_err_pending = false;
    if (tc_read_error(c))
        return set_err(c, WC4D_ETIMEOUT, "a bounded wait on an asynchronous copy timed out (FP32 Lorenz-96 sweep or "
                                         "tensor-core kernel)");
    return WC4D_OK;
}

extern "C" wc4d_status wc4d_sync(wc4d_ctx *c)
{
    if (!c) return WC4D_EINVAL;
    WC4D_TRY(sync(c, "wc4d_sync"));
    if (const int e = sweep_error(c)) return set_err(c, WC4D_ETIMEOUT, "persistent sweep failed (code %d)", e);
    return pending_wait_error(c);
}

// W (nA x K, ld) <- L^{-1} W in place: W_{t+1} += M_t W_t.
template <typename T>
static wc4d_status forward_sweep(wc4d_ctx *c, int K, T *W, int64_t ld, bool allow_tc)
{
    const int n = c->prob.n, N = c->prob.N;
    if (c->prob.model == WC4D_MODEL_L96) {
        ProfScope ps(c, PROF_L96_TLM);
        int *err = sizeof(T) == 4 ? wait_err_word(c) : nullptr;
        launch_l96_tlm_sweep<T>(c->stream, n, N, c->prob.steps, c->prob.dt, Ops<T>::stages(c), K, W, ld, err,
                                c->wait_limit);
        if (err) c->tc_err_pending = true;
        return check_launch(c, "l96 tlm sweep");
    }
    if constexpr (sizeof(T) == 4) {
        if (allow_tc && tc_sweep_supported(c, K) && tc_sweep_forward(c, K, (float *)W, ld))
            return check_launch(c, "tc forward sweep");
    }
    if (K == 1) {
        ProfScope ps(c, sizeof(T) == 4 ? PROF_GEMV : PROF_GEMV64);
        if (persistent_sweep<T>(c, W, 0)) return check_launch(c, "forward sweep");
    }
    Epi e{0, 1.0, 1.0, 0.0, 1};
    for (int t = 0; t < N; ++t) {
        ProfScope ps(c, K == 1 ? PROF_GEMV : PROF_GEMM);
        launch_sweep_gemm<T>(c->stream, n, K, Ops<T>::M(c, t), W + (int64_t)t * n, ld, W + (int64_t)(t + 1) * n, ld,
                             e);
    }
    return check_launch(c, "forward sweep");
}

// W <- L^{-T} H^T R^{-1} H W in place: W_N = obs_N(W_N); W_t = obs_t(W_t) + M_t^T W_{t+1}.
template <typename T>
static wc4d_status adjoint_obs_sweep(wc4d_ctx *c, int K, T *W, int64_t ld, bool allow_tc)
{
    const int n = c->prob.n, N = c->prob.N;
    if (c->prob.model == WC4D_MODEL_L96) {
        ProfScope ps(c, PROF_L96_ADJ);
        int *err = sizeof(T) == 4 ? wait_err_word(c) : nullptr;
        launch_l96_adj_sweep<T>(c->stream, n, N, c->prob.steps, c->prob.dt, Ops<T>::stages(c), K, W, ld, 1,
                                1.0 / c->prob.sigma_o2, c->prob.obs_stride, c->prob.obs_t0, c->prob.obs_tstride, err,
                                c->wait_limit);
        if (err) c->tc_err_pending = true;
        return check_launch(c, "l96 adjoint sweep");
    }
    if constexpr (sizeof(T) == 4) {
        if (allow_tc && tc_sweep_supported(c, K) && tc_sweep_adjoint(c, K, (float *)W, ld))
            return check_launch(c, "tc adjoint sweep");
    }
    launch_obs_block<T>(c->stream, n, K, W + (int64_t)N * n, ld, obs_scale(c, N), c->prob.obs_stride);
    if (K == 1) {
        ProfScope ps(c, sizeof(T) == 4 ? PROF_GEMV : PROF_GEMV64);
        if (persistent_sweep<T>(c, W, 1)) return check_launch(c, "adjoint sweep");
    }
    for (int t = N - 1; t >= 0; --t) {
        Epi e{1, 1.0, 0.0, obs_scale(c, t), c->prob.obs_stride};
        ProfScope ps(c, K == 1 ? PROF_GEMV : PROF_GEMM);
        launch_sweep_gemm<T>(c->stream, n, K, Ops<T>::MT(c, t), W + (int64_t)(t + 1) * n, ld, W + (int64_t)t * n, ld,
                             e);
    }
    return check_launch(c, "adjoint sweep");
}

template <typename T>
static wc4d_status hvp_impl(wc4d_ctx *c, const T *X, T *Y, int K, int64_t ld, bool allow_tc = true)
{
    const int64_t nA = c->nA;
    DevBuf &wb = Ops<T>::work(c);
    WC4D_TRY(ensure(c, wb, sizeof(T) * (size_t)nA * K));
    T *W = P<T>(wb);
    WC4D_TRY(apply_circ<T>(c, K, X, ld, W, nA, nullptr, 0));            // W = D^{1/2} X
    WC4D_TRY(forward_sweep<T>(c, K, W, nA, allow_tc));                  // W = L^{-1} W
    WC4D_TRY(adjoint_obs_sweep<T>(c, K, W, nA, allow_tc));              // W = L^{-T} H^T R^{-1} H W
    WC4D_TRY(apply_circ<T>(c, K, W, nA, Y, ld, X, ld));                 // Y = X + D^{1/2} W
    c->hvp_count++;
    if constexpr (sizeof(T) == 4) {
        if (allow_tc && tc_sweep_supported(c, K) && tc_read_error(c))
            return set_err(c, WC4D_ETIMEOUT, "tensor-core sweep: a bounded wait timed out");
    }
    return WC4D_OK;
}

static wc4d_status prep_precision(wc4d_ctx *c, int precision)
{
    if (precision == WC4D_MIXED && c->prob.model == WC4D_MODEL_DENSE) WC4D_TRY(ensure_M32(c));
    return WC4D_OK;
}

extern "C" wc4d_status wc4d_hvp(wc4d_ctx *c, const void *X, void *Y, int32_t K, int64_t ld, int32_t precision)
{
    if (!c || !X || !Y || K < 1 || ld < c->nA) return WC4D_EINVAL;
    if (precision != WC4D_FP64 && precision != WC4D_MIXED) return WC4D_EINVAL;
    WC4D_TRY(require_operator(c));
    WC4D_TRY(prep_precision(c, precision));
    wc4d_status st = (precision == WC4D_FP64) ? hvp_impl<double>(c, (const double *)X, (double *)Y, K, ld)
                                              : hvp_impl<float>(c, (const float *)X, (float *)Y, K, ld);
    int e = 0;
    if (st == WC4D_OK && K == 1 && (e = sweep_error(c)) != 0)
        return set_err(c, WC4D_ETIMEOUT, "persistent sweep failed (code %d: 1 grid barrier timeout, 2 misaligned "
                                         "operand, 3/4 copy pipeline wait timeout)", e);
    return st;
}

template <typename T>
static wc4d_status plain_adjoint_sweep(wc4d_ctx *c, int K, T *W, int64_t ld)
{
    const int n = c->prob.n, N = c->prob.N;
    if (c->prob.model == WC4D_MODEL_L96) {
        int *err = sizeof(T) == 4 ? wait_err_word(c) : nullptr;
        launch_l96_adj_sweep<T>(c->stream, n, N, c->prob.steps, c->prob.dt, Ops<T>::stages(c), K, W, ld, 0, 0.0, 1,
                                0, 1, err, c->wait_limit);
        if (err) c->tc_err_pending = true;
        return check_launch(c, "l96 adjoint sweep");
    }
    Epi e{0, 1.0, 1.0, 0.0, 1};
    for (int t = N - 1; t >= 0; --t)
        launch_sweep_gemm<T>(c->stream, n, K, Ops<T>::MT(c, t), W + (int64_t)(t + 1) * n, ld, W + (int64_t)t * n, ld,
                             e);
    return check_launch(c, "adjoint sweep");
}

extern "C" wc4d_status wc4d_apply_dsqrt(wc4d_ctx *c, const void *X, void *Y, int32_t K, int64_t ld, int32_t precision)
{
    if (!c || !X || !Y || K < 1 || ld < c->nA) return WC4D_EINVAL;
    if (!c->have_cov[0] || !c->have_cov[1]) return set_err(c, WC4D_ESTATE, "covariances are not set");
    if (precision == WC4D_FP64) return apply_circ<double>(c, K, (const double *)X, ld, (double *)Y, ld, nullptr, 0);
    if (precision == WC4D_MIXED) return apply_circ<float>(c, K, (const float *)X, ld, (float *)Y, ld, nullptr, 0);
    return WC4D_EINVAL;
}

extern "C" wc4d_status wc4d_apply_linv(wc4d_ctx *c, void *W, int32_t K, int64_t ld, int32_t precision)
{
    if (!c || !W || K < 1 || ld < c->nA) return WC4D_EINVAL;
    WC4D_TRY(require_operator(c));
    WC4D_TRY(prep_precision(c, precision));
    if (precision == WC4D_FP64) return forward_sweep<double>(c, K, (double *)W, ld, false);
    if (precision == WC4D_MIXED) return forward_sweep<float>(c, K, (float *)W, ld, true);
    return WC4D_EINVAL;
}

extern "C" wc4d_status wc4d_apply_linvT(wc4d_ctx *c, void *W, int32_t K, int64_t ld, int32_t precision)
{
    if (!c || !W || K < 1 || ld < c->nA) return WC4D_EINVAL;
    WC4D_TRY(require_operator(c));
    WC4D_TRY(prep_precision(c, precision));
    if (precision == WC4D_FP64) return plain_adjoint_sweep<double>(c, K, (double *)W, ld);
    if (precision == WC4D_MIXED) return plain_adjoint_sweep<float>(c, K, (float *)W, ld);
    return WC4D_EINVAL;
}

extern "C" wc4d_status wc4d_get_propagator(wc4d_ctx *c, int32_t t, double *M)
{
    if (!c || !M) return WC4D_EINVAL;
    if (c->prob.model != WC4D_MODEL_DENSE || !c->have_M) return set_err(c, WC4D_ESTATE, "no dense propagator");
    if (t < 0 || t >= c->prob.N) return WC4D_EINVAL;
    size_t nn = (size_t)c->prob.n * c->prob.n;
    WC4D_CUDA(c, cudaMemcpyAsync(M, P<double>(c->M64) + mblk(c, t), nn * sizeof(double), cudaMemcpyDeviceToDevice,
                                 c->stream));
    return sync(c, "get_propagator");
}

// ============================================================================
// Outer-loop quantities: innovations and right-hand side
// ============================================================================
// Model run from the stored linearisation point p = (x_0, eta), innovations
// d_t = y_t - H_t x_t and rhs = D^{1/2} L^{-T} H^T R^{-1} d (+ D^{-1/2} b).
// rhs = D^{1/2} L^{-T} H^T R^{-1} d (+ D^{-1/2} b) from the innovations in c->d.
static wc4d_status compute_rhs(wc4d_ctx *c)
{
    const int n = c->prob.n;
    const int64_t nA = c->nA;
    WC4D_TRY(ensure(c, c->blkB, sizeof(double) * nA));
    WC4D_TRY(ensure(c, c->rhs, sizeof(double) * nA));
    double *v = P<double>(c->blkB);
    WC4D_CUDA(c, cudaMemsetAsync(v, 0, sizeof(double) * nA, c->stream));
    if (c->nobs > 0)
        WC4D_LAUNCH(k_scatter_obs<<<ceil_div(c->nobs, 256), 256, 0, c->stream>>>(c->nobs, c->obs_per_time, c->prob.obs_t0,
                                                                      c->prob.obs_tstride, c->prob.obs_stride, n,
                                                                      P<double>(c->d), 1.0 / c->prob.sigma_o2, v));
    WC4D_TRY(check_launch(c, "innovation"));
    WC4D_TRY(plain_adjoint_sweep<double>(c, 1, v, nA));    // S = L^{-T} H^T R^{-1} d
    WC4D_TRY(apply_circ<double>(c, 1, v, nA, P<double>(c->rhs), nA, c->have_Dm12b ? P<double>(c->Dm12b) : nullptr,
                                nA));
    c->have_rhs = true;
    return sync(c, "rhs");
}

static wc4d_status relinearise(wc4d_ctx *c)
{
    const int n = c->prob.n, N = c->prob.N;
    const int64_t nA = c->nA;
    WC4D_TRY(ensure(c, c->blkA, sizeof(double) * nA));
    WC4D_TRY(ensure(c, c->blkB, sizeof(double) * nA));
    WC4D_TRY(ensure(c, c->d, sizeof(double) * std::max<int64_t>(c->nobs, 1)));
    WC4D_TRY(ensure(c, c->rhs, sizeof(double) * nA));
    double *xs = P<double>(c->blkA);
    const double *lin = P<double>(c->lin);
    if (c->prob.model == WC4D_MODEL_L96) {
        const int64_t nsteps = (int64_t)N * c->prob.steps;
        WC4D_TRY(ensure(c, c->traj64, sizeof(double) * (size_t)(nsteps + 1) * n));
        WC4D_TRY(ensure(c, c->stage64, sizeof(double) * (size_t)4 * nsteps * n));
        WC4D_TRY(ensure(c, c->stage32, sizeof(float) * (size_t)4 * nsteps * n));
        WC4D_CUDA(c, cudaMemcpyAsync(c->traj64.p, lin, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
        launch_l96_run(c->stream, n, (int)nsteps, c->prob.F, c->prob.dt, P<double>(c->traj64), P<double>(c->stage64),
                       lin, c->prob.steps);
        launch_convert_f64_f32(c->stream, 4 * nsteps * n, P<double>(c->stage64), P<float>(c->stage32));
        WC4D_TRY(check_launch(c, "l96 run"));
        for (int t = 0; t <= N; ++t)
            WC4D_CUDA(c, cudaMemcpyAsync(xs + (int64_t)t * n, P<double>(c->traj64) + (int64_t)t * c->prob.steps * n,
                                         sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
        c->have_traj = true;
    } else {
        if (!c->have_M) return set_err(c, WC4D_ESTATE, "propagator not set");
        // x_{t+1} = M_t x_t + eta_{t+1}: the sweep adds M_t x_t to block t+1
        WC4D_CUDA(c, cudaMemcpyAsync(xs, lin, sizeof(double) * nA, cudaMemcpyDeviceToDevice, c->stream));
        WC4D_TRY(forward_sweep<double>(c, 1, xs, nA, false));
    }
    // innovations
    if (c->nobs > 0)
        WC4D_LAUNCH(k_innovation<<<ceil_div(c->nobs, 256), 256, 0, c->stream>>>(c->nobs, c->obs_per_time, c->prob.obs_t0,
                                                                     c->prob.obs_tstride, c->prob.obs_stride, n,
                                                                     P<double>(c->ydev), xs, P<double>(c->d)));
    return compute_rhs(c);
}

extern "C" wc4d_status wc4d_set_background_obs(wc4d_ctx *c, const double *xb, const double *y, const double *Dm12b)
{
    if (!c || !xb || !y) return WC4D_EINVAL;
    if (!c->have_cov[0] || !c->have_cov[1]) return set_err(c, WC4D_ESTATE, "covariances are not set");
    const int n = c->prob.n;
    const int64_t nA = c->nA;
    WC4D_TRY(ensure(c, c->lin, sizeof(double) * nA));
    WC4D_TRY(ensure(c, c->ydev, sizeof(double) * std::max<int64_t>(c->nobs, 1)));
    WC4D_CUDA(c, cudaMemsetAsync(c->lin.p, 0, sizeof(double) * nA, c->stream));   // eta = 0
    WC4D_CUDA(c, cudaMemcpyAsync(c->lin.p, xb, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    if (c->nobs > 0)
        WC4D_CUDA(c, cudaMemcpyAsync(c->ydev.p, y, sizeof(double) * c->nobs, cudaMemcpyHostToDevice, c->stream));
    c->have_Dm12b = Dm12b != nullptr;
    if (Dm12b) {
        WC4D_TRY(ensure(c, c->Dm12b, sizeof(double) * nA));
        WC4D_CUDA(c, cudaMemcpyAsync(c->Dm12b.p, Dm12b, sizeof(double) * nA, cudaMemcpyHostToDevice, c->stream));
    }
    c->have_lin = true;
    return relinearise(c);
}

extern "C" wc4d_status wc4d_set_trajectory(wc4d_ctx *c, const double *X)
{
    if (!c || !X) return WC4D_EINVAL;
    if (c->prob.model != WC4D_MODEL_L96) return set_err(c, WC4D_EINVAL, "set_trajectory: Lorenz-96 model only");
    const int n = c->prob.n;
    const int64_t nsteps = (int64_t)c->prob.N * c->prob.steps;
    WC4D_TRY(ensure(c, c->traj64, sizeof(double) * (size_t)(nsteps + 1) * n));
    WC4D_TRY(ensure(c, c->stage64, sizeof(double) * (size_t)4 * nsteps * n));
    WC4D_TRY(ensure(c, c->stage32, sizeof(float) * (size_t)4 * nsteps * n));
    WC4D_CUDA(c, cudaMemcpyAsync(c->traj64.p, X, sizeof(double) * (size_t)(nsteps + 1) * n, cudaMemcpyDeviceToDevice,
                                 c->stream));
    launch_l96_stages(c->stream, n, (int)nsteps, c->prob.F, c->prob.dt, P<double>(c->traj64), P<double>(c->stage64));
    launch_convert_f64_f32(c->stream, 4 * nsteps * n, P<double>(c->stage64), P<float>(c->stage32));
    WC4D_TRY(check_launch(c, "set_trajectory"));
    c->have_traj = true;
    return sync(c, "set_trajectory");
}

extern "C" wc4d_status wc4d_set_innovation(wc4d_ctx *c, const double *d, const double *Dm12b)
{
    if (!c || (!d && c->nobs > 0)) return WC4D_EINVAL;
    WC4D_TRY(require_operator(c));
    const int64_t nA = c->nA;
    WC4D_TRY(ensure(c, c->d, sizeof(double) * std::max<int64_t>(c->nobs, 1)));
    if (c->nobs > 0)
        WC4D_CUDA(c, cudaMemcpyAsync(c->d.p, d, sizeof(double) * c->nobs, cudaMemcpyDeviceToDevice, c->stream));
    c->have_Dm12b = Dm12b != nullptr;
    if (Dm12b) {
        WC4D_TRY(ensure(c, c->Dm12b, sizeof(double) * nA));
        WC4D_CUDA(c, cudaMemcpyAsync(c->Dm12b.p, Dm12b, sizeof(double) * nA, cudaMemcpyDeviceToDevice, c->stream));
    }
    return compute_rhs(c);
}

extern "C" wc4d_status wc4d_outer_update(wc4d_ctx *c, const double *x)
{
    if (!c || !x) return WC4D_EINVAL;
    if (!c->have_lin) return set_err(c, WC4D_ESTATE, "no linearisation point (call wc4d_set_background_obs)");
    const int64_t nA = c->nA;
    WC4D_TRY(ensure(c, c->blkC, sizeof(double) * nA));
    WC4D_TRY(ensure(c, c->Dm12b, sizeof(double) * nA));
    if (!c->have_Dm12b) WC4D_CUDA(c, cudaMemsetAsync(c->Dm12b.p, 0, sizeof(double) * nA, c->stream));
    double *dp = P<double>(c->blkC);
    WC4D_TRY(apply_circ<double>(c, 1, x, nA, dp, nA, nullptr, 0));                       // dp = D^{1/2} x
    launch_axpby<double>(c->stream, nA, 1.0, dp, 1.0, P<double>(c->lin));                  // p += dp (eq. 3)
    launch_axpby<double>(c->stream, nA, -1.0, x, 1.0, P<double>(c->Dm12b));               // D^{-1/2} b -= x
    WC4D_TRY(check_launch(c, "outer update"));
    c->have_Dm12b = true;
    return relinearise(c);
}

extern "C" wc4d_status wc4d_get_rhs(wc4d_ctx *c, double *rhs)
{
    if (!c || !rhs) return WC4D_EINVAL;
    if (!c->have_rhs) return set_err(c, WC4D_ESTATE, "rhs not set");
    WC4D_CUDA(c, cudaMemcpyAsync(rhs, c->rhs.p, sizeof(double) * c->nA, cudaMemcpyDeviceToDevice, c->stream));
    return sync(c, "get_rhs");
}

extern "C" wc4d_status wc4d_gaussian(wc4d_ctx *c, uint64_t seed, int64_t rows, int32_t cols, int64_t ld, double *G)
{
    if (!c || !G || rows < 1 || cols < 1 || ld < rows) return WC4D_EINVAL;
    launch_gaussian(c->stream, seed, rows, cols, ld, G);
    return check_launch(c, "gaussian");
}

extern "C" wc4d_status wc4d_gaussian_f32(wc4d_ctx *c, uint64_t seed, int64_t rows, int32_t cols, int64_t ld,
                                         float *G)
{
    if (!c || !G || rows < 1 || cols < 1 || ld < rows) return WC4D_EINVAL;
    launch_gaussian_f32(c->stream, seed, rows, cols, ld, G);
    return check_launch(c, "gaussian f32");
}

// ============================================================================
// CholeskyQR2 and the small symmetric eigenproblem
// ============================================================================
// Y (rows x m, ld) <- Y R^{-1} with Y = Z R; Rout (m x m, device FP64) = R.
template <typename T>
static wc4d_status cholqr_pass(wc4d_ctx *c, T *Y, int64_t rows, int m, int64_t ld, T *tmp, double *R,
                               bool *shifted = nullptr)
{
    const size_t mm = (size_t)m * m;
    WC4D_TRY(ensure(c, c->small0, sizeof(double) * mm));
    WC4D_TRY(ensure(c, c->small1, sizeof(double) * mm));
    const size_t part_need = atb_part_doubles(c->num_sms, rows, m, m, 1);
    WC4D_TRY(ensure(c, c->part, sizeof(double) * part_need));
    int S = 0;
    double *G = P<double>(c->small0);
    unsigned *rs_work = reinterpret_cast<unsigned *>(P<int>(c->counter) + 12);   // counter words 12, 13
    if constexpr (sizeof(T) == 4) {
        ProfScope ps(c, PROF_GRAM);
        launch_range_scale_f32(c->stream, c->num_sms, rows, m, ld, Y, rs_work);
    }
    {
        ProfScope ps(c, PROF_GRAM);
        if (gram_sym<T>(c, rows, m, Y, ld, Y, ld, G, &S) != 0)   // G = Y^T Y
            return set_err(c, WC4D_EINVAL, "internal: Gram partial buffer too small");
    }
    double *Rinv = P<double>(c->small1);
    int info = 0;
    {
        ProfScope psc(c, PROF_CHOL);
        chol_upper(c, m, G, R);                            // G = R^T R
        launch_trinv_upper(c->stream, m, R, Rinv);
        WC4D_TRY(check_launch(c, "cholqr"));
        WC4D_CUDA(c, cudaMemcpyAsync(&info, c->counter.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    }
    WC4D_TRY(sync(c, "cholqr info"));
    if (info < 0) return set_err(c, WC4D_ETIMEOUT, "Cholesky: a grid barrier timed out");
    WC4D_TRY(pending_wait_error(c));
    // Numerically rank-deficient Y (the Gram is accurate to FP64 rounding --
    // to ~1e-12 relative on the tensor-core path -- so this happens when its
    // condition exceeds ~1e16 (~1e12), e.g. sketches of a
    // Hessian whose eigenvalues span 1e17): shifted CholeskyQR -- factor
    // G + s I with s = f trace(G), f from m 2^-52 up by factors of 100.  Y
    // R^{-1} is then well conditioned but not orthonormal; the caller runs
    // one more pass (shifted CholeskyQR3).  Y = (Y R^{-1}) R holds exactly
    // whatever the shift.
    for (double f = m * 0x1p-52; info != 0 && shifted && f < 1e-4; f *= 100.0) {
        *shifted = true;
        {
            ProfScope psc(c, PROF_CHOL);
            launch_shift_diag(c->stream, m, G, f);
            chol_upper(c, m, G, R);
            launch_trinv_upper(c->stream, m, R, Rinv);
            WC4D_TRY(check_launch(c, "shifted cholqr"));
            WC4D_CUDA(c, cudaMemcpyAsync(&info, c->counter.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        }
        WC4D_TRY(sync(c, "shifted cholqr info"));
        if (info < 0) return set_err(c, WC4D_ETIMEOUT, "Cholesky: a grid barrier timed out");
    }
    if (info != 0) return set_err(c, WC4D_ENOTSPD, "CholeskyQR: Gram matrix not positive definite at pivot %d", info);
    ProfScope psl(c, PROF_LA);
    Epi e{0, 1.0, 0.0, 0.0, 1};
    if constexpr (sizeof(T) == 8) {
        launch_gemm<double>(c->stream, (int)rows, m, m, Y, 1, ld, Rinv, m, tmp, rows, e);
    } else {
        if (!tall_product_tc(c, rows, m, m, Y, ld, Rinv, m, tmp, rows)) {
            float *Rinv32 = reinterpret_cast<float *>(G);   // G is no longer needed
            launch_convert_f64_f32(c->stream, (int64_t)mm, Rinv, Rinv32);
            launch_gemm<float>(c->stream, (int)rows, m, m, Y, 1, ld, Rinv32, m, tmp, rows, e);
        }
    }
    WC4D_TRY(check_launch(c, "cholqr gemm"));
    WC4D_CUDA(c, cudaMemcpy2DAsync(Y, sizeof(T) * ld, tmp, sizeof(T) * rows, sizeof(T) * rows, m,
                                   cudaMemcpyDeviceToDevice, c->stream));
    if constexpr (sizeof(T) == 4) launch_unscale_R(c->stream, m, R, rs_work);   // R of the unscaled Y
    return WC4D_OK;
}

// CholeskyQR2: Y = Z R with orthonormal Z (in place), R = R2 R1 (device, m x m).
template <typename T>
static wc4d_status cholqr2(wc4d_ctx *c, T *Y, int64_t rows, int m, int64_t ld, T *tmp, double *R)
{
    const size_t mm = (size_t)m * m;
    WC4D_TRY(ensure(c, c->small2, sizeof(double) * mm * 3));
    double *R1 = P<double>(c->small2), *R2 = R1 + mm, *R3 = R2 + mm;
    bool shifted = false;
    WC4D_TRY(cholqr_pass<T>(c, Y, rows, m, ld, tmp, R1, &shifted));
    WC4D_TRY(cholqr_pass<T>(c, Y, rows, m, ld, tmp, R2, &shifted));
    if (shifted) WC4D_TRY(cholqr_pass<T>(c, Y, rows, m, ld, tmp, R3));   // shifted CholeskyQR3
    if (R) {
        Epi e{0, 1.0, 0.0, 0.0, 1};
        if (shifted) {   // R = R3 R2 R1
            launch_gemm<double>(c->stream, m, m, m, R3, 1, m, R2, m, R, m, e);
            launch_gemm<double>(c->stream, m, m, m, R, 1, m, R1, m, R3, m, e);
            WC4D_CUDA(c, cudaMemcpyAsync(R, R3, sizeof(double) * mm, cudaMemcpyDeviceToDevice, c->stream));
        } else {
            launch_gemm<double>(c->stream, m, m, m, R2, 1, m, R1, m, R, m, e);   // R = R2 R1
        }
        WC4D_TRY(check_launch(c, "R2R1"));
    }
    return WC4D_OK;
}

// One-sided Jacobi in FP64 on X0 (m x m, device): X0 V = U Sigma.  m <= 256
// runs as one persistent cooperative launch; larger m (or a refused
// cooperative launch) as one launch per round of the round-robin ordering.
// On return *X holds U Sigma and *V the accumulated rotations, both with
// leading dimension *ld (columns in the order of X0).
static wc4d_status jacobi_run(wc4d_ctx *c, int m, const double *X0, double **Xo, double **Vo, int *ld,
                              bool want_v = true)
{
    const int mp = m + (m & 1);
    const double tol = 4.0 * 2.220446049250313e-16 * std::sqrt((double)mp);
    c->jacobi_sweeps32 = 0;
    c->jacobi_kernel32 = 0;
    if (const int Pq = c->allow_coop ? jacobi_coop_size(m) : 0) {
        // Without V (the left singular vectors only): an FP32 pre-rotation
        // phase first.  One-sided Jacobi in FP32 (about 1.6 FP64 operations
        // per clock per SM make the FP64 rounds several times dearer) runs
        // until a sweep's largest rotation has |cos| <= 1e-4; its accumulated
        // V is made orthogonal to FP64 rounding (two Newton-Schulz steps) and
        // X0 V -- the same left singular vectors and singular values, columns
        // orthogonal to ~1e-6 -- goes to the FP64 solve, which then needs one
        // or two sweeps.  Any failure of the FP32 phase leaves X0 as it is.
        if (!want_v) {
            const size_t P2 = (size_t)Pq * Pq, mm = (size_t)m * m;
            const size_t fbytes = sizeof(float) * 4 * P2, dbytes = sizeof(double) * (P2 + 3 * mm + 8);
            const size_t ibytes = sizeof(int) * 128 + sizeof(unsigned long long) * 64;
            if (ensure(c, c->jq32, fbytes + dbytes + ibytes) == WC4D_OK) {
                float *XV32 = P<float>(c->jq32);
                double *V64 = reinterpret_cast<double *>(P<char>(c->jq32) + fbytes);
                double *X1 = V64 + P2, *tmp = X1 + mm, *scale = tmp + 2 * mm;
                int *rot = reinterpret_cast<int *>(scale + 8);
                unsigned *bar = reinterpret_cast<unsigned *>(rot + 64);
                int *err = rot + 65, *status = rot + 66;
                unsigned long long *maxm = reinterpret_cast<unsigned long long *>(rot + 128);
                WC4D_CUDA(c, cudaMemsetAsync(err, 0, sizeof(int), c->stream));
                // one 16-CTA cluster (V written to XV32 + P^2); else the cooperative form
                const bool on_cluster =
                    launch_jacobi_cluster_f32(c->stream, m, X0, XV32 + P2, 1e-6, 30, status, 1e-8, scale);
                if (on_cluster || launch_jacobi_coop_f32(c->stream, m, X0, XV32, 1e-6, 30, rot, bar, err, status,
                                                         1e-8, maxm, scale)) {
                    int *h = P<int>(c->pinned);
                    WC4D_CUDA(c, cudaMemcpyAsync(h, err, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
                    WC4D_TRY(sync(c, "jacobi fp32 phase"));
                    if (h[0] == 0) {
                        c->jacobi_kernel32 = on_cluster ? 1 : 2;
                        launch_convert_f32_f64(c->stream, (int64_t)P2, XV32 + P2, V64);     // V (ld P)
                        launch_orthogonalise_ns(c->stream, m, V64, Pq, tmp);
                        launch_small_gemm64(c->stream, m, X0, m, false, V64, Pq, X1, m, 1.0, 0.0);   // X0 V
                        WC4D_TRY(check_launch(c, "jacobi fp32 phase"));
                        c->jacobi_sweeps32 = h[1];
                        X0 = X1;
                    }
                }
            }
        }
        const size_t nd = jacobi_coop_doubles(m);
        // XV | rot[64] | bar, err, status | maxm[64] (64-bit words)
        WC4D_TRY(ensure(c, c->small3, sizeof(double) * nd + sizeof(int) * 128 + sizeof(unsigned long long) * 64));
        double *XV = P<double>(c->small3);
        int *rot = reinterpret_cast<int *>(XV + nd);
        unsigned *bar = reinterpret_cast<unsigned *>(rot + 64);
        int *err = rot + 65;
        int *status = rot + 66;
        unsigned long long *maxm = reinterpret_cast<unsigned long long *>(rot + 128);
        WC4D_CUDA(c, cudaMemsetAsync(err, 0, sizeof(int), c->stream));
        if (launch_jacobi_coop(c->stream, m, X0, XV, tol, 60, rot, bar, err, status, want_v, c->jacobi_stop2, maxm)) {
            int *h = P<int>(c->pinned);
            WC4D_CUDA(c, cudaMemcpyAsync(h, err, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
            WC4D_TRY(sync(c, "jacobi"));
            if (h[0]) return set_err(c, WC4D_ETIMEOUT, "Jacobi: a grid barrier timed out");
            if (h[1] < 0) return set_err(c, WC4D_ETIMEOUT, "one-sided Jacobi did not converge in 60 sweeps");
            c->jacobi_sweeps = h[1];
            *Xo = XV;
            *Vo = XV + (size_t)Pq * Pq;
            *ld = Pq;
            return WC4D_OK;
        }
    }
    size_t mpmp = (size_t)mp * mp;
    DevBuf &xb = c->small3;
    WC4D_TRY(ensure(c, xb, sizeof(double) * mpmp * 2));
    double *X = P<double>(xb), *V = X + mpmp;
    launch_jacobi_init(c->stream, m, mp, X0, X, V);
    WC4D_TRY(check_launch(c, "jacobi init"));
    if (mp >= 2) {
        int *rot = P<int>(c->counter) + 1;
        int *hrot = P<int>(c->pinned);
        bool conv = false;
        for (int sweep = 0; sweep < 60; ++sweep) {
            WC4D_CUDA(c, cudaMemsetAsync(rot, 0, sizeof(int), c->stream));
            for (int r = 0; r < mp - 1; ++r) launch_jacobi_round(c->stream, mp, X, V, r, tol, rot);
            WC4D_TRY(check_launch(c, "jacobi round"));
            WC4D_CUDA(c, cudaMemcpyAsync(hrot, rot, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
            WC4D_TRY(sync(c, "jacobi sweep"));
            if (*hrot == 0) { conv = true; c->jacobi_sweeps = sweep + 1; break; }
        }
        if (!conv) return set_err(c, WC4D_ETIMEOUT, "one-sided Jacobi did not converge in 60 sweeps");
    }
    *Xo = X;
    *Vo = V;
    *ld = mp;
    return WC4D_OK;
}

// SVD by one-sided Jacobi: w (device, 2m doubles) receives the singular
// values of X0 decreasing in w[0..m), Vout (m x m) the matching right
// singular vectors.  For symmetric positive semi-definite X0 these are its
// eigenvalues and eigenvectors.
static wc4d_status jacobi_svd(wc4d_ctx *c, int m, const double *X0, double *w, double *Vout)
{
    ProfScope ps(c, PROF_JACOBI);
    double *X, *V;
    int ld;
    WC4D_TRY(jacobi_run(c, m, X0, &X, &V, &ld));
    launch_jacobi_finish(c->stream, m, ld, X, V, w, Vout);
    return check_launch(c, "jacobi finish");
}

// Eigenpairs of a symmetric positive definite S (m x m, device): with
// S = R^T R (Cholesky), one-sided Jacobi on R^T gives R^T = U Sigma V^T,
// so S = U Sigma^2 U^T.  w receives Sigma^2 decreasing, Vout the matching U.
// The Cholesky factor's columns are far closer to orthogonal than S's own
// (about half the Jacobi sweeps on the sketch matrices).  Falls back to
// Jacobi on S when S is not numerically positive definite.
static wc4d_status spd_evd(wc4d_ctx *c, int m, const double *S, double *w, double *Vout)
{
    DevBuf &rb = c->evd_r;
    WC4D_TRY(ensure(c, rb, sizeof(double) * 2 * (size_t)m * m));
    double *R = P<double>(rb), *RT = R + (size_t)m * m;
    int info = 0;
    {
        ProfScope psc(c, PROF_CHOL);
        chol_upper(c, m, S, R);
        launch_rrt(c->stream, m, R, RT);
        wc4d_status st = check_launch(c, "spd_evd chol");
        if (st != WC4D_OK) return st;
        cudaMemcpyAsync(&info, c->counter.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    }
    wc4d_status st = sync(c, "spd_evd chol");
    if (st == WC4D_OK && info < 0) return set_err(c, WC4D_ETIMEOUT, "Cholesky: a grid barrier timed out");
    if (st == WC4D_OK && info == 0) {
        ProfScope ps(c, PROF_JACOBI);
        double *X, *V;
        int ld;
        st = jacobi_run(c, m, RT, &X, &V, &ld, false);
        if (st == WC4D_OK) {
            launch_jacobi_finish_left(c->stream, m, ld, X, w, Vout);
            st = check_launch(c, "jacobi finish");
        }
    } else if (st == WC4D_OK) {
        st = jacobi_svd(c, m, S, w, Vout);
    }
    return st;
}

extern "C" wc4d_status wc4d_orthonormalize(wc4d_ctx *c, void *Y, int64_t rows, int32_t m, int64_t ld, double *R_host,
                                           int32_t precision)
{
    if (!c || !Y || rows < m || m < 1 || ld < rows) return WC4D_EINVAL;
    if (precision != WC4D_FP64 && precision != WC4D_MIXED) return WC4D_EINVAL;
    const size_t esz = (precision == WC4D_FP64) ? sizeof(double) : sizeof(float);
    WC4D_TRY(ensure(c, c->blkD, esz * (size_t)rows * m));
    WC4D_TRY(ensure(c, c->small1, sizeof(double) * (size_t)m * m));
    DevBuf Rb;
    double *R = nullptr;
    if (R_host) {
        WC4D_TRY(ensure(c, Rb, sizeof(double) * (size_t)m * m));
        R = P<double>(Rb);
    }
    wc4d_status s = (precision == WC4D_FP64)
                        ? cholqr2<double>(c, static_cast<double *>(Y), rows, m, ld, P<double>(c->blkD), R)
                        : cholqr2<float>(c, static_cast<float *>(Y), rows, m, ld, P<float>(c->blkD), R);
    if (s == WC4D_OK && R_host) {
        cudaMemcpyAsync(R_host, R, sizeof(double) * (size_t)m * m, cudaMemcpyDeviceToHost, c->stream);
        s = sync(c, "orthonormalize");
    }
    free_buf(Rb);
    return s;
}

extern "C" wc4d_status wc4d_symeig(wc4d_ctx *c, int32_t m, const double *S, double *w_host, double *V)
{
    if (!c || !S || !w_host || !V || m < 1) return WC4D_EINVAL;
    DevBuf wb;
    WC4D_TRY(ensure(c, wb, sizeof(double) * 2 * m));
    wc4d_status s = jacobi_svd(c, m, S, P<double>(wb), V);
    if (s == WC4D_OK) {
        cudaMemcpyAsync(w_host, wb.p, sizeof(double) * m, cudaMemcpyDeviceToHost, c->stream);
        s = sync(c, "symeig");
    }
    free_buf(wb);
    return s;
}

// Pieces of the orthonormalisation and Rayleigh-Ritz steps of Alg. 3-5 for
// callers that distribute the rows of a block over several devices and sum
// the partial Gram matrices themselves (the column-sharded sketch).
extern "C" wc4d_status wc4d_gram(wc4d_ctx *c, const void *A, int64_t lda, const void *B, int64_t ldb, int64_t rows,
                                 int32_t ma, int32_t mb, double *C, int32_t precision)
{
    if (!c || !A || !B || !C || rows < 1 || ma < 1 || mb < 1 || lda < rows || ldb < rows) return WC4D_EINVAL;
    if (precision != WC4D_FP64 && precision != WC4D_MIXED) return WC4D_EINVAL;
    const size_t need = atb_part_doubles(c->num_sms, rows, ma, mb, 0);
    WC4D_TRY(ensure(c, c->part, sizeof(double) * need));
    int S = 0;
    ProfScope ps(c, PROF_GRAM);
    int r;
    if (precision == WC4D_FP64)
        r = launch_atb<double>(c->stream, c->num_sms, rows, ma, mb, static_cast<const double *>(A), lda,
                               static_cast<const double *>(B), ldb, P<double>(c->part), c->part.bytes / 8, &S, C, 0);
    else
        r = launch_atb<float>(c->stream, c->num_sms, rows, ma, mb, static_cast<const float *>(A), lda,
                              static_cast<const float *>(B), ldb, P<double>(c->part), c->part.bytes / 8, &S, C, 0);
    if (r != 0) return set_err(c, WC4D_EINVAL, "internal: Gram partial buffer too small");
    return check_launch(c, "gram");
}

extern "C" wc4d_status wc4d_gram_sym(wc4d_ctx *c, const void *A, int64_t lda, const void *B, int64_t ldb, int64_t rows,
                                     int32_t m, double *C, int32_t precision)
{
    if (!c || !A || !B || !C || rows < 1 || m < 1 || lda < rows || ldb < rows) return WC4D_EINVAL;
    if (precision != WC4D_FP64 && precision != WC4D_MIXED) return WC4D_EINVAL;
    WC4D_TRY(ensure(c, c->part, sizeof(double) * atb_part_doubles(c->num_sms, rows, m, m, 1)));
    int S = 0, r;
    {
        ProfScope ps(c, PROF_GRAM);
        if (precision == WC4D_FP64)
            r = gram_sym<double>(c, rows, m, static_cast<const double *>(A), lda, static_cast<const double *>(B), ldb,
                                 C, &S);
        else
            r = gram_sym<float>(c, rows, m, static_cast<const float *>(A), lda, static_cast<const float *>(B), ldb, C,
                                &S);
    }
    if (r != 0) return set_err(c, WC4D_EINVAL, "internal: Gram partial buffer too small");
    WC4D_TRY(check_launch(c, "gram_sym"));
    WC4D_TRY(sync(c, "gram_sym"));
    WC4D_TRY(pending_wait_error(c));
    return WC4D_OK;
}

extern "C" wc4d_status wc4d_chol_inverse(wc4d_ctx *c, int32_t m, const double *G, double *Rinv)
{
    if (!c || !G || !Rinv || m < 1) return WC4D_EINVAL;
    WC4D_TRY(ensure(c, c->small1, sizeof(double) * (size_t)m * m));
    double *R = P<double>(c->small1);
    int info = 0;
    {
        ProfScope psc(c, PROF_CHOL);
        chol_upper(c, m, G, R);
        launch_trinv_upper(c->stream, m, R, Rinv);
        WC4D_TRY(check_launch(c, "chol_inverse"));
        WC4D_CUDA(c, cudaMemcpyAsync(&info, c->counter.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    }
    WC4D_TRY(sync(c, "chol_inverse"));
    if (info < 0) return set_err(c, WC4D_ETIMEOUT, "Cholesky: a grid barrier timed out");
    if (info != 0) return set_err(c, WC4D_ENOTSPD, "Cholesky: matrix not positive definite at pivot %d", info);
    return WC4D_OK;
}

extern "C" wc4d_status wc4d_tall_times_small(wc4d_ctx *c, const void *Y, int64_t ldy, int64_t rows, int32_t m,
                                             const double *W, int32_t k, void *Z, int64_t ldz, int32_t precision)
{
    if (!c || !Y || !W || !Z || rows < 1 || m < 1 || k < 1 || ldy < rows || ldz < rows) return WC4D_EINVAL;
    if (rows > INT32_MAX) return set_err(c, WC4D_EINVAL, "tall_times_small: more than 2^31 - 1 rows");
    if (precision != WC4D_FP64 && precision != WC4D_MIXED) return WC4D_EINVAL;
    ProfScope psl(c, PROF_LA);
    Epi e{0, 1.0, 0.0, 0.0, 1};
    if (precision == WC4D_FP64) {
        launch_gemm<double>(c->stream, (int)rows, k, m, static_cast<const double *>(Y), 1, ldy, W, m,
                            static_cast<double *>(Z), ldz, e);
    } else {
        WC4D_TRY(ensure(c, c->small3, sizeof(float) * (size_t)m * k));
        float *W32 = P<float>(c->small3);
        launch_convert_f64_f32(c->stream, (int64_t)m * k, W, W32);
        launch_gemm<float>(c->stream, (int)rows, k, m, static_cast<const float *>(Y), 1, ldy, W32, m,
                           static_cast<float *>(Z), ldz, e);
    }
    return check_launch(c, "tall_times_small");
}

// ============================================================================
// Randomised eigensolvers (Section 4)
// ============================================================================
template <typename T>
static wc4d_status sketch_impl(wc4d_ctx *c, int method, int k, int l, int q, uint64_t seed, const double *Gdev)
{
    const int m = k + l;
    const int64_t nA = c->nA;
    const size_t blk = sizeof(T) * (size_t)nA * m;
    WC4D_TRY(ensure(c, c->blkA, blk));
    WC4D_TRY(ensure(c, c->blkB, blk));
    WC4D_TRY(ensure(c, c->blkC, blk));
    WC4D_TRY(ensure(c, c->blkD, std::max(blk, sizeof(double) * (size_t)nA * m)));
    WC4D_TRY(ensure(c, c->theta64, sizeof(double) * 2 * m));
    const size_t mm = (size_t)m * m;
    DevBuf &kb = c->sk_k, &wb = c->sk_w, &Rb = c->sk_r;
    WC4D_TRY(ensure(c, kb, sizeof(double) * mm * 2));
    WC4D_TRY(ensure(c, wb, sizeof(double) * 2 * m));
    WC4D_TRY(ensure(c, Rb, sizeof(double) * mm));
    double *Kmat = P<double>(kb), *Wv = Kmat + mm, *w = P<double>(wb), *R = P<double>(Rb);
    T *A_ = P<T>(c->blkA), *B_ = P<T>(c->blkB), *C_ = P<T>(c->blkC), *D_ = P<T>(c->blkD);
    wc4d_status st = WC4D_OK;
    auto fail = [&](wc4d_status s) { return s; };
    // Mixed sketch: the small FP64 eigensolves stop after a sweep whose
    // largest rotation had |cos| <= 1e-5 (columns then orthogonal to about
    // 1e-10, far below the TF32 error of the sketch products) instead of
    // running a last sweep that only confirms convergence.
    struct StopGuard {
        wc4d_ctx *c;
        ~StopGuard() { c->jacobi_stop2 = 0.0; }
    } stop_guard{c};
    c->jacobi_stop2 = (sizeof(T) == 4) ? 1e-10 : 0.0;

    // step 1: Gaussian probes G in the working precision (given probes are
    // FP64 and cast; the mixed path draws its own in FP32 arithmetic)
    double *G64 = P<double>(c->blkD);
    if constexpr (sizeof(T) == 8) {
        if (Gdev) WC4D_CUDA(c, cudaMemcpyAsync(A_, Gdev, blk, cudaMemcpyDeviceToDevice, c->stream));
        else launch_gaussian(c->stream, seed, nA, m, nA, (double *)A_);
    } else if (Gdev) {
        WC4D_CUDA(c, cudaMemcpyAsync(G64, Gdev, sizeof(double) * nA * m, cudaMemcpyDeviceToDevice, c->stream));
        launch_convert_f64_f32(c->stream, nA * m, G64, (float *)A_);
    } else {
        launch_gaussian_f32(c->stream, seed, nA, m, nA, (float *)A_);
    }
    if ((st = check_launch(c, "probes")) != WC4D_OK) return fail(st);

    // U (nA x k) in the working precision, theta in c->theta64
    T *U = nullptr;
    if (method == WC4D_REVD || method == WC4D_NYSTROM) {
        // Y = A G; Z = orth(Y)  (+ q power iterations for REVD)
        if ((st = hvp_impl<T>(c, A_, B_, m, nA)) != WC4D_OK) return fail(st);
        // A basis of span(A G) that only feeds the power iteration needs one
        // CholeskyQR pass; the basis used for Rayleigh-Ritz gets two.
        if (method == WC4D_REVD && q > 0) {
            WC4D_TRY(ensure(c, c->small2, sizeof(double) * mm));
            bool shifted = false;   // a well-conditioned basis suffices here
            if ((st = cholqr_pass<T>(c, B_, nA, m, nA, D_, P<double>(c->small2), &shifted)) != WC4D_OK)
                return fail(st);
        } else if ((st = cholqr2<T>(c, B_, nA, m, nA, D_, nullptr)) != WC4D_OK) {
            return fail(st);
        }
        T *Z = B_, *Y = A_;
        if (method == WC4D_REVD)
            for (int it = 0; it < q; ++it) {
                if ((st = hvp_impl<T>(c, Z, Y, m, nA)) != WC4D_OK) return fail(st);
                if ((st = cholqr2<T>(c, Y, nA, m, nA, D_, nullptr)) != WC4D_OK) return fail(st);
                std::swap(Z, Y);
            }
        // E = A Z
        T *E = Y;
        if ((st = hvp_impl<T>(c, Z, E, m, nA)) != WC4D_OK) return fail(st);
        if ((st = ensure(c, c->part, sizeof(double) * atb_part_doubles(c->num_sms, nA, m, m, 1))) != WC4D_OK)
            return fail(st);
        int S = 0;
        {
            // Z^T A Z is symmetric: upper tiles only, mirrored
            ProfScope psg(c, PROF_GRAM);
            if (gram_sym<T>(c, nA, m, Z, nA, E, nA, Kmat, &S) != 0)
                return fail(set_err(c, WC4D_EINVAL, "internal: Gram partial buffer too small"));
        }
        launch_symmetrize(c->stream, m, Kmat);
        if ((st = check_launch(c, "ZtAZ")) != WC4D_OK) return fail(st);
        if (method == WC4D_REVD) {
            // EVD of K_1 (Alg. 3 step 5); U = Z W[:, :k]
            if ((st = spd_evd(c, m, Kmat, w, Wv)) != WC4D_OK) return fail(st);
            U = C_;
            ProfScope psl(c, PROF_LA);
            Epi e{0, 1.0, 0.0, 0.0, 1};
            if constexpr (sizeof(T) == 8) {
                launch_gemm<double>(c->stream, (int)nA, k, m, Z, 1, nA, Wv, m, U, nA, e);
            } else {
                // FP32 pipe: the LMP needs the Ritz vectors orthonormal to
                // FP32 rounding (their loss of orthonormality is amplified by
                // the largest Ritz values); the 3xTF32 product cost ~12 %
                // more CG iterations on the n = 4096, N = 40 window
                float *W32 = reinterpret_cast<float *>(Kmat);
                launch_convert_f64_f32(c->stream, (int64_t)mm, Wv, W32);
                launch_gemm<float>(c->stream, (int)nA, k, m, Z, 1, nA, W32, m, U, nA, e);
            }
            WC4D_CUDA(c, cudaMemcpyAsync(P<double>(c->theta64), w, sizeof(double) * k, cudaMemcpyDeviceToDevice,
                                         c->stream));
        } else {
            // Nystrom (Alg. 4): E2 = C^T C; F = E1 C^{-1}; F = U Sigma V^T
            double *Cc = R;
            chol_upper(c, m, Kmat, Cc);
            int info = 0;
            WC4D_CUDA(c, cudaMemcpyAsync(&info, c->counter.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
            if ((st = sync(c, "nystrom chol")) != WC4D_OK) return fail(st);
            if (info < 0) return fail(set_err(c, WC4D_ETIMEOUT, "Cholesky: a grid barrier timed out"));
            if (info) return fail(set_err(c, WC4D_ENOTSPD, "Nystrom: Z^T A Z not positive definite (pivot %d)", info));
            launch_trinv_upper(c->stream, m, Cc, Wv);              // Wv = C^{-1}
            T *F = C_;
            Epi e{0, 1.0, 0.0, 0.0, 1};
            if constexpr (sizeof(T) == 8) {
                launch_gemm<double>(c->stream, (int)nA, m, m, E, 1, nA, Wv, m, F, nA, e);
            } else {
                float *Ci32 = reinterpret_cast<float *>(Kmat);
                launch_convert_f64_f32(c->stream, (int64_t)mm, Wv, Ci32);
                launch_gemm<float>(c->stream, (int)nA, m, m, E, 1, nA, Ci32, m, F, nA, e);
            }
            if (gram_sym<T>(c, nA, m, F, nA, F, nA, Kmat, &S) != 0)   // F^T F
                return fail(set_err(c, WC4D_EINVAL, "internal: Gram partial buffer too small"));
            launch_symmetrize(c->stream, m, Kmat);
            if ((st = check_launch(c, "nystrom F")) != WC4D_OK) return fail(st);
            if ((st = spd_evd(c, m, Kmat, w, Wv)) != WC4D_OK) return fail(st);   // F^T F = V Sigma^2 V^T
            // U = F V[:, :k] Sigma^{-1}
            U = E;
            if constexpr (sizeof(T) == 8) {
                launch_gemm<double>(c->stream, (int)nA, k, m, F, 1, nA, Wv, m, U, nA, e);
                launch_scale_cols(c->stream, nA, k, (double *)U, nA, w, 1);
            } else {
                float *V32 = reinterpret_cast<float *>(Kmat);
                launch_convert_f64_f32(c->stream, (int64_t)mm, Wv, V32);
                launch_gemm<float>(c->stream, (int)nA, k, m, F, 1, nA, V32, m, U, nA, e);
                // scale in FP64 via a temporary copy
                double *U64t = reinterpret_cast<double *>(c->blkD.p);
                launch_convert_f32_f64(c->stream, nA * k, (const float *)U, U64t);
                launch_scale_cols(c->stream, nA, k, U64t, nA, w, 1);
                launch_convert_f64_f32(c->stream, nA * k, U64t, (float *)U);
            }
            WC4D_CUDA(c, cudaMemcpyAsync(P<double>(c->theta64), w, sizeof(double) * k, cudaMemcpyDeviceToDevice,
                                         c->stream));   // Theta = Sigma^2 (eigenvalues of F^T F)
        }
    } else if (method == WC4D_NYSTROM1) {
        // Single-pass Nystrom (Tropp, Yurtsever, Udell, Cevher 2017; named as
        // future work in Section 6): Omega = orth(G); Y = A Omega (the only
        // product with A); Y_nu = Y + nu Omega; Omega^T Y_nu = C^T C;
        // E = Y_nu C^{-1} = U Sigma V^T; Theta = max(Sigma^2 - nu, 0).
        T *Om = A_, *Yb = B_;
        if ((st = cholqr2<T>(c, Om, nA, m, nA, D_, nullptr)) != WC4D_OK) return fail(st);
        if ((st = hvp_impl<T>(c, Om, Yb, m, nA)) != WC4D_OK) return fail(st);
        // nu = scale ||Y||_F: sqrt(n_A) 2^-52 in FP64 (Tropp et al.), in the mixed
        // path 2^-22 (FP32 storage of Y rounds each entry by up to 2^-24)
        const int gridn = std::min<int64_t>(2 * c->num_sms, std::max<int64_t>(1, (nA * m + 255) / 256));
        WC4D_TRY(ensure(c, c->small1, sizeof(double) * 4 * 1024));
        launch_dot_partial<T>(c->stream, gridn, nA * m, Yb, Yb, P<double>(c->small1));
        std::vector<double> hp(gridn);
        WC4D_CUDA(c, cudaMemcpyAsync(hp.data(), c->small1.p, sizeof(double) * gridn, cudaMemcpyDeviceToHost,
                                     c->stream));
        if ((st = sync(c, "nystrom1 norm")) != WC4D_OK) return fail(st);
        double yy = 0.0;
        for (double v : hp) yy += v;
        const double nu = ((sizeof(T) == 8) ? std::sqrt((double)nA) * 0x1p-52 : 0x1p-22) * std::sqrt(yy);
        launch_axpy_block<T>(c->stream, c->num_sms, nA * m, nu, Om, Yb);                  // Y_nu
        if ((st = ensure(c, c->part, sizeof(double) * atb_part_doubles(c->num_sms, nA, m, m, 1))) != WC4D_OK)
            return fail(st);
        int S = 0;
        {
            ProfScope psg(c, PROF_GRAM);
            if (gram_sym<T>(c, nA, m, Om, nA, Yb, nA, Kmat, &S) != 0)   // Omega^T Y_nu, symmetric up to rounding: upper tiles
                return fail(set_err(c, WC4D_EINVAL, "internal: Gram partial buffer too small"));
        }
        launch_symmetrize(c->stream, m, Kmat);
        double *Cc = R;
        chol_upper(c, m, Kmat, Cc);
        int info = 0;
        WC4D_CUDA(c, cudaMemcpyAsync(&info, c->counter.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        if ((st = sync(c, "nystrom1 chol")) != WC4D_OK) return fail(st);
        if (info < 0) return fail(set_err(c, WC4D_ETIMEOUT, "Cholesky: a grid barrier timed out"));
        if (info)
            return fail(set_err(c, WC4D_ENOTSPD, "single-pass Nystrom: Omega^T Y_nu not positive definite (pivot %d)",
                                info));
        launch_trinv_upper(c->stream, m, Cc, Wv);              // Wv = C^{-1}
        T *E = C_;
        Epi e{0, 1.0, 0.0, 0.0, 1};
        if constexpr (sizeof(T) == 8) {
            launch_gemm<double>(c->stream, (int)nA, m, m, Yb, 1, nA, Wv, m, E, nA, e);
        } else {
            float *Ci32 = reinterpret_cast<float *>(Kmat);
            launch_convert_f64_f32(c->stream, (int64_t)mm, Wv, Ci32);
            launch_gemm<float>(c->stream, (int)nA, m, m, Yb, 1, nA, Ci32, m, E, nA, e);
        }
        if (gram_sym<T>(c, nA, m, E, nA, E, nA, Kmat, &S) != 0)   // E^T E
            return fail(set_err(c, WC4D_EINVAL, "internal: Gram partial buffer too small"));
        launch_symmetrize(c->stream, m, Kmat);
        if ((st = check_launch(c, "nystrom1 E")) != WC4D_OK) return fail(st);
        if ((st = spd_evd(c, m, Kmat, w, Wv)) != WC4D_OK) return fail(st);   // E^T E = V Sigma^2 V^T
        // U = E V[:, :k] Sigma^{-1}
        U = Yb;
        if constexpr (sizeof(T) == 8) {
            launch_gemm<double>(c->stream, (int)nA, k, m, E, 1, nA, Wv, m, U, nA, e);
            launch_scale_cols(c->stream, nA, k, (double *)U, nA, w, 1);
        } else {
            float *V32 = reinterpret_cast<float *>(Kmat);
            launch_convert_f64_f32(c->stream, (int64_t)mm, Wv, V32);
            launch_gemm<float>(c->stream, (int)nA, k, m, E, 1, nA, V32, m, U, nA, e);
            double *U64t = reinterpret_cast<double *>(c->blkD.p);
            launch_convert_f32_f64(c->stream, nA * k, (const float *)U, U64t);
            launch_scale_cols(c->stream, nA, k, U64t, nA, w, 1);
            launch_convert_f64_f32(c->stream, nA * k, U64t, (float *)U);
        }
        launch_theta_unshift(c->stream, k, w, nu, P<double>(c->theta64));          // Theta = max(Sigma^2 - nu, 0)
    } else {
        // REVD_ritzit (Alg. 5): G_3 = orth(G); Y_3 = A G_3 = Z_3 R_3; K_3 = R_3 R_3^T
        if ((st = cholqr2<T>(c, A_, nA, m, nA, D_, nullptr)) != WC4D_OK) return fail(st);
        if ((st = hvp_impl<T>(c, A_, B_, m, nA)) != WC4D_OK) return fail(st);
        if ((st = cholqr2<T>(c, B_, nA, m, nA, D_, R)) != WC4D_OK) return fail(st);
        // left singular vectors of R_3 = eigenvectors of R_3 R_3^T: one-sided Jacobi on R_3^T
        launch_rrt(c->stream, m, R, Kmat);
        if ((st = check_launch(c, "R^T")) != WC4D_OK) return fail(st);
        if ((st = jacobi_svd(c, m, Kmat, w, Wv)) != WC4D_OK) return fail(st);   // singular values = Theta_3
        U = C_;
        ProfScope psl(c, PROF_LA);
        Epi e{0, 1.0, 0.0, 0.0, 1};
        if constexpr (sizeof(T) == 8) {
            launch_gemm<double>(c->stream, (int)nA, k, m, B_, 1, nA, Wv, m, U, nA, e);
        } else {
            float *W32 = reinterpret_cast<float *>(Kmat);
            launch_convert_f64_f32(c->stream, (int64_t)mm, Wv, W32);
            launch_gemm<float>(c->stream, (int)nA, k, m, B_, 1, nA, W32, m, U, nA, e);
        }
        WC4D_CUDA(c, cudaMemcpyAsync(P<double>(c->theta64), w, sizeof(double) * k, cudaMemcpyDeviceToDevice,
                                     c->stream));
    }
    if ((st = check_launch(c, "ritz vectors")) != WC4D_OK) return fail(st);
    // keep U in both precisions
    WC4D_TRY(ensure(c, c->U64, sizeof(double) * (size_t)nA * k));
    WC4D_TRY(ensure(c, c->U32, sizeof(float) * (size_t)nA * k));
    if constexpr (sizeof(T) == 8) {
        WC4D_CUDA(c, cudaMemcpyAsync(c->U64.p, U, sizeof(double) * nA * k, cudaMemcpyDeviceToDevice, c->stream));
        launch_convert_f64_f32(c->stream, nA * k, (const double *)U, P<float>(c->U32));
    } else {
        WC4D_CUDA(c, cudaMemcpyAsync(c->U32.p, U, sizeof(float) * nA * k, cudaMemcpyDeviceToDevice, c->stream));
        launch_convert_f32_f64(c->stream, nA * k, (const float *)U, P<double>(c->U64));
    }
    WC4D_TRY(ensure(c, c->c64, sizeof(double) * k));
    launch_lmp_coeffs(c->stream, k, P<double>(c->theta64), P<double>(c->c64));
    if ((st = check_launch(c, "lmp coeffs")) != WC4D_OK) return fail(st);
    c->kU = k;
    c->theta_host.assign(k, 0.0);
    cudaMemcpyAsync(c->theta_host.data(), c->theta64.p, sizeof(double) * k, cudaMemcpyDeviceToHost, c->stream);
    WC4D_TRY(sync(c, "sketch"));
    WC4D_TRY(pending_wait_error(c));
    return WC4D_OK;
}

// Row-major, zero-padded copies of the Ritz vectors for the LMP kernels.
static wc4d_status build_rowmajor_U(wc4d_ctx *c)
{
    const int k = c->kU, kp = (k + 3) / 4 * 4;
    const int64_t nA = c->nA;
    WC4D_TRY(ensure(c, c->Urm64, sizeof(double) * (size_t)nA * kp));
    WC4D_TRY(ensure(c, c->Urm32, sizeof(float) * (size_t)nA * kp));
    launch_to_rowmajor<double>(c->stream, nA, k, kp, P<double>(c->U64), P<double>(c->Urm64));
    launch_to_rowmajor<float>(c->stream, nA, k, kp, P<float>(c->U32), P<float>(c->Urm32));
    c->kp = kp;
    return check_launch(c, "row-major U");
}

extern "C" wc4d_status wc4d_sketch(wc4d_ctx *c, int32_t method, int32_t k, int32_t l, int32_t q, uint64_t seed,
                                   const double *G, double *theta_host, int32_t precision)
{
    if (!c || k < 1 || l < 0 || q < 0 || method < 0 || method > 3) return WC4D_EINVAL;
    if (k + l > 1024 || k + l > c->nA) return set_err(c, WC4D_EINVAL, "k + l = %d too large", k + l);
    if (precision != WC4D_FP64 && precision != WC4D_MIXED) return WC4D_EINVAL;
    WC4D_TRY(require_operator(c));
    WC4D_TRY(prep_precision(c, precision));
    wc4d_status s = (precision == WC4D_FP64) ? sketch_impl<double>(c, method, k, l, q, seed, G)
                                             : sketch_impl<float>(c, method, k, l, q, seed, G);
    if (s != WC4D_OK) return s;
    WC4D_TRY(build_rowmajor_U(c));
    if (theta_host) std::memcpy(theta_host, c->theta_host.data(), sizeof(double) * k);
    return sync(c, "sketch");
}

extern "C" wc4d_status wc4d_get_ritz(wc4d_ctx *c, double *U, double *theta_host)
{
    if (!c) return WC4D_EINVAL;
    if (c->kU == 0) return set_err(c, WC4D_ESTATE, "no Ritz pairs");
    if (U) WC4D_CUDA(c, cudaMemcpyAsync(U, c->U64.p, sizeof(double) * c->nA * c->kU, cudaMemcpyDeviceToDevice,
                                        c->stream));
    if (theta_host) std::memcpy(theta_host, c->theta_host.data(), sizeof(double) * c->kU);
    return sync(c, "get_ritz");
}

extern "C" wc4d_status wc4d_set_ritz(wc4d_ctx *c, int32_t k, const double *U, const double *theta_host)
{
    if (!c || k < 0 || (k > 0 && (!U || !theta_host))) return WC4D_EINVAL;
    if (k == 0) { c->kU = 0; return WC4D_OK; }
    const int64_t nA = c->nA;
    WC4D_TRY(ensure(c, c->U64, sizeof(double) * (size_t)nA * k));
    WC4D_TRY(ensure(c, c->U32, sizeof(float) * (size_t)nA * k));
    WC4D_TRY(ensure(c, c->theta64, sizeof(double) * 2 * k));
    WC4D_TRY(ensure(c, c->c64, sizeof(double) * k));
    WC4D_CUDA(c, cudaMemcpyAsync(c->U64.p, U, sizeof(double) * nA * k, cudaMemcpyDeviceToDevice, c->stream));
    launch_convert_f64_f32(c->stream, nA * k, P<double>(c->U64), P<float>(c->U32));
    WC4D_CUDA(c, cudaMemcpyAsync(c->theta64.p, theta_host, sizeof(double) * k, cudaMemcpyHostToDevice, c->stream));
    launch_lmp_coeffs(c->stream, k, P<double>(c->theta64), P<double>(c->c64));
    WC4D_TRY(check_launch(c, "set_ritz"));
    c->kU = k;
    c->theta_host.assign(theta_host, theta_host + k);
    WC4D_TRY(build_rowmajor_U(c));
    return sync(c, "set_ritz");
}

// ============================================================================
// Spectral LMP (eq. 16) and PCG (Alg. 1)
// ============================================================================
template <typename T> static T *Urm(wc4d_ctx *c);
template <> double *Urm<double>(wc4d_ctx *c) { return P<double>(c->Urm64); }
template <> float *Urm<float>(wc4d_ctx *c) { return P<float>(c->Urm32); }
template <typename T> static T *Ucm(wc4d_ctx *c);   // column-major Ritz vectors, ld nA
template <> double *Ucm<double>(wc4d_ctx *c) { return P<double>(c->U64); }
template <> float *Ucm<float>(wc4d_ctx *c) { return P<float>(c->U32); }

// y = C v (C^T = C for the closed form); skip: optional device flag
template <typename T>
static wc4d_status lmp_apply_impl(wc4d_ctx *c, const T *v, T *y, const int *skip)
{
    const int k = c->kU;
    const int64_t nA = c->nA;
    ProfScope ps(c, PROF_LMP);
    const int kp = c->kp;
    int splits = utv_rm_splits(nA);
    WC4D_TRY(ensure(c, c->part, sizeof(double) * ((size_t)splits * kp + kp) + 64));
    launch_utv_rm<T>(c->stream, nA, kp, Urm<T>(c), v, P<double>(c->part), &splits);
    // the reduced t = U^T v sits after the partials
    launch_lmp_combine_rm<T>(c->stream, c->num_sms, nA, k, kp, Urm<T>(c), P<double>(c->part) + (size_t)splits * kp,
                             P<double>(c->c64), v, y, skip);
    return check_launch(c, "lmp apply");
}

extern "C" wc4d_status wc4d_lmp_apply(wc4d_ctx *c, const double *v, double *y, int32_t transpose)
{
    (void)transpose;   // C is symmetric in the closed form
    if (!c || !v || !y) return WC4D_EINVAL;
    if (c->kU == 0) {
        WC4D_CUDA(c, cudaMemcpyAsync(y, v, sizeof(double) * c->nA, cudaMemcpyDeviceToDevice, c->stream));
        return WC4D_OK;
    }
    return lmp_apply_impl<double>(c, v, y, nullptr);
}

struct PcgOut {
    int iters = 0;
    int breakdown = 0;
    bool done = false;
    double relres_rec = 0.0;
};

// The LMP half of one CG iteration after q = A p (alpha; x += alpha p,
// r -= alpha q; rhat -= alpha C q; t = C rhat; beta), fused into two passes
// over the Ritz vectors.  qcf_dev may be null.
template <typename T>
static wc4d_status lmp_cg_step(wc4d_ctx *c, T *x, T *r, T *rh, const T *p, const T *q, T *t, double tol_k,
                               double *qcf_dev)
{
    const int64_t nA = c->nA;
    const int kp = c->kp;
    const int S = lmp_pass_a_splits(nA, c->num_sms), G = std::max(S, lmp_pass_b_grid(nA));   // second-pass CTAs
    WC4D_TRY(ensure(c, c->part, sizeof(double) * ((size_t)S * (2 * kp + 1))));
    WC4D_TRY(ensure(c, c->small2, sizeof(double) * (4 * (size_t)kp + 1 + 2 * (size_t)G)));
    double *w = P<double>(c->small2), *partB = w + 4 * kp + 1;
    double *scal = P<double>(c->scal);
    int *flags = P<int>(c->counter) + 4;
    unsigned *done = reinterpret_cast<unsigned *>(P<int>(c->counter) + 8);
    ProfScope ps(c, PROF_LMP);
    launch_lmp_fused<T>(c->stream, c->num_sms, nA, c->kU, kp, Urm<T>(c), Ucm<T>(c), P<double>(c->c64), q, p, rh, t,
                        x, r, scal, flags, P<double>(c->part), w, partB, done, tol_k, qcf_dev);
    return WC4D_OK;
}

// CG on A x = b from x = 0 in precision T; b, x device vectors of the context.
template <typename T>
static wc4d_status pcg_core(wc4d_ctx *c, const T *b, T *x, double tol, int maxit, int force, bool use_lmp,
                            double *qcf_dev, PcgOut &out)
{
    const int64_t nA = c->nA;
    DevBuf *vb = (sizeof(T) == 8) ? c->pcg64 : c->pcg32;
    for (int i = 1; i < 6; ++i) WC4D_TRY(ensure(c, vb[i], sizeof(T) * nA));
    T *r = P<T>(vb[1]), *rh = P<T>(vb[2]), *p = P<T>(vb[3]), *q = P<T>(vb[4]), *t = P<T>(vb[5]);
    const int grid = std::min<int64_t>(2 * c->num_sms, std::max<int64_t>(1, (nA + 255) / 256));
    WC4D_TRY(ensure(c, c->small1, sizeof(double) * 4 * 1024));
    double *pa = P<double>(c->small1), *pb = pa + 1024, *pc = pb + 1024;
    double *scal = P<double>(c->scal);
    int *flags = P<int>(c->counter) + 4;
    const bool lmp = use_lmp && c->kU > 0;

    WC4D_CUDA(c, cudaMemsetAsync(x, 0, sizeof(T) * nA, c->stream));
    launch_copy<T>(c->stream, nA, b, r);                                    // r_0 = b
    if (lmp) WC4D_TRY(lmp_apply_impl<T>(c, r, rh, nullptr));                // rhat_0 = C^T r_0
    else launch_copy<T>(c->stream, nA, r, rh);
    if (lmp) WC4D_TRY(lmp_apply_impl<T>(c, rh, p, nullptr));                // p_0 = C rhat_0
    else launch_copy<T>(c->stream, nA, rh, p);
    launch_dot_partial<T>(c->stream, grid, nA, b, b, pa);
    launch_dot_partial<T>(c->stream, grid, nA, rh, rh, pb);
    launch_pcg_init(c->stream, grid, pa, pb, scal, flags);
    WC4D_TRY(check_launch(c, "pcg init"));
    int *hflags = P<int>(c->pinned);
    const double tol_k = (force > 0) ? 0.0 : tol;
    const int nit = (force > 0) ? force : maxit;
    out = PcgOut();
    IterGraph graph;
    auto body = [&]() -> wc4d_status {
        WC4D_TRY(hvp_impl<T>(c, p, q, 1, nA, false));                       // q = A p
        if (lmp) {
            WC4D_TRY(lmp_cg_step<T>(c, x, r, rh, p, q, t, tol_k, qcf_dev));
            launch_pcg_p<T>(c->stream, grid, nA, scal, p, t);               // p = C rhat + beta p
        } else {
            launch_dot_partial<T>(c->stream, grid, nA, p, q, pa);
            launch_pcg_alpha(c->stream, grid, pa, scal, flags);             // alpha = rho / p^T A p
            launch_pcg_xr<T>(c->stream, grid, nA, scal, x, r, p, q, pb);    // x += alpha p; r -= alpha q
            launch_pcg_rh<T>(c->stream, grid, nA, scal, rh, q, pc);         // rhat -= alpha A p
            launch_pcg_beta(c->stream, grid, pc, pb, scal, flags, tol_k, qcf_dev);
            launch_pcg_p<T>(c->stream, grid, nA, scal, p, rh);              // p = rhat + beta p
        }
        return check_launch(c, "pcg iteration");
    };
    LoopGraph loop;
    for (int it = 0; it < nit;) {
        if (it > 0 && build_loop(c, loop, body, nit, false)) {   // the remaining iterations on the device
            double hrel_unused;
            WC4D_TRY(run_loop(c, loop, nit - it, it, hflags, &hrel_unused, &it));
            break;
        }
        WC4D_TRY(run_iteration(c, graph, it, body));
        WC4D_CUDA(c, cudaMemcpyAsync(hflags, flags, sizeof(int) * 3, cudaMemcpyDeviceToHost, c->stream));
        WC4D_TRY(sync(c, "pcg iteration"));
        ++it;
        if (hflags[0]) break;
    }
    c->iter_mode = loop.exec ? 2 : graph.exec ? 1 : 0;
    double hs[8];
    WC4D_CUDA(c, cudaMemcpyAsync(hflags, flags, sizeof(int) * 3, cudaMemcpyDeviceToHost, c->stream));
    WC4D_CUDA(c, cudaMemcpyAsync(hs, scal, sizeof(double) * 8, cudaMemcpyDeviceToHost, c->stream));
    WC4D_TRY(sync(c, "pcg end"));
    out.done = hflags[0] != 0;
    if (const int e = sweep_error(c)) return set_err(c, WC4D_ETIMEOUT, "persistent sweep failed (code %d)", e);
    WC4D_TRY(pending_wait_error(c));
    out.breakdown = hflags[1];
    out.iters = hflags[2];
    out.relres_rec = hs[4];
    return WC4D_OK;
}

// FP64 true relative residual |rhs - A x| / |rhs|; r64 receives rhs - A x.
static wc4d_status true_residual(wc4d_ctx *c, const double *x, double *r64, double *rel, double *bnorm_out,
                                 bool df = false)
{
    const int64_t nA = c->nA;
    WC4D_TRY(ensure(c, c->pcg64[6], sizeof(double) * nA));
    double *Ax = P<double>(c->pcg64[6]);
    {
        // df (the mixed CG): the one-column sweeps of this product in
        // double-float (48-bit propagators, ~2^-44 sums), FP64 accuracy at
        // the HBM rate; the FP64 path keeps FP64 arithmetic
        struct DfScope {
            wc4d_ctx *c;
            DfScope(wc4d_ctx *ctx, bool on) : c(ctx) { c->sweep_df = on && c->prob.model == WC4D_MODEL_DENSE; }
            ~DfScope() { c->sweep_df = false; }
        } df_scope(c, df);
        WC4D_TRY(hvp_impl<double>(c, x, Ax, 1, nA, false));
    }
    launch_sub_f64(c->stream, nA, P<double>(c->rhs), Ax, r64);
    const int grid = std::min<int64_t>(2 * c->num_sms, std::max<int64_t>(1, (nA + 255) / 256));
    WC4D_TRY(ensure(c, c->small0, sizeof(double) * 2048));
    double *pa = P<double>(c->small0), *pb = pa + 1024;
    launch_dot_partial<double>(c->stream, grid, nA, r64, r64, pa);
    launch_dot_partial<double>(c->stream, grid, nA, P<double>(c->rhs), P<double>(c->rhs), pb);
    WC4D_TRY(check_launch(c, "true residual"));
    std::vector<double> h(2 * grid);
    WC4D_CUDA(c, cudaMemcpyAsync(h.data(), pa, sizeof(double) * grid, cudaMemcpyDeviceToHost, c->stream));
    WC4D_CUDA(c, cudaMemcpyAsync(h.data() + grid, pb, sizeof(double) * grid, cudaMemcpyDeviceToHost, c->stream));
    WC4D_TRY(sync(c, "true residual"));
    double rr = 0.0, bb = 0.0;
    for (int i = 0; i < grid; ++i) { rr += h[i]; bb += h[grid + i]; }
    // non-finite sums give a non-finite relative residual (a zero rhs gives 0)
    *rel = !(std::isfinite(rr) && std::isfinite(bb)) ? std::nan("") : (bb > 0.0 ? std::sqrt(rr / bb) : 0.0);
    if (bnorm_out) *bnorm_out = std::sqrt(bb);
    return WC4D_OK;
}

// Mixed-precision CG with reliable updates (Sleijpen and van der Vorst,
// "Reliable updated residuals in hybrid Bi-CG methods", Computing 56, 1996):
// the recurrences of Alg. 1 run in FP32 on a correction d.  When the
// recurrence residual has fallen by kReliableDelta since the last update, or
// claims convergence, the FP64 solution absorbs d (x += d, d = 0) and the
// FP32 residual is replaced by the FP64 true residual rhs - A x, while the
// search direction p is kept.  Unlike restarted refinement this keeps the
// Krylov space, so the iteration count stays close to the FP64 solver's.
// The factor (default 1e-3) is c->reliable_delta (wc4d_set_reliable_delta).

static wc4d_status pcg_reliable(wc4d_ctx *c, double *x, double tol, int maxit, int force, bool use_lmp,
                                double *qcf_dev, int *iters_out, double *rel_out, bool *breakdown_out)
{
    const int64_t nA = c->nA;
    DevBuf *vb = c->pcg32;
    for (int i = 0; i < 6; ++i) WC4D_TRY(ensure(c, vb[i], sizeof(float) * nA));
    WC4D_TRY(ensure(c, c->pcg64[7], sizeof(double) * nA));
    float *d = P<float>(vb[0]), *r = P<float>(vb[1]), *rh = P<float>(vb[2]), *p = P<float>(vb[3]);
    float *q = P<float>(vb[4]), *t = P<float>(vb[5]);
    double *r64 = P<double>(c->pcg64[7]);
    const int grid = std::min<int64_t>(2 * c->num_sms, std::max<int64_t>(1, (nA + 255) / 256));
    WC4D_TRY(ensure(c, c->small1, sizeof(double) * 4 * 1024));
    double *pa = P<double>(c->small1), *pb = pa + 1024, *pc = pb + 1024;
    double *scal = P<double>(c->scal);
    int *flags = P<int>(c->counter) + 4;
    const bool lmp = use_lmp && c->kU > 0;
    int *hflags = P<int>(c->pinned);
    double *hrel = reinterpret_cast<double *>(P<char>(c->pinned) + 64);

    // x = 0, d = 0, r = rhs; rhat = C^T r, p = C rhat
    WC4D_CUDA(c, cudaMemsetAsync(x, 0, sizeof(double) * nA, c->stream));
    WC4D_CUDA(c, cudaMemsetAsync(d, 0, sizeof(float) * nA, c->stream));
    launch_convert_f64_f32(c->stream, nA, P<double>(c->rhs), r);
    auto precondition_residual = [&]() -> wc4d_status {
        if (lmp) {
            WC4D_TRY(lmp_apply_impl<float>(c, r, rh, nullptr));
            WC4D_TRY(lmp_apply_impl<float>(c, rh, p, nullptr));
        } else {
            launch_copy<float>(c->stream, nA, r, rh);
            launch_copy<float>(c->stream, nA, rh, p);
        }
        return WC4D_OK;
    };
    WC4D_TRY(precondition_residual());
    launch_dot_partial<double>(c->stream, grid, nA, P<double>(c->rhs), P<double>(c->rhs), pa);
    launch_dot_partial<float>(c->stream, grid, nA, rh, rh, pb);
    launch_pcg_init(c->stream, grid, pa, pb, scal, flags);
    WC4D_TRY(check_launch(c, "pcg init"));
    WC4D_CUDA(c, cudaMemcpyAsync(hflags, flags, sizeof(int) * 3, cudaMemcpyDeviceToHost, c->stream));
    WC4D_TRY(sync(c, "pcg init"));
    const bool init_bad = hflags[1] != 0;   // non-finite rhs: a breakdown, no iteration
    double rel = init_bad ? std::nan("") : (hflags[0] ? 0.0 : 1.0);   // |rhs| = 0: x = 0 is exact
    double rmax = rel;
    bool converged = (force == 0 && rel <= tol), breakdown = init_bad, pending = false;
    const double tol_k = (force > 0) ? 0.0 : tol;
    const int nit = init_bad ? 0 : ((force > 0) ? force : maxit);
    int it = 0;
    IterGraph graph;
    auto body = [&]() -> wc4d_status {
        WC4D_TRY(hvp_impl<float>(c, p, q, 1, nA, false));                    // q = A p
        if (lmp) {
            WC4D_TRY(lmp_cg_step<float>(c, d, r, rh, p, q, t, tol_k, qcf_dev));
            ProfScope ps(c, PROF_VEC);
            launch_pcg_p<float>(c->stream, grid, nA, scal, p, t);            // p = C rhat + beta p
        } else {
            ProfScope ps(c, PROF_VEC);
            launch_dot_partial<float>(c->stream, grid, nA, p, q, pa);
            launch_pcg_alpha(c->stream, grid, pa, scal, flags);              // alpha = rho / p^T A p
            launch_pcg_xr<float>(c->stream, grid, nA, scal, d, r, p, q, pb); // d += alpha p; r -= alpha q
            launch_pcg_rh<float>(c->stream, grid, nA, scal, rh, q, pc);      // rhat -= alpha A p
            launch_pcg_beta(c->stream, grid, pc, pb, scal, flags, tol_k, qcf_dev);
            launch_pcg_p<float>(c->stream, grid, nA, scal, p, rh);           // p = rhat + beta p
        }
        return check_launch(c, "pcg iteration");
    };
    LoopGraph loop;
    for (; it < nit && !converged; ++it) {
        const double thresh = c->reliable_delta * rmax;
        if (it > 0 && build_loop(c, loop, body, nit, true)) {
            // iterations on the device until an update is due, CG ends or the limit
            double *hth = reinterpret_cast<double *>(P<char>(c->pinned) + 192);
            *hth = thresh;
            WC4D_CUDA(c, cudaMemcpyAsync(scal + 8, hth, sizeof(double), cudaMemcpyHostToDevice, c->stream));
            int after = it;
            WC4D_TRY(run_loop(c, loop, nit - it, it, hflags, hrel, &after));
            it = after - 1;   // the loop's ++it makes it the device count
        } else {
            WC4D_TRY(run_iteration(c, graph, it, body));
            WC4D_CUDA(c, cudaMemcpyAsync(hflags, flags, sizeof(int) * 3, cudaMemcpyDeviceToHost, c->stream));
            WC4D_CUDA(c, cudaMemcpyAsync(hrel, scal + 4, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
            WC4D_TRY(sync(c, "pcg iteration"));
        }
        pending = true;
        if (hflags[1]) { breakdown = true; ++it; break; }
        if (!(hflags[0] || *hrel < thresh)) continue;
        // reliable update
        launch_add_f32_to_f64(c->stream, nA, d, x);
        WC4D_CUDA(c, cudaMemsetAsync(d, 0, sizeof(float) * nA, c->stream));
        pending = false;
        WC4D_TRY(true_residual(c, x, r64, &rel, nullptr, true));
        rmax = rel;
        if (force == 0 && rel <= tol) { converged = true; ++it; break; }
        launch_convert_f64_f32(c->stream, nA, r64, r);
        if (lmp) WC4D_TRY(lmp_apply_impl<float>(c, r, rh, nullptr));
        else launch_copy<float>(c->stream, nA, r, rh);
        launch_dot_partial<float>(c->stream, grid, nA, rh, rh, pb);
        launch_dot_partial<float>(c->stream, grid, nA, r, r, pc);
        launch_pcg_restart(c->stream, grid, pb, pc, scal, flags);
        WC4D_TRY(check_launch(c, "reliable update"));
    }
    c->iter_mode = loop.exec ? 2 : graph.exec ? 1 : 0;
    if (pending) {   // iteration budget spent (or breakdown) between updates
        launch_add_f32_to_f64(c->stream, nA, d, x);
        WC4D_TRY(true_residual(c, x, r64, &rel, nullptr, true));
    }
    if (const int e = sweep_error(c)) return set_err(c, WC4D_ETIMEOUT, "persistent sweep failed (code %d)", e);
    WC4D_TRY(pending_wait_error(c));
    *iters_out = it;
    *rel_out = rel;
    *breakdown_out = breakdown;
    return WC4D_OK;
}

// ============================================================================
// Ritz pairs from CG (Section 3.3): the deterministic LMP of the previous
// inner loop.  FP64 CG without a preconditioner (Alg. 1 with C = I) keeps
// alpha_j, beta_j and the normalised residuals as Lanczos vectors
// f_j = (-1)^j r_j / |r_j|, optionally reorthogonalised against all previous
// f (classical Gram-Schmidt, twice; the complete reorthogonalisation the
// paper cites against ghost values).  The tridiagonal T_J of eq. 18-20 is
// then formed on the host, its eigenpairs come from the FP64 one-sided
// Jacobi of the sketches, and u_i = F_J w_i.
// ============================================================================
extern "C" wc4d_status wc4d_lanczos_cg(wc4d_ctx *c, double *x, double tol, int32_t maxit, int32_t reorth,
                                       int32_t *iters_out, double *relres_out)
{
    if (!c || !x || maxit < 1) return WC4D_EINVAL;
    if (!c->have_rhs) return set_err(c, WC4D_ESTATE, "rhs not set (call wc4d_set_background_obs)");
    WC4D_TRY(require_operator(c));
    const int64_t nA = c->nA;
    DevBuf *vb = c->pcg64;
    for (int i = 1; i < 6; ++i) WC4D_TRY(ensure(c, vb[i], sizeof(double) * nA));
    double *r = P<double>(vb[1]), *rh = P<double>(vb[2]), *p = P<double>(vb[3]), *q = P<double>(vb[4]);
    const int cap = maxit + 1;
    WC4D_TRY(ensure(c, c->lz_F, sizeof(double) * (size_t)nA * cap));
    WC4D_TRY(ensure(c, c->lz_ab, sizeof(double) * 2 * (size_t)maxit));
    WC4D_TRY(ensure(c, c->lz_h, sizeof(double) * (size_t)cap));
    double *F = P<double>(c->lz_F), *ab = P<double>(c->lz_ab), *h = P<double>(c->lz_h);
    const int grid = std::min<int64_t>(2 * c->num_sms, std::max<int64_t>(1, (nA + 255) / 256));
    WC4D_TRY(ensure(c, c->small1, sizeof(double) * 4 * 1024));
    double *pa = P<double>(c->small1), *pb = pa + 1024, *pc = pb + 1024;
    double *scal = P<double>(c->scal);
    int *flags = P<int>(c->counter) + 4;
    const double *b = P<double>(c->rhs);
    c->lz_J = 0;

    WC4D_CUDA(c, cudaMemsetAsync(x, 0, sizeof(double) * nA, c->stream));
    launch_copy<double>(c->stream, nA, b, r);
    launch_copy<double>(c->stream, nA, r, rh);
    launch_copy<double>(c->stream, nA, rh, p);
    launch_dot_partial<double>(c->stream, grid, nA, b, b, pa);
    launch_dot_partial<double>(c->stream, grid, nA, rh, rh, pb);
    launch_pcg_init(c->stream, grid, pa, pb, scal, flags);
    launch_lanczos_first(c->stream, grid, nA, b, scal, F);
    WC4D_TRY(check_launch(c, "lanczos cg init"));
    int *hflags = P<int>(c->pinned);
    int it = 0;
    for (; it < maxit; ++it) {
        WC4D_TRY(hvp_impl<double>(c, p, q, 1, nA, false));                   // q = A p
        launch_dot_partial<double>(c->stream, grid, nA, p, q, pa);
        launch_pcg_alpha(c->stream, grid, pa, scal, flags);                  // alpha = rho / p^T A p
        launch_pcg_xr<double>(c->stream, grid, nA, scal, x, r, p, q, pb);    // x += alpha p; r -= alpha q
        if (reorth) {
            // r -= F_{0..j} (F_{0..j}^T r), twice
            const int cols = it + 1;
            const size_t need = atb_part_doubles(c->num_sms, nA, cols, 1, 0);
            WC4D_TRY(ensure(c, c->part, sizeof(double) * need));
            for (int pass = 0; pass < 2; ++pass) {
                if (launch_atb<double>(c->stream, c->num_sms, nA, cols, 1, F, nA, r, nA, P<double>(c->part),
                                       c->part.bytes / 8, nullptr, h, 0) != 0)
                    return set_err(c, WC4D_EINVAL, "internal: partial buffer too small");
                Epi e{0, -1.0, 1.0, 0.0, 1};
                launch_gemm<double>(c->stream, (int)nA, 1, cols, F, 1, nA, h, cols, r, nA, e);
            }
            launch_copy<double>(c->stream, nA, r, rh);
            launch_dot_partial<double>(c->stream, grid, nA, r, r, pb);
            launch_dot_partial<double>(c->stream, grid, nA, rh, rh, pc);
        } else {
            launch_pcg_rh<double>(c->stream, grid, nA, scal, rh, q, pc);     // rhat -= alpha A p (= r)
        }
        launch_pcg_beta(c->stream, grid, pc, pb, scal, flags, tol, nullptr);
        launch_lanczos_record(c->stream, grid, nA, r, scal, flags, F, ab, cap);
        launch_pcg_p<double>(c->stream, grid, nA, scal, p, rh);              // p = r + beta p
        WC4D_TRY(check_launch(c, "lanczos cg iteration"));
        WC4D_CUDA(c, cudaMemcpyAsync(hflags, flags, sizeof(int) * 3, cudaMemcpyDeviceToHost, c->stream));
        WC4D_TRY(sync(c, "lanczos cg iteration"));
        if (hflags[1]) return set_err(c, WC4D_EBREAKDOWN, "Lanczos CG: breakdown at iteration %d", it + 1);
        if (hflags[0]) { ++it; break; }
    }
    double hs[8];
    WC4D_CUDA(c, cudaMemcpyAsync(hflags, flags, sizeof(int) * 3, cudaMemcpyDeviceToHost, c->stream));
    WC4D_CUDA(c, cudaMemcpyAsync(hs, scal, sizeof(double) * 8, cudaMemcpyDeviceToHost, c->stream));
    WC4D_TRY(sync(c, "lanczos cg end"));
    if (const int e = sweep_error(c)) return set_err(c, WC4D_ETIMEOUT, "persistent sweep failed (code %d)", e);
    WC4D_TRY(pending_wait_error(c));
    c->lz_J = hflags[2];
    if (iters_out) *iters_out = hflags[2];
    if (relres_out) *relres_out = hs[4];
    return WC4D_OK;
}

// gamma (J) and tau (J - 1) of T_J (eq. 19-20) from the recorded alpha, beta.
static wc4d_status lanczos_tridiag_host(wc4d_ctx *c, std::vector<double> &gam, std::vector<double> &tau)
{
    const int J = c->lz_J;
    if (J < 1) return set_err(c, WC4D_ESTATE, "no Lanczos data (call wc4d_lanczos_cg)");
    std::vector<double> ab(2 * (size_t)J);
    WC4D_CUDA(c, cudaMemcpyAsync(ab.data(), c->lz_ab.p, sizeof(double) * 2 * J, cudaMemcpyDeviceToHost, c->stream));
    WC4D_TRY(sync(c, "lanczos coefficients"));
    gam.assign(J, 0.0);
    tau.assign(J > 1 ? J - 1 : 0, 0.0);
    for (int j = 0; j < J; ++j) {
        const double al = ab[2 * j];
        gam[j] = 1.0 / al + (j > 0 ? ab[2 * (j - 1) + 1] / ab[2 * (j - 1)] : 0.0);
        if (j + 1 < J) tau[j] = std::sqrt(ab[2 * j + 1]) / al;
    }
    return WC4D_OK;
}

extern "C" wc4d_status wc4d_lanczos_tridiag(wc4d_ctx *c, double *gamma_host, double *tau_host)
{
    if (!c || !gamma_host) return WC4D_EINVAL;
    std::vector<double> gam, tau;
    WC4D_TRY(lanczos_tridiag_host(c, gam, tau));
    std::copy(gam.begin(), gam.end(), gamma_host);
    if (tau_host) std::copy(tau.begin(), tau.end(), tau_host);
    return WC4D_OK;
}

extern "C" wc4d_status wc4d_lanczos_ritz(wc4d_ctx *c, int32_t k, double *theta_host)
{
    if (!c || k < 1) return WC4D_EINVAL;
    std::vector<double> gam, tau;
    WC4D_TRY(lanczos_tridiag_host(c, gam, tau));
    const int J = c->lz_J;
    if (k > J) return set_err(c, WC4D_EINVAL, "lanczos_ritz: k = %d exceeds the %d CG iterations", k, J);
    const int64_t nA = c->nA;
    const size_t JJ = (size_t)J * J;
    std::vector<double> T(JJ, 0.0);   // column-major, symmetric
    for (int j = 0; j < J; ++j) {
        T[(size_t)j * J + j] = gam[j];
        if (j + 1 < J) T[(size_t)j * J + j + 1] = T[(size_t)(j + 1) * J + j] = tau[j];
    }
    WC4D_TRY(ensure(c, c->sk_k, sizeof(double) * JJ * 2));
    WC4D_TRY(ensure(c, c->sk_w, sizeof(double) * 2 * J));
    double *Td = P<double>(c->sk_k), *V = Td + JJ, *w = P<double>(c->sk_w);
    WC4D_CUDA(c, cudaMemcpyAsync(Td, T.data(), sizeof(double) * JJ, cudaMemcpyHostToDevice, c->stream));
    {
        ProfScope ps(c, PROF_JACOBI);
        WC4D_TRY(spd_evd(c, J, Td, w, V));   // T_J = W Theta W^T, decreasing
    }
    WC4D_TRY(ensure(c, c->blkC, sizeof(double) * (size_t)nA * k));
    double *U = P<double>(c->blkC);
    Epi e{0, 1.0, 0.0, 0.0, 1};
    launch_gemm<double>(c->stream, (int)nA, k, J, P<double>(c->lz_F), 1, nA, V, J, U, nA, e);   // u_i = F_J w_i
    WC4D_TRY(check_launch(c, "lanczos ritz vectors"));
    std::vector<double> th(k);
    WC4D_CUDA(c, cudaMemcpyAsync(th.data(), w, sizeof(double) * k, cudaMemcpyDeviceToHost, c->stream));
    WC4D_TRY(sync(c, "lanczos ritz values"));
    if (theta_host) std::copy(th.begin(), th.end(), theta_host);
    return wc4d_set_ritz(c, k, U, th.data());
}

extern "C" wc4d_status wc4d_pcg(wc4d_ctx *c, double *x, double tol, int32_t maxit, int32_t use_lmp, int32_t force,
                                int32_t precision, int32_t *iters, double *relres, double *qcf_host)
{
    if (!c || !x || maxit < 0 || force < 0) return WC4D_EINVAL;
    if (precision != WC4D_FP64 && precision != WC4D_MIXED) return WC4D_EINVAL;
    if (!c->have_rhs) return set_err(c, WC4D_ESTATE, "rhs not set (call wc4d_set_background_obs)");
    WC4D_TRY(require_operator(c));
    WC4D_TRY(prep_precision(c, precision));
    const int64_t nA = c->nA;
    const int cap = std::max(1, std::max(maxit, force));
    DevBuf &qcf = c->qcf;
    WC4D_TRY(ensure(c, qcf, sizeof(double) * cap));
    WC4D_CUDA(c, cudaMemsetAsync(qcf.p, 0, sizeof(double) * cap, c->stream));
    wc4d_status st = WC4D_OK;
    int total_it = 0;
    bool breakdown = false;
    double rel = 0.0;
    if (precision == WC4D_FP64) {
        PcgOut o;
        st = pcg_core<double>(c, P<double>(c->rhs), x, tol, maxit, force, use_lmp != 0, P<double>(qcf), o);
        if (st == WC4D_OK) {
            total_it = o.iters;
            breakdown = o.breakdown != 0;
            WC4D_TRY(ensure(c, c->pcg64[7], sizeof(double) * nA));
            st = true_residual(c, x, P<double>(c->pcg64[7]), &rel, nullptr);
        }
    } else {
        st = pcg_reliable(c, x, tol, maxit, force, use_lmp != 0, P<double>(qcf), &total_it, &rel, &breakdown);
    }
    if (st == WC4D_OK && qcf_host) {
        cudaMemcpyAsync(qcf_host, qcf.p, sizeof(double) * std::min(cap, std::max(total_it, 0)),
                        cudaMemcpyDeviceToHost, c->stream);
        st = sync(c, "qcf");
    }
    if (st != WC4D_OK) return st;
    if (iters) *iters = total_it;
    if (relres) *relres = rel;
    if (breakdown) return set_err(c, WC4D_EBREAKDOWN, "CG breakdown: p^T A p <= 0 or non-finite");
    if (!std::isfinite(rel)) return set_err(c, WC4D_ENAN, "non-finite residual");
    if (force == 0 && rel > tol) return set_err(c, WC4D_ENOCONV, "CG: relres %.3e > tol after %d iterations", rel,
                                                total_it);
    return WC4D_OK;
}

extern "C" wc4d_status wc4d_inner_loop(wc4d_ctx *c, int32_t method, int32_t k, int32_t l, int32_t q, uint64_t seed,
                                       double tol, int32_t maxit, int32_t precision, double *x, int32_t *iters,
                                       double *relres)
{
    WC4D_TRY(wc4d_sketch(c, method, k, l, q, seed, nullptr, nullptr, precision));
    return wc4d_pcg(c, x, tol, maxit, 1, 0, precision, iters, relres, nullptr);
}
