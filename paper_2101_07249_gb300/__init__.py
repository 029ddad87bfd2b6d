"""GB300-native inner loop of forcing-formulation weak-constraint 4D-Var with
randomised spectral-LMP preconditioning.

All arithmetic runs in libwc4d.so (hand-written CUDA for sm_103a, C-ABI in
include/wc4d.h).  This module is its thin ctypes binding: the functions keep
the C names and only marshal arguments (torch CUDA tensors -> device
pointers, numpy arrays -> host pointers).  A block of K control vectors is a
torch tensor of shape (K, nA): row j is vector j, i.e. the column-major
nA x K matrix of the C-ABI with leading dimension nA.

There is no CPU fallback: if the library cannot be loaded every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import inputs  # noqa: F401  (seeded synthetic inputs; no method arithmetic)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwc4d.so")

OK, EINVAL, ENOMEM, ECUDA, ENOTSPD, EBREAKDOWN, ENOCONV, ETIMEOUT, ENAN, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9
FP64, MIXED = 0, 1
REVD, NYSTROM, RITZIT, NYSTROM1 = 0, 1, 2, 3
MODEL_DENSE, MODEL_L96 = 0, 1
CORR_SOAR, CORR_GAUSS, CORR_DIAG = 0, 1, 2
METHODS = {"revd": REVD, "nystrom": NYSTROM, "ritzit": RITZIT, "nystrom1": NYSTROM1}
_STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENOTSPD", -5: "EBREAKDOWN",
           -6: "ENOCONV", -7: "ETIMEOUT", -8: "ENAN", -9: "ESTATE"}


class WC4DError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"wc4d status {_STATUS.get(status, status)}: {msg}")
        self.status = status


class Problem(C.Structure):
    """wc4d_problem (include/wc4d.h)."""
    _fields_ = [("n", C.c_int32), ("N", C.c_int32), ("model", C.c_int32), ("steps", C.c_int32),
                ("dt", C.c_double), ("F", C.c_double), ("sigma_o2", C.c_double),
                ("obs_stride", C.c_int32), ("obs_t0", C.c_int32), ("obs_tstride", C.c_int32),
                ("M_shared", C.c_int32)]


_V = C.c_void_p
_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_SIGS = {
    "wc4d_create": (C.c_int, [C.POINTER(_V), C.POINTER(Problem), _V]),
    "wc4d_destroy": (None, [_V]),
    "wc4d_last_error": (C.c_char_p, [_V]),
    "wc4d_set_stream": (C.c_int, [_V, _V]),
    "wc4d_set_propagator": (C.c_int, [_V, C.c_int32, _V]),
    "wc4d_build_advdiff_propagator": (C.c_int, [_V, C.c_double, C.c_double, C.c_double, C.c_int32]),
    "wc4d_set_covariance": (C.c_int, [_V, C.c_int32, C.c_int32, C.c_double, C.c_double]),
    "wc4d_set_covariance_row": (C.c_int, [_V, C.c_int32, _D]),
    "wc4d_set_cov_sqrt": (C.c_int, [_V, C.c_int32, C.c_int32, _V]),
    "wc4d_get_problem": (C.c_int, [_V, C.c_void_p]),
    "wc4d_set_trajectory": (C.c_int, [_V, _V]),
    "wc4d_set_innovation": (C.c_int, [_V, _V, _V]),
    "wc4d_set_background_obs": (C.c_int, [_V, _D, _D, _D]),
    "wc4d_outer_update": (C.c_int, [_V, _V]),
    "wc4d_learned_probes": (C.c_int, [_V, _V, _V, C.c_int32, _V, C.c_int64]),
    "wc4d_batch_inner_loop": (C.c_int, [_V, C.c_int32, C.c_int32, _V, _V, C.c_int32, _V, C.c_double, C.c_int32,
                                        C.c_int32, _V, _V, _V, _V, C.c_int32]),
    "wc4d_nobs": (C.c_int64, [_V]),
    "wc4d_control_dim": (C.c_int64, [_V]),
    "wc4d_ritz_count": (C.c_int32, [_V]),
    "wc4d_get_rhs": (C.c_int, [_V, _V]),
    "wc4d_hvp": (C.c_int, [_V, _V, _V, C.c_int32, C.c_int64, C.c_int32]),
    "wc4d_gaussian": (C.c_int, [_V, C.c_uint64, C.c_int64, C.c_int32, C.c_int64, _V]),
    "wc4d_gaussian_f32": (C.c_int32, [_V, C.c_uint64, C.c_int64, C.c_int32, C.c_int64, _V]),
    "wc4d_sketch": (C.c_int, [_V, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, _V, _D, C.c_int32]),
    "wc4d_get_ritz": (C.c_int, [_V, _V, _D]),
    "wc4d_set_ritz": (C.c_int, [_V, C.c_int32, _V, _D]),
    "wc4d_lmp_apply": (C.c_int, [_V, _V, _V, C.c_int32]),
    "wc4d_pcg": (C.c_int, [_V, _V, C.c_double, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _I32, _D, _D]),
    "wc4d_inner_loop": (C.c_int, [_V, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.c_double,
                                  C.c_int32, C.c_int32, _V, _I32, _D]),
    "wc4d_orthonormalize": (C.c_int, [_V, _V, C.c_int64, C.c_int32, C.c_int64, _D, C.c_int32]),
    "wc4d_symeig": (C.c_int, [_V, C.c_int32, _V, _D, _V]),
    "wc4d_set_wait_limit": (C.c_int, [_V, C.c_int64]),
    "wc4d_sync": (C.c_int, [_V]),
    "wc4d_gram": (C.c_int, [_V, _V, C.c_int64, _V, C.c_int64, C.c_int64, C.c_int32, C.c_int32, _V, C.c_int32]),
    "wc4d_chol_inverse": (C.c_int, [_V, C.c_int32, _V, _V]),
    "wc4d_tall_times_small": (C.c_int, [_V, _V, C.c_int64, C.c_int64, C.c_int32, _V, C.c_int32, _V, C.c_int64,
                                        C.c_int32]),
    "wc4d_hvp_count": (C.c_int64, [_V, C.c_int32]),
    "wc4d_jacobi_sweeps": (C.c_int32, [_V]),
    "wc4d_jacobi_sweeps_fp32": (C.c_int32, [_V]),
    "wc4d_jacobi_fp32_kernel": (C.c_int32, [_V]),
    "wc4d_lanczos_cg": (C.c_int32, [_V, _V, C.c_double, C.c_int32, C.c_int32, C.POINTER(C.c_int32),
                                    C.POINTER(C.c_double)]),
    "wc4d_lanczos_tridiag": (C.c_int32, [_V, _V, _V]),
    "wc4d_lanczos_ritz": (C.c_int32, [_V, C.c_int32, _V]),
    "wc4d_set_graphs": (C.c_int32, [_V, C.c_int32]),
    "wc4d_iteration_mode": (C.c_int32, [_V, C.c_char_p, C.c_int32]),
    "wc4d_set_gram_path": (C.c_int32, [_V, C.c_int32]),
    "wc4d_gram_sym": (C.c_int32, [_V, _V, C.c_int64, _V, C.c_int64, C.c_int64, C.c_int32, _V, C.c_int32]),
    "wc4d_stream_create": (C.c_int32, [C.POINTER(C.c_void_p)]),
    "wc4d_stream_destroy": (C.c_int32, [_V]),
    "wc4d_set_reliable_delta": (C.c_int32, [_V, C.c_double]),
    "wc4d_set_autotune": (None, [C.c_int32]),
    "wc4d_autotune_choice": (C.c_int32, [C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    "wc4d_apply_dsqrt": (C.c_int, [_V, _V, _V, C.c_int32, C.c_int64, C.c_int32]),
    "wc4d_apply_linv": (C.c_int, [_V, _V, C.c_int32, C.c_int64, C.c_int32]),
    "wc4d_apply_linvT": (C.c_int, [_V, _V, C.c_int32, C.c_int64, C.c_int32]),
    "wc4d_get_propagator": (C.c_int, [_V, C.c_int32, _V]),
    "wc4d_launch_count": (C.c_int64, [C.c_int32]),
    "wc4d_profile": (C.c_int, [_V, C.c_int32]),
    "wc4d_profile_read": (C.c_int, [_V, C.c_int32, _D, C.POINTER(C.c_int64)]),
    "wc4d_lmp_apply_static": (C.c_int, [_V, _V, C.c_int32, C.c_int64, _V, _V, _V]),
}
PROF_CLASSES = ("gemv_sweep", "gemm", "tc_gemm", "circulant", "lmp", "gram", "tall_gemm", "l96_tlm", "l96_adj",
                "pcg_vec", "gemv_sweep_f64", "jacobi", "chol")
EXPORTS = tuple(_SIGS)

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libwc4d.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"libwc4d.so is not built ({p}); run __graft_entry__.build() first")
            L = C.CDLL(p)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def build(force: bool = False) -> str:
    from ._build import build as _b
    return _b(force=force)


# --------------------------------------------------------------------------
# marshalling helpers
# --------------------------------------------------------------------------
def _ptr(t):
    if t is None:
        return None
    import torch
    if isinstance(t, torch.Tensor):
        if not t.is_cuda:
            raise ValueError("device argument must be a CUDA tensor")
        if not t.is_contiguous():
            raise ValueError("device argument must be contiguous")
        return C.c_void_p(t.data_ptr())
    return C.c_void_p(int(t))


def _dev(t, dtype, count, name):
    """_ptr after checking what the C ABI cannot see behind a bare pointer: the
    element type (None: any) and at least `count` elements (count <= 0: left to
    the library's own argument checks).  Raw integer addresses pass unchecked."""
    import torch
    if isinstance(t, torch.Tensor):
        if dtype is not None and t.dtype != dtype:
            raise ValueError(f"{name}: expected {dtype}, got {t.dtype}")
        if count > 0 and t.numel() < count:
            raise ValueError(f"{name}: needs at least {count} elements, has {t.numel()}")
    return _ptr(t)


def _fdtype(precision):
    """Element type of the blocks of a call in this precision (None: invalid,
    left to the library's EINVAL)."""
    import torch
    return {FP64: torch.float64, MIXED: torch.float32}.get(int(precision))


def _block(ctx, K, ld):
    """Elements an n_A x K block with leading dimension ld spans (0 when K or
    ld are invalid: the library rejects those itself)."""
    nA = int(load().wc4d_control_dim(ctx))
    K, ld = int(K), int(ld)
    return (K - 1) * ld + nA if K >= 1 and nA >= 1 and ld >= nA else 0


def _hp(a):
    """Host float64 pointer (keeps a contiguous copy alive via the caller)."""
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _hv(a):
    """Host pointer of a contiguous numpy array of any dtype."""
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


def torch_f64():
    import torch
    return torch.float64


def _stream(stream=None):
    if stream is not None:
        return C.c_void_p(int(stream))
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(ctx, status):
    if status != OK:
        msg = load().wc4d_last_error(ctx)
        raise WC4DError(status, msg.decode() if msg else "")
    return status


# --------------------------------------------------------------------------
# C-ABI, one Python function per entry point
# --------------------------------------------------------------------------
def wc4d_create(prob: Problem, stream=None):
    ctx = C.c_void_p()
    st = load().wc4d_create(C.byref(ctx), C.byref(prob), _stream(stream))
    if st != OK:
        raise WC4DError(st, "wc4d_create rejected the problem")
    return ctx


def wc4d_destroy(ctx):
    load().wc4d_destroy(ctx)


def wc4d_last_error(ctx):
    msg = load().wc4d_last_error(ctx)
    return msg.decode() if msg else ""


def wc4d_set_stream(ctx, stream=None):
    _check(ctx, load().wc4d_set_stream(ctx, _stream(stream)))


def wc4d_set_propagator(ctx, t, M):
    _check(ctx, load().wc4d_set_propagator(ctx, int(t), _ptr(M)))


def wc4d_build_advdiff_propagator(ctx, kappa, c, dt, steps):
    _check(ctx, load().wc4d_build_advdiff_propagator(ctx, float(kappa), float(c), float(dt), int(steps)))


def wc4d_set_covariance(ctx, block, corr, variance, length):
    _check(ctx, load().wc4d_set_covariance(ctx, int(block), int(corr), float(variance), float(length)))


COV_SQRT_CIRCULANT, COV_SQRT_DENSE, COV_SQRT_SCALAR = 0, 1, 2


def wc4d_set_cov_sqrt(ctx, block, kind, data):
    """Covariance block given by its square root: kind 0 circulant first row
    (host, n values), 1 dense n x n row-major (device FP64 tensor), 2 scalar
    sigma (host)."""
    import torch
    kind = int(kind)
    n = wc4d_get_problem(ctx).n
    if kind == COV_SQRT_DENSE:
        ptr = _dev(data, torch.float64, n * n, "data")
    elif kind == COV_SQRT_SCALAR:
        buf = np.array([float(data)], dtype=np.float64)
        ptr = buf.ctypes.data_as(_D)
    else:
        buf = np.ascontiguousarray(data, dtype=np.float64)
        if buf.size < n:
            raise ValueError(f"data: needs at least {n} values, has {buf.size}")
        ptr = buf.ctypes.data_as(_D)
    _check(ctx, load().wc4d_set_cov_sqrt(ctx, int(block), kind, ptr))


def wc4d_get_problem(ctx):
    """The context's problem statement (a Problem structure)."""
    pr = Problem()
    _check(ctx, load().wc4d_get_problem(ctx, C.byref(pr)))
    return pr


def wc4d_set_trajectory(ctx, X):
    """External Lorenz-96 linearisation trajectory (device FP64, (N steps + 1) x n)."""
    import torch
    pr = wc4d_get_problem(ctx)
    _check(ctx, load().wc4d_set_trajectory(ctx, _dev(X, torch.float64, (pr.N * pr.steps + 1) * pr.n, "X")))


def wc4d_set_innovation(ctx, d, Dm12b=None):
    """Innovations d (device FP64, nobs) and optional D^{-1/2} b (device FP64, nA); forms the rhs."""
    import torch
    _check(ctx, load().wc4d_set_innovation(ctx, _dev(d, torch.float64, int(load().wc4d_nobs(ctx)), "d"),
                                           _dev(Dm12b, torch.float64, int(load().wc4d_control_dim(ctx)), "Dm12b")))


def wc4d_set_covariance_row(ctx, block, row):
    row = np.ascontiguousarray(row, dtype=np.float64)
    _check(ctx, load().wc4d_set_covariance_row(ctx, int(block), _hp(row)))


def wc4d_set_background_obs(ctx, xb, y, Dm12b=None):
    xb = np.ascontiguousarray(xb, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    Dm = None if Dm12b is None else np.ascontiguousarray(Dm12b, dtype=np.float64)
    _check(ctx, load().wc4d_set_background_obs(ctx, _hp(xb), _hp(y), _hp(Dm)))


def wc4d_outer_update(ctx, x):
    _check(ctx, load().wc4d_outer_update(ctx, _ptr(x)))


def wc4d_batch_inner_loop(ctxs, method, ks, ls, q_power, seeds, tol, maxit, precision, xs, workers=0):
    """Inner loops of independent contexts (each with its own stream) run
    concurrently; returns (iters, relres, statuses) as lists."""
    cnt = len(ctxs)
    arr_ctx = (C.c_void_p * cnt)(*[C.c_void_p(c.value if isinstance(c, C.c_void_p) else c) for c in ctxs])
    arr_x = (C.c_void_p * cnt)(*[_ptr(x).value for x in xs])
    k = np.ascontiguousarray(ks, dtype=np.int32)
    l = np.ascontiguousarray(ls, dtype=np.int32)
    sd = np.ascontiguousarray(seeds, dtype=np.uint64)
    it = np.zeros(cnt, dtype=np.int32)
    rr = np.zeros(cnt)
    st = np.zeros(cnt, dtype=np.int32)
    s = load().wc4d_batch_inner_loop(C.cast(arr_ctx, C.c_void_p), int(cnt), int(method), _hv(k), _hv(l),
                                     int(q_power), _hv(sd), float(tol), int(maxit), int(precision),
                                     C.cast(arr_x, C.c_void_p), _hv(it), _hv(rr), _hv(st), int(workers))
    if s != OK and s != ENOCONV:
        bad = [i for i in range(cnt) if st[i] != OK]
        _check(ctxs[bad[0]] if bad else ctxs[0], s)
    return it.tolist(), rr.tolist(), st.tolist()


def wc4d_learned_probes(ctx, w_bf16, bias, m, S, ld):
    """S (m x ld device tensor, FP64) = learned start columns; w_bf16: device
    int16/bfloat16 tensor of the packed weights, bias: device float32."""
    _check(ctx, load().wc4d_learned_probes(ctx, _ptr(w_bf16), _ptr(bias), int(m), _ptr(S), int(ld)))


def wc4d_nobs(ctx):
    return int(load().wc4d_nobs(ctx))


def wc4d_control_dim(ctx):
    return int(load().wc4d_control_dim(ctx))


def wc4d_ritz_count(ctx):
    return int(load().wc4d_ritz_count(ctx))


def wc4d_get_rhs(ctx, rhs):
    _check(ctx, load().wc4d_get_rhs(ctx, _ptr(rhs)))


def wc4d_hvp(ctx, X, Y, K, ld, precision=FP64):
    dt, n = _fdtype(precision), _block(ctx, K, ld)
    _check(ctx, load().wc4d_hvp(ctx, _dev(X, dt, n, "X"), _dev(Y, dt, n, "Y"), int(K), int(ld), int(precision)))


def wc4d_gaussian(ctx, seed, rows, cols, ld, G):
    _check(ctx, load().wc4d_gaussian(ctx, int(seed), int(rows), int(cols), int(ld), _ptr(G)))


def wc4d_gaussian_f32(ctx, seed, rows, cols, ld, G):
    """The mixed sketch's FP32 probes (same Philox stream as wc4d_gaussian) into FP32 G."""
    import torch
    rows, cols, ld = int(rows), int(cols), int(ld)
    if cols < 1 or rows < 1 or ld < rows:
        raise WC4DError(EINVAL, "wc4d_gaussian_f32: bad shape")
    _check(ctx, load().wc4d_gaussian_f32(ctx, int(seed), rows, cols, ld,
                                         _dev(G, torch.float32, (cols - 1) * ld + rows, "G")))


def wc4d_sketch(ctx, method, k, l, q_power, seed, G=None, precision=FP64):
    import torch
    th = np.zeros(max(int(k), 0))
    Gp = _dev(G, torch.float64, _block(ctx, int(k) + int(l), load().wc4d_control_dim(ctx)), "G")
    _check(ctx, load().wc4d_sketch(ctx, int(method), int(k), int(l), int(q_power), int(seed), Gp,
                                   _hp(th), int(precision)))
    return th


def wc4d_get_ritz(ctx, U, k):
    """Ritz values (the first k) and, into U, all installed Ritz vectors."""
    import torch
    kU = int(load().wc4d_ritz_count(ctx))
    th = np.zeros(max(int(k), kU, 0))     # the library writes all kU values
    nA = int(load().wc4d_control_dim(ctx))
    _check(ctx, load().wc4d_get_ritz(ctx, _dev(U, torch.float64, kU * nA, "U"), _hp(th)))
    return th[:int(k)]


def wc4d_set_ritz(ctx, k, U, theta):
    import torch
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    if theta.size < int(k):
        raise ValueError(f"theta: needs {int(k)} values, has {theta.size}")
    n = int(k) * int(load().wc4d_control_dim(ctx))
    _check(ctx, load().wc4d_set_ritz(ctx, int(k), _dev(U, torch.float64, n, "U"), _hp(theta)))


def wc4d_lmp_apply(ctx, v, y, transpose=0):
    import torch
    n = int(load().wc4d_control_dim(ctx))
    _check(ctx, load().wc4d_lmp_apply(ctx, _dev(v, torch.float64, n, "v"), _dev(y, torch.float64, n, "y"),
                                      int(transpose)))


def wc4d_pcg(ctx, x, tol=1e-6, maxit=5000, use_lmp=1, force_iters=0, precision=FP64, qcf=False,
             raise_on_noconv=True):
    """Returns (iters, relres, qcf_drop or None, status)."""
    it = C.c_int32(0)
    rr = C.c_double(0.0)
    cap = max(int(maxit), int(force_iters), 1)
    q = np.zeros(cap) if qcf else None
    import torch
    xp = _dev(x, torch.float64, int(load().wc4d_control_dim(ctx)), "x")
    st = load().wc4d_pcg(ctx, xp, float(tol), int(maxit), int(use_lmp), int(force_iters), int(precision),
                         C.byref(it), C.byref(rr), _hp(q))
    if st != OK and (raise_on_noconv or st != ENOCONV):
        _check(ctx, st)
    return it.value, rr.value, (q[:it.value] if qcf else None), st


def wc4d_inner_loop(ctx, method, k, l, q_power, seed, tol, maxit, precision, x):
    it = C.c_int32(0)
    rr = C.c_double(0.0)
    import torch
    xp = _dev(x, torch.float64, int(load().wc4d_control_dim(ctx)), "x")
    _check(ctx, load().wc4d_inner_loop(ctx, int(method), int(k), int(l), int(q_power), int(seed), float(tol),
                                       int(maxit), int(precision), xp, C.byref(it), C.byref(rr)))
    return it.value, rr.value


def wc4d_orthonormalize(ctx, Y, rows, m, ld, want_R=True, precision=FP64):
    R = np.zeros(int(m) * int(m)) if want_R else None
    _check(ctx, load().wc4d_orthonormalize(ctx, _ptr(Y), int(rows), int(m), int(ld), _hp(R), int(precision)))
    return None if R is None else R.reshape(int(m), int(m)).T.copy()   # ordinary (row, col) indexing


def wc4d_symeig(ctx, m, S, V):
    w = np.zeros(int(m))
    _check(ctx, load().wc4d_symeig(ctx, int(m), _ptr(S), _hp(w), _ptr(V)))
    return w


def wc4d_set_wait_limit(ctx, polls):
    """Polls of a bounded device-side wait (grid barriers of the persistent
    sweeps, staged-copy waits of the FP32 Lorenz-96 sweeps) before it gives
    up (< 0: default; 0: fail at once)."""
    _check(ctx, load().wc4d_set_wait_limit(ctx, int(polls)))


def wc4d_sync(ctx):
    """Synchronise the context's stream; raises WC4DError (ETIMEOUT) if a
    bounded wait of queued work gave up."""
    _check(ctx, load().wc4d_sync(ctx))


def wc4d_gram(ctx, A, lda, B, ldb, rows, ma, mb, C_out, precision=FP64):
    """C_out = A^T B (ma x mb FP64, column-major) for column-major blocks A
    (rows x ma, lda) and B (rows x mb, ldb) of the given precision."""
    import torch
    dt, rows, ma, mb, lda, ldb = _fdtype(precision), int(rows), int(ma), int(mb), int(lda), int(ldb)
    _check(ctx, load().wc4d_gram(ctx, _dev(A, dt, (ma - 1) * lda + rows, "A"), lda,
                                 _dev(B, dt, (mb - 1) * ldb + rows, "B"), ldb, rows, ma, mb,
                                 _dev(C_out, torch.float64, ma * mb, "C"), int(precision)))


def wc4d_gram_sym(ctx, A, lda, B, ldb, rows, m, C_out, precision=FP64):
    """C_out = A^T B (m x m FP64) for a product known to be symmetric (B = A,
    or Z^T A Z): upper 64 x 64 tiles, mirrored.  FP32 blocks (MIXED) take
    the path wc4d_set_gram_path selects."""
    import torch
    dt, rows, m, lda, ldb = _fdtype(precision), int(rows), int(m), int(lda), int(ldb)
    _check(ctx, load().wc4d_gram_sym(ctx, _dev(A, dt, (m - 1) * lda + rows, "A"), lda,
                                     _dev(B, dt, (m - 1) * ldb + rows, "B"), ldb, rows, m,
                                     _dev(C_out, torch.float64, m * m, "C"), int(precision)))


def wc4d_chol_inverse(ctx, m, G, Rinv):
    """G = R^T R (m x m FP64 SPD): Rinv = R^{-1} (FP64, m x m)."""
    import torch
    m = int(m)
    _check(ctx, load().wc4d_chol_inverse(ctx, m, _dev(G, torch.float64, m * m, "G"),
                                         _dev(Rinv, torch.float64, m * m, "Rinv")))


def wc4d_tall_times_small(ctx, Y, ldy, rows, m, W, k, Z, ldz, precision=FP64):
    """Z = Y W: Y (rows x m, ldy) in the given precision, W (m x k FP64), Z (rows x k, ldz)."""
    import torch
    dt, rows, m, k, ldy, ldz = _fdtype(precision), int(rows), int(m), int(k), int(ldy), int(ldz)
    _check(ctx, load().wc4d_tall_times_small(ctx, _dev(Y, dt, (m - 1) * ldy + rows, "Y"), ldy, rows, m,
                                             _dev(W, torch.float64, m * k, "W"), k,
                                             _dev(Z, dt, (k - 1) * ldz + rows, "Z"), ldz, int(precision)))


def wc4d_apply_dsqrt(ctx, X, Y, K, ld, precision=FP64):
    dt, n = _fdtype(precision), _block(ctx, K, ld)
    _check(ctx, load().wc4d_apply_dsqrt(ctx, _dev(X, dt, n, "X"), _dev(Y, dt, n, "Y"), int(K), int(ld),
                                        int(precision)))


def wc4d_apply_linv(ctx, W, K, ld, precision=FP64):
    Wp = _dev(W, _fdtype(precision), _block(ctx, K, ld), "W")
    _check(ctx, load().wc4d_apply_linv(ctx, Wp, int(K), int(ld), int(precision)))


def wc4d_apply_linvT(ctx, W, K, ld, precision=FP64):
    Wp = _dev(W, _fdtype(precision), _block(ctx, K, ld), "W")
    _check(ctx, load().wc4d_apply_linvT(ctx, Wp, int(K), int(ld), int(precision)))


def wc4d_get_propagator(ctx, t, M):
    _check(ctx, load().wc4d_get_propagator(ctx, int(t), _ptr(M)))


def wc4d_launch_count(reset=False):
    return int(load().wc4d_launch_count(1 if reset else 0))


def wc4d_profile(ctx, enable=True):
    _check(ctx, load().wc4d_profile(ctx, 1 if enable else 0))


def wc4d_profile_read(ctx, cls):
    """(total device ms, number of timed launch groups) of one kernel class."""
    ms = C.c_double(0.0)
    n = C.c_int64(0)
    _check(ctx, load().wc4d_profile_read(ctx, int(cls), C.byref(ms), C.byref(n)))
    return ms.value, n.value


def wc4d_lmp_apply_static(U, theta, k, nA, v, y, stream=None):
    """y = C v without any device allocation (shared fixed scratch; see wc4d.h).
    U: FP64, k*nA elements (column-major nA x k); theta: FP64, k; v, y: FP64, nA."""
    k, nA = int(k), int(nA)
    args = (_dev(U, torch_f64(), k * nA, "U"), _dev(theta, torch_f64(), k, "theta"), k, nA,
            _dev(v, torch_f64(), nA, "v"), _dev(y, torch_f64(), nA, "y"), _stream(stream))
    st = load().wc4d_lmp_apply_static(*args)
    if st != OK:
        raise WC4DError(st, "wc4d_lmp_apply_static")


def wc4d_hvp_count(ctx, reset=False):
    return int(load().wc4d_hvp_count(ctx, 1 if reset else 0))


def wc4d_lanczos_cg(ctx, x, tol, maxit, reorth=True):
    """FP64 CG without a preconditioner recording the Lanczos data; returns (J, relres)."""
    it = C.c_int32(0)
    rr = C.c_double(0.0)
    _check(ctx, load().wc4d_lanczos_cg(ctx, _ptr(x), float(tol), int(maxit), 1 if reorth else 0, C.byref(it),
                                       C.byref(rr)))
    return it.value, rr.value


def wc4d_lanczos_tridiag(ctx, J):
    g = np.zeros(int(J))
    t = np.zeros(max(int(J) - 1, 1))
    _check(ctx, load().wc4d_lanczos_tridiag(ctx, _hp(g), _hp(t)))
    return g, t[:max(int(J) - 1, 0)]


def wc4d_lanczos_ritz(ctx, k):
    th = np.zeros(int(k))
    _check(ctx, load().wc4d_lanczos_ritz(ctx, int(k), _hp(th)))
    return th


def wc4d_jacobi_sweeps(ctx):
    return int(load().wc4d_jacobi_sweeps(ctx))


def wc4d_jacobi_sweeps_fp32(ctx):
    return int(load().wc4d_jacobi_sweeps_fp32(ctx))


def wc4d_jacobi_fp32_kernel(ctx):
    """1 = one 16-CTA cluster, 2 = cooperative grid, 0 = no FP32 phase."""
    return int(load().wc4d_jacobi_fp32_kernel(ctx))


def wc4d_set_graphs(ctx, enable):
    """enable: True / 1 device-side loop graph, 2 one graph per iteration, False / 0 eager."""
    _check(ctx, load().wc4d_set_graphs(ctx, int(enable)))


def wc4d_set_gram_path(ctx, tensor_cores):
    """True: FP32 Gram products on the tensor cores (sliced, exact chunks) where the shape allows; False: FP32 pipe."""
    _check(ctx, load().wc4d_set_gram_path(ctx, 1 if tensor_cores else 0))


ITER_EAGER, ITER_GRAPH_PER_ITERATION, ITER_DEVICE_LOOP = 0, 1, 2


def wc4d_iteration_mode(ctx):
    """(mode, note): how the last solve ran its CG iterations (ITER_*) and,
    if the device-side loop graph could not be built, the failing call."""
    buf = C.create_string_buffer(256)
    mode = load().wc4d_iteration_mode(ctx, buf, len(buf))
    if mode < 0:
        raise WC4DError(EINVAL, "wc4d_iteration_mode: null context")
    return mode, buf.value.decode(errors="replace")


def wc4d_stream_create():
    """A new non-blocking CUDA stream (integer handle) for one batched instance."""
    h = C.c_void_p()
    st = load().wc4d_stream_create(C.byref(h))
    if st != OK:
        raise WC4DError(st, "wc4d_stream_create failed")
    return h.value


def wc4d_stream_destroy(handle):
    load().wc4d_stream_destroy(C.c_void_p(handle))


def wc4d_set_reliable_delta(ctx, delta):
    _check(ctx, load().wc4d_set_reliable_delta(ctx, float(delta)))


def wc4d_set_autotune(enable):
    load().wc4d_set_autotune(1 if enable else 0)


def wc4d_autotune_choice(fp64, rows, cols, kdim, tall=False):
    kind = (1 if fp64 else 0) + (2 if tall else 0)
    return int(load().wc4d_autotune_choice(kind, int(rows), int(cols), int(kdim)))


# --------------------------------------------------------------------------
# Convenience: a context set up from a configuration of the inputs module
# --------------------------------------------------------------------------
class Solver:
    """Owns one wc4d context for an inputs.Config: covariances, model and the
    background/observations of the synthetic twin (all on the device)."""

    def __init__(self, cfg, twin=None, M_shared=False, stream=None):
        self.cfg = cfg
        prob = Problem()
        prob.n, prob.N = cfg.n, cfg.N
        prob.model = MODEL_L96 if cfg.model == inputs.MODEL_L96 else MODEL_DENSE
        prob.steps, prob.dt, prob.F, prob.sigma_o2 = cfg.steps, cfg.dt, cfg.F, cfg.sigma_o2
        prob.obs_stride, prob.obs_t0, prob.obs_tstride = cfg.obs_stride, cfg.obs_t0, 1
        prob.M_shared = 1 if M_shared else 0
        self.prob = prob
        self.ctx = wc4d_create(prob, stream)
        self.nA = cfg.nA
        wc4d_set_covariance(self.ctx, 0, cfg.b_kind, cfg.b_var, cfg.b_L)
        wc4d_set_covariance(self.ctx, 1, cfg.q_kind, cfg.q_var, cfg.q_L)
        if prob.model == MODEL_DENSE:
            wc4d_build_advdiff_propagator(self.ctx, cfg.kappa, cfg.u, cfg.dt, cfg.steps)
        if twin is not None:
            wc4d_set_background_obs(self.ctx, twin.xb, twin.y)

    def close(self):
        if self.ctx:
            wc4d_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
