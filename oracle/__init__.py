"""FP64 CPU oracle (plain C, loaded with ctypes).

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, plain reference that the
CUDA library is checked against.  Only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the library never does
and shares no code with it.

Each wrapper names the passage of the paper the C routine follows; the C file
states what every routine is pinned to.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODEL_DENSE, MODEL_ADVDIFF, MODEL_L96 = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, -O2, OpenMP)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(f) > os.path.getmtime(_LIB) for f in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class OProblem(C.Structure):
    _fields_ = [
        ("n", C.c_int32), ("N", C.c_int32), ("model", C.c_int32), ("steps", C.c_int32),
        ("M_shared", C.c_int32), ("obs_stride", C.c_int32), ("obs_t0", C.c_int32),
        ("obs_tstride", C.c_int32),
        ("dt", C.c_double), ("kappa", C.c_double), ("u", C.c_double), ("F", C.c_double),
        ("sigma_o2", C.c_double),
        ("M", C.POINTER(C.c_double)), ("Bsqrt", C.POINTER(C.c_double)),
        ("Qsqrt", C.POINTER(C.c_double)), ("traj", C.POINTER(C.c_double)),
    ]


_D = C.POINTER(C.c_double)
_U32 = C.POINTER(C.c_uint32)
_I32 = C.POINTER(C.c_int32)
_P = C.POINTER(OProblem)

_SIGS = {
    "o_threads": (C.c_int, [C.c_int]),
    "o_philox4x32_10": (None, [_U32, _U32, _U32]),
    "o_philox_words": (None, [C.c_uint64, C.c_int64, _U32]),
    "o_gaussian": (None, [C.c_uint64, C.c_int64, C.c_int64, C.c_int64, _D]),
    "o_corr_row": (None, [C.c_int32, C.c_int32, C.c_double, C.c_double, _D]),
    "o_circulant_sqrt_row": (C.c_int, [C.c_int32, _D, _D, _D]),
    "o_cov_eigs": (None, [C.c_int32, C.c_int32, C.c_double, C.c_double, _D]),
    "o_cov_sqrt_row": (C.c_int, [C.c_int32, C.c_int32, C.c_double, C.c_double, _D, _D]),
    "o_circulant_apply": (None, [C.c_int32, _D, _D, _D]),
    "o_advdiff_step": (None, [C.c_int32, C.c_double, C.c_double, C.c_double, _D, _D]),
    "o_advdiff_step_T": (None, [C.c_int32, C.c_double, C.c_double, C.c_double, _D, _D]),
    "o_advdiff_dense": (None, [C.c_int32, C.c_double, C.c_double, C.c_double, C.c_int32, _D]),
    "o_l96_tendency": (None, [C.c_int32, C.c_double, _D, _D]),
    "o_l96_rk4": (None, [C.c_int32, C.c_double, C.c_double, _D, _D]),
    "o_l96_tlm": (None, [C.c_int32, C.c_double, C.c_double, _D, _D, _D]),
    "o_l96_adj": (None, [C.c_int32, C.c_double, C.c_double, _D, _D, _D]),
    "o_l96_run": (None, [C.c_int32, C.c_double, C.c_double, C.c_int32, _D, _D]),
    "o_nobs": (C.c_int64, [_P]),
    "o_model_apply": (None, [_P, C.c_int32, _D, _D]),
    "o_model_apply_T": (None, [_P, C.c_int32, _D, _D]),
    "o_Linv": (None, [_P, C.c_int32, _D, C.c_int64, _D]),
    "o_LinvT": (None, [_P, C.c_int32, _D, C.c_int64, _D]),
    "o_Dsqrt": (None, [_P, C.c_int32, _D, C.c_int64, _D]),
    "o_obs_adjoint": (None, [_P, C.c_int32, _D, C.c_int64, _D]),
    "o_hvp": (None, [_P, C.c_int32, _D, C.c_int64, _D]),
    "o_hvp_count": (C.c_int64, [C.c_int]),
    "o_forward_run": (None, [_P, _D, _D, _D]),
    "o_innovation": (None, [_P, _D, _D, _D, _D]),
    "o_rhs": (None, [_P, _D, _D, _D]),
    "o_qcf": (C.c_double, [_P, _D, _D, _D]),
    "o_householder_qr": (None, [C.c_int64, C.c_int32, _D, C.c_int64, _D, C.c_int64, _D]),
    "o_jacobi_eig": (C.c_int, [C.c_int32, _D, _D, _D]),
    "o_cholesky_upper": (C.c_int, [C.c_int32, _D, _D]),
    "o_solve_right_upper": (None, [C.c_int64, C.c_int32, _D, _D, C.c_int64]),
    "o_jacobi_svd": (C.c_int, [C.c_int64, C.c_int32, _D, C.c_int64, _D, _D, _D]),
    "o_revd": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, _D, _D, _D]),
    "o_nystrom": (C.c_int, [_P, C.c_int32, C.c_int32, _D, _D, _D]),
    "o_ritzit": (C.c_int, [_P, C.c_int32, C.c_int32, _D, _D, _D]),
    "o_lmp_apply": (None, [C.c_int64, C.c_int32, _D, _D, C.c_int32, _D, _D]),
    "o_pcg": (C.c_int, [_P, _D, C.c_int32, _D, _D, C.c_double, C.c_int32, C.c_int32, _D,
                        _I32, _D, _D, _D]),
}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _dp(a):
    """Pointer to a C-contiguous float64 array (None -> NULL)."""
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle wants contiguous float64"
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Problem description
# --------------------------------------------------------------------------
class Problem:
    """An inner-loop problem (Section 2): model, D^{1/2} = diag(B^{1/2}, Q^{1/2}, ...),
    H (every obs_stride-th point at times t >= obs_t0), R = sigma_o2 I.

    Column blocks of the control space are column-major (n*(N+1)) x K arrays,
    i.e. numpy arrays of shape (K, nA) in C order (one row per vector)."""

    def __init__(self, n, N, model, Bsqrt, Qsqrt, sigma_o2, obs_stride, obs_t0=1, obs_tstride=1,
                 steps=1, dt=0.0, kappa=0.0, u=0.0, F=8.0, M=None, M_shared=False, traj=None):
        self.n, self.N = int(n), int(N)
        self.nA = self.n * (self.N + 1)
        self._keep = {}
        self.Bsqrt = _f64(Bsqrt)
        self.Qsqrt = _f64(Qsqrt)
        self.M = None if M is None else _f64(M)
        self.traj = None if traj is None else _f64(traj)
        s = OProblem()
        s.n, s.N, s.model, s.steps = self.n, self.N, int(model), int(steps)
        s.M_shared = 1 if M_shared else 0
        s.obs_stride, s.obs_t0, s.obs_tstride = int(obs_stride), int(obs_t0), int(obs_tstride)
        s.dt, s.kappa, s.u, s.F, s.sigma_o2 = float(dt), float(kappa), float(u), float(F), float(sigma_o2)
        s.M = _dp(self.M)
        s.Bsqrt = _dp(self.Bsqrt)
        s.Qsqrt = _dp(self.Qsqrt)
        s.traj = _dp(self.traj)
        self.s = s
        self.model = int(model)

    @property
    def ptr(self):
        return C.byref(self.s)

    @property
    def nobs(self):
        return int(lib().o_nobs(self.ptr))


# --------------------------------------------------------------------------
# Wrappers
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().o_philox4x32_10(c.ctypes.data_as(_U32), k.ctypes.data_as(_U32), out.ctypes.data_as(_U32))
    return out


def philox_words(seed, count):
    out = np.zeros(4 * count, dtype=np.uint32)
    lib().o_philox_words(int(seed), int(count), out.ctypes.data_as(_U32))
    return out


def gaussian(seed, rows, cols):
    """Probe matrix (Alg. 3-5 step 1); returned as (cols, rows) = column-major."""
    G = np.zeros((cols, rows))
    lib().o_gaussian(int(seed), int(rows), int(cols), int(rows), _dp(G))
    return G


def threads(n=0):
    """Set (n > 0) the threads of the oracle's column loops; returns the count
    the next loop will use."""
    return int(lib().o_threads(int(n)))


def corr_row(kind, n, L, variance):
    row = np.zeros(n)
    lib().o_corr_row(int(kind), int(n), float(L), float(variance), _dp(row))
    return row


def circulant_sqrt_row(row):
    """First row of the symmetric square root of the circulant with first row
    `row` (Section 5 covariances): eigenvalues by an extended-precision DFT of
    the row, negative ones clamped to zero.  Returns (row, clamped, min_eig)."""
    row = _f64(row)
    out = np.zeros_like(row)
    mn = C.c_double(0.0)
    clamped = lib().o_circulant_sqrt_row(len(row), _dp(row), _dp(out), C.byref(mn))
    return out, int(clamped), mn.value


def cov_eigs(kind, n, L, variance):
    """Eigenvalues of variance * C(kind, L) (the circulant of corr_row), from
    the correlation function: extended-precision DFT for SOAR, the Poisson
    summation closed form for the Gaussian."""
    lam = np.zeros(n)
    lib().o_cov_eigs(int(kind), int(n), float(L), float(variance), _dp(lam))
    return lam


def cov_sqrt_row(kind, n, L, variance):
    """First row of (variance * C(kind, L))^{1/2} from cov_eigs, negative
    eigenvalues clamped to zero.  Returns (row, clamped, min_eig)."""
    out = np.zeros(n)
    mn = C.c_double(0.0)
    clamped = lib().o_cov_sqrt_row(int(kind), int(n), float(L), float(variance), _dp(out), C.byref(mn))
    return out, int(clamped), mn.value


def circulant_apply(row, x):
    row, x = _f64(row), _f64(x)
    y = np.zeros_like(x)
    lib().o_circulant_apply(len(row), _dp(row), _dp(x), _dp(y))
    return y


def advdiff_step(x, kappa, u, dt, transpose=False):
    x = _f64(x)
    y = np.zeros_like(x)
    f = lib().o_advdiff_step_T if transpose else lib().o_advdiff_step
    f(len(x), float(kappa), float(u), float(dt), _dp(x), _dp(y))
    return y


def advdiff_dense(n, kappa, u, dt, steps):
    M = np.zeros((n, n))
    lib().o_advdiff_dense(int(n), float(kappa), float(u), float(dt), int(steps), _dp(M))
    return M


def l96_tendency(x, F):
    x = _f64(x)
    f = np.zeros_like(x)
    lib().o_l96_tendency(len(x), float(F), _dp(x), _dp(f))
    return f


def l96_rk4(x, F, dt):
    x = _f64(x)
    y = np.zeros_like(x)
    lib().o_l96_rk4(len(x), float(F), float(dt), _dp(x), _dp(y))
    return y


def l96_tlm(x, dx, F, dt):
    x, dx = _f64(x), _f64(dx)
    y = np.zeros_like(x)
    lib().o_l96_tlm(len(x), float(F), float(dt), _dp(x), _dp(dx), _dp(y))
    return y


def l96_adj(x, ly, F, dt):
    x, ly = _f64(x), _f64(ly)
    y = np.zeros_like(x)
    lib().o_l96_adj(len(x), float(F), float(dt), _dp(x), _dp(ly), _dp(y))
    return y


def l96_run(x0, F, dt, nsteps):
    x0 = _f64(x0)
    traj = np.zeros((nsteps + 1, len(x0)))
    lib().o_l96_run(len(x0), float(F), float(dt), int(nsteps), _dp(x0), _dp(traj))
    return traj


def _block(p, X):
    X = _f64(np.atleast_2d(X))
    assert X.shape[1] == p.nA
    return X


def model_apply(p, t, x, transpose=False):
    x = _f64(x)
    y = np.zeros(p.n)
    (lib().o_model_apply_T if transpose else lib().o_model_apply)(p.ptr, int(t), _dp(x), _dp(y))
    return y


def Linv(p, Z):
    Z = _block(p, Z)
    W = np.zeros_like(Z)
    lib().o_Linv(p.ptr, Z.shape[0], _dp(Z), p.nA, _dp(W))
    return W


def LinvT(p, V):
    V = _block(p, V)
    S = np.zeros_like(V)
    lib().o_LinvT(p.ptr, V.shape[0], _dp(V), p.nA, _dp(S))
    return S


def Dsqrt(p, X):
    X = _block(p, X)
    Z = np.zeros_like(X)
    lib().o_Dsqrt(p.ptr, X.shape[0], _dp(X), p.nA, _dp(Z))
    return Z


def obs_adjoint(p, W):
    W = _block(p, W)
    V = np.zeros_like(W)
    lib().o_obs_adjoint(p.ptr, W.shape[0], _dp(W), p.nA, _dp(V))
    return V


def hvp(p, X):
    """Y = A X (eq. 10), X given as (K, nA)."""
    X = _block(p, X)
    Y = np.zeros_like(X)
    lib().o_hvp(p.ptr, X.shape[0], _dp(X), p.nA, _dp(Y))
    return Y


def hvp_count(reset=False):
    return int(lib().o_hvp_count(1 if reset else 0))


def forward_run(p, xb, eta=None):
    out = np.zeros((p.N + 1, p.n))
    lib().o_forward_run(p.ptr, _dp(_f64(xb)), _dp(None if eta is None else _f64(eta)), _dp(out))
    return out


def innovation(p, xb, y, eta=None):
    d = np.zeros(p.nobs)
    lib().o_innovation(p.ptr, _dp(_f64(xb)), _dp(None if eta is None else _f64(eta)),
                       _dp(_f64(y)), _dp(d))
    return d


def rhs(p, d, Dm12b=None):
    out = np.zeros(p.nA)
    lib().o_rhs(p.ptr, _dp(_f64(d)), _dp(None if Dm12b is None else _f64(Dm12b)), _dp(out))
    return out


def qcf(p, x, d, Dm12b=None):
    return float(lib().o_qcf(p.ptr, _dp(_f64(x)), _dp(_f64(d)),
                             _dp(None if Dm12b is None else _f64(Dm12b))))


def householder_qr(A):
    """A given as (k, m) rows = columns; returns Q (k, m) and R (k x k, column-major as (k,k) rows=cols)."""
    A = _f64(A)
    k, m = A.shape
    Q = np.zeros_like(A)
    R = np.zeros((k, k))
    lib().o_householder_qr(m, k, _dp(A), m, _dp(Q), m, _dp(R))
    return Q, R.T.copy()   # R returned in ordinary (row, col) indexing


def jacobi_eig(A):
    """Symmetric EVD; returns w (decreasing) and V with eigenvectors as columns."""
    A = _f64(A)
    m = A.shape[0]
    w = np.zeros(m)
    V = np.zeros((m, m))
    sweeps = lib().o_jacobi_eig(m, _dp(_f64(A.T)), _dp(w), _dp(V))
    return w, V.T.copy(), sweeps


def cholesky_upper(A):
    A = _f64(A)
    m = A.shape[0]
    R = np.zeros((m, m))
    rc = lib().o_cholesky_upper(m, _dp(_f64(A.T)), _dp(R))
    return R.T.copy(), rc


def solve_right_upper(B, R):
    """Solve X R = B; B given as ordinary (rows, m) matrix."""
    Bc = _f64(np.asarray(B).T)        # column-major storage
    rows, m = B.shape
    lib().o_solve_right_upper(rows, m, _dp(_f64(np.asarray(R).T)), _dp(Bc), rows)
    return Bc.T.copy()


def jacobi_svd(A):
    """Thin SVD of an ordinary (rows, m) matrix; returns U (rows, m), s, V (m, m)."""
    A = np.asarray(A)
    rows, m = A.shape
    Ac = _f64(A.T)
    U = np.zeros((m, rows))
    s = np.zeros(m)
    V = np.zeros((m, m))
    rc = lib().o_jacobi_svd(rows, m, _dp(Ac), rows, _dp(U), _dp(s), _dp(V))
    return U.T.copy(), s, V.T.copy(), rc


def _method(fn, p, k, G, *extra):
    G = _block(p, G)
    m = G.shape[0]
    U = np.zeros((k, p.nA))
    th = np.zeros(k)
    rc = fn(p.ptr, int(k), int(m - k), *extra, _dp(G), _dp(U), _dp(th))
    if rc != 0:
        raise RuntimeError(f"oracle eigensolver failed with status {rc}")
    return U, th


def revd(p, k, G, q=0):
    """REVD (Alg. 3) with q power iterations; G is (k+l, nA).  Returns U (k, nA), theta."""
    G = _block(p, G)
    m = G.shape[0]
    U = np.zeros((k, p.nA))
    th = np.zeros(k)
    rc = lib().o_revd(p.ptr, int(k), int(m - k), int(q), _dp(G), _dp(U), _dp(th))
    if rc != 0:
        raise RuntimeError(f"oracle REVD failed with status {rc}")
    return U, th


def nystrom(p, k, G):
    """Randomised Nystrom (Alg. 4)."""
    return _method(lib().o_nystrom, p, k, G)


def ritzit(p, k, G):
    """REVD_ritzit (Alg. 5)."""
    return _method(lib().o_ritzit, p, k, G)


def nystrom_single_pass_core(apply_A, G, k, nu_scale):
    """Single-pass randomised Nystrom approximation of a symmetric positive
    semi-definite operator (Tropp, Yurtsever, Udell, Cevher, SIAM J. Matrix
    Anal. Appl. 2017, fixed-rank PSD approximation from one sketch; the paper
    names a single-pass Nystrom method as future work in Section 6).  Written
    out step by step from that definition:

        Omega = orth(G)                        Householder QR, m columns
        Y     = A Omega                        the only product with A
        nu    = nu_scale * ||Y||_F             stabilising shift
        Y_nu  = Y + nu Omega
        B     = Omega^T Y_nu, symmetrised      m x m
        B     = C^T C                          Cholesky, C upper triangular
        E     = Y_nu C^{-1}                    n x m
        E     = U Sigma V^T                    thin SVD
        theta = max(Sigma^2 - nu, 0)

    apply_A maps a (m, n) block of rows to A applied to each row.  G is
    (m, n).  Returns U (k, n) and theta (k) in decreasing order."""
    G = _f64(np.atleast_2d(G))
    Omega, _ = householder_qr(G)                    # rows = orthonormal columns
    Y = np.asarray(apply_A(Omega), dtype=np.float64)
    nu = nu_scale * np.linalg.norm(Y)
    Ynu = Y + nu * Omega
    B = Omega @ Ynu.T                               # Omega^T Y_nu (m x m)
    B = 0.5 * (B + B.T)
    Cu, rc = cholesky_upper(B)
    if rc != 0:
        raise RuntimeError(f"single-pass Nystrom: Omega^T Y_nu not positive definite (pivot {rc})")
    E = solve_right_upper(Ynu.T, Cu)                # (n, m) = Y_nu C^{-1}
    Ue, s, _, rc = jacobi_svd(E)                    # rc: sweeps used, < 0 if not converged
    if rc < 0:
        raise RuntimeError("single-pass Nystrom: SVD did not converge")
    theta = np.maximum(s * s - nu, 0.0)
    return Ue[:, :k].T.copy(), theta[:k].copy()


NU_SCALE_FP64 = 2.0 ** -52   # times sqrt(n): the shift Tropp et al. use in double precision


def nystrom_single_pass(p, k, G):
    """Single-pass Nystrom on the preconditioned Hessian A of eq. 10 (one
    product with A); nu = sqrt(n_A) 2^-52 ||Y||_F."""
    G = _block(p, G)
    return nystrom_single_pass_core(lambda X: hvp(p, X), G, k, NU_SCALE_FP64 * np.sqrt(p.nA))


def lanczos_cg(p, b, iters, reorth=True, tol=0.0):
    """Unpreconditioned CG (Alg. 1 with C = I) on A x = b from x_0 = 0 that
    keeps what Section 3.3 needs for the Lanczos Ritz pairs: alpha_j, beta_j
    and the normalised residuals, signed as Lanczos vectors: f_j = (-1)^j
    r_j / ||r_j|| (f_0 = b / ||b||).  Section 3.3 writes f_j = r_j / ||r_j||
    with tau_j = sqrt(beta_j) / alpha_j > 0; consecutive CG residuals point
    in opposite senses along the Lanczos basis, so the unsigned vectors give
    F^T A F with off-diagonals -tau_j (same eigenvalues, eigenvectors with
    alternating signs) and the alternation is needed for u_i = F_J w_i.  With
    reorth, every new residual is orthogonalised against all previous f
    (classical Gram-Schmidt, twice) before its norm is taken -- the complete
    reorthogonalisation the paper cites against ghost Ritz values.  Stops
    after `iters` iterations or at relative residual tol.  Returns dict with
    alpha, beta (length J), F (J + 1, n) and x."""
    b = _f64(b)
    n = b.size
    x = np.zeros(n)
    r = b.copy()
    pdir = r.copy()
    rho = float(r @ r)
    bn = np.sqrt(rho)
    F = [r / bn]
    al, be = [], []
    for _ in range(iters):
        q = hvp(p, pdir[None, :])[0]
        alpha = rho / float(pdir @ q)
        x += alpha * pdir
        r = r - alpha * q
        if reorth:
            Fm = np.array(F)
            for _ in range(2):
                r = r - Fm.T @ (Fm @ r)
        rho_new = float(r @ r)
        beta = rho_new / rho
        al.append(alpha)
        be.append(beta)
        F.append((-1.0) ** len(al) * r / np.sqrt(rho_new))
        pdir = r + beta * pdir
        rho = rho_new
        if tol > 0 and np.sqrt(rho) / bn <= tol:
            break
    return dict(alpha=np.array(al), beta=np.array(be), F=np.array(F), x=x)


def lanczos_tridiag(alpha, beta):
    """T_J of Section 3.3 from the CG coefficients (eq. 19-20): gamma_1 =
    1/alpha_1, gamma_j = 1/alpha_j + beta_{j-1}/alpha_{j-1}; tau_j =
    sqrt(beta_j)/alpha_j."""
    J = len(alpha)
    gam = np.empty(J)
    gam[0] = 1.0 / alpha[0]
    for j in range(1, J):
        gam[j] = 1.0 / alpha[j] + beta[j - 1] / alpha[j - 1]
    tau = np.sqrt(beta[:J - 1]) / alpha[:J - 1]
    return np.diag(gam) + np.diag(tau, 1) + np.diag(tau, -1)


def lanczos_ritz(alpha, beta, F, k):
    """Ritz pairs from CG (Section 3.3): the eigenpairs (theta_i, w_i) of T_J,
    decreasing, and u_i = F_J w_i with F_J = (f_0 .. f_{J-1}).  Returns U
    (k, n) and theta (k)."""
    T = lanczos_tridiag(alpha, beta)
    w, V, _ = jacobi_eig(T)             # the oracle's own cyclic Jacobi (numpy's eigh stays a test cross-check)
    order = np.argsort(w)[::-1][:k]
    J = len(alpha)
    U = V[:, order].T @ np.asarray(F)[:J]
    return U, w[order]


def lmp_apply(U, theta, v, transpose=False):
    """C v (or C^T v) for the spectral-LMP factor of eq. 16; U is (k, nA)."""
    U = _f64(np.atleast_2d(U)) if U is not None and len(theta) else np.zeros((0, len(v)))
    theta = _f64(theta)
    v = _f64(v)
    y = np.zeros_like(v)
    lib().o_lmp_apply(len(v), len(theta), _dp(U) if len(theta) else None, _dp(theta) if len(theta) else None,
                      1 if transpose else 0, _dp(v), _dp(y))
    return y


def pcg(p, b, U=None, theta=None, tol=1e-6, maxit=5000, force_iters=0):
    """Split-preconditioned CG (Alg. 1) from x_0 = 0.  Returns dict with x, iters,
    relres, status, qcf_drop (per iteration) and relres_hist."""
    b = _f64(b)
    k = 0 if theta is None else len(theta)
    Uc = _f64(U) if k else None
    th = _f64(theta) if k else None
    x = np.zeros(p.nA)
    iters = C.c_int32(0)
    rr = C.c_double(0.0)
    cap = max(maxit, force_iters, 1)
    drop = np.zeros(cap)
    hist = np.zeros(cap)
    rc = lib().o_pcg(p.ptr, _dp(b), k, _dp(Uc), _dp(th), float(tol), int(maxit), int(force_iters),
                     _dp(x), C.byref(iters), C.byref(rr), _dp(drop), _dp(hist))
    it = iters.value
    return dict(x=x, iters=it, relres=rr.value, status=int(rc), qcf_drop=drop[:it].copy(),
                relres_hist=hist[:it].copy())


# ---------------------------------------------------------------------------
# Learned sketch proposal (not in the paper): the same fixed 4-layer periodic
# 1D convolutional encoder the library runs, written out plainly in numpy
# FP64 from its definition (input: states at the subwindow boundaries / F and
# the observation masks; layers 2(N+1)->64 (width 5, ReLU), 64->64 (width 5,
# ReLU) twice, 64->m(N+1) (width 1); output channel j(N+1)+t = time block t of
# column j).  Pinned by the periodic-convolution identities in the tests.
# ---------------------------------------------------------------------------
def bf16_to_f64(u16):
    """BF16 bit patterns (uint16) to float64: the top 16 bits of an FP32."""
    u = np.asarray(u16, dtype=np.uint16).astype(np.uint32) << 16
    return u.view(np.float32).astype(np.float64)


def periodic_conv1d(x, W, b):
    """y[o, s] = b[o] + sum_{i,k} W[o, i, k] x[i, (s + k - width//2) mod n]."""
    cout, cin, width = W.shape
    n = x.shape[1]
    h = width // 2
    y = np.repeat(np.asarray(b, dtype=np.float64)[:, None], n, axis=1)
    for k in range(width):
        xs = np.roll(x, -(k - h), axis=1)           # xs[i, s] = x[i, (s + k - h) mod n]
        y += W[:, :, k] @ xs
    return y


def learned_probes(traj_boundaries, F, mask, weights, biases, m):
    """traj_boundaries: (N+1, n) states at the subwindow boundaries; mask:
    (N+1, n) observation mask; weights: the four (out, in, width) arrays;
    biases: the four bias vectors.  Returns S (m, (N+1) n)."""
    Np1, n = traj_boundaries.shape
    x = np.concatenate([np.asarray(traj_boundaries, dtype=np.float64) / F, np.asarray(mask, dtype=np.float64)])
    for li in range(4):
        x = periodic_conv1d(x, weights[li], biases[li])
        if li < 3:
            x = np.maximum(x, 0.0)
    return x.reshape(m, Np1, n).reshape(m, Np1 * n)
