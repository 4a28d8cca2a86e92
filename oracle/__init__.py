"""CPU oracle for sparse-sign sketch-and-precondition least squares.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this package; the CUDA library and its
Python binding never do.  It is a ctypes wrapper around ``lsq_oracle.c``: plain,
slow, single-threaded FP64 C written from the paper (arXiv 2506.03070):

* ``philox4x64_10``      -- the counter-based generator both sides implement
                           from its published definition (Salmon et al., SC'11).
* ``sketch_indices``     -- Sec. 3.1.2 rejection sampling + Algorithm 3 signs.
* ``sketch_apply``       -- Y = S [A | b] (Sec. 2.1 definition, Algorithm 1).
* ``householder_qr``     -- Algorithm 1 "QR(Y)" (textbook unblocked Householder).
* ``tri_inverse``        -- Algorithm 1 "M = R^{-1}", explicit (Sec. 3.2).
* ``lsqr``               -- Algorithm 2, preconditioned LSQR.
* ``backward_error``     -- Stewart's normal-equation bound ||A^T r|| / (||A||_F ||r||).
* ``backward_error_kw``  -- Karlson-Waldén estimate of the optimal normwise
                           backward error (the acceptance metric).
* ``solve``              -- Algorithm 1 end to end.
* ``hbm``, ``hbm_params``  -- Algorithm 6 (gradient descent with heavy-ball
                           momentum) with the step/momentum rule of App. C.2,
                           plain numpy.

Pins: every function is checked in ``tests/test_oracle_*.py`` against facts
fixed by the paper or by mathematics (numpy's Philox, closed-form redraw
probabilities, uniformity over subsets, dense S@A, numpy QR/lstsq, scipy
LSQR iterates, the App. A bounds).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lsq_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblsq_oracle.so")
_lib = None

ORC_OK, ORC_ERR_ARG, ORC_ERR_SKETCH, ORC_ERR_RANK, ORC_ERR_NOCONV, ORC_ERR_OOM = 0, -1, -2, -3, -4, -5


_OMP_PATH = os.path.join(_BUILD, "liblsq_oracle_omp.so")


def build(force: bool = False) -> str:
    """Compile lsq_oracle.c with gcc (plain -O2, no fast-math, no OpenMP): the
    single-threaded checker every test uses."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def build_parallel(force: bool = False) -> str:
    """The same source with -O3 -fopenmp: the CPU-baseline build that the
    benchmark times on all host cores (row loops on every thread, per-thread
    partial sums added in thread order).  Tests never load it."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_OMP_PATH) or os.path.getmtime(_OMP_PATH) < os.path.getmtime(_SRC):
        tmp = _OMP_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp", "-o", tmp, _SRC,
               "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _OMP_PATH)
    return _OMP_PATH


def use_parallel(threads: int) -> None:
    """Switch this process's oracle calls to the OpenMP build on `threads`
    threads (the benchmark's CPU baseline only)."""
    global _lib
    os.environ["OMP_NUM_THREADS"] = str(int(threads))
    _lib = None
    _load(build_parallel())
    set_threads(threads)


def set_threads(threads: int) -> None:
    """Threads of the OpenMP build's loops from now on (the checker build
    ignores it)."""
    if _lib is not None and hasattr(_lib, "orc_set_threads"):
        _lib.orc_set_threads(int(threads))


class LsqrInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("stop", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("anorm_est", ctypes.c_double), ("normal_rel", ctypes.c_double), ("rnorm_est", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("stop", ctypes.c_int32), ("sketch_rounds_max", ctypes.c_int32),
                ("backward_error", ctypes.c_double), ("anorm_est", ctypes.c_double)]


def lib():
    if _lib is None:
        _load(build())
    return _lib


def _load(path):
    global _lib
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i64, i32, u64, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
    L.orc_philox4x64_10.argtypes = [P, P, P]
    L.orc_philox4x64_10.restype = None
    L.orc_sketch_row.argtypes = [u64, i64, i64, i32, P, P]
    L.orc_sketch_indices.argtypes = [u64, i64, i64, i64, i32, P, P, P]
    L.orc_sketch_apply.argtypes = [P, i64, i64, i64, P, i64, i32, u64, i64, P, i64]
    L.orc_householder_qr.argtypes = [P, i64, i64, i64, P]
    L.orc_tri_inverse.argtypes = [P, i64, i64, P, i64]
    L.orc_lsqr.argtypes = [P, i64, i64, i64, P, P, P, f64, i64, P, P, P, P]
    L.orc_backward_error.argtypes = [P, i64, i64, i64, P, P, f64, P]
    L.orc_backward_error.restype = f64
    L.orc_solve.argtypes = [P, i64, i64, i64, P, i64, i32, u64, f64, i64, P, P, P, P, P]
    L.orc_set_threads.argtypes = [i32]
    L.orc_set_threads.restype = None
    _lib = L


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    def __init__(self, rc, what):
        super().__init__(f"oracle {what} failed with status {rc}")
        self.rc = rc


def philox4x64_10(counter, key):
    c = np.asarray(counter, dtype=np.uint64).copy()
    k = np.asarray(key, dtype=np.uint64).copy()
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(_p(c), _p(k), _p(out))
    return out


def sketch_indices(seed, row0, rows, d, zeta, with_rounds=False):
    """(idx int32 rows x zeta, sign int8 rows x zeta[, rounds int32 rows])."""
    idx = np.zeros((rows, zeta), dtype=np.int32)
    sgn = np.zeros((rows, zeta), dtype=np.int8)
    rnd = np.zeros(rows, dtype=np.int32)
    rc = lib().orc_sketch_indices(seed, row0, rows, d, zeta, _p(idx), _p(sgn), _p(rnd))
    if rc != ORC_OK:
        raise OracleError(rc, "sketch_indices")
    return (idx, sgn, rnd) if with_rounds else (idx, sgn)


def sketch_apply(A, b, d, zeta, seed, row0=0):
    """Y = S [A | b] (d x (n+1)), or S A (d x n) when b is None."""
    A = _f64(A)
    m, n = A.shape
    bb = None if b is None else _f64(b)
    ncol = n + (0 if b is None else 1)
    Y = np.zeros((d, ncol), dtype=np.float64)
    rc = lib().orc_sketch_apply(_p(A), m, n, n, _p(bb), d, zeta, seed, row0, _p(Y), ncol)
    if rc != ORC_OK:
        raise OracleError(rc, "sketch_apply")
    return Y


def householder_qr(Y):
    """Returns (R_full, tau): R_full holds R in its upper triangle (rows x cols)."""
    W = _f64(Y).copy()
    rows, cols = W.shape
    tau = np.zeros(min(rows, cols), dtype=np.float64)
    rc = lib().orc_householder_qr(_p(W), rows, cols, cols, _p(tau))
    if rc != ORC_OK:
        raise OracleError(rc, "householder_qr")
    return np.triu(W[: min(rows, cols)]), W, tau


def tri_inverse(R):
    R = _f64(R)
    n = R.shape[0]
    M = np.zeros((n, n), dtype=np.float64)
    rc = lib().orc_tri_inverse(_p(R), n, n, _p(M), n)
    if rc != ORC_OK:
        raise OracleError(rc, "tri_inverse")
    return M


def lsqr(A, b, M, x0, tol, maxit, trace=False):
    A, b, M, x0 = _f64(A), _f64(b), _f64(M), _f64(x0)
    m, n = A.shape
    x = np.zeros(n, dtype=np.float64)
    info = LsqrInfo()
    tr = np.zeros((max(maxit, 1), n), dtype=np.float64) if trace else None
    ab = np.zeros((maxit + 2, 2), dtype=np.float64) if trace else None
    rc = lib().orc_lsqr(_p(A), m, n, n, _p(b), _p(M), _p(x0), tol, maxit, _p(x), ctypes.byref(info), _p(tr), _p(ab))
    if rc not in (ORC_OK, ORC_ERR_NOCONV):
        raise OracleError(rc, "lsqr")
    out = {"x": x, "iters": info.iters, "stop": info.stop, "anorm_est": info.anorm_est,
           "normal_rel": info.normal_rel, "rnorm_est": info.rnorm_est, "status": rc}
    if trace:
        out["trace"] = tr[: info.iters]
        out["alpha_beta"] = ab[: info.iters + 1]
    return out


def backward_error(A, b, x, tol=1e-12, parts=False):
    A, b, x = _f64(A), _f64(b), _f64(x)
    m, n = A.shape
    out = np.zeros(3, dtype=np.float64)
    eta = lib().orc_backward_error(_p(A), m, n, n, _p(b), _p(x), tol, _p(out))
    if parts:
        return eta, {"rnorm": out[0], "normal": out[1], "fro": out[2]}
    return eta


def backward_error_kw(A, b, x):
    """Karlson-Waldén estimate of the optimal backward error of x as a
    least-squares solution, relative to ||A||_F:

        mu~(x) = || (||x||^2 A^T A + ||r||^2 I)^{-1/2} A^T r || / ||A||_F,  r = b - A x.

    Grcar, Saunders & Su (2007) show mu~ agrees with the optimal
    Waldén-Karlson-Sun backward error to within a small factor (asymptotically
    exactly as x -> x_star).  Computed without an SVD: with K = [||x|| A ; ||r|| I]
    and K = Q_K R_K, K^T K = ||x||^2 A^T A + ||r||^2 I, so mu~ = ||R_K^{-T} A^T r||.
    Works on numpy arrays (LAPACK QR) or on torch tensors of any device."""
    try:
        import torch
        is_torch = isinstance(A, torch.Tensor)
    except ImportError:  # pragma: no cover
        is_torch = False
    if is_torch:
        import torch
        r = b - A @ x
        g = A.T @ r
        nx, nr = torch.linalg.vector_norm(x), torch.linalg.vector_norm(r)
        n = A.shape[1]
        K = torch.cat([nx * A, nr * torch.eye(n, dtype=A.dtype, device=A.device)], dim=0)
        R = torch.linalg.qr(K, mode="r")[1]
        del K
        y = torch.linalg.solve_triangular(R.T, g[:, None], upper=False)[:, 0]
        return float(torch.linalg.vector_norm(y) / torch.linalg.matrix_norm(A))
    import scipy.linalg as sl
    A, b, x = _f64(A), _f64(b), _f64(x)
    r = b - A @ x
    g = A.T @ r
    n = A.shape[1]
    K = np.vstack([np.linalg.norm(x) * A, np.linalg.norm(r) * np.eye(n)])
    R = np.linalg.qr(K, mode="r")
    y = sl.solve_triangular(R, g, trans="T")
    return float(np.linalg.norm(y) / np.linalg.norm(A))


def solve(A, b, d, zeta, seed, tol, maxit):
    A, b = _f64(A), _f64(b)
    m, n = A.shape
    x = np.zeros(n)
    R = np.zeros((n, n))
    M = np.zeros((n, n))
    x0 = np.zeros(n)
    info = SolveInfo()
    rc = lib().orc_solve(_p(A), m, n, n, _p(b), d, zeta, seed, tol, maxit, _p(x), _p(R), _p(M), _p(x0),
                         ctypes.byref(info))
    if rc not in (ORC_OK, ORC_ERR_NOCONV):
        raise OracleError(rc, "solve")
    return {"x": x, "R": R, "M": M, "x0": x0, "iters": info.iters, "stop": info.stop,
            "backward_error": info.backward_error, "status": rc}


def default_maxit(n, d, tol):
    """10 * ceil(log(tol) / log(sqrt(n/d))): ten times the rate estimate of
    Sec. 4.3 (error ~ (n/d)^{t/2})."""
    rate = np.sqrt(n / d)
    return int(10 * np.ceil(np.log(tol) / np.log(rate)))


def hbm_params(eta_hat):
    """App. C.2 ("Gradient methods"): step alpha = (1 - eta^2)^2 and momentum
    beta = eta^2, rate sqrt(beta).  These are the optimal heavy-ball
    parameters 4/(sqrt(L)+sqrt(mu))^2 and ((sqrt(L)-sqrt(mu))/(sqrt(L)+sqrt(mu)))^2
    for singular values of AM in [1/(1+eta), 1/(1-eta)] -- what a sketch with
    distortion eta leaves (||S A x|| within (1 +- eta) ||A x||, M from QR(SA)),
    and a condition number (1 + eta)/(1 - eta)."""
    eta2 = float(eta_hat) ** 2
    return (1.0 - eta2) ** 2, eta2


def hbm(A, b, M, x0, alpha, beta, tol, maxit, trace=False):
    """Algorithm 6, gradient descent with heavy-ball momentum, in FP64:

        x_{-1} = x_0
        for t = 1, 2, ...:
            g_t = M M^T A^T (b - A x_{t-1})      (= v - M M^T A^T A x_{t-1})
            x_t = x_{t-1} + alpha g_t + beta (x_{t-1} - x_{t-2})

    The algorithm leaves the convergence test open; here, before each update,
    with r = b - A x_{t-1}: stop (1) when ||M^T A^T r|| <= tol ||b||, which
    bounds ||A (x - x_*)|| by tol ||b|| / sigma_min(AM) -- the accuracy target
    of the Sec. 4.3 experiments, ||A (x_* - x)|| <= eps ||b|| (a test relative
    to ||r|| instead has a rounding floor u ||A|| ||x|| / ||r|| far above small
    tolerances when the residual is small); (2) when ||r|| <= tol ||b||; (3)
    after maxit updates."""
    A, b, M, x = _f64(A), _f64(b), _f64(M), _f64(x0).copy()
    x_prev = x.copy()
    bn = float(np.linalg.norm(b))
    iters, stop, rel = 0, 3, 0.0
    tr = []
    while True:
        r = b - A @ x
        q = M.T @ (A.T @ r)
        rn, qn = float(np.linalg.norm(r)), float(np.linalg.norm(q))
        rel = qn / bn if bn > 0 else 0.0
        if qn <= tol * bn:
            stop = 1
            break
        if rn <= tol * bn:
            stop = 2
            break
        if iters >= maxit:
            stop = 3
            break
        x_new = x + alpha * (M @ q) + beta * (x - x_prev)
        x_prev, x = x, x_new
        iters += 1
        if trace:
            tr.append(x.copy())
    out = {"x": x, "iters": iters, "stop": stop, "normal_rel": rel}
    if trace:
        out["trace"] = np.array(tr).reshape(len(tr), -1)
    return out


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
