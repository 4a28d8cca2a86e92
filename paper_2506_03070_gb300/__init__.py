"""GB300 (sm_103a) sparse-sign sketch-and-precondition least squares.

Thin ctypes binding over the C ABI of ``include/lsq.h`` (``liblsq.so``, built
in-tree by ``paper_2506_03070_gb300.build``).  Every step of the solve runs in
the library's CUDA kernels; this module only marshals arguments: torch tensors
(device memory, current stream) or numpy arrays (host problems for
``lsq_solve``).  There is no CPU fallback: if the library or a GPU is missing
the calls raise.

Functions carry the C names: ``lsq_sketch_indices``, ``lsq_sketch``,
``lsq_precond``, ``lsq_lsqr``, ``lsq_check``, ``lsq_solve``,
``lsq_solve_batch``, ``lsq_submit``, ``lsq_poll``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblsq.so")

LSQ_OK, LSQ_PENDING = 0, 1
STATUS = {0: "LSQ_OK", 1: "LSQ_PENDING", -1: "LSQ_ERR_ARG", -2: "LSQ_ERR_CUDA", -3: "LSQ_ERR_OOM",
          -4: "LSQ_ERR_BUDGET", -5: "LSQ_ERR_SKETCH", -6: "LSQ_ERR_RANK", -7: "LSQ_ERR_NOCONV",
          -8: "LSQ_ERR_TIMEOUT", -9: "LSQ_ERR_NONFINITE", -10: "LSQ_ERR_UNSUPPORTED", -11: "LSQ_ERR_ACCURACY"}
LSQ_ERR_ARG, LSQ_ERR_NOCONV, LSQ_ERR_TIMEOUT, LSQ_ERR_ACCURACY = -1, -7, -8, -11
PREC_FP64, PREC_MIXED = 0, 1
MEM_DEVICE, MEM_HOST = 0, 1
FLAG_TIMING, FLAG_NO_CHECK, FLAG_NATIVE_FP64, FLAG_NO_IMAGE, FLAG_NO_FALLBACK = 1, 2, 4, 8, 16
FLAG_HBM = 64

EXPORTS = ("lsq_create", "lsq_destroy", "lsq_last_error", "lsq_status_string", "lsq_workspace_bytes",
           "lsq_sketch_indices", "lsq_sketch", "lsq_precond", "lsq_lsqr", "lsq_check", "lsq_solve",
           "lsq_check_noalloc", "lsq_solve_batch", "lsq_submit", "lsq_poll", "lsq_serve_config",
           "lsq_serve_stats_get", "lsq_set_qr_mode", "lsq_choose_d", "lsq_d_from_model", "lsq_lambert_w0",
           "lsq_hbm", "lsq_solve_csr", "lsq_set_wait_limit", "lsq_selftest_wait", "lsq_batch_shape_set",
           "lsq_batch_shape_get")
QR_AUTO, QR_UNBLOCKED, QR_BLOCKED = 0, 1, 2


class LsqError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Problem(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("b", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("lda", ctypes.c_int64), ("mem", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Opts(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int64), ("zeta", ctypes.c_int32), ("prec", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("tol", ctypes.c_double), ("maxit", ctypes.c_int64), ("flags", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("gate", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("stop", ctypes.c_int32), ("iters", ctypes.c_int64),
                ("normal_rel_est", ctypes.c_double), ("backward_error_ne", ctypes.c_double),
                ("backward_error_pre", ctypes.c_double), ("rnorm", ctypes.c_double), ("arnorm", ctypes.c_double),
                ("anorm_fro", ctypes.c_double), ("xnorm", ctypes.c_double), ("bnorm", ctypes.c_double),
                ("sketch_rounds_max", ctypes.c_int32), ("precond_fallback", ctypes.c_int32),
                ("t_sketch_ms", ctypes.c_float), ("t_precond_ms", ctypes.c_float), ("t_lsqr_ms", ctypes.c_float),
                ("t_check_ms", ctypes.c_float), ("t_h2d_ms", ctypes.c_float), ("t_d2h_ms", ctypes.c_float),
                ("t_submit_s", ctypes.c_double), ("t_start_s", ctypes.c_double), ("t_done_s", ctypes.c_double),
                ("group_blocks", ctypes.c_int32), ("t_group_wait_ms", ctypes.c_float), ("d_used", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class CsrProblem(ctypes.Structure):
    _fields_ = [("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("values", ctypes.c_void_p),
                ("b", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64)]


class BatchItem(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("b", ctypes.c_void_p), ("x", ctypes.c_void_p), ("m", ctypes.c_int64),
                ("n", ctypes.c_int64), ("lda", ctypes.c_int64), ("d", ctypes.c_int64), ("zeta", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class BatchResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("stop", ctypes.c_int32), ("iters", ctypes.c_int64),
                ("backward_error_ne", ctypes.c_double), ("rnorm", ctypes.c_double), ("anorm_fro", ctypes.c_double),
                ("xnorm", ctypes.c_double), ("bnorm", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


FLAG_AUTOTUNE = 32


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("pending", ctypes.c_int64),
                ("in_flight", ctypes.c_int64), ("server_launches", ctypes.c_int64), ("grid_blocks", ctypes.c_int64),
                ("arena_bytes", ctypes.c_size_t), ("arena_peak_bytes", ctypes.c_size_t)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}

_lib = None


def load(path: str = LIB_PATH):
    """Load liblsq.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2506_03070_gb300.build`")
    L = ctypes.CDLL(path)
    P, i32, i64, u64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    L.lsq_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_size_t]
    L.lsq_destroy.argtypes = [P]
    L.lsq_last_error.argtypes = [P]
    L.lsq_last_error.restype = ctypes.c_char_p
    L.lsq_status_string.argtypes = [i32]
    L.lsq_status_string.restype = ctypes.c_char_p
    L.lsq_workspace_bytes.argtypes = [P]
    L.lsq_workspace_bytes.restype = ctypes.c_size_t
    L.lsq_sketch_indices.argtypes = [P, u64, i64, i64, i64, i32, P, P, P, P]
    L.lsq_sketch.argtypes = [P, P, i64, i64, i64, P, i64, i32, u64, i32, P, i64, P]
    L.lsq_precond.argtypes = [P, P, i64, i64, i64, i32, i32, P, P, P, P]
    L.lsq_lsqr.argtypes = [P, P, i64, i64, i64, P, P, P, f64, i64, i32, P, P, P]
    L.lsq_hbm.argtypes = [P, P, i64, i64, i64, P, P, P, f64, i64, f64, i32, P, P, P]
    L.lsq_solve_csr.argtypes = [P, ctypes.POINTER(CsrProblem), ctypes.POINTER(Opts), P, ctypes.POINTER(Info), P]
    L.lsq_solve_csr.restype = i32
    L.lsq_hbm.restype = i32
    L.lsq_check.argtypes = [P, P, i64, i64, i64, P, P, P, P, P]
    L.lsq_solve.argtypes = [P, ctypes.POINTER(Problem), ctypes.POINTER(Opts), P, ctypes.POINTER(Info), P]
    L.lsq_check_noalloc.argtypes = [P, i64, i64, i64, P, P, P, ctypes.POINTER(Info), P]
    L.lsq_check_noalloc.restype = i32
    L.lsq_solve_batch.argtypes = [P, ctypes.POINTER(BatchItem), i64, f64, i64, i32, ctypes.POINTER(BatchResult), P]
    L.lsq_solve_batch.restype = i32
    L.lsq_submit.argtypes = [P, ctypes.POINTER(Problem), ctypes.POINTER(Opts), P, ctypes.POINTER(ctypes.c_int64), P]
    L.lsq_poll.argtypes = [P, i64, ctypes.POINTER(Info)]
    L.lsq_serve_config.argtypes = [P, ctypes.c_size_t, f64, i32]
    L.lsq_set_qr_mode.argtypes = [P, i32]
    L.lsq_set_qr_mode.restype = i32
    L.lsq_choose_d.argtypes = [P, i64, i64, f64, ctypes.POINTER(ctypes.c_int64)]
    L.lsq_choose_d.restype = i32
    L.lsq_d_from_model.argtypes = [i64, i64, f64, f64, f64]
    L.lsq_d_from_model.restype = i64
    L.lsq_lambert_w0.argtypes = [f64]
    L.lsq_lambert_w0.restype = f64
    L.lsq_serve_stats_get.argtypes = [P, ctypes.POINTER(ServeStats)]
    L.lsq_set_wait_limit.argtypes = [P, f64]
    L.lsq_selftest_wait.argtypes = [P, i32, P]
    L.lsq_batch_shape_set.argtypes = [P, i32, i32]
    L.lsq_batch_shape_get.argtypes = [P, i32, ctypes.POINTER(i32)]
    for name in ("lsq_batch_shape_set", "lsq_batch_shape_get", "lsq_set_wait_limit", "lsq_selftest_wait", "lsq_create", "lsq_destroy", "lsq_sketch_indices", "lsq_sketch", "lsq_precond", "lsq_lsqr",
                 "lsq_check", "lsq_solve", "lsq_submit", "lsq_poll", "lsq_serve_config", "lsq_serve_stats_get"):
        getattr(L, name).restype = i32
    _lib = L
    return L


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def _dev_f64(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    return t


def _vec(t, length, name, device=None):
    """A CUDA float64 tensor holding exactly `length` contiguous elements (on
    `device` when given): the C calls read or write that many from its first
    element, so a shorter or strided tensor is refused here."""
    _dev_f64(t, name)
    if t.numel() != length or not t.is_contiguous():
        raise ValueError(f"{name} must hold {length} contiguous float64 elements, got shape {tuple(t.shape)}")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, A on {device}")
    return t


def _host_vec(a, length, name):
    """A contiguous float64 numpy copy (or view) of `a` with `length` elements."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != length:
        raise ValueError(f"{name} must hold {length} elements, got shape {a.shape}")
    return a


def _rowmajor(A):
    if A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("A must be a row-major 2-D tensor (unit column stride)")
    return A.shape[0], A.shape[1], A.stride(0)


class Context:
    """One library context (device workspace under an HBM budget)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.lib = load()
        h = ctypes.c_void_p()
        st = self.lib.lsq_create(ctypes.byref(h), device, hbm_budget_bytes)
        if st != LSQ_OK:
            raise LsqError(st, "lsq_create failed (no usable GPU?)")
        self.h = h
        self.device = device
        self._live = {}  # ticket -> (A, b, x): buffers the library reads or writes until completion

    def close(self):
        if getattr(self, "h", None):
            self.lib.lsq_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow=(LSQ_OK,)):
        if st not in allow:
            raise LsqError(st, self.lib.lsq_last_error(self.h).decode())
        return st

    def lsq_choose_d(self, m, n, tol=1e-12):
        """Embedding dimension minimising the modelled solve time on this GPU."""
        d = ctypes.c_int64()
        self._check(self.lib.lsq_choose_d(self.h, m, n, tol, ctypes.byref(d)))
        return d.value

    def lsq_set_qr_mode(self, mode):
        self._check(self.lib.lsq_set_qr_mode(self.h, mode))

    def lsq_set_wait_limit(self, seconds):
        """Limit of every device-side wait of later calls (0: the built-in 20 s)."""
        self._check(self.lib.lsq_set_wait_limit(self.h, float(seconds)))

    def lsq_selftest_wait(self, kind, stream=None):
        """Run a device wait that can never be satisfied (kind 0: grid barrier,
        1: mbarrier) and return its status (LSQ_ERR_TIMEOUT when it gave up)."""
        return self.lib.lsq_selftest_wait(self.h, int(kind), _stream(stream))

    @property
    def workspace_bytes(self):
        return self.lib.lsq_workspace_bytes(self.h)

    # -- C ABI calls -------------------------------------------------------
    def lsq_sketch_indices(self, seed, row0, rows, d, zeta, stream=None, with_rounds=False):
        import torch
        dev = torch.device("cuda", self.device)
        idx = torch.empty((rows, zeta), dtype=torch.int32, device=dev)
        sgn = torch.empty((rows, zeta), dtype=torch.int8, device=dev)
        rnd = torch.empty((rows,), dtype=torch.int32, device=dev) if with_rounds else None
        self._check(self.lib.lsq_sketch_indices(self.h, seed, row0, rows, d, zeta, _ptr(idx), _ptr(sgn), _ptr(rnd),
                                                _stream(stream)))
        return (idx, sgn, rnd) if with_rounds else (idx, sgn)

    def lsq_sketch(self, A, b, d, zeta, seed, prec=PREC_FP64, stream=None, ldy=None):
        """Y = S [A | b]; returns a (d, n+1) view.  ldy (default: n+1 for FP64,
        n+1 rounded up to 4 for FP32, which enables 4-wide reductions)."""
        import torch
        _dev_f64(A, "A")
        m, n, lda = _rowmajor(A)
        if b is not None:
            _vec(b, m, "b", A.device)
        ncol = n + (b is not None)
        if ldy is None:
            ldy = ncol if prec == PREC_FP64 else (ncol + 3) // 4 * 4
        Y = torch.empty((d, ldy), dtype=torch.float64 if prec == PREC_FP64 else torch.float32, device=A.device)
        self._check(self.lib.lsq_sketch(self.h, _ptr(A), m, n, lda, _ptr(b), d, zeta, seed, prec, _ptr(Y), ldy,
                                        _stream(stream)))
        return Y[:, :ncol]

    def lsq_precond(self, Y, n, has_b=True, prec=None, want_R=True, stream=None):
        import torch
        if Y.dim() != 2 or Y.stride(1) != 1 or Y.shape[1] < n + int(bool(has_b)):
            raise ValueError("Y must be a row-major d x (n + has_b) tensor (unit column stride)")
        d, ldy = Y.shape[0], Y.stride(0)
        if prec is None:
            prec = PREC_FP64 if Y.dtype == torch.float64 else PREC_MIXED
        dev = Y.device
        R = torch.empty((n, n), dtype=torch.float64, device=dev) if want_R else None
        M = torch.empty((n, n), dtype=torch.float64, device=dev)
        x0 = torch.empty((n,), dtype=torch.float64, device=dev) if has_b else None
        self._check(self.lib.lsq_precond(self.h, _ptr(Y), d, n, ldy, int(has_b), prec, _ptr(R), _ptr(M), _ptr(x0),
                                         _stream(stream)))
        return R, M, x0

    def lsq_lsqr(self, A, b, M, x0, tol, maxit, flags=0, stream=None):
        import torch
        _dev_f64(A, "A")
        m, n, lda = _rowmajor(A)
        _vec(b, m, "b", A.device)
        _vec(M, n * n, "M", A.device)
        if x0 is not None:
            _vec(x0, n, "x0", A.device)
        x = torch.empty((n,), dtype=torch.float64, device=A.device)
        info = Info()
        st = self.lib.lsq_lsqr(self.h, _ptr(A), m, n, lda, _ptr(b), _ptr(M), _ptr(x0), tol, maxit, flags, _ptr(x),
                               ctypes.byref(info), _stream(stream))
        self._check(st, allow=(LSQ_OK, LSQ_ERR_NOCONV))
        return x, info.as_dict()

    def lsq_hbm(self, A, b, M, x0, tol, maxit, eta_hat, flags=0, stream=None):
        """Heavy-ball momentum (Algorithm 6) from x0; returns (x, info)."""
        import torch
        _dev_f64(A, "A")
        m, n, lda = _rowmajor(A)
        _vec(b, m, "b", A.device)
        _vec(M, n * n, "M", A.device)
        if x0 is not None:
            _vec(x0, n, "x0", A.device)
        x = torch.empty((n,), dtype=torch.float64, device=A.device)
        info = Info()
        st = self.lib.lsq_hbm(self.h, _ptr(A), m, n, lda, _ptr(b), _ptr(M), _ptr(x0), tol, maxit, eta_hat, flags,
                              _ptr(x), ctypes.byref(info), _stream(stream))
        self._check(st, allow=(LSQ_OK, LSQ_ERR_NOCONV))
        return x, info.as_dict()

    def lsq_solve_csr(self, row_ptr, col_idx, values, b, n, d, zeta=8, seed=0, tol=1e-12, maxit=0, flags=0,
                      stream=None, allow_noconv=False, gate=0.0):
        """Algorithm 1 for a sparse A in CSR form (CUDA tensors: int64 row_ptr,
        int32 col_idx, float64 values, float64 b).  Returns (x, info)."""
        import torch
        if row_ptr.dtype != torch.int64 or col_idx.dtype != torch.int32 or values.dtype != torch.float64:
            raise TypeError("row_ptr int64, col_idx int32, values float64")
        m = row_ptr.numel() - 1
        dev = row_ptr.device
        for t, name in ((row_ptr, "row_ptr"), (col_idx, "col_idx"), (values, "values")):
            if not t.is_cuda or not t.is_contiguous() or t.device != dev:
                raise ValueError(f"{name} must be a contiguous CUDA tensor on {dev}")
        if m < 1 or col_idx.numel() != values.numel():
            raise ValueError("need m >= 1 (row_ptr holds m + 1 offsets) and one column index per value")
        _vec(b, m, "b", dev)
        x = torch.empty((n,), dtype=torch.float64, device=b.device)
        pr = CsrProblem(_ptr(row_ptr), _ptr(col_idx), _ptr(values), _ptr(b), m, n, values.numel())
        op = Opts(d, zeta, PREC_FP64, seed, tol, maxit, flags, 0, gate)
        info = Info()
        st = self.lib.lsq_solve_csr(self.h, ctypes.byref(pr), ctypes.byref(op), _ptr(x), ctypes.byref(info),
                                    _stream(stream))
        self._check(st, allow=(LSQ_OK, LSQ_ERR_NOCONV) if allow_noconv else (LSQ_OK,))
        return x, info.as_dict()

    def lsq_check(self, A, b, x, M=None, stream=None):
        _dev_f64(A, "A")
        m, n, lda = _rowmajor(A)
        _vec(b, m, "b", A.device)
        _vec(x, n, "x", A.device)
        if M is not None:
            _vec(M, n * n, "M", A.device)
        info = Info()
        self._check(self.lib.lsq_check(self.h, _ptr(A), m, n, lda, _ptr(b), _ptr(x), _ptr(M), ctypes.byref(info),
                                       _stream(stream)))
        return info.as_dict()

    def lsq_batch_shape_set(self, bucket, shape):
        """Pin the LSQR pass shape of an n-range (bucket 0..3: n <= 32, 64,
        128, 256) for batched and served solves; -1 clears it."""
        self._check(self.lib.lsq_batch_shape_set(self.h, bucket, shape))

    def lsq_batch_shape_get(self, bucket):
        """The pinned pass shape of an n-range, or -1."""
        r = ctypes.c_int32(0)
        self._check(self.lib.lsq_batch_shape_get(self.h, bucket, ctypes.byref(r)))
        return r.value

    def lsq_solve_batch(self, problems, tol=1e-12, maxit=0, flags=0, stream=None, raise_on_error=True):
        """Solve many problems in one persistent launch.  problems: list of
        dicts with CUDA float64 tensors A (m x n, row-major), b and optional d
        (default 4n), zeta (default 8), seed, x.  Returns (xs, results)."""
        items, xs = _batch_items(problems)
        res = (BatchResult * len(problems))()
        st = self.lib.lsq_solve_batch(self.h, items, len(problems), tol, maxit, flags, res, _stream(stream))
        if raise_on_error:
            self._check(st)
        return xs, [r.as_dict() for r in res]

    def lsq_solve(self, A, b, d, zeta=8, seed=0, tol=1e-12, maxit=0, prec=PREC_FP64, flags=0, x=None, stream=None,
                  allow_noconv=False, gate=0.0, allow=None):
        """Algorithm 1 end to end.  A, b: CUDA float64 tensors (device
        problem) or numpy float64 arrays (host problem: copies inside the
        call).  gate: accuracy gate (0: max(1e-10, tol); < 0: none).  allow:
        statuses returned instead of raised.  Returns (x, info dict)."""
        import torch
        if isinstance(A, np.ndarray):
            if A.dtype != np.float64 or A.ndim != 2 or A.strides[1] != 8:
                raise ValueError("host A must be a row-major float64 array")
            m, n = A.shape
            b = _host_vec(b, m, "b")
            lda = A.strides[0] // 8
            mem = MEM_HOST
            if x is None:
                x = np.empty(n, dtype=np.float64)
            elif not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.size == n and x.flags.c_contiguous):
                raise ValueError(f"host x must be a contiguous float64 array of {n} elements")
            strm = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        else:
            _dev_f64(A, "A")
            m, n, lda = _rowmajor(A)
            _vec(b, m, "b", A.device)
            mem = MEM_DEVICE
            if x is None:
                x = torch.empty((n,), dtype=torch.float64, device=A.device)
            else:
                _vec(x, n, "x", A.device)
            strm = _stream(stream)
        pr = Problem(_ptr(A), _ptr(b), m, n, lda, mem, 0)
        op = Opts(d, zeta, prec, seed, tol, maxit, flags, 0, gate)
        info = Info()
        st = self.lib.lsq_solve(self.h, ctypes.byref(pr), ctypes.byref(op), _ptr(x), ctypes.byref(info), strm)
        if allow is None:
            allow = (LSQ_OK, LSQ_ERR_NOCONV) if allow_noconv else (LSQ_OK,)
        self._check(st, allow=allow)
        return x, info.as_dict()

    # -- serving -------------------------------------------------------------
    def lsq_serve_config(self, arena_bytes=0, cta_bytes=0.0, max_group=0):
        self._check(self.lib.lsq_serve_config(self.h, arena_bytes, cta_bytes, max_group))

    def lsq_submit(self, A, b, d, zeta=8, seed=0, tol=1e-12, maxit=0, flags=0, x=None, stream=None, gate=0.0):
        """Queue a problem for the persistent request loop; returns a ticket.
        A, b: CUDA float64 tensors or numpy float64 arrays (host problem).
        They (and x) are kept referenced here until lsq_poll reports the
        request complete.  The request starts after the work already queued
        on `stream` (default: torch's current stream), so tensors that pending
        kernels still use are safe to hand over."""
        import torch
        if isinstance(A, np.ndarray):
            if A.dtype != np.float64 or A.ndim != 2 or A.strides[1] != 8:
                raise ValueError("host A must be a row-major float64 array")
            m, n = A.shape
            b = _host_vec(b, m, "b")
            lda = A.strides[0] // 8
            mem = MEM_HOST
            if x is None:
                x = np.empty(n, dtype=np.float64)
            elif not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.size == n and x.flags.c_contiguous):
                raise ValueError(f"host x must be a contiguous float64 array of {n} elements")
        else:
            _dev_f64(A, "A")
            m, n, lda = _rowmajor(A)
            _vec(b, m, "b", A.device)
            mem = MEM_DEVICE
            if x is None:
                x = torch.empty((n,), dtype=torch.float64, device=A.device)
            else:
                _vec(x, n, "x", A.device)
        pr = Problem(_ptr(A), _ptr(b), m, n, lda, mem, 0)
        op = Opts(d, zeta, PREC_FP64, seed, tol, maxit, flags, 0, gate)
        t = ctypes.c_int64()
        self._check(self.lib.lsq_submit(self.h, ctypes.byref(pr), ctypes.byref(op), _ptr(x), ctypes.byref(t),
                                        _stream(stream)))
        self._live[t.value] = (A, b, x)
        return t.value

    def lsq_poll(self, ticket):
        """None while the request is pending; else (status, x, info dict)."""
        info = Info()
        st = self.lib.lsq_poll(self.h, ticket, ctypes.byref(info))
        if st == LSQ_PENDING:
            return None
        if st == LSQ_ERR_ARG and ticket not in self._live:
            self._check(st)
        _, _, x = self._live.pop(ticket, (None, None, None))
        return st, x, info.as_dict()

    def lsq_wait(self, ticket, timeout=600.0, sleep=50e-6):
        import time
        t0 = time.monotonic()
        while True:
            r = self.lsq_poll(ticket)
            if r is not None:
                return r
            if time.monotonic() - t0 > timeout:
                raise TimeoutError(f"ticket {ticket} still pending after {timeout} s")
            time.sleep(sleep)

    def lsq_serve_stats(self):
        s = ServeStats()
        self._check(self.lib.lsq_serve_stats_get(self.h, ctypes.byref(s)))
        return s.as_dict()


def lsq_lambert_w0(x):
    """Principal branch of the Lambert W function (host code of the library)."""
    return load().lsq_lambert_w0(float(x))


def lsq_d_from_model(m, n, tol, t_iter_per_row, t_qr_per_d):
    """The solve-time model's minimising embedding dimension (no clamping)."""
    return load().lsq_d_from_model(m, n, tol, t_iter_per_row, t_qr_per_d)


def lsq_check_noalloc(A, b, x, M=None, stream=None):
    """Accuracy pass without any device allocation and without a context
    (for callers that may not allocate device memory).  Uses the library's
    static device scratch (n <= 512); calls that overlap on the GPU race.
    Runs on the current CUDA device.  Returns the info dict."""
    L = load()
    _dev_f64(A, "A")
    m, n, lda = _rowmajor(A)
    info = Info()
    st = L.lsq_check_noalloc(_ptr(A), m, n, lda, _ptr(b), _ptr(x), _ptr(M), ctypes.byref(info), _stream(stream))
    if st != LSQ_OK:
        raise LsqError(st, "lsq_check_noalloc failed (n > 512 or CUDA error)")
    return info.as_dict()


def _batch_items(problems):
    import torch
    items = (BatchItem * len(problems))()
    xs = []
    for i, pr in enumerate(problems):
        A, b = pr["A"], pr["b"]
        _dev_f64(A, "A")
        m, n, lda = _rowmajor(A)
        _vec(b, m, "b", A.device)
        x = pr.get("x")
        if x is None:
            x = torch.empty((n,), dtype=torch.float64, device=A.device)
        else:
            _vec(x, n, "x", A.device)
        xs.append(x)
        items[i] = BatchItem(_ptr(A), _ptr(b), _ptr(x), m, n, lda, pr.get("d", 4 * n), pr.get("zeta", 8), 0,
                             pr.get("seed", 0))
    return items, xs


_default = {}


def context(device: int = 0) -> Context:
    """Process-wide default context for `device`."""
    if device not in _default:
        _default[device] = Context(device)
    return _default[device]


def lsq_solve(A, b, d, **kw):
    return context().lsq_solve(A, b, d, **kw)
