"""lsq_check_noalloc: the accuracy pass for callers that may not allocate
device memory (an allocator owned by someone else, a memory plan fixed at
start-up), so they have no lsq_ctx either.  It must give the same results as
lsq_check through the C ABI, call after call, although every call reuses the
same static device scratch.  This file sorts last so that a run stopping at
the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ("rnorm", "arnorm", "anorm_fro", "xnorm", "bnorm", "backward_error_ne", "backward_error_pre")


@pytest.fixture(scope="module")
def lib_and_ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2506_03070_gb300 import build
    build.build()
    import paper_2506_03070_gb300 as P
    return P, P.load(), P.Context(0)


def _problem(m, n, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    A = U * np.geomspace(1, 1e-6, n)
    x = rng.standard_normal(n)
    b = A @ x + 1e-3 * rng.standard_normal(m)
    R = np.linalg.qr(A[: 4 * n], mode="r")
    M = np.linalg.inv(R)
    return [torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (A, b, x + 1e-5, np.triu(M))]


def _noalloc(P, L, A, b, x, M):
    info = P.Info()
    m, n = A.shape
    st = L.lsq_check_noalloc(A.data_ptr(), m, n, A.stride(0), b.data_ptr(), x.data_ptr(),
                             None if M is None else M.data_ptr(), ctypes.byref(info),
                             torch.cuda.current_stream().cuda_stream)
    assert st == 0
    return info.as_dict()


def _same(a, ref):
    for k in FIELDS:
        assert abs(a[k] - ref[k]) <= 1e-12 * max(abs(ref[k]), 1e-300), (k, a[k], ref[k])


def test_noalloc_matches_lsq_check_twice_in_a_row(lib_and_ctx):
    P, L, ctx = lib_and_ctx
    A1, b1, x1, M1 = _problem(5003, 37, 1)   # odd n: unaligned-row path
    A2, b2, x2, M2 = _problem(20000, 200, 2)  # even n: vector path, another M
    first = _noalloc(P, L, A1, b1, x1, M1)
    second = _noalloc(P, L, A2, b2, x2, M2)
    _same(first, ctx.lsq_check(A1, b1, x1, M1))
    _same(second, ctx.lsq_check(A2, b2, x2, M2))
    # a call after a larger one: nothing left over from the 200-column call
    third = _noalloc(P, L, A1, b1, x1, M1)
    _same(third, first)
    no_m = _noalloc(P, L, A2, b2, x2, None)
    _same(no_m, ctx.lsq_check(A2, b2, x2))


def test_noalloc_rejects_n_beyond_its_scratch(lib_and_ctx):
    P, L, _ = lib_and_ctx
    A = torch.zeros((600, 513), dtype=torch.float64, device="cuda")
    b = torch.zeros(600, dtype=torch.float64, device="cuda")
    x = torch.zeros(513, dtype=torch.float64, device="cuda")
    info = P.Info()
    st = L.lsq_check_noalloc(A.data_ptr(), 600, 513, 513, b.data_ptr(), x.data_ptr(), None, ctypes.byref(info),
                             torch.cuda.current_stream().cuda_stream)
    assert st == -1
