"""Inputs the double-float LSQR passes must handle like FP64 does, the
accuracy gate of the final check, and the bounded device waits.

The passes split A 2^-sa and b 2^-sb into float pairs, with exact power-of-two
shifts taken from the largest entries, so a problem scaled by any power of two
has the same iterates as the unscaled one (scaled back); entries below
2^-103 of the largest are flushed, a normwise perturbation far below the
1e-10 backward-error bar.  Every solution is compared with the oracle's in the
A-norm, ||A (x - x_oracle)|| <= 1e-10 ||b||, and its Karlson-Walden backward
error (oracle, FP64) must be <= 1e-10."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2506_03070_gb300 import build
    build.build()
    import paper_2506_03070_gb300 as P
    return P.Context(0)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _problem(m, n, cond, seed, resid=1e-6):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (U * np.geomspace(1, 1 / cond, n)) @ V.T
    x = rng.standard_normal(n)
    g = rng.standard_normal(m)
    g -= U @ (U.T @ g)
    g -= U @ (U.T @ g)
    b = A @ x + resid * g / np.linalg.norm(g)
    return A, b, x


NATIVE = 4


@pytest.mark.parametrize("ka,kb", [(-120, -120), (130, 130), (130, 0), (-120, 40), (300, -300), (-400, -400)])
def test_solve_power_of_two_scaled_problem(ctx, orc, ka, kb):
    """A 2^ka, b 2^kb (outside the FP32 range for |k| > 127): the solution is
    x 2^(kb-ka) with the unscaled problem's iterations."""
    m, n, d = 20000, 200, 800
    A, b, xt = _problem(m, n, 1e8, 5)
    ref = orc.solve(A, b, d, 8, 42, 1e-12, orc.default_maxit(n, d, 1e-12))
    As, bs = np.ldexp(A, ka), np.ldexp(b, kb)
    for flags in (0, NATIVE):
        x, info = ctx.lsq_solve(_dev(As), _dev(bs), d, zeta=8, seed=42, tol=1e-12, flags=flags)
        x = np.ldexp(x.cpu().numpy(), ka - kb)  # back to the unscaled problem
        assert info["status"] == 0, info
        assert abs(info["iters"] - ref["iters"]) <= 2, (flags, info, ref["iters"])
        assert np.linalg.norm(A @ (x - ref["x"])) <= 1e-10 * np.linalg.norm(b)
        assert orc.backward_error_kw(A, b, x) <= 1e-10


@pytest.mark.parametrize("ka,kb", [(-130, -130), (140, 0)])
def test_lsqr_power_of_two_scaled_problem(ctx, orc, ka, kb):
    """lsq_lsqr without a sketch first: its range scan sets the shifts."""
    m, n, d = 8000, 100, 400
    A, b, _ = _problem(m, n, 1e6, 6)
    Yo = orc.sketch_apply(A, b, d, 8, 3)
    Ro, _, _ = orc.householder_qr(Yo)
    Mo = orc.tri_inverse(Ro[:n, :n])
    x0 = Mo @ Ro[:n, n]
    maxit = orc.default_maxit(n, d, 1e-12)
    ref = orc.lsqr(A, b, Mo, x0, 1e-12, maxit)
    s = 2.0 ** (ka - kb)  # M of A 2^ka is M 2^-ka; x of (A 2^ka, b 2^kb) is x 2^(kb-ka)
    x, info = ctx.lsq_lsqr(_dev(np.ldexp(A, ka)), _dev(np.ldexp(b, kb)), _dev(np.ldexp(Mo, -ka)),
                           _dev(np.ldexp(x0, kb - ka)), 1e-12, maxit)
    x = x.cpu().numpy() * s
    assert abs(info["iters"] - ref["iters"]) <= 2
    assert np.linalg.norm(A @ (x - ref["x"])) <= 1e-10 * np.linalg.norm(b)


def test_solve_rows_spanning_sixty_decades(ctx, orc):
    """Row scales 10^u, u uniform on [-30, 30]: the largest rows fix x; rows
    below 2^-103 of the largest entry are flushed in the double-float passes
    (a relative perturbation ~1e-31 of A), the FP64 check sees them all."""
    m, n, d = 20000, 50, 400
    rng = np.random.default_rng(11)
    A0 = rng.standard_normal((m, n))
    D = 10.0 ** rng.uniform(-30, 30, m)
    A = A0 * D[:, None]
    xt = rng.standard_normal(n)
    b = A @ xt + 1e-6 * D * rng.standard_normal(m)
    ref = orc.solve(A, b, d, 8, 9, 1e-12, orc.default_maxit(n, d, 1e-12))
    for flags in (0, NATIVE):
        x, info = ctx.lsq_solve(_dev(A), _dev(b), d, zeta=8, seed=9, tol=1e-12, flags=flags)
        x = x.cpu().numpy()
        assert info["status"] == 0, info
        assert np.linalg.norm(A @ (x - ref["x"])) <= 1e-10 * np.linalg.norm(b)
        assert orc.backward_error_kw(A, b, x) <= 1e-10


def test_solve_coherent_rows_like_config1(ctx, orc):
    """The config-1 recipe at 20000 x 200: singular values 1..1e-10, then 1%
    of the rows scaled x1e4, ||r_perp|| = 1e-6 orthogonal to range(A)."""
    from paper_2506_03070_gb300 import synth
    p = synth.dense_problem(20000, 200, 1e10, resid_norm=1e-6, coherent_frac=0.01, coherent_scale=1e4, seed=3)
    A, b, xt = p["A"].numpy(), p["b"].numpy(), p["x_true"].numpy()
    d = 800
    ref = orc.solve(A, b, d, 8, 43, 1e-12, orc.default_maxit(200, d, 1e-12))
    x, info = ctx.lsq_solve(_dev(A), _dev(b), d, zeta=8, seed=43, tol=1e-12)
    x = x.cpu().numpy()
    bn = np.linalg.norm(b)
    assert info["status"] == 0
    assert abs(info["iters"] - ref["iters"]) <= 2, (info["iters"], ref["iters"])
    assert np.linalg.norm(A @ (x - ref["x"])) <= 1e-10 * bn
    assert np.linalg.norm(A @ (x - xt)) <= 1e-10 * bn
    assert orc.backward_error_kw(A, b, x) <= 1e-10


def test_accuracy_gate(ctx, orc):
    """A gate no solution can meet gives LSQ_ERR_ACCURACY with x written
    (the same x as an ungated solve); a disabled gate gives LSQ_OK."""
    import paper_2506_03070_gb300 as P
    A, b, _ = _problem(6000, 60, 1e6, 12)
    x_ok, i_ok = ctx.lsq_solve(_dev(A), _dev(b), 240, seed=4, tol=1e-12)
    assert i_ok["status"] == 0
    # the default gate max(1e-10, tol) holds: min of the two bounds
    assert min(i_ok["backward_error_ne"], i_ok["backward_error_pre"]) <= 1e-10
    x_g, i_g = ctx.lsq_solve(_dev(A), _dev(b), 240, seed=4, tol=1e-12, gate=1e-300, allow=(P.LSQ_ERR_ACCURACY,))
    assert i_g["status"] == P.LSQ_ERR_ACCURACY
    assert np.linalg.norm(A @ (x_g.cpu().numpy() - x_ok.cpu().numpy())) <= 1e-11 * np.linalg.norm(b)
    with pytest.raises(P.LsqError) as e:
        ctx.lsq_solve(_dev(A), _dev(b), 240, seed=4, tol=1e-12, gate=1e-300)
    assert e.value.status == P.LSQ_ERR_ACCURACY
    _, i_off = ctx.lsq_solve(_dev(A), _dev(b), 240, seed=4, tol=1e-12, gate=-1.0)
    assert i_off["status"] == 0


def test_bounded_waits_time_out_and_context_stays_usable(ctx, orc):
    """A grid barrier that can never fill and an mbarrier phase nothing
    completes, each with a 1 ms limit, return LSQ_ERR_TIMEOUT; the same
    context then solves a problem correctly."""
    import time

    import paper_2506_03070_gb300 as P
    ctx.lsq_set_wait_limit(1e-3)
    try:
        for kind in (0, 1):
            t0 = time.perf_counter()
            st = ctx.lsq_selftest_wait(kind)
            dt = time.perf_counter() - t0
            assert st == P.LSQ_ERR_TIMEOUT, (kind, st)
            assert dt < 5.0, dt  # gave up after ~1 ms, not the built-in 20 s
    finally:
        ctx.lsq_set_wait_limit(0.0)
    A, b, xt = _problem(8000, 64, 1e6, 13)
    x, info = ctx.lsq_solve(_dev(A), _dev(b), 256, seed=5, tol=1e-12)
    assert info["status"] == 0
    ref = orc.solve(A, b, 256, 8, 5, 1e-12, orc.default_maxit(64, 256, 1e-12))
    assert np.linalg.norm(A @ (x.cpu().numpy() - ref["x"])) <= 1e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("m,n,lda_pad", [(7001, 700, 0), (5003, 1500, 3), (4001, 3000, 0), (3000, 2049, 1)])
def test_check_wide_rows_native_fp64(ctx, orc, m, n, lda_pad):
    """The accuracy pass for n > 512 (2, 4 or 8 warps per row) is native FP64:
    it matches the oracle's FP64 residual to rounding."""
    A, b, xt = _problem(m, n, 1e5, n)
    x = xt + 1e-7 * np.random.default_rng(0).standard_normal(n)
    if lda_pad:
        Ap = np.zeros((m, n + lda_pad))
        Ap[:, :n] = A
        Ad = _dev(Ap)[:, :n]
    else:
        Ad = _dev(A)
    info = ctx.lsq_check(Ad, _dev(b), _dev(x))
    eta, parts = orc.backward_error(A, b, x, parts=True)
    # r = b - A x cancels ~6 digits; both sides round each entry of A x to
    # ~sqrt(n) u ||A_i|| ||x|| in their own summation order
    bound = 4 * np.sqrt(n) * 2.0 ** -53 * parts["fro"] * np.linalg.norm(x) / parts["rnorm"]
    assert abs(info["rnorm"] - parts["rnorm"]) <= bound * parts["rnorm"]
    assert abs(info["backward_error_ne"] - eta) <= 4 * bound * eta
    assert abs(info["anorm_fro"] - parts["fro"]) <= 1e-13 * parts["fro"]
    assert abs(info["xnorm"] - np.linalg.norm(x)) <= 1e-14 * np.linalg.norm(x)
