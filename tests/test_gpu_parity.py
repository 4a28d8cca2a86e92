"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Sketch indices and signs: bit-exact.  Sketch Y, R, M, x: FP64 tolerances
derived from the summation lengths and condition numbers (each test states
its bound).  Solutions: Karlson-Waldén backward error <= 1e-10 and the
residual-norm distance ||A (x_gpu - x_oracle)|| / ||b|| <= 1e-10."""
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ---------------------------------------------------------------- sketch ---
@pytest.mark.parametrize("d,zeta,row0,rows", [(800, 8, 0, 20011), (2000, 8, 123456789, 5000), (9, 8, 0, 3001),
                                              (8, 8, 17, 1000), (64, 64, 0, 777), (100, 1, 5, 999),
                                              (40, 16, 2**40, 1234), (3000, 33, 7, 2049)])
def test_sketch_indices_bit_exact(ctx, orc, d, zeta, row0, rows):
    idx, sgn, rnd = ctx.lsq_sketch_indices(42, row0, rows, d, zeta, with_rounds=True)
    oi, os_, orr = orc.sketch_indices(42, row0, rows, d, zeta, with_rounds=True)
    assert np.array_equal(idx.cpu().numpy(), oi)
    assert np.array_equal(sgn.cpu().numpy(), os_)
    assert np.array_equal(rnd.cpu().numpy(), orr)


# larger m: many row blocks, ragged last warp block (70001), wide d, zeta < 8, no b
@pytest.mark.parametrize("m,n,d,zeta,has_b", [(20000, 200, 800, 8, True), (3001, 37, 120, 8, True),
                                              (513, 1, 16, 3, False), (1000, 129, 400, 16, True),
                                              (257, 64, 300, 64, True), (80000, 50, 300, 8, True),
                                              (70001, 33, 2560, 5, True), (66000, 16, 64, 8, False)])
def test_sketch_apply_fp64(ctx, orc, m, n, d, zeta, has_b):
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m) if has_b else None
    Y = ctx.lsq_sketch(_dev(A), _dev(b) if has_b else None, d, zeta, 7).cpu().numpy()
    Yo = orc.sketch_apply(A, b, d, zeta, 7)
    # each entry sums ~m*zeta/d terms of size ~1/sqrt(zeta) in a different order:
    # |error| <= (terms) * eps * max partial sum; bound it by 64 * eps * sum|terms|
    k = m * zeta / d
    tol = 64 * 2.2e-16 * k / np.sqrt(zeta) * 4
    assert np.max(np.abs(Y - Yo)) <= tol, np.max(np.abs(Y - Yo))


@pytest.mark.parametrize("ldy_pad", [None, 201])
def test_sketch_apply_mixed_fp32(ctx, orc, ldy_pad):
    """FP32 accumulation (mixed form): every term added in FP32 into chunk
    sums, the chunk sums combined in FP64, the result rounded once to FP32
    into Y (any row stride).  Against the oracle's FP64 sketch: within the
    FP32 rounding of Yo times the growth of a chunk's FP32 sum (here at most
    m zeta / d = 200 terms per entry in all: sqrt(200) u32 relative in norm
    bounds it)."""
    A, b, _ = _problem(20000, 200, 1e8, 3)
    Y = ctx.lsq_sketch(_dev(A), _dev(b), 800, 8, 9, prec=1, ldy=ldy_pad).cpu().numpy().astype(np.float64)
    Yo = orc.sketch_apply(A, b, 800, 8, 9)
    u32 = 2.0 ** -24
    assert np.linalg.norm(Y - Yo) <= (1 + np.sqrt(200)) * u32 * np.linalg.norm(Yo)


@pytest.mark.parametrize("m,n,d,zeta,has_b", [(20011, 33, 120, 16, False), (7777, 64, 300, 32, True),
                                              (3001, 5, 64, 64, True), (90001, 129, 2600, 8, True),
                                              (257, 17, 40, 3, True)])
def test_sketch_apply_mixed_variants(ctx, orc, m, n, d, zeta, has_b):
    """The FP32 chunk-sum sketch for every zeta register width (8, 16, 32, 64),
    without b, with ragged last chunks and rows per warp from 1 to 32: within
    the FP32 error of one sum over all m zeta / d terms of each entry (the
    chunk sums can only be better) plus the final rounding."""
    rng = np.random.default_rng(m + d)
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m) if has_b else None
    Y = ctx.lsq_sketch(_dev(A), _dev(b) if has_b else None, d, zeta, 17, prec=1).cpu().numpy().astype(np.float64)
    Yo = orc.sketch_apply(A, b, d, zeta, 17)
    u32 = 2.0 ** -24
    assert np.linalg.norm(Y - Yo) <= (1 + np.sqrt(m * zeta / d)) * u32 * np.linalg.norm(Yo)


def test_sketch_apply_column_slabs(ctx, orc):
    """A sketch larger than one L2-sized column slab (6400 x 1001: 51 MB in
    FP64, 77 MB of pairs and chunk sums) is built slab by slab in both forms:
    every column, b's included, against the oracle's sketch."""
    m, n, d = 4000, 1000, 6400
    rng = np.random.default_rng(77)
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    Ad, bd = _dev(A), _dev(b)
    Yo = orc.sketch_apply(A, b, d, 8, 23)
    Y64 = ctx.lsq_sketch(Ad, bd, d, 8, 23, prec=0).cpu().numpy()
    k = m * 8 / d
    assert np.max(np.abs(Y64 - Yo)) <= 64 * 2.2e-16 * k / np.sqrt(8) * 4
    Y32 = ctx.lsq_sketch(Ad, bd, d, 8, 23, prec=1).cpu().numpy().astype(np.float64)
    u32 = 2.0 ** -24
    assert np.linalg.norm(Y32 - Yo) <= (1 + np.sqrt(k)) * u32 * np.linalg.norm(Yo)
    # per column: no slab left out or added twice
    col = np.linalg.norm(Y32 - Yo, axis=0) / np.linalg.norm(Yo, axis=0)
    assert col.max() <= 8 * u32, col.max()


def test_sketch_apply_mixed_blocked_large(ctx, orc):
    """~5000 terms per entry (m zeta / d at 2.5e6 rows, d = 4000): one FP32
    sum over all of them would be off by ~0.3 sqrt(5000) u32 = 1.3e-6
    relative (measured with plain FP32 accumulation); the chunked sum (about
    16-20 terms per chunk sum) stays within 6 u32 of the FP64 sketch in norm,
    near the 0.3 u32 of rounding Yo once."""
    m, n, d = 2_500_000, 8, 4000
    rng = np.random.default_rng(21)
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    Ad, bd = _dev(A), _dev(b)
    Y = ctx.lsq_sketch(Ad, bd, d, 8, 13, prec=1).cpu().numpy().astype(np.float64)
    Y64 = ctx.lsq_sketch(Ad, bd, d, 8, 13, prec=0).cpu().numpy()
    Yo = orc.sketch_apply(A, b, d, 8, 13)
    assert np.max(np.abs(Y64 - Yo)) <= 1e-12 * np.abs(Yo).max()
    u32 = 2.0 ** -24
    err = np.linalg.norm(Y - Yo) / np.linalg.norm(Yo)
    assert err <= 6 * u32, err


def test_precond_fp32_from_fp32_sketch(ctx, orc):
    """Mixed form: FP32 sketch and FP32 Householder QR still precondition a
    cond-1e6 problem to cond(AM) near the FP64 value (same iterations +-2)."""
    A, b, _ = _problem(6000, 64, 1e6, 31)
    Y32 = ctx.lsq_sketch(_dev(A), _dev(b), 256, 8, 5, prec=1)
    R, M, x0 = ctx.lsq_precond(Y32, 64, has_b=True)
    M = M.cpu().numpy()
    sv = np.linalg.svd(A @ M, compute_uv=False)
    Yo = orc.sketch_apply(A, b, 256, 8, 5)
    Ro, _, _ = orc.householder_qr(Yo)
    svo = np.linalg.svd(A @ orc.tri_inverse(Ro[:64, :64]), compute_uv=False)
    assert sv[0] / sv[-1] <= 1.05 * svo[0] / svo[-1]
    Mo = orc.tri_inverse(Ro[:64, :64])
    assert np.linalg.norm(A @ (x0.cpu().numpy() - Mo @ Ro[:64, 64])) <= 1e-5 * np.linalg.norm(b)


@pytest.mark.parametrize("m,n,d", [(20000, 300, 1200), (8000, 130, 300)])
def test_precond_fp32_blocked(ctx, orc, m, n, d):
    """Mixed form, blocked FP32 QR (one-block panels of 64, trailing updates as
    FP32-accurate tensor-core GEMMs): cond(AM) stays at the FP64 value."""
    A, b, _ = _problem(m, n, 1e5, n + 7)
    Y32 = ctx.lsq_sketch(_dev(A), _dev(b), d, 8, 5, prec=1)
    ctx.lsq_set_qr_mode(2)
    try:
        R, M, x0 = ctx.lsq_precond(Y32, n, has_b=True)
    finally:
        ctx.lsq_set_qr_mode(0)
    M = M.cpu().numpy()
    sv = np.linalg.svd(A @ M, compute_uv=False)
    Yo = orc.sketch_apply(A, b, d, 8, 5)
    Ro, _, _ = orc.householder_qr(Yo)
    Mo = orc.tri_inverse(Ro[:n, :n])
    svo = np.linalg.svd(A @ Mo, compute_uv=False)
    assert sv[0] / sv[-1] <= 1.05 * svo[0] / svo[-1]
    assert np.linalg.norm(A @ (x0.cpu().numpy() - Mo @ Ro[:n, n])) <= 1e-4 * np.linalg.norm(b)


@pytest.mark.parametrize("mode", [1, 2])
def test_solve_mixed_matches_plain_wide(ctx, orc, mode):
    A, b, xt = _problem(40000, 600, 1e6, 45)
    ctx.lsq_set_qr_mode(mode)
    try:
        xp, ip = ctx.lsq_solve(_dev(A), _dev(b), 2400, seed=3, tol=1e-12, prec=0)
        xm, im = ctx.lsq_solve(_dev(A), _dev(b), 2400, seed=3, tol=1e-12, prec=1)
    finally:
        ctx.lsq_set_qr_mode(0)
    assert ip["status"] == 0 and im["status"] == 0 and im["precond_fallback"] == 0
    bn = np.linalg.norm(b)
    assert np.linalg.norm(A @ (xm.cpu().numpy() - xp.cpu().numpy())) <= 1e-10 * bn
    assert orc.backward_error_kw(A, b, xp.cpu().numpy()) <= 1e-10


def test_solve_mixed_falls_back_when_fp32_sketch_is_too_coarse(ctx, orc):
    """cond 1e12: the FP32 sketch cannot precondition; the mixed solve stalls,
    re-solves in FP64 and still meets the accuracy bar."""
    A, b, xt = _problem(20000, 64, 1e12, 43)
    x, info = ctx.lsq_solve(_dev(A), _dev(b), 256, seed=3, tol=1e-12, prec=1)
    assert info["status"] == 0 and info["precond_fallback"] == 1
    assert orc.backward_error_kw(A, b, x.cpu().numpy()) <= 1e-10
    import paper_2506_03070_gb300 as P
    with pytest.raises(P.LsqError) as e:
        ctx.lsq_solve(_dev(A), _dev(b), 256, seed=3, tol=1e-12, prec=1, flags=P.FLAG_NO_FALLBACK)
    assert e.value.status == -7


def test_solve_mixed_matches_plain(ctx, orc):
    A, b, xt = _problem(30000, 128, 1e7, 41)
    xp, ip = ctx.lsq_solve(_dev(A), _dev(b), 512, seed=3, tol=1e-12, prec=0)
    xm, im = ctx.lsq_solve(_dev(A), _dev(b), 512, seed=3, tol=1e-12, prec=1)
    assert im["precond_fallback"] == 0
    bn = np.linalg.norm(b)
    # the FP32 chunk sums leave the sketch ~1e-7 off the FP64 one: kappa(AM)
    # and the counts stay within 10% of the plain form's
    assert abs(ip["iters"] - im["iters"]) <= max(2, int(0.1 * ip["iters"])), (ip["iters"], im["iters"])
    assert np.linalg.norm(A @ (xm.cpu().numpy() - xp.cpu().numpy())) <= 1e-10 * bn
    assert orc.backward_error_kw(A, b, xm.cpu().numpy()) <= 1e-10


def test_sketch_apply_row_stride(ctx, orc):
    rng = np.random.default_rng(1)
    Afull = rng.standard_normal((1000, 41))
    A = Afull[:, :37]
    b = rng.standard_normal(1000)
    At = _dev(Afull)[:, :37]
    Y = ctx.lsq_sketch(At, _dev(b), 100, 8, 5).cpu().numpy()
    Yo = orc.sketch_apply(A, b, 100, 8, 5)
    assert np.max(np.abs(Y - Yo)) <= 1e-13


def test_sketch_rejects_bad_arguments(ctx):
    import paper_2506_03070_gb300 as P
    A = torch.zeros((10, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(P.LsqError) as e:
        ctx.lsq_sketch(A, None, 4, 8, 1)
    assert e.value.status == -1
    with pytest.raises(P.LsqError):
        ctx.lsq_sketch(A, None, 10, 65, 1)


def test_sketch_detects_nonfinite(ctx):
    import paper_2506_03070_gb300 as P
    A = torch.ones((300, 5), dtype=torch.float64, device="cuda")
    A[123, 2] = float("nan")
    with pytest.raises(P.LsqError) as e:
        ctx.lsq_sketch(A, None, 20, 8, 1)
    assert e.value.status == -9


# ---------------------------------------------------------- precondition ---
# mode 2 forces the blocked QR (panels of 32 in FP64, rows spread over blocks;
# 700 = 21 panels + a remainder of 28; 129 = 4 panels + 1), mode 1 the unblocked
@pytest.mark.parametrize("m,n,d,cond,mode", [(20000, 200, 800, 1e8, 1), (3000, 31, 124, 1e4, 0),
                                             (500, 1, 8, 1.0, 0), (4000, 64, 65, 1e6, 0),
                                             (20000, 200, 800, 1e8, 2), (12000, 700, 1400, 1e6, 2),
                                             (6000, 129, 600, 1e8, 2)])
def test_precond_matches_oracle(ctx, orc, m, n, d, cond, mode):
    A, b, _ = _problem(m, n, cond, n)
    Yo = orc.sketch_apply(A, b, d, 8, 11)
    ctx.lsq_set_qr_mode(mode)
    try:
        R, M, x0 = ctx.lsq_precond(_dev(Yo), n, has_b=True)
    finally:
        ctx.lsq_set_qr_mode(0)
    R, M, x0 = R.cpu().numpy(), M.cpu().numpy(), x0.cpu().numpy()
    Ro, _, _ = orc.householder_qr(Yo)
    Ro = Ro[:n, :n]
    # same reflector sign convention -> same signs; backward-stable QR of the
    # same Y: |R - Ro| <~ d * eps * cond * ||Y||
    nrm = np.linalg.norm(Yo)
    assert np.linalg.norm(R - Ro) <= 50 * d * 2.2e-16 * cond * nrm
    assert np.linalg.norm(R.T @ R - Yo[:, :n].T @ Yo[:, :n]) <= 50 * d * 2.2e-16 * nrm ** 2
    assert np.allclose(np.tril(M, -1), 0.0)
    assert np.linalg.norm(M @ R - np.eye(n)) <= 100 * n * 2.2e-16 * cond * 10
    Mo = orc.tri_inverse(Ro)
    xo = Mo @ orc.householder_qr(Yo)[1][:n, n]
    assert np.linalg.norm(A @ (x0 - xo)) <= 1e-9 * np.linalg.norm(b) * max(1.0, cond * 1e-8)


def test_precond_rank_deficient(ctx, orc):
    import paper_2506_03070_gb300 as P
    rng = np.random.default_rng(4)
    A = rng.standard_normal((2000, 10))
    A[:, 3] = 0.0
    b = rng.standard_normal(2000)
    Y = orc.sketch_apply(A, b, 40, 8, 1)
    with pytest.raises(P.LsqError) as e:
        ctx.lsq_precond(_dev(Y), 10, has_b=True)
    assert e.value.status == -6


# ------------------------------------------------------------------ LSQR ---
@pytest.mark.parametrize("m,n,d,zeta,cond,tol", [(20000, 200, 800, 8, 1e8, 1e-12), (5003, 33, 132, 8, 1e10, 1e-12),
                                                 (777, 1, 4, 3, 1.0, 1e-12), (9000, 512, 2048, 8, 1e6, 1e-12),
                                                 (4000, 64, 256, 8, 1e3, 1e-14)])
def test_lsqr_matches_oracle(ctx, orc, m, n, d, zeta, cond, tol):
    A, b, xt = _problem(m, n, cond, m)
    Yo = orc.sketch_apply(A, b, d, zeta, 3)
    Ro, _, _ = orc.householder_qr(Yo)
    Mo = orc.tri_inverse(Ro[:n, :n])
    x0 = Mo @ Ro[:n, n]
    maxit = orc.default_maxit(n, d, tol)
    ref = orc.lsqr(A, b, Mo, x0, tol, maxit)
    x, info = ctx.lsq_lsqr(_dev(A), _dev(b), _dev(Mo), _dev(x0), tol, maxit)
    x = x.cpu().numpy()
    bn = np.linalg.norm(b)
    assert abs(info["iters"] - ref["iters"]) <= 2, (info["iters"], ref["iters"])
    assert np.linalg.norm(A @ (x - ref["x"])) <= 1e-10 * bn
    assert orc.backward_error_kw(A, b, x) <= 1e-10


def test_lsqr_maxit_reports_noconv(ctx, orc):
    A, b, _ = _problem(3000, 20, 1e4, 5)
    Yo = orc.sketch_apply(A, b, 80, 8, 3)
    Ro, _, _ = orc.householder_qr(Yo)
    Mo = orc.tri_inverse(Ro[:20, :20])
    x0 = Mo @ Ro[:20, 20]
    ref = orc.lsqr(A, b, Mo, x0, 1e-30, 4, trace=True)
    x, info = ctx.lsq_lsqr(_dev(A), _dev(b), _dev(Mo), _dev(x0), 1e-30, 4)
    assert info["status"] == -7 and info["iters"] == 4 and info["stop"] == 3
    # after exactly 4 iterations the iterates agree with the oracle's x_4
    assert np.linalg.norm(A @ (x.cpu().numpy() - ref["trace"][3])) <= 1e-12 * np.linalg.norm(b)


# ----------------------------------------------------------------- check ---
def test_check_matches_oracle(ctx, orc):
    A, b, xt = _problem(6007, 45, 1e5, 8)
    x = xt + 1e-7 * np.random.default_rng(0).standard_normal(45)
    info = ctx.lsq_check(_dev(A), _dev(b), _dev(x))
    eta, parts = orc.backward_error(A, b, x, parts=True)
    assert abs(info["backward_error_ne"] - eta) <= 1e-8 * eta
    assert abs(info["rnorm"] - parts["rnorm"]) <= 1e-10 * parts["rnorm"]
    assert abs(info["anorm_fro"] - parts["fro"]) <= 1e-13 * parts["fro"]
    assert abs(info["xnorm"] - np.linalg.norm(x)) <= 1e-14 * np.linalg.norm(x)


# ------------------------------------------------------------------ solve ---
def test_solve_config0_matches_oracle(ctx, orc):
    """20000 x 200, cond 1e8, ||r_perp|| = 1e-6, d = 800, zeta = 8, tol 1e-12."""
    from paper_2506_03070_gb300 import synth
    p = synth.config0()
    A, b, xt = p["A"].numpy(), p["b"].numpy(), p["x_true"].numpy()
    x, info = ctx.lsq_solve(_dev(A), _dev(b), 800, zeta=8, seed=42, tol=1e-12)
    x = x.cpu().numpy()
    ref = orc.solve(A, b, 800, 8, 42, 1e-12, orc.default_maxit(200, 800, 1e-12))
    bn = np.linalg.norm(b)
    assert info["status"] == 0 and info["stop"] == 1
    assert abs(info["iters"] - ref["iters"]) <= 2
    assert np.linalg.norm(A @ (x - ref["x"])) <= 1e-10 * bn
    assert np.linalg.norm(A @ (x - xt)) <= 1e-10 * bn
    assert orc.backward_error_kw(A, b, x) <= 1e-10
    # the device-side accuracy pass agrees with the oracle's.  r = b - A x
    # cancels ~6 digits here (||r|| / ||b|| ~ 2e-6) and A^T r cancels again,
    # so both sides carry only ~2 significant digits of eta_NE.
    eta = orc.backward_error(A, b, x)
    assert abs(info["backward_error_ne"] - eta) <= 5e-2 * eta
    assert abs(info["rnorm"] - np.linalg.norm(b - A @ x)) <= 1e-8 * info["rnorm"]


@pytest.mark.parametrize("prec", [0, 1])
def test_solve_host_memory_equals_device(ctx, orc, prec):
    A, b, xt = _problem(8000, 100, 1e8, 21)
    xd, infod = ctx.lsq_solve(_dev(A), _dev(b), 400, seed=5, tol=1e-12, prec=prec)
    xh, infoh = ctx.lsq_solve(np.ascontiguousarray(A), b, 400, seed=5, tol=1e-12, prec=prec)
    bn = np.linalg.norm(b)
    assert np.linalg.norm(A @ (xd.cpu().numpy() - xh)) <= 1e-10 * bn
    assert orc.backward_error_kw(A, b, xh) <= 1e-10
    # FP64: the two runs differ only in the order of the sketch's L2 reductions
    # (Y moves at the 1e-16 level), so the iteration counts agree to one.  Mixed
    # form: Y is accumulated in FP32 in that arbitrary order (1e-7 relative) and
    # the FP32 QR carries it into M, so kappa(AM) -- about 4 here, where
    # cond(A) = 1e8 meets FP32's 6e-8 unit roundoff -- moves by a few percent
    # between runs and LSQR's count (~55) with it.
    slack = 1 if prec == 0 else max(1, int(0.1 * infod["iters"]))
    assert abs(infod["iters"] - infoh["iters"]) <= slack, (infod["iters"], infoh["iters"])


@pytest.mark.parametrize("m,n,lda_pad,zeta", [(8000, 100, 0, 8), (6001, 77, 5, 16), (5000, 600, 0, 8),
                                              (3001, 1, 3, 5), (4001, 40, 0, 33)])
def test_solve_pinned_host_memory_read_in_place(ctx, orc, m, n, lda_pad, zeta):
    """Pinned host A and b: the FP64 sketch reads them in place and writes the
    device copy in the same pass.  The solution equals the device-memory
    solve's up to the order of the sketch's reductions (iterations within
    one), the host arrays are untouched, and the accuracy bar holds."""
    A, b, xt = _problem(m, n, 1e6, 500 + n)
    Ap = torch.zeros((m, n + lda_pad), dtype=torch.float64).pin_memory()
    Ap[:, :n] = torch.from_numpy(A)
    bp = torch.from_numpy(b).pin_memory()
    Ah, bh = Ap.numpy()[:, :n], bp.numpy()
    d = max(4 * n + 4, zeta)
    xd, infod = ctx.lsq_solve(_dev(A), _dev(b), d, zeta=zeta, seed=5, tol=1e-12)
    xh, infoh = ctx.lsq_solve(Ah, bh, d, zeta=zeta, seed=5, tol=1e-12)
    bn = np.linalg.norm(b)
    assert infoh["status"] == 0
    assert abs(infod["iters"] - infoh["iters"]) <= 1, (infod["iters"], infoh["iters"])
    assert np.linalg.norm(A @ (xd.cpu().numpy() - xh)) <= 1e-10 * bn
    assert orc.backward_error_kw(A, b, xh) <= 1e-10
    assert np.array_equal(Ah, A) and np.array_equal(bh, b)


def test_solve_edge_shapes(ctx, orc):
    import paper_2506_03070_gb300 as P
    # n = 1, tiny d, ragged m
    A, b, xt = _problem(1001, 1, 1.0, 2)
    x, info = ctx.lsq_solve(_dev(A), _dev(b), 4, zeta=3, seed=1, tol=1e-12)
    assert orc.backward_error_kw(A, b, x.cpu().numpy()) <= 1e-10
    # n beyond the built kernels
    A2 = torch.zeros((600, 4097), dtype=torch.float64, device="cuda")
    with pytest.raises(P.LsqError) as e:
        ctx.lsq_solve(A2, torch.zeros(600, dtype=torch.float64, device="cuda"), 4200)
    assert e.value.status == -10
    # d < n + 1
    with pytest.raises(P.LsqError) as e:
        ctx.lsq_solve(_dev(A), _dev(b), 1)
    assert e.value.status == -1


def test_solve_degenerate_inputs(ctx):
    """Fewer rows than columns: the sketch has rank <= m < n and the rank test
    refuses it (LSQ_ERR_RANK); no rows at all: the sketch is zero in both forms."""
    import paper_2506_03070_gb300 as P
    rng = np.random.default_rng(12)
    A = rng.standard_normal((10, 20))
    b = rng.standard_normal(10)
    with pytest.raises(P.LsqError) as e:
        ctx.lsq_solve(_dev(A), _dev(b), 64, seed=1)
    assert e.value.status == -6
    A0 = torch.zeros((0, 5), dtype=torch.float64, device="cuda")
    b0 = torch.zeros(0, dtype=torch.float64, device="cuda")
    for prec in (0, 1):
        Y = ctx.lsq_sketch(A0, b0, 16, 8, 3, prec=prec)
        assert Y.shape == (16, 6) and not Y.abs().any().item()


def test_solve_largest_n(ctx, orc):
    """n = 4096, the widest rows built (8 warps per row, 512 columns each; 64
    panels of the blocked QR): the solution is the least-squares one (LAPACK's
    pivoted QR on the same A and b) to 1e-10 in the A-norm, KW backward error
    <= 1e-10."""
    import scipy.linalg as sl
    m, n = 12000, 4096
    A, b, xt = _problem(m, n, 1e6, 4096)
    x, info = ctx.lsq_solve(_dev(A), _dev(b), 2 * n + 8, seed=3, tol=1e-12)
    x = x.cpu().numpy()
    assert info["status"] == 0 and info["stop"] in (1, 2)
    xs = sl.lstsq(A, b, lapack_driver="gelsy")[0]
    assert np.linalg.norm(A @ (x - xs)) <= 1e-10 * np.linalg.norm(b)
    assert orc.backward_error_kw(A, b, x) <= 1e-10


def test_solve_tall_matches_oracle(ctx, orc):
    """A taller solve (100000 x 64, d = 256) against the oracle end to end."""
    A, b, xt = _problem(100000, 64, 1e8, 17)
    x, info = ctx.lsq_solve(_dev(A), _dev(b), 256, seed=4, tol=1e-12)
    x = x.cpu().numpy()
    ref = orc.solve(A, b, 256, 8, 4, 1e-12, orc.default_maxit(64, 256, 1e-12))
    assert info["status"] == 0
    assert abs(info["iters"] - ref["iters"]) <= 2
    assert np.linalg.norm(A @ (x - ref["x"])) <= 1e-10 * np.linalg.norm(b)
    assert orc.backward_error_kw(A, b, x) <= 1e-10


def test_solve_automatic_embedding_dimension(ctx, orc):
    """d = 0: lsq_choose_d calibrates on this GPU and picks d from the model."""
    A, b, xt = _problem(60000, 100, 1e8, 51)
    d = ctx.lsq_choose_d(60000, 100, 1e-12)
    assert 125 <= d <= 60000
    x, info = ctx.lsq_solve(_dev(A), _dev(b), 0, seed=3, tol=1e-12)
    assert info["status"] == 0 and info["d_used"] == d
    assert orc.backward_error_kw(A, b, x.cpu().numpy()) <= 1e-10
    assert np.linalg.norm(A @ (x.cpu().numpy() - xt)) <= 1e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("m,n,d,flags", [(20000, 100, 400, 0), (12000, 600, 2400, 0), (12000, 600, 2400, 4),
                                         (8000, 100, 400, 4)])
def test_hbm_matches_oracle(ctx, orc, m, n, d, flags):
    """Heavy-ball momentum (Algorithm 6): the iterates after k updates follow
    the oracle's, and the converged solve takes the oracle's iteration count;
    flags 4 (LSQ_FLAG_NATIVE_FP64): every pass on the FP64 pipe, one warp per
    row (n = 100) or column panels (n = 600)."""
    A, b, xt = _problem(m, n, 1e6, m + n + 1)
    Yo = orc.sketch_apply(A, b, d, 8, 3)
    Ro = np.linalg.qr(Yo, mode="r")
    Mo = orc.tri_inverse(Ro[:n, :n])
    x0 = Mo @ Ro[:n, n]
    eta = np.sqrt(n / d)
    a, beta = orc.hbm_params(eta)
    bn = np.linalg.norm(b)
    for k in (3, 12):
        ref = orc.hbm(A, b, Mo, x0, a, beta, 1e-30, k)
        x, info = ctx.lsq_hbm(_dev(A), _dev(b), _dev(Mo), _dev(x0), 1e-30, k, eta, flags=flags)
        assert info["iters"] == k and info["status"] == -7 and info["stop"] == 3
        assert np.linalg.norm(A @ (x.cpu().numpy() - ref["x"])) <= 1e-10 * bn
    ref = orc.hbm(A, b, Mo, x0, a, beta, 1e-12, 500)
    x, info = ctx.lsq_hbm(_dev(A), _dev(b), _dev(Mo), _dev(x0), 1e-12, 500, eta, flags=flags)
    assert ref["stop"] in (1, 2) and info["status"] == 0
    assert abs(info["iters"] - ref["iters"]) <= 2, (info["iters"], ref["iters"])
    assert orc.backward_error_kw(A, b, x.cpu().numpy()) <= 1e-10


def test_solve_with_hbm_flag(ctx, orc):
    import paper_2506_03070_gb300 as P
    A, b, xt = _problem(30000, 128, 1e8, 62)
    x, info = ctx.lsq_solve(_dev(A), _dev(b), 512, seed=4, tol=1e-12, flags=P.FLAG_HBM)
    assert info["status"] == 0
    assert orc.backward_error_kw(A, b, x.cpu().numpy()) <= 1e-10


@pytest.mark.parametrize("m,n,density,d", [(20000, 50, 0.02, 200), (30000, 120, 0.05, 480), (12000, 300, 0.06, 1200),
                                          (8000, 600, 0.1, 2400)])
def test_solve_csr_matches_oracle_and_dense(ctx, orc, m, n, density, d):
    """Sparse A in CSR form (the paper's random-sign sparse recipe; (20000, 50,
    0.02) leaves most rows empty): the same sketch columns as the dense path, so
    the solve follows the oracle run on the dense form of A.  Mean row lengths
    1, 6, 18 and 60 take the pass with 1, 1, 4 and 32 lanes per row."""
    from paper_2506_03070_gb300 import synth
    p = synth.sparse_sign_problem(m, n, density, seed=m + n, device="cuda")
    A = synth.csr_to_dense(p).cpu().numpy()
    b = p["b"].cpu().numpy()
    x, info = ctx.lsq_solve_csr(p["row_ptr"], p["col_idx"], p["values"], p["b"], n, d, seed=6, tol=1e-12)
    x = x.cpu().numpy()
    ref = orc.solve(A, b, d, 8, 6, 1e-12, orc.default_maxit(n, d, 1e-12))
    bn = np.linalg.norm(b)
    assert info["status"] == 0 and info["d_used"] == d
    assert abs(info["iters"] - ref["iters"]) <= 2, (info["iters"], ref["iters"])
    assert np.linalg.norm(A @ (x - ref["x"])) <= 1e-10 * bn
    assert orc.backward_error_kw(A, b, x) <= 1e-10
    xd, _ = ctx.lsq_solve(_dev(A), _dev(b), d, seed=6, tol=1e-12)
    assert np.linalg.norm(A @ (x - xd.cpu().numpy())) <= 1e-10 * bn
    # heavy-ball momentum and automatic d on the same sparse problem
    import paper_2506_03070_gb300 as P
    xh, ih = ctx.lsq_solve_csr(p["row_ptr"], p["col_idx"], p["values"], p["b"], n, 0, seed=6, tol=1e-12,
                               flags=P.FLAG_HBM)
    assert ih["status"] == 0 and ih["d_used"] > n
    assert orc.backward_error_kw(A, b, xh.cpu().numpy()) <= 1e-10


def test_solve_csr_rejects_malformed_structure(ctx):
    """Row offsets and column indices are checked on the device before any
    kernel indexes by them: a column index out of [0, n), offsets that
    decrease or that do not end at nnz give LSQ_ERR_ARG."""
    import paper_2506_03070_gb300 as P
    from paper_2506_03070_gb300 import synth
    p = synth.sparse_sign_problem(3000, 40, 0.05, seed=8, device="cuda")
    x, info = ctx.lsq_solve_csr(p["row_ptr"], p["col_idx"], p["values"], p["b"], 40, 160, seed=1)
    assert info["status"] == 0
    for what in ("col_n", "col_neg", "rp_dec", "rp_end"):
        rp, ci = p["row_ptr"].clone(), p["col_idx"].clone()
        if what == "col_n":
            ci[len(ci) // 2] = 40
        elif what == "col_neg":
            ci[7] = -1
        elif what == "rp_dec":
            k = 1500
            rp[k] = rp[k + 1] + 1
        else:
            rp[-1] = rp[-1] - 1
        with pytest.raises(P.LsqError) as e:
            ctx.lsq_solve_csr(rp, ci, p["values"], p["b"], 40, 160, seed=1)
        assert e.value.status == -1, what


def test_solve_consistent_system(ctx, orc):
    rng = np.random.default_rng(3)
    A = rng.standard_normal((4000, 30))
    b = A @ rng.standard_normal(30)
    x, info = ctx.lsq_solve(_dev(A), _dev(b), 120, seed=2, tol=1e-12)
    assert info["status"] == 0
    assert np.linalg.norm(b - A @ x.cpu().numpy()) <= 1e-10 * np.linalg.norm(b)


# ------------------------------------------- double-float vs native pass ---
NATIVE = 4  # LSQ_FLAG_NATIVE_FP64
NO_IMAGE = 8  # LSQ_FLAG_NO_IMAGE


@pytest.mark.parametrize("m,n,lda_pad", [(20000, 200, 0), (1001, 64, 0), (150, 8, 0), (7001, 128, 2), (3000, 512, 6),
                                         (5003, 33, 0), (4001, 101, 1), (2000, 1, 0), (3001, 511, 0)])
def test_lsqr_double_float_pass_matches_native_and_oracle(ctx, orc, m, n, lda_pad):
    A, b, xt = _problem(m, n, 1e6, m + n)
    d = 4 * n if 4 * n < m else n + 1
    zeta = min(8, d)
    Yo = orc.sketch_apply(A, b, d, zeta, 3)
    Ro, _, _ = orc.householder_qr(Yo)
    Mo = orc.tri_inverse(Ro[:n, :n])
    x0 = Mo @ Ro[:n, n]
    maxit = orc.default_maxit(n, d, 1e-12)
    ref = orc.lsqr(A, b, Mo, x0, 1e-12, maxit)
    if lda_pad:
        Ap = np.zeros((m, n + lda_pad))
        Ap[:, :n] = A
        Ad = _dev(Ap)[:, :n]
    else:
        Ad = _dev(A)
    x_df, info_df = ctx.lsq_lsqr(Ad, _dev(b), _dev(Mo), _dev(x0), 1e-12, maxit)
    x_nv, info_nv = ctx.lsq_lsqr(Ad, _dev(b), _dev(Mo), _dev(x0), 1e-12, maxit, flags=NATIVE)
    x_ni, info_ni = ctx.lsq_lsqr(Ad, _dev(b), _dev(Mo), _dev(x0), 1e-12, maxit, flags=NO_IMAGE)
    bn = np.linalg.norm(b)
    if n % 2 == 0 and not lda_pad % 2:
        # the float-pair image holds exactly the values the on-the-fly split makes
        assert np.array_equal(x_df.cpu().numpy(), x_ni.cpu().numpy())
    for x, info in ((x_df, info_df), (x_nv, info_nv)):
        x = x.cpu().numpy()
        assert abs(info["iters"] - ref["iters"]) <= 2, (info["iters"], ref["iters"])
        assert np.linalg.norm(A @ (x - ref["x"])) <= 1e-10 * bn
        assert orc.backward_error_kw(A, b, x) <= 1e-10


def test_solve_double_float_repeatable(ctx):
    """The LSQR kernel reduces in a fixed order, so solving the same problem
    twice gives the same iterations; x differs only through the sketch's
    atomic summation order."""
    A, b, _ = _problem(30000, 100, 1e6, 77)
    x1, i1 = ctx.lsq_solve(_dev(A), _dev(b), 400, seed=9, tol=1e-12)
    x2, i2 = ctx.lsq_solve(_dev(A), _dev(b), 400, seed=9, tol=1e-12)
    assert abs(i1["iters"] - i2["iters"]) <= 1
    assert np.linalg.norm(A @ (x1.cpu().numpy() - x2.cpu().numpy())) <= 1e-11 * np.linalg.norm(b)


# ------------------------------------------------ wide rows (n > 512) ---
@pytest.mark.parametrize("m,n,d,lda_pad", [(6000, 513, 1100, 0), (8000, 1000, 2400, 0), (5000, 1100, 2300, 3),
                                           (6000, 1025, 2100, 1), (7000, 2048, 4200, 0), (9000, 2100, 4300, 0)])
def test_lsqr_wide_rows_match_oracle(ctx, orc, m, n, d, lda_pad):
    """Rows shared by 2, 4 or 8 warps (column panels; n = 1025 and 2048 are
    the edges of the 4-warp band).  M comes from LAPACK's
    QR of the oracle's sketch (any upper triangular M is a valid input); the
    iterates must follow the oracle's LSQR."""
    A, b, xt = _problem(m, n, 1e6, m + n)
    Yo = orc.sketch_apply(A, b, d, 8, 3)
    Ro = np.linalg.qr(Yo, mode="r")
    Mo = orc.tri_inverse(Ro[:n, :n])
    x0 = Mo @ Ro[:n, n]
    maxit = orc.default_maxit(n, d, 1e-12)
    ref = orc.lsqr(A, b, Mo, x0, 1e-12, maxit)
    if lda_pad:
        Ap = np.zeros((m, n + lda_pad))
        Ap[:, :n] = A
        Ad = _dev(Ap)[:, :n]
    else:
        Ad = _dev(A)
    x, info = ctx.lsq_lsqr(Ad, _dev(b), _dev(Mo), _dev(x0), 1e-12, maxit)
    x_ni, info_ni = ctx.lsq_lsqr(Ad, _dev(b), _dev(Mo), _dev(x0), 1e-12, maxit, flags=NO_IMAGE)
    bn = np.linalg.norm(b)
    if n % 2 == 0 and not lda_pad % 2:
        assert np.array_equal(x.cpu().numpy(), x_ni.cpu().numpy())
    for xx, inf in ((x, info), (x_ni, info_ni)):
        xx = xx.cpu().numpy()
        assert inf["status"] == 0
        assert abs(inf["iters"] - ref["iters"]) <= 2, (inf["iters"], ref["iters"])
        assert np.linalg.norm(A @ (xx - ref["x"])) <= 1e-10 * bn
        assert orc.backward_error_kw(A, b, xx) <= 1e-10
    # the same rows on the FP64 pipe (LSQ_FLAG_NATIVE_FP64: every pass native,
    # same panel layout): the oracle's iterates too
    x_nv, info_nv = ctx.lsq_lsqr(Ad, _dev(b), _dev(Mo), _dev(x0), 1e-12, maxit, flags=NATIVE)
    assert info_nv["status"] == 0
    assert abs(info_nv["iters"] - ref["iters"]) <= 2, (info_nv["iters"], ref["iters"])
    x_nv = x_nv.cpu().numpy()
    assert np.linalg.norm(A @ (x_nv - ref["x"])) <= 1e-10 * bn
    assert orc.backward_error_kw(A, b, x_nv) <= 1e-10


def test_check_wide_rows_matches_oracle(ctx, orc):
    """Accuracy pass for n > 512 (two warps per row, column panels) in
    native FP64: rnorm and eta agree with the oracle's FP64 residual to
    rounding (r cancels ~1 digit here), ||A||_F to a few ulps."""
    A, b, xt = _problem(7001, 700, 1e5, 8)
    x = xt + 1e-7 * np.random.default_rng(0).standard_normal(700)
    info = ctx.lsq_check(_dev(A), _dev(b), _dev(x))
    eta, parts = orc.backward_error(A, b, x, parts=True)
    assert abs(info["backward_error_ne"] - eta) <= 1e-8 * eta
    assert abs(info["rnorm"] - parts["rnorm"]) <= 1e-10 * parts["rnorm"]
    assert abs(info["anorm_fro"] - parts["fro"]) <= 1e-13 * parts["fro"]


@pytest.mark.parametrize("flags", [0, NATIVE])
def test_solve_wide_rows(ctx, orc, flags):
    """Whole solve (sketch, QR, inverse, LSQR, check) at n = 1000, d = 4n, with
    the double-float passes and with native FP64 ones."""
    A, b, xt = _problem(20000, 1000, 1e8, 31)
    x, info = ctx.lsq_solve(_dev(A), _dev(b), 4000, zeta=8, seed=11, tol=1e-12, flags=flags)
    x = x.cpu().numpy()
    assert info["status"] == 0 and info["stop"] in (1, 2)
    assert orc.backward_error_kw(A, b, x) <= 1e-10
    assert np.linalg.norm(A @ (x - xt)) <= 1e-10 * np.linalg.norm(b)
