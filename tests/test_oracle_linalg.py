"""Pins for the oracle's sketch apply, Householder QR, triangular inverse,
sketch-and-solve start, LSQR (Algorithm 2) and backward error, each against
numpy/scipy routines, closed forms or the bounds of App. A."""
import numpy as np
import pytest


def _dense_S(idx, sgn, d, zeta):
    m = idx.shape[0]
    S = np.zeros((d, m))
    for i in range(m):
        for k in range(zeta):
            S[idx[i, k], i] = sgn[i, k] / np.sqrt(zeta)
    return S


def _problem(m, n, cond, seed, resid=1e-6):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = np.geomspace(1, 1 / cond, n)
    A = (U * s) @ V.T
    x = rng.standard_normal(n)
    g = rng.standard_normal(m)
    g -= U @ (U.T @ g)
    g -= U @ (U.T @ g)
    b = A @ x + resid * g / np.linalg.norm(g)
    return A, b, x, U


@pytest.mark.parametrize("m,n,d,zeta", [(300, 7, 40, 8), (257, 16, 64, 3), (50, 5, 8, 8)])
def test_sketch_apply_equals_dense_product(orc, m, n, d, zeta):
    rng = np.random.default_rng(m)
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    Y = orc.sketch_apply(A, b, d, zeta, seed=11)
    idx, sgn = orc.sketch_indices(11, 0, m, d, zeta)
    S = _dense_S(idx, sgn, d, zeta)
    ref = S @ np.column_stack([A, b])
    assert np.allclose(Y, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    Y2 = orc.sketch_apply(A, None, d, zeta, seed=11)
    assert np.array_equal(Y2, Y[:, :n])


def test_sketch_columns_unit_norm_and_isometry_in_mean(orc):
    m, d, zeta = 200, 50, 8
    Y = orc.sketch_apply(np.eye(m), None, d, zeta, seed=3)  # = S itself
    assert np.allclose(np.linalg.norm(Y, axis=0), 1.0, atol=1e-15)
    assert np.count_nonzero(Y) == m * zeta
    z = np.random.default_rng(0).standard_normal((m, 1))
    vals = [np.linalg.norm(orc.sketch_apply(z, None, d, zeta, seed=s)) ** 2 for s in range(400)]
    # E ||S z||^2 = ||z||^2; the per-seed variance is ~2||z||^4/d
    assert abs(np.mean(vals) / np.linalg.norm(z) ** 2 - 1) < 5 * np.sqrt(2 / d / 400)


def test_sketch_row_partition_sums(orc):
    """App. B: S A = S[:, I1] A[I1] + S[:, I2] A[I2] with S keyed by global row."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((500, 9))
    b = rng.standard_normal(500)
    Y = orc.sketch_apply(A, b, 60, 8, seed=9)
    Y1 = orc.sketch_apply(A[:173], b[:173], 60, 8, seed=9, row0=0)
    Y2 = orc.sketch_apply(A[173:], b[173:], 60, 8, seed=9, row0=173)
    assert np.allclose(Y1 + Y2, Y, atol=1e-13)


def _q_from_reflectors(W, tau):
    rows, cols = W.shape
    k = len(tau)
    Q = np.eye(rows)
    for j in reversed(range(k)):
        v = np.zeros(rows)
        v[j] = 1.0
        v[j + 1:] = W[j + 1:, j]
        Q -= tau[j] * np.outer(v, v @ Q)
    return Q[:, :k]


@pytest.mark.parametrize("rows,cols,cond", [(40, 10, 1e2), (120, 31, 1e8), (25, 25, 1e3), (60, 1, 1)])
def test_householder_qr(orc, rows, cols, cond):
    rng = np.random.default_rng(rows + cols)
    U, _ = np.linalg.qr(rng.standard_normal((rows, cols)))
    V, _ = np.linalg.qr(rng.standard_normal((cols, cols)))
    Y = (U * np.geomspace(1, 1 / cond, cols)) @ V.T
    R, W, tau = orc.householder_qr(Y)
    Q = _q_from_reflectors(W, tau)
    nrm = np.linalg.norm(Y)
    assert np.linalg.norm(Q.T @ Q - np.eye(cols)) < 1e-14 * rows
    assert np.linalg.norm(Q @ R - Y) < 1e-15 * rows * nrm
    assert np.linalg.norm(R.T @ R - Y.T @ Y) < 1e-15 * rows * nrm ** 2
    Rn = np.linalg.qr(Y, mode="r")
    sg = np.sign(np.diag(R)) * np.sign(np.diag(Rn))
    assert np.linalg.norm(sg[:, None] * R - Rn) < 1e-15 * rows * cond * nrm
    assert np.all(np.abs(np.diag(R)) > 0)


def test_householder_zero_column_below_diagonal(orc):
    Y = np.array([[2.0, 1.0], [0.0, 3.0], [0.0, 4.0]])
    R, W, tau = orc.householder_qr(Y)
    assert tau[0] == 0.0
    assert R[0, 0] == 2.0 and R[0, 1] == 1.0
    assert abs(abs(R[1, 1]) - 5.0) < 1e-15


@pytest.mark.parametrize("n,cond", [(1, 1), (7, 10), (40, 1e6), (100, 1e3)])
def test_tri_inverse(orc, n, cond):
    rng = np.random.default_rng(n)
    R = np.linalg.qr((rng.standard_normal((3 * n, n)) * np.geomspace(1, 1 / cond, n)), mode="r")
    M = orc.tri_inverse(R)
    assert np.allclose(np.tril(M, -1), 0)
    assert np.linalg.norm(R @ M - np.eye(n)) < 1e-15 * n * cond * 10
    Mi = np.linalg.inv(R)
    assert np.linalg.norm(M - Mi) <= 1e-14 * n * cond * np.linalg.norm(Mi)


def test_tri_inverse_rank_error(orc):
    R = np.array([[1.0, 2.0], [0.0, 0.0]])
    with pytest.raises(orc.OracleError):
        orc.tri_inverse(R)


def test_sketch_and_solve_start_equals_lstsq(orc):
    """x0 = M z from the augmented QR of S[A|b] equals argmin ||Sb - SAx||."""
    A, b, _, _ = _problem(2000, 20, 1e6, 1)
    d, zeta = 80, 8
    Y = orc.sketch_apply(A, b, d, zeta, seed=42)
    R, _, _ = orc.householder_qr(Y)
    M = orc.tri_inverse(R[:20, :20])
    x0 = M @ R[:20, 20]
    ref = np.linalg.lstsq(Y[:, :20], Y[:, 20], rcond=None)[0]
    assert np.linalg.norm(A @ (x0 - ref)) < 1e-9 * np.linalg.norm(b)


def test_preconditioned_condition_number(orc):
    """cond(A M) = smax(S U) / smin(S U) when S A M has orthonormal columns
    (App. A.1), and it is close to the Gaussian estimate for d = 4n."""
    A, b, _, U = _problem(4000, 25, 1e8, 2)
    d = 100
    Y = orc.sketch_apply(A, None, d, 8, seed=5)
    R, _, _ = orc.householder_qr(Y)
    M = orc.tri_inverse(R)
    sv = np.linalg.svd(A @ M, compute_uv=False)
    S_U = orc.sketch_apply(U, None, d, 8, seed=5)
    su = np.linalg.svd(S_U, compute_uv=False)
    assert abs(sv[0] / sv[-1] - su[0] / su[-1]) < 1e-6 * su[0] / su[-1]
    eta = max(su[0] - 1, 1 - su[-1])
    assert sv[0] / sv[-1] <= (1 + eta) / (1 - eta) * (1 + 1e-8)
    assert sv[0] / sv[-1] < 6.0


def _sketch_precond(orc, A, b, d, zeta, seed):
    n = A.shape[1]
    Y = orc.sketch_apply(A, b, d, zeta, seed=seed)
    R, _, _ = orc.householder_qr(Y)
    M = orc.tri_inverse(R[:n, :n])
    x0 = M @ R[:n, n]
    return R[:n, :n], M, x0


def test_lsqr_iterates_match_scipy(orc):
    """Algorithm 2 from x0 equals scipy's LSQR on the operator A M started from
    y0 = R x0, iterate by iterate (x_t = M y_t)."""
    from scipy.sparse.linalg import LinearOperator, lsqr
    A, b, _, _ = _problem(1500, 30, 1e7, 3)
    R, M, x0 = _sketch_precond(orc, A, b, 120, 8, 1)
    out = orc.lsqr(A, b, M, x0, tol=0.0, maxit=25, trace=True)
    assert out["iters"] == 25
    op = LinearOperator(A.shape, matvec=lambda y: A @ (M @ y), rmatvec=lambda r: M.T @ (A.T @ r), dtype=np.float64)
    y0 = R @ x0
    for t in (1, 2, 5, 10, 25):
        y = lsqr(op, b, x0=y0, iter_lim=t, atol=0, btol=0, conlim=0)[0]
        xt = M @ y
        err = np.linalg.norm(A @ (out["trace"][t - 1] - xt)) / np.linalg.norm(b)
        assert err < 1e-12, (t, err)


def test_lsqr_converges_to_least_squares_solution(orc):
    """App. A.3: with r_perp orthogonal to range(A), x_true is the LS solution
    and ||A(x - x_true)|| = (||b - A x||^2 - ||r_perp||^2)^{1/2}."""
    A, b, xt, _ = _problem(3000, 30, 1e8, 4, resid=1e-6)
    R, M, x0 = _sketch_precond(orc, A, b, 120, 8, 2)
    maxit = orc.default_maxit(30, 120, 1e-12)
    out = orc.lsqr(A, b, M, x0, tol=1e-12, maxit=maxit)
    assert out["status"] == 0 and out["stop"] == 1
    x = out["x"]
    assert np.linalg.norm(A @ (x - xt)) < 1e-10 * np.linalg.norm(b)
    assert orc.backward_error_kw(A, b, x) < 1e-10
    # iteration count: rate ~ sqrt(n/d) per iteration (Sec. 4.3)
    assert out["iters"] <= 2 * np.log(1e-12) / np.log(np.sqrt(30 / 120))
    # the sketch-and-solve start already satisfies the App. A.2 residual bound
    # with a constant-distortion embedding
    r0 = np.linalg.norm(b - A @ x0)
    assert r0 <= 3.0 * 1e-6


def test_lsqr_consistent_system_stops_on_residual(orc):
    rng = np.random.default_rng(8)
    A = rng.standard_normal((400, 10))
    b = A @ rng.standard_normal(10)
    R, M, x0 = _sketch_precond(orc, A, b, 40, 8, 3)
    x0 = x0 + 1e-3  # perturb so LSQR has work to do
    out = orc.lsqr(A, b, M, x0, tol=1e-12, maxit=200)
    assert out["stop"] in (1, 2)
    assert np.linalg.norm(b - A @ out["x"]) < 1e-10 * np.linalg.norm(b)


def test_lsqr_maxit_status(orc):
    A, b, _, _ = _problem(500, 10, 1e3, 9)
    R, M, x0 = _sketch_precond(orc, A, b, 40, 8, 4)
    out = orc.lsqr(A, b, M, x0, tol=1e-30, maxit=3)
    assert out["iters"] == 3 and out["stop"] == 3 and out["status"] == orc.ORC_ERR_NOCONV


def test_backward_error_is_an_exact_perturbation(orc):
    """x solves the LS problem for A + E with E = -r (A^T r)^T / ||r||^2 and
    ||E||_2 / ||A||_F equals the reported backward error."""
    rng = np.random.default_rng(6)
    A = rng.standard_normal((60, 5))
    b = rng.standard_normal(60)
    x = np.linalg.lstsq(A, b, rcond=None)[0] + 1e-4 * rng.standard_normal(5)
    eta, parts = orc.backward_error(A, b, x, parts=True)
    r = b - A @ x
    g = A.T @ r
    E = -np.outer(r, g) / (r @ r)
    xe = np.linalg.lstsq(A + E, b, rcond=None)[0]
    assert np.linalg.norm(xe - x) < 1e-10 * np.linalg.norm(x)
    assert abs(np.linalg.norm(E, 2) / np.linalg.norm(A) - eta) < 1e-12 * eta
    assert abs(parts["fro"] - np.linalg.norm(A)) < 1e-13 * parts["fro"]
    # the exact LS solution has backward error at rounding level
    assert orc.backward_error(A, b, np.linalg.lstsq(A, b, rcond=None)[0]) < 1e-14


def _wks_optimal_backward_error(A, b, x):
    """Waldén-Karlson-Sun (1995) optimal normwise backward error (A perturbed):
    min(eta, sigma_min([A, eta (I - r r^T/||r||^2)])), eta = ||r||/||x||."""
    r = b - A @ x
    eta = np.linalg.norm(r) / np.linalg.norm(x)
    m = A.shape[0]
    B = np.hstack([A, eta * (np.eye(m) - np.outer(r, r) / (r @ r))])
    return min(eta, np.linalg.svd(B, compute_uv=False)[m - 1]) / np.linalg.norm(A)


def test_backward_error_kw_matches_optimal(orc):
    rng = np.random.default_rng(21)
    for trial in range(12):
        m, n = 14, 5
        A = rng.standard_normal((m, n)) * np.geomspace(1, 10.0 ** -float(trial % 6), n)
        b = rng.standard_normal(m)
        x = np.linalg.lstsq(A, b, rcond=None)[0] + 10.0 ** -float(1 + trial % 7) * rng.standard_normal(n)
        kw = orc.backward_error_kw(A, b, x)
        opt = _wks_optimal_backward_error(A, b, x)
        assert 0.5 * kw <= opt <= 2.0 * kw
        # Stewart's normal-equation quantity is an upper bound on the optimum
        assert opt <= orc.backward_error(A, b, x) * (1 + 1e-8)


def test_solve_end_to_end(orc):
    A, b, xt, _ = _problem(4000, 40, 1e8, 12)
    out = orc.solve(A, b, d=160, zeta=8, seed=42, tol=1e-12, maxit=400)
    assert out["status"] == 0
    assert orc.backward_error_kw(A, b, out["x"]) < 1e-10
    # the loose normal-equation bound stays within a few 1e-10 on this
    # small-residual (||r|| / ||b|| ~ 2e-6), cond 1e8 problem
    assert out["backward_error"] < 1e-9
    assert np.linalg.norm(A @ (out["x"] - xt)) < 1e-10 * np.linalg.norm(b)
    n = 40
    assert np.allclose(out["M"] @ out["R"], np.eye(n), atol=1e-6)


def test_default_maxit_is_ten_times_the_rate_estimate(orc):
    """Reading of the stopping rule: ten times the Sec. 4.3 estimate
    t = log(tol) / log(sqrt(n/d)) iterations, rounded up."""
    assert orc.default_maxit(200, 800, 1e-12) == 400  # sqrt(1/4) = 1/2: 39.9 -> 40
    assert orc.default_maxit(500, 2000, 1e-12) == 400
    assert orc.default_maxit(100, 400, 1e-10) == 340  # 33.2 -> 34
    assert orc.default_maxit(2000, 8000, 1e-12) == 400
    for n, d, tol in [(50, 200, 1e-12), (300, 1200, 1e-8), (64, 1000, 1e-14)]:
        k = orc.default_maxit(n, d, tol) // 10
        assert np.sqrt(n / d) ** k <= tol < np.sqrt(n / d) ** (k - 1)
