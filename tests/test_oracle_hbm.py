"""Pins of the oracle's heavy-ball momentum (Algorithm 6, App. C.2 parameters)
by facts the mathematics fixes: an orthonormal preconditioned matrix is solved
in one step; iterates lie in LSQR's Krylov space, so LSQR's error bounds
theirs from below at every step; the asymptotic rate is sqrt(beta)."""
import numpy as np


def _qr_problem(m, n, seed, sv=None):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((m, n)))
    if sv is not None:
        V, _ = np.linalg.qr(rng.standard_normal((n, n)))
        A = (Q * sv) @ V.T
    else:
        A = Q @ np.triu(rng.standard_normal((n, n)) + 3 * np.eye(n))
    b = rng.standard_normal(m)
    return A, b


def test_params_rule(orc):
    a, b = orc.hbm_params(0.5)
    assert a == (1 - 0.25) ** 2 and b == 0.25
    assert orc.hbm_params(0.0) == (1.0, 0.0)


def test_orthonormal_am_one_step(orc):
    """A = Q R0, M = R0^{-1}: AM = Q, eta = 0 -> alpha = 1, beta = 0, and
    x_1 = x_0 + M M^T A^T (b - A x_0) = R0^{-1} Q^T b is the LS solution."""
    rng = np.random.default_rng(2)
    m, n = 300, 20
    Q, _ = np.linalg.qr(rng.standard_normal((m, n)))
    R0 = np.triu(rng.standard_normal((n, n))) + 4 * np.eye(n)
    A = Q @ R0
    b = rng.standard_normal(m)
    M = np.linalg.inv(R0)
    a, beta = orc.hbm_params(0.0)
    out = orc.hbm(A, b, M, rng.standard_normal(n), a, beta, 1e-12, 5)
    xs = np.linalg.lstsq(A, b, rcond=None)[0]
    assert out["iters"] == 1 and out["stop"] == 1
    assert np.linalg.norm(out["x"] - xs) <= 1e-12 * np.linalg.norm(xs)


def test_lsqr_error_bounds_hbm_error(orc):
    """Both iterate in x_0 + M K_t(M^T A^T A M, M^T A^T r_0); LSQR minimises
    ||A (x - x_*)|| there, so it is never worse than heavy-ball momentum."""
    m, n, eta = 2000, 40, 0.5
    sv = 1.0 / np.linspace(1 - eta, 1 + eta, n)
    A, b = _qr_problem(m, n, 7, sv)
    M = np.eye(n)
    x0 = np.zeros(n)
    xs = np.linalg.lstsq(A, b, rcond=None)[0]
    a, beta = orc.hbm_params(eta)
    T = 25
    h = orc.hbm(A, b, M, x0, a, beta, 1e-30, T, trace=True)
    l = orc.lsqr(A, b, M, x0, 1e-30, T, trace=True)
    for t in range(T):
        eh = np.linalg.norm(A @ (h["trace"][t] - xs))
        el = np.linalg.norm(A @ (l["trace"][t] - xs))
        assert el <= eh * (1 + 1e-9) + 1e-14, (t, el, eh)


def test_rate_is_sqrt_beta(orc):
    """Singular values of AM spread over [1/(1+eta), 1/(1-eta)] (what a sketch
    with distortion eta leaves: ||S A x|| within (1 +- eta) ||A x||): the error
    decays like t eta^t (rate sqrt(beta) = eta, with the double root's factor t)."""
    m, n, eta = 3000, 60, 0.4
    sv = 1.0 / np.linspace(1 - eta, 1 + eta, n)
    A, b = _qr_problem(m, n, 9, sv)
    xs = np.linalg.lstsq(A, b, rcond=None)[0]
    a, beta = orc.hbm_params(eta)
    T = 30
    h = orc.hbm(A, b, np.eye(n), np.zeros(n), a, beta, 1e-30, T, trace=True)
    e0 = np.linalg.norm(A @ xs)
    for t in (10, 20, 30):
        et = np.linalg.norm(A @ (h["trace"][t - 1] - xs))
        assert et <= 4 * t * eta ** t * e0, (t, et / e0, t * eta ** t)
    # and not much faster than eta^t: the rate is sqrt(beta), not better
    e30 = np.linalg.norm(A @ (h["trace"][T - 1] - xs))
    assert e30 >= 1e-3 * eta ** T * e0
