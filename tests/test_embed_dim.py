"""Embedding-dimension selection (Sec. 4.3): the library's Lambert W and the
closed-form minimiser of its solve-time model, checked on the CPU (host code
of liblsq, no GPU needed) against scipy's Lambert W, the defining identity,
brute-force minimisation of the same model, and the balance identity the
paper prints for its unit-constant version."""
import math

import numpy as np
import pytest

P = pytest.importorskip("paper_2506_03070_gb300")


@pytest.fixture(scope="module")
def lib():
    from paper_2506_03070_gb300 import build
    build.build()
    return P


def test_lambert_w0_matches_scipy_and_identity(lib):
    special = pytest.importorskip("scipy.special")
    # the branch point: W0(-1/e) = -1 (scipy returns NaN for the rounded -1/e)
    assert abs(lib.lsq_lambert_w0(-1 / math.e) + 1.0) <= 1e-7
    xs = [-0.3678, -0.3, -0.1, -1e-6, 1e-9, 0.5, 1.0, math.e, 10.0, 1e3, 1e8, 1e15]
    for x in xs:
        w = lib.lsq_lambert_w0(x)
        ref = float(special.lambertw(x, 0).real)
        assert abs(w - ref) <= 1e-12 * max(1.0, abs(ref)), (x, w, ref)
        if x > -1 / math.e:
            assert abs(w * math.exp(w) - x) <= 1e-13 * max(1.0, abs(x))
    assert lib.lsq_lambert_w0(0.0) == 0.0
    assert math.isnan(lib.lsq_lambert_w0(-0.5))


def _model(d, m, n, tol, ti, tq):
    return tq * d + (2 * abs(math.log(tol)) / math.log(d / n) + 2) * ti * m


@pytest.mark.parametrize("m,n,tol,ti,tq", [(2_000_000, 500, 1e-12, 9e-10, 1.2e-6), (20000, 200, 1e-12, 2e-9, 3e-7),
                                           (5_000_000, 2000, 1e-12, 1.3e-10, 1e-5), (10**6, 50, 1e-8, 5e-11, 1e-7)])
def test_model_minimiser_matches_brute_force(lib, m, n, tol, ti, tq):
    d = lib.lsq_d_from_model(m, n, tol, ti, tq)
    assert d > n
    grid = np.unique(np.round(np.geomspace(n * 1.001, n * 1e4, 200000)).astype(np.int64))
    grid = grid[grid > n]
    vals = [_model(float(g), m, n, tol, ti, tq) for g in grid]
    best = grid[int(np.argmin(vals))]
    # same minimum to within the grid's spacing and a flat optimum
    assert abs(_model(d, m, n, tol, ti, tq) - min(vals)) <= 1e-6 * min(vals), (d, best)


def test_paper_balance_identity(lib):
    """Sec. 4.3: d = n exp(W(-m log(eps) / n^2)) equalises (log eps / log(n/d)) m n and d n^2."""
    for m, n, eps in [(600000, 300, 1e-5), (600000, 5000, 1e-5), (2_000_000, 500, 1e-12)]:
        d = n * math.exp(lib.lsq_lambert_w0(-m * math.log(eps) / n ** 2))
        lhs = math.log(eps) / math.log(n / d) * m * n
        assert abs(lhs - d * n ** 2) <= 1e-9 * d * n ** 2
