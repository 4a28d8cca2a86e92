"""Batched solves (many independent problems, one persistent launch) against
standalone solves and the CPU oracle."""
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


def _problem(m, n, cond, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (U * np.geomspace(1, 1 / cond, n)) @ V.T
    xt = rng.standard_normal(n)
    g = rng.standard_normal(m)
    g -= U @ (U.T @ g)
    b = A @ xt + 1e-6 * g / np.linalg.norm(g)
    return A, b


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


SHAPES = [(3000, 16), (2001, 17), (5000, 33), (1500, 64), (4099, 65), (2500, 100), (3001, 128), (800, 1),
          (6000, 129), (2000, 200), (1200, 255), (5000, 256), (900, 2), (4000, 127)]


def test_batch_matches_standalone_and_oracle(ctx, orc):
    probs, host = [], []
    for k, (m, n) in enumerate(SHAPES):
        A, b = _problem(m, n, 10.0 ** (2 + k % 7), 100 + k)
        d = max(4 * n, n + 1)
        host.append((A, b, d))
        probs.append({"A": _dev(A), "b": _dev(b), "d": d, "zeta": 8 if d >= 8 else d, "seed": 7 + k})
    xs, res = ctx.lsq_solve_batch(probs, tol=1e-12)
    for k, ((A, b, d), x, r) in enumerate(zip(host, xs, res)):
        x = x.cpu().numpy()
        bn = np.linalg.norm(b)
        assert r["status"] == 0 and r["stop"] in (1, 2), (k, r)
        assert orc.backward_error_kw(A, b, x) <= 1e-10, k
        xs1, info = ctx.lsq_solve(probs[k]["A"], probs[k]["b"], d, zeta=probs[k]["zeta"], seed=probs[k]["seed"],
                                  tol=1e-12)
        assert np.linalg.norm(A @ (x - xs1.cpu().numpy())) <= 1e-10 * bn, k
        assert abs(r["iters"] - info["iters"]) <= 2, (k, r["iters"], info["iters"])
        if k < 4:
            ref = orc.solve(A, b, d, probs[k]["zeta"], probs[k]["seed"], 1e-12, orc.default_maxit(A.shape[1], d, 1e-12))
            assert np.linalg.norm(A @ (x - ref["x"])) <= 1e-10 * bn, k
        assert abs(r["rnorm"] - np.linalg.norm(b - A @ x)) <= 1e-6 * r["rnorm"] + 1e-20


def test_batch_each_result_same_alone_and_in_the_mix(ctx):
    """A problem solved inside a large mixed batch gives the same iterate as
    solved alone in a batch of one (fixed-order arithmetic within a block)."""
    probs = []
    for k in range(40):
        m, n = 1000 + 97 * k, 16 + (k * 7) % 100
        A, b = _problem(m, n, 1e6, 300 + k)
        probs.append({"A": _dev(A), "b": _dev(b), "seed": k})
    xs_mix, _ = ctx.lsq_solve_batch(probs, tol=1e-12)
    for k in (0, 13, 39):
        xs_one, _ = ctx.lsq_solve_batch([dict(probs[k], x=None)], tol=1e-12)
        # the sketch accumulates with atomics (order may differ); everything after is deterministic
        A = probs[k]["A"].cpu().numpy()
        b = probs[k]["b"].cpu().numpy()
        assert np.linalg.norm(A @ (xs_mix[k].cpu().numpy() - xs_one[0].cpu().numpy())) <= 1e-12 * np.linalg.norm(b)


def test_batch_autotune_and_reuse(ctx, orc):
    import paper_2506_03070_gb300 as P
    probs, host = [], []
    for k in range(24):
        m, n = 3000 + 11 * k, [24, 48, 96][k % 3]
        A, b = _problem(m, n, 1e5, 500 + k)
        host.append((A, b))
        probs.append({"A": _dev(A), "b": _dev(b), "seed": k})
    xs, res = ctx.lsq_solve_batch(probs, tol=1e-12, flags=P.FLAG_AUTOTUNE)
    for (A, b), x, r in zip(host, xs, res):
        assert r["status"] == 0
        assert orc.backward_error_kw(A, b, x.cpu().numpy()) <= 1e-10


# every pass shape of every n-range, pinned: n at the edges of the range and
# inside it (odd n, a single column pair, rows that do not fill a buffer)
BUCKET_NS = {0: [1, 2, 16, 17, 31, 32], 1: [33, 50, 63, 64], 2: [65, 100, 127, 128], 3: [129, 200, 255, 256]}
SHAPE_CASES = [(0, 0), (0, 2), (0, 5), (1, 1), (1, 2), (1, 3), (2, 3), (2, 4), (2, 5), (3, 5)]


@pytest.mark.parametrize("bucket,shape", SHAPE_CASES)
def test_batch_every_pass_shape(ctx, orc, bucket, shape):
    """Batched solves with the bucket's pass shape pinned (lsq_batch_shape_set):
    each result matches the oracle's solve on the same sketch, and the first
    of the bucket's n also at another row count."""
    probs, host = [], []
    for k, n in enumerate(BUCKET_NS[bucket]):
        for m in (1500 + 37 * k, 803):
            A, b = _problem(m, n, 10.0 ** (3 + k % 5), 900 + 10 * k + m % 7)
            d = max(4 * n, n + 1)
            host.append((A, b, d))
            probs.append({"A": _dev(A), "b": _dev(b), "d": d, "zeta": min(8, d), "seed": 40 + k})
    ctx.lsq_batch_shape_set(bucket, shape)
    try:
        assert ctx.lsq_batch_shape_get(bucket) == shape
        xs, res = ctx.lsq_solve_batch(probs, tol=1e-12)
    finally:
        ctx.lsq_batch_shape_set(bucket, -1)
    assert ctx.lsq_batch_shape_get(bucket) == -1
    for k, ((A, b, d), x, r) in enumerate(zip(host, xs, res)):
        x = x.cpu().numpy()
        bn = np.linalg.norm(b)
        assert r["status"] == 0 and r["stop"] in (1, 2), (k, r)
        assert orc.backward_error_kw(A, b, x) <= 1e-10, k
        ref = orc.solve(A, b, d, probs[k]["zeta"], probs[k]["seed"], 1e-12, orc.default_maxit(A.shape[1], d, 1e-12))
        assert np.linalg.norm(A @ (x - ref["x"])) <= 1e-10 * bn, k
        assert abs(r["iters"] - ref["iters"]) <= 2, (k, r["iters"], ref["iters"])


def test_batch_shape_set_refuses_bad_shapes(ctx):
    """A shape too narrow for the bucket's n, an unknown shape or bucket: LSQ_ERR_ARG, nothing changed."""
    import paper_2506_03070_gb300 as P
    before = [ctx.lsq_batch_shape_get(k) for k in range(4)]
    for bucket, shape in ((0, 6), (1, 0), (2, 2), (3, 4), (4, 0), (-1, 0), (0, -2)):
        with pytest.raises(P.LsqError) as e:
            ctx.lsq_batch_shape_set(bucket, shape)
        assert e.value.status == -1
    assert [ctx.lsq_batch_shape_get(k) for k in range(4)] == before
    with pytest.raises(P.LsqError):
        ctx.lsq_batch_shape_get(4)


def test_batch_item_errors(ctx):
    import paper_2506_03070_gb300 as P
    A, b = _problem(500, 10, 10.0, 1)
    good = {"A": _dev(A), "b": _dev(b)}
    with pytest.raises(P.LsqError) as e:
        ctx.lsq_solve_batch([good, dict(good, zeta=9)])
    assert e.value.status == -1
    with pytest.raises(P.LsqError):
        ctx.lsq_solve_batch([dict(good, d=10)])
    big = torch.zeros((600, 257), dtype=torch.float64, device="cuda")
    with pytest.raises(P.LsqError):
        ctx.lsq_solve_batch([{"A": big, "b": torch.zeros(600, dtype=torch.float64, device="cuda")}])
    # a rank-deficient item reports LSQ_ERR_RANK; the others still solve
    Ar = A.copy()
    Ar[:, 4] = 0.0
    xs, res = ctx.lsq_solve_batch([good, {"A": _dev(Ar), "b": _dev(b)}], raise_on_error=False)
    assert res[0]["status"] == 0 and res[1]["status"] == -6
