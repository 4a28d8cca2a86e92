"""Serving form: lsq_submit / lsq_poll on the persistent request loop.

Each request runs Algorithm 1 on a group of blocks sized from the problem;
the checks: every solution reaches Karlson-Waldén backward error <= 1e-10,
a request gives the same solution alone and in a mix of concurrent requests
(same sketch, same group size, same pass shape: only the order of the
sketch's L2 reductions differs, so ||A (x_alone - x_mix)|| <= 1e-10 ||b||),
small cases agree with the oracle, and admission respects the arena."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (m, n): chunked shapes (n <= 256, one or more blocks), one warp per row
# (n <= 512) and two warps per row (n <= 1024); small to 1.2e8-byte A
MIX = [(5000, 20), (12000, 50), (30001, 100), (8000, 200), (60000, 64), (40000, 300), (20000, 700),
       (150000, 130), (3001, 1000), (100000, 33)]


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2506_03070_gb300 import build
    build.build()
    import paper_2506_03070_gb300 as P
    return P


@pytest.fixture(scope="module")
def sctx(P):
    c = P.Context(0, 24 << 30)
    c.lsq_serve_config(arena_bytes=16 << 30)
    yield c
    c.close()


def _mix(device="cuda"):
    from paper_2506_03070_gb300 import synth
    out = []
    for k, (m, n) in enumerate(MIX):
        cond = 10.0 ** (2 + 8 * k / (len(MIX) - 1))
        out.append(synth.batched_problem(m, n, cond, seed=1000 + k, device=device))
    return out


def test_serve_each_result_same_alone_and_in_the_mix(sctx, orc):
    probs = _mix()
    alone = []
    for k, p in enumerate(probs):
        n = p["A"].shape[1]
        st, x, info = sctx.lsq_wait(sctx.lsq_submit(p["A"], p["b"], 4 * n, seed=k))
        assert st == 0, (k, st)
        alone.append((x.clone(), info))
    tickets = []
    for k, p in enumerate(probs):
        tickets.append(sctx.lsq_submit(p["A"], p["b"], 4 * p["A"].shape[1], seed=k))
        if k == len(probs) // 2:
            time.sleep(0.003)  # the second half arrives while the first is on the GPU
    mixed = [sctx.lsq_wait(t) for t in tickets]
    for k, p in enumerate(probs):
        A, b = p["A"].cpu().numpy(), p["b"].cpu().numpy()
        bn = np.linalg.norm(b)
        st, xm, im = mixed[k]
        assert st == 0, (k, st)
        xa, ia = alone[k][0].cpu().numpy(), alone[k][1]
        xm = xm.cpu().numpy()
        assert orc.backward_error_kw(A, b, xa) <= 1e-10, k
        assert im["group_blocks"] == ia["group_blocks"]
        assert abs(im["iters"] - ia["iters"]) <= 1, (k, im["iters"], ia["iters"])
        assert np.linalg.norm(A @ (xa - xm)) <= 1e-10 * bn, k
        assert orc.backward_error_kw(A, b, xm) <= 1e-10, k
    # the mix really overlapped: some request started before an earlier one finished
    iv = sorted((r[2]["t_start_s"], r[2]["t_done_s"]) for r in mixed)
    assert any(iv[j][0] < iv[i][1] for i in range(len(iv)) for j in range(i + 1, len(iv)))
    # both one-block groups and multi-block groups were exercised
    groups = [r[2]["group_blocks"] for r in mixed]
    assert min(groups) == 1 and max(groups) > 8


def test_serve_matches_oracle_and_plain_solve(sctx, orc):
    from paper_2506_03070_gb300 import synth
    for k, (m, n, d) in enumerate([(5000, 20, 80), (9001, 37, 148), (7000, 300, 1200)]):
        p = synth.batched_problem(m, n, 1e6, seed=77 + k, device="cpu")
        A, b = p["A"].numpy(), p["b"].numpy()
        st, x, info = sctx.lsq_wait(sctx.lsq_submit(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), d,
                                                     seed=5 + k))
        assert st == 0
        x = x.cpu().numpy()
        ref = orc.solve(A, b, d, 8, 5 + k, 1e-12, orc.default_maxit(n, d, 1e-12))
        bn = np.linalg.norm(b)
        assert abs(info["iters"] - ref["iters"]) <= 2, (info["iters"], ref["iters"])
        assert np.linalg.norm(A @ (x - ref["x"])) <= 1e-10 * bn
        # the device's accuracy pass (native FP64) agrees with the oracle's on
        # the same x.  Both evaluate eta = ||A^T r|| / (||A||_F ||r||) after
        # r = b - A x cancelled ~6 digits, each summing in its own order, so r
        # moves by up to ~sqrt(n) u ||A||_F ||x|| and eta by that over ||r||:
        # that is the bound, however small eta is.
        eta = orc.backward_error(A, b, x)
        r = b - A @ x
        fro = np.linalg.norm(A)
        bound = 4 * np.sqrt(n) * 2.0 ** -53 * fro * np.linalg.norm(x) / np.linalg.norm(r)
        assert abs(info["backward_error_ne"] - eta) <= bound, (info["backward_error_ne"], eta, bound)
        assert abs(info["rnorm"] - np.linalg.norm(r)) <= bound * info["rnorm"]


@pytest.mark.parametrize("shapes", [(2, 2, 4, 5), (5, 5, 5, 5)])
def test_serve_pinned_pass_shapes(sctx, orc, shapes):
    """Requests with n <= 256 on pinned pass shapes other than the defaults
    (0, 1, 3, 5; the wider shape of each range, and the widest shape for every
    range) agree with the oracle; one request spans several blocks."""
    from paper_2506_03070_gb300 import synth
    for bucket, shape in enumerate(shapes):
        sctx.lsq_batch_shape_set(bucket, shape)
    try:
        cases = [(5000, 20, 80), (9001, 37, 148), (30001, 100, 400), (7000, 200, 800), (400000, 64, 256)]
        tickets, host = [], []
        for k, (m, n, d) in enumerate(cases):
            p = synth.batched_problem(m, n, 1e5, seed=600 + k, device="cpu")
            A, b = p["A"].numpy(), p["b"].numpy()
            host.append((A, b, d))
            tickets.append(sctx.lsq_submit(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), d, seed=20 + k))
        res = [sctx.lsq_wait(t) for t in tickets]
    finally:
        for bucket in range(4):
            sctx.lsq_batch_shape_set(bucket, -1)
    assert max(r[2]["group_blocks"] for r in res) > 1
    for k, ((A, b, d), (st, x, info)) in enumerate(zip(host, res)):
        assert st == 0, (k, st)
        x = x.cpu().numpy()
        ref = orc.solve(A, b, d, 8, 20 + k, 1e-12, orc.default_maxit(A.shape[1], d, 1e-12))
        assert abs(info["iters"] - ref["iters"]) <= 2, (k, info["iters"], ref["iters"])
        assert np.linalg.norm(A @ (x - ref["x"])) <= 1e-10 * np.linalg.norm(b), k


def test_serve_host_problems(sctx, orc):
    from paper_2506_03070_gb300 import synth
    p = synth.batched_problem(20000, 80, 1e6, seed=5, device="cpu")
    A, b = p["A"].numpy(), p["b"].numpy()
    Ap = np.zeros((20000, 83))
    Ap[:, :80] = A  # strided host rows (lda = 83) are packed on the way in
    st, xh, info = sctx.lsq_wait(sctx.lsq_submit(Ap[:, :80], b, 320, seed=3))
    assert st == 0 and isinstance(xh, np.ndarray)
    assert orc.backward_error_kw(A, b, xh) <= 1e-10
    st, xd, _ = sctx.lsq_wait(sctx.lsq_submit(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), 320, seed=3))
    assert st == 0
    assert np.linalg.norm(A @ (xh - xd.cpu().numpy())) <= 1e-10 * np.linalg.norm(b)


def test_serve_admits_by_budget(P, orc):
    from paper_2506_03070_gb300 import synth
    c = P.Context(0, 2 << 30)
    arena = 120 << 20
    c.lsq_serve_config(arena_bytes=arena)
    try:
        # each request holds ~53 MB of slot (float-pair image of A, u, sketch):
        # at most two fit at once
        probs = [synth.batched_problem(100000, 64, 1e4, seed=300 + k, device="cuda") for k in range(6)]
        tickets = [c.lsq_submit(p["A"], p["b"], 256, seed=k) for k, p in enumerate(probs)]
        res = [c.lsq_wait(t) for t in tickets]
        for (st, x, info), p in zip(res, probs):
            assert st == 0
            assert orc.backward_error_kw(p["A"].cpu().numpy(), p["b"].cpu().numpy(), x.cpu().numpy()) <= 1e-10
        s = c.lsq_serve_stats()
        assert s["completed"] == 6 and s["arena_bytes"] == arena
        assert 53e6 < s["arena_peak_bytes"] <= arena
        iv = [(r[2]["t_start_s"], r[2]["t_done_s"]) for r in res]
        for t0, _ in iv:
            assert sum(1 for a, z in iv if a <= t0 < z) <= 2
        # a problem that alone exceeds the arena is refused at submission
        big = synth.batched_problem(400000, 64, 1e2, seed=9, device="cuda")
        with pytest.raises(P.LsqError) as e:
            c.lsq_submit(big["A"], big["b"], 256)
        assert e.value.status == -4
    finally:
        c.close()


def test_serve_poll_and_errors(sctx, P):
    from paper_2506_03070_gb300 import synth
    good = synth.batched_problem(6000, 30, 1e3, seed=1, device="cuda")
    bad = torch.randn(6000, 30, dtype=torch.float64, device="cuda")
    bad[:, 3] = 0.0  # rank deficient: R_33 = 0
    nanA = good["A"].clone()
    nanA[17, 5] = float("nan")
    wide = torch.zeros((2000, 1025), dtype=torch.float64, device="cuda")
    bvec = torch.randn(6000, dtype=torch.float64, device="cuda")
    t_bad = sctx.lsq_submit(bad, bvec, 120)
    t_good = sctx.lsq_submit(good["A"], good["b"], 120)
    t_nan = sctx.lsq_submit(nanA, good["b"], 120)
    assert sctx.lsq_wait(t_bad)[0] == -6
    assert sctx.lsq_wait(t_good)[0] == 0
    assert sctx.lsq_wait(t_nan)[0] == -9
    with pytest.raises(P.LsqError) as e:  # a finished ticket is gone after its final poll
        sctx.lsq_poll(t_good)
    assert e.value.status == -1
    with pytest.raises(P.LsqError) as e:
        sctx.lsq_poll(123456789)
    assert e.value.status == -1
    with pytest.raises(P.LsqError) as e:
        sctx.lsq_submit(wide, torch.zeros(2000, dtype=torch.float64, device="cuda"), 2000)
    assert e.value.status == -10
    with pytest.raises(P.LsqError) as e:
        sctx.lsq_submit(good["A"], good["b"], 120, zeta=9)
    assert e.value.status == -1
    with pytest.raises(P.LsqError) as e:
        sctx.lsq_submit(good["A"], good["b"], 30)  # d < n + 1
    assert e.value.status == -1
