"""Two CPU ranks (gloo): the row-sharded arithmetic of App. B and the bench's
replica timing.  This build runs replicas only (one problem per GPU), but the
path shards by rows: the sketch is keyed by the global row index, so the
partial sketches of row blocks sum to the sketch of the whole matrix, and the
one-synchronisation LSQR step reduces per-rank partials of A^T u and ||u||^2.
Both are checked here with the oracle on each rank and an all-reduce between
them; the bench's max-over-ranks timing goes through its own helper."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        rng = np.random.default_rng(5)  # same problem on every rank
        m, n, d, zeta, seed = 3001, 23, 96, 8, 17
        A = rng.standard_normal((m, n))
        b = rng.standard_normal(m)
        r0, r1 = m * rank // world, m * (rank + 1) // world
        # sketch of my rows, keyed by their global indices
        Yp = torch.from_numpy(oracle.sketch_apply(np.ascontiguousarray(A[r0:r1]), b[r0:r1], d, zeta, seed, row0=r0))
        dist.all_reduce(Yp)
        Yfull = oracle.sketch_apply(A, b, d, zeta, seed)
        sketch_err = float(np.max(np.abs(Yp.numpy() - Yfull)))
        # one-sync LSQR partials: A_p^T u_p and ||u_p||^2
        u = rng.standard_normal(m)
        gp = torch.from_numpy(A[r0:r1].T @ u[r0:r1])
        sp = torch.tensor([float(u[r0:r1] @ u[r0:r1])], dtype=torch.float64)
        dist.all_reduce(gp)
        dist.all_reduce(sp)
        g_err = float(np.max(np.abs(gp.numpy() - A.T @ u)))
        s_err = abs(float(sp[0]) - float(u @ u))
        # replica timing: each rank its own time, every rank gets the slowest
        t_max = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
        q.put((rank, sketch_err, g_err, s_err, t_max))
    finally:
        dist.destroy_process_group()


def test_row_sharded_sketch_and_lsqr_partials_two_ranks(orc):
    import multiprocessing as mpl
    ctx = mpl.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, sketch_err, g_err, s_err, t_max in out:
        # sums of 2 partials vs one pass: reordering error only
        assert sketch_err <= 1e-12, (rank, sketch_err)
        assert g_err <= 1e-11 and s_err <= 1e-9
        assert t_max == 15.0
