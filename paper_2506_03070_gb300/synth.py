"""Seeded synthetic least-squares problems shaped like the paper's dense test
problems (tall, dense, controlled condition number, optional coherent rows;
Sec. 4.1 and Table 1).  The paper's own matrices (MNIST, SuiteSparse, Krylov
bases) are not available; these stand in for them.

This module holds input generation only -- none of the solver's arithmetic --
so both the CUDA path's tests and the CPU oracle can take their inputs from it.

Recipe (``dense_problem``):
  U = Q of QR(G1), G1 ~ N(0,1)^{m x n}        (seed)
  V = Q of QR(G2), G2 ~ N(0,1)^{n x n}        (seed + 1)
  s = geomspace(1, 1/cond, n)
  A = U diag(s) V^T
  optionally: a seeded fraction of rows scaled by ``coherent_scale`` (seed + 4)
  x_true ~ N(0,1)^n                            (seed + 2)
  r_perp = (I - Q Q^T) g, g ~ N(0,1)^m         (seed + 3), Q = orthonormal basis
           of range(A) (U itself when no rows were scaled), scaled to norm
           ``resid_norm``
  b = A x_true + r_perp

Because r_perp is orthogonal to range(A), x_true is the exact least-squares
solution and ||b - A x_true|| = resid_norm (up to rounding of the construction).

``batched_problem`` is the cheap construction used for many small problems:
  A = (G / sqrt(m)) diag(s) H1 H2 with H1, H2 random Householder reflectors,
  b = A x_true + 1e-6 g/||g||.
``large_problem`` builds the same construction in place, in row chunks, for
matrices too large to hold twice (the 5e6 x 2000, 80 GB case).
"""
from __future__ import annotations

import math

import torch


def _gen(device, seed):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _orth(G):
    Q, R = torch.linalg.qr(G, mode="reduced")
    # fix signs so the construction does not depend on the QR's sign convention
    d = torch.sign(torch.diagonal(R))
    d[d == 0] = 1
    return Q * d


def dense_problem(m, n, cond, *, resid_norm=1e-6, coherent_frac=0.0, coherent_scale=1e4, seed=0,
                  device="cpu", dtype=torch.float64):
    dev = torch.device(device)
    G1 = torch.randn(m, n, generator=_gen(dev, seed), device=dev, dtype=dtype)
    U = _orth(G1)
    del G1
    G2 = torch.randn(n, n, generator=_gen(dev, seed + 1), device=dev, dtype=dtype)
    V = _orth(G2)
    s = torch.logspace(0.0, -math.log10(cond), n, device=dev, dtype=dtype)
    A = (U * s) @ V.T
    Q = U
    if coherent_frac > 0:
        k = max(1, int(round(coherent_frac * m)))
        perm = torch.randperm(m, generator=_gen("cpu", seed + 4))[:k].to(dev)
        A[perm] *= coherent_scale
        del U
        Q = _orth(A)
    x_true = torch.randn(n, generator=_gen(dev, seed + 2), device=dev, dtype=dtype)
    g = torch.randn(m, generator=_gen(dev, seed + 3), device=dev, dtype=dtype)
    for _ in range(2):  # project twice for orthogonality to rounding level
        g = g - Q @ (Q.T @ g)
    r_perp = g * (resid_norm / torch.linalg.vector_norm(g))
    del Q
    b = A @ x_true + r_perp
    return {"A": A.contiguous(), "b": b, "x_true": x_true, "resid_norm": resid_norm, "cond": cond}


def config0(device="cpu"):
    """A 20000 x 200, s geometric 1..1e-8, ||r_perp|| = 1e-6; d = 800, zeta = 8."""
    p = dense_problem(20000, 200, 1e8, resid_norm=1e-6, seed=0, device=device)
    p.update(d=800, zeta=8, tol=1e-12, seed_sketch=42, name="dense_20000x200_cond1e8")
    return p


def config1(device="cuda"):
    """A 2,000,000 x 500 (8 GB), s geometric 1..1e-10, 1% of rows scaled x1e4;
    d = 2000, zeta = 8."""
    p = dense_problem(2_000_000, 500, 1e10, resid_norm=1e-6, coherent_frac=0.01, coherent_scale=1e4, seed=10,
                      device=device)
    p.update(d=2000, zeta=8, tol=1e-12, seed_sketch=43, name="dense_2000000x500_cond1e10_coherent")
    return p


def _householder(n, gen, device, dtype):
    v = torch.randn(n, generator=gen, device=device, dtype=dtype)
    v = v / torch.linalg.vector_norm(v)
    return v


def batched_problem(m, n, cond, *, seed, device="cpu", dtype=torch.float64):
    """Cheap construction: A = (G/sqrt(m)) diag(s) H1 H2, H = I - 2 v v^T.
    cond(A) is within (1+sqrt(n/m))/(1-sqrt(n/m)) of ``cond``."""
    dev = torch.device(device)
    gen = _gen(dev, seed)
    G = torch.randn(m, n, generator=gen, device=dev, dtype=dtype) / math.sqrt(m)
    s = torch.logspace(0.0, -math.log10(cond), n, device=dev, dtype=dtype)
    A = G * s
    for _ in range(2):
        v = _householder(n, gen, dev, dtype)
        A = A - 2.0 * (A @ v)[:, None] * v[None, :]
    x_true = torch.randn(n, generator=gen, device=dev, dtype=dtype)
    g = torch.randn(m, generator=gen, device=dev, dtype=dtype)
    b = A @ x_true + 1e-6 * g / torch.linalg.vector_norm(g)
    return {"A": A.contiguous(), "b": b, "x_true": x_true, "cond": cond}


def large_problem(m, n, cond, *, seed, device="cuda", chunk_rows=1 << 18, dtype=torch.float64, rows=None):
    """Cheap construction of ``batched_problem`` built in place: A (m x n) is the
    only full-size allocation; G, diag(s) and the two reflectors are applied
    chunk by chunk of rows.  cond(A) is within (1+sqrt(n/m))/(1-sqrt(n/m)) of
    ``cond``.  With ``rows``, only the first ``rows`` rows of the m-row problem
    are built (A, b), the same values as the full construction's first rows on
    the same device (a bounded sample of the workload)."""
    dev = torch.device(device)
    gen = _gen(dev, seed)
    mr = m if rows is None else min(int(rows), m)
    A = torch.empty((mr, n), device=dev, dtype=dtype)
    s = torch.logspace(0.0, -math.log10(cond), n, device=dev, dtype=dtype) / math.sqrt(m)
    vs = [_householder(n, _gen(dev, seed + 1 + k), dev, dtype) for k in range(2)]
    for r0 in range(0, mr, chunk_rows):
        blk = A[r0:r0 + chunk_rows]
        if blk.shape[0] < chunk_rows and mr < m:
            # a partial last chunk of a sample: draw the full chunk so the
            # generator's stream (and so every value) matches the full build
            full = torch.empty((min(chunk_rows, m - r0), n), device=dev, dtype=dtype)
            full.normal_(generator=gen)
            blk.copy_(full[: blk.shape[0]])
            del full
        else:
            blk.normal_(generator=gen)
        blk.mul_(s)
        for v in vs:
            blk.addr_(blk @ v, v, alpha=-2.0)
    x_true = torch.randn(n, generator=_gen(dev, seed + 3), device=dev, dtype=dtype)
    g = torch.randn(m, generator=_gen(dev, seed + 4), device=dev, dtype=dtype)
    b = A @ x_true
    b.add_(g[:mr], alpha=1e-6 / float(torch.linalg.vector_norm(g)))
    del g
    return {"A": A, "b": b, "x_true": x_true, "cond": cond}


def sparse_sign_problem(m, n, density, *, seed, device="cpu"):
    """The paper's 5e5_500_sparse recipe (Sec. 4.1): each entry independently
    nonzero with probability ``density``, nonzero values random signs; plus one
    nonzero per column at a seeded row so no column is empty.  CSR arrays
    (int64 row_ptr, int32 col_idx, float64 values) and b = A x_true +
    1e-6 g / ||g||, x_true ~ N(0, 1)."""
    dev = torch.device(device)
    gen = _gen(dev, seed)
    mask = torch.rand(m, n, generator=gen, device=dev) < density
    rows = torch.randint(0, m, (n,), generator=gen, device=dev)
    mask[rows, torch.arange(n, device=dev)] = True
    r, cidx = torch.nonzero(mask, as_tuple=True)  # row-major order
    del mask
    vals = torch.where(torch.rand(r.numel(), generator=gen, device=dev) < 0.5, -1.0, 1.0).to(torch.float64)
    counts = torch.bincount(r, minlength=m)
    row_ptr = torch.zeros(m + 1, dtype=torch.int64, device=dev)
    row_ptr[1:] = torch.cumsum(counts, 0)
    x_true = torch.randn(n, generator=gen, device=dev, dtype=torch.float64)
    Ax = torch.zeros(m, dtype=torch.float64, device=dev)
    Ax.index_add_(0, r, vals * x_true[cidx])
    g = torch.randn(m, generator=gen, device=dev, dtype=torch.float64)
    b = Ax + 1e-6 * g / torch.linalg.vector_norm(g)
    return {"row_ptr": row_ptr, "col_idx": cidx.to(torch.int32), "values": vals, "b": b, "x_true": x_true,
            "m": m, "n": n, "rows": r}


def csr_to_dense(p):
    A = torch.zeros(p["m"], p["n"], dtype=torch.float64, device=p["values"].device)
    A[p["rows"], p["col_idx"].long()] = p["values"]
    return A
