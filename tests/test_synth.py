"""The seeded input generators against the recipes they state (no GPU): the
singular values and residual of the dense problems, the condition-number bound
of the cheap construction, and the CSR structure of the sparse recipe (Sec. 4.1,
`5e5_500_sparse`), cross-checked with scipy.sparse."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_dense_problem_singular_values_and_orthogonal_residual():
    from paper_2506_03070_gb300 import synth
    p = synth.dense_problem(3000, 40, 1e6, resid_norm=1e-6, seed=5)
    A, b, xt = p["A"].numpy(), p["b"].numpy(), p["x_true"].numpy()
    s = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(s, np.geomspace(1.0, 1e-6, 40), rtol=1e-9)
    r = b - A @ xt
    assert abs(np.linalg.norm(r) - 1e-6) <= 1e-12
    # x_true is the exact LS solution: r is orthogonal to range(A)
    U = np.linalg.svd(A, full_matrices=False)[0]
    assert np.linalg.norm(U.T @ r) <= 1e-12 * np.linalg.norm(r) * 1e3


def test_dense_problem_coherent_rows_keep_x_true_exact():
    from paper_2506_03070_gb300 import synth
    p0 = synth.dense_problem(2000, 20, 1e4, seed=7)
    p = synth.dense_problem(2000, 20, 1e4, coherent_frac=0.01, coherent_scale=1e4, seed=7)
    A0, A = p0["A"].numpy(), p["A"].numpy()
    ratio = np.linalg.norm(A, axis=1) / np.linalg.norm(A0, axis=1)
    assert np.sum(np.isclose(ratio, 1e4, rtol=1e-12)) == 20  # 1% of the rows, x1e4
    assert np.sum(np.isclose(ratio, 1.0, rtol=1e-12)) == 1980
    b, xt = p["b"].numpy(), p["x_true"].numpy()
    r = b - A @ xt
    Q = np.linalg.qr(A)[0]
    # r is recomputed here from b = A x_true + r_perp: b's rounding (A x_true is
    # ~1e4 on the scaled rows) leaves ~u ||A|| ||x|| in r; a residual that was not
    # projected out of range(A) would leave ~||r|| = 1e-6
    tol = 64 * np.finfo(float).eps * (np.linalg.norm(A, 2) * np.linalg.norm(xt) + np.linalg.norm(b))
    assert np.linalg.norm(Q.T @ r) <= tol < 1e-3 * np.linalg.norm(r)


@pytest.mark.parametrize("build", ["batched", "large"])
def test_cheap_construction_condition_bound(build):
    from paper_2506_03070_gb300 import synth
    m, n, cond = 6000, 30, 1e5
    if build == "batched":
        p = synth.batched_problem(m, n, cond, seed=3)
    else:  # built in place chunk by chunk: chunks of 1000 rows exercise the loop
        p = synth.large_problem(m, n, cond, seed=3, device="cpu", chunk_rows=1000)
    A = p["A"].numpy()
    s = np.linalg.svd(A, compute_uv=False)
    bound = (1 + math.sqrt(n / m)) / (1 - math.sqrt(n / m))
    assert cond / bound <= s[0] / s[-1] <= cond * bound
    r = p["b"].numpy() - A @ p["x_true"].numpy()
    assert abs(np.linalg.norm(r) - 1e-6) <= 1e-12


def test_sparse_sign_problem_structure():
    from paper_2506_03070_gb300 import synth
    sp = pytest.importorskip("scipy.sparse")
    m, n, p_nz = 20000, 60, 0.02
    p = synth.sparse_sign_problem(m, n, p_nz, seed=11)
    rp, ci, va = p["row_ptr"].numpy(), p["col_idx"].numpy(), p["values"].numpy()
    nnz = va.size
    assert rp[0] == 0 and rp[-1] == nnz and np.all(np.diff(rp) >= 0)
    assert ci.dtype == np.int32 and ci.min() >= 0 and ci.max() < n
    assert set(np.unique(va)) <= {-1.0, 1.0}
    # column indices increase within each row (row-major order of the mask)
    for i in range(0, m, 997):
        assert np.all(np.diff(ci[rp[i]:rp[i + 1]]) > 0)
    # density: each entry nonzero with probability p, plus at most one guard per column
    mean, sd = p_nz * m * n, math.sqrt(m * n * p_nz * (1 - p_nz))
    assert abs(nnz - mean) <= 5 * sd + n
    # no empty column (reading: the guard entry)
    assert np.all(np.bincount(ci, minlength=n) > 0)
    # signs balanced
    assert abs(np.mean(va)) <= 5 / math.sqrt(nnz)
    # the dense form agrees with scipy's CSR reading of the same arrays
    D = synth.csr_to_dense(p).numpy()
    S = sp.csr_matrix((va, ci, rp), shape=(m, n)).toarray()
    assert np.array_equal(D, S)
    r = p["b"].numpy() - D @ p["x_true"].numpy()
    assert abs(np.linalg.norm(r) - 1e-6) <= 1e-12


def test_sparse_guard_fills_an_otherwise_empty_column():
    from paper_2506_03070_gb300 import synth
    # density 0: every nonzero is a guard, one per column
    p = synth.sparse_sign_problem(500, 12, 0.0, seed=2)
    ci = p["col_idx"].numpy()
    assert np.array_equal(np.sort(ci), np.arange(12))
