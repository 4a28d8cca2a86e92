"""Pins for the oracle's counter-based generator and rejection sampler
(Sec. 3.1.2 and Algorithm 3 of arXiv 2506.03070; Philox from Salmon et al. SC'11).

The oracle is checked against things it does not share code with: numpy's own
Philox4x64-10, the published known-answer vectors, the closed-form probability
that a column needs a redraw, uniformity over all zeta-subsets, and a
brute-force restatement of the procedure for tiny inputs that draws its random
words from numpy."""
import itertools
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MASK64 = (1 << 64) - 1


def _numpy_block(counter, key):
    """Philox4x64-10 block for `counter` via numpy, whose generator increments
    the 256-bit counter before producing a block (established by this test)."""
    c = 0
    for w, x in enumerate(counter):
        c |= int(x) << (64 * w)
    c = (c - 1) % (1 << 256)
    ctr = np.array([(c >> (64 * w)) & MASK64 for w in range(4)], dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=ctr)
    return [int(v) for v in bg.random_raw(4)]


def test_philox_known_answers(orc):
    rows = 0
    with open(os.path.join(GOLDEN, "philox4x64_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(t, 16) for t in line.split()]
            out = orc.philox4x64_10(w[0:4], w[4:6])
            assert [int(v) for v in out] == w[6:10]
            rows += 1
    assert rows == 3


def test_philox_matches_numpy(orc):
    rng = np.random.default_rng(7)
    cases = [([0, 0, 0, 0], [0, 0]), ([MASK64, 0, 0, 0], [1, 2]), ([5, MASK64, 3, 1], [42, 0])]
    for _ in range(40):
        cases.append(([int(x) for x in rng.integers(0, 2**63, 4, dtype=np.int64)],
                      [int(x) for x in rng.integers(0, 2**63, 2, dtype=np.int64)]))
    for ctr, key in cases:
        assert [int(v) for v in orc.philox4x64_10(ctr, key)] == _numpy_block(ctr, key)


def _index(word, d):
    return (word * d) >> 64


def _brute_force_row(seed, i, d, zeta):
    """Sec. 3.1.2 steps (i)-(iv) restated with Python lists, random words from
    numpy's Philox under the stream layout (counter (i, r, j//4, 0), word j%4;
    signs from counter (i, 0, 0, 1), bit k of word 0)."""
    def draw(r, j):
        return _index(_numpy_block([i, r, j // 4, 0], [seed, 0])[j % 4], d)

    C = sorted(draw(0, j) for j in range(zeta))
    r = 0
    while True:
        bad = [j for j in range(zeta - 1) if C[j] == C[j + 1]]
        if not bad:
            break
        r += 1
        for j in bad:
            C[j] = draw(r, j)
        C = sorted(C)
    sw = _numpy_block([i, 0, 0, 1], [seed, 0])[0]
    signs = [1 if (sw >> k) & 1 else -1 for k in range(zeta)]
    return C, signs, r


@pytest.mark.parametrize("d,zeta", [(5, 4), (12, 8), (40, 8), (9, 9), (64, 3)])
def test_rejection_sampler_brute_force(orc, d, zeta):
    seed = 1234
    idx, sgn, rnd = orc.sketch_indices(seed, 100, 60, d, zeta, with_rounds=True)
    for t in range(60):
        C, signs, r = _brute_force_row(seed, 100 + t, d, zeta)
        assert list(idx[t]) == C
        assert list(sgn[t]) == signs
        assert rnd[t] == r


@pytest.mark.parametrize("d,zeta", [(8, 8), (16, 8), (800, 8), (2000, 8), (100, 1), (70, 64)])
def test_sketch_column_invariants(orc, d, zeta):
    idx, sgn = orc.sketch_indices(99, 0, 3000, d, zeta)
    assert idx.min() >= 0 and idx.max() < d
    assert np.all(np.diff(idx, axis=1) > 0)  # sorted and pairwise distinct
    assert set(np.unique(sgn)) <= {-1, 1}


def test_redraw_rate_closed_form(orc):
    """P(first draw has a repeat) = 1 - prod_{k<zeta}(1 - k/d) (Sec. 3.1.2)."""
    d, zeta, rows = 64, 8, 40000
    _, _, rnd = orc.sketch_indices(5, 0, rows, d, zeta, with_rounds=True)
    p = 1.0 - np.prod([1.0 - k / d for k in range(zeta)])
    frac = np.mean(rnd > 0)
    sd = math.sqrt(p * (1 - p) / rows)
    assert abs(frac - p) < 5 * sd
    # the paper's lower bound p_norepeat >= (1 - zeta/d)^zeta >= 1 - zeta^2/d
    assert 1 - frac >= (1 - zeta / d) ** zeta - 5 * sd


def test_uniform_over_subsets(orc):
    """Rejection with partial redraw is exactly uniform over zeta-subsets:
    chi-square over all C(10,3) = 120 subsets."""
    d, zeta, rows = 10, 3, 120000
    idx, _ = orc.sketch_indices(2024, 0, rows, d, zeta)
    cells = {c: 0 for c in itertools.combinations(range(d), zeta)}
    for row in map(tuple, idx):
        cells[row] += 1
    exp = rows / len(cells)
    chi2 = sum((v - exp) ** 2 / exp for v in cells.values())
    from scipy.stats import chi2 as chi2dist
    assert chi2dist.sf(chi2, len(cells) - 1) > 1e-4


def test_sign_balance_and_independence_of_rows(orc):
    idx, sgn = orc.sketch_indices(77, 0, 20000, 800, 8)
    frac = np.mean(sgn > 0)
    assert abs(frac - 0.5) < 5 * math.sqrt(0.25 / sgn.size)
    # keyed by global column: a slice reproduces the same columns
    idx2, sgn2 = orc.sketch_indices(77, 12345, 100, 800, 8)
    assert np.array_equal(idx2, idx[12345:12445]) and np.array_equal(sgn2, sgn[12345:12445])


def test_sketch_argument_errors(orc):
    with pytest.raises(orc.OracleError):
        orc.sketch_indices(1, 0, 4, 4, 8)  # zeta > d
    with pytest.raises(orc.OracleError):
        orc.sketch_indices(1, 0, 4, 100, 0)
    with pytest.raises(orc.OracleError):
        orc.sketch_indices(1, 0, 4, 100, 65)
