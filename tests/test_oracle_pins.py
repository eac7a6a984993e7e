"""Pins of the CPU oracle against facts that do not come from the oracle itself:
a hand-enumerated fixture, exact integer arithmetic on dyadic lattices, an
independent library (scipy's k-d tree), invariants of the definition, a closed
form for uniform points in the unit square, and exact rational arithmetic for
the double-double band classifier.  CPU only.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2209_11287_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_tiny():
    pts, cases, cur = [], {}, None
    with open(os.path.join(GOLDEN, "tiny2d.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            if line == "points":
                cur = "points"
                continue
            if line.startswith("eps"):
                cur = float(line.split()[1])
                cases[cur] = set()
                continue
            if cur == "points":
                pts.append([float(v) for v in line.split()])
            elif line.startswith("all"):
                ids = [int(v) for v in line.split()[1:]]
                cases[cur] |= {(a, b) for a in ids for b in ids}
            else:
                a, b = (int(v) for v in line.split())
                cases[cur].add((a, b))
    return np.array(pts), cases


def _pairs(orc, x, eps):
    return {tuple(int(v) for v in p) for p in orc.keys_to_pairs(orc.join(x, eps))}


def test_hand_enumerated_fixture(orc):
    """Sec. II-A, Eq. 1, on seven points worked out by hand (tests/golden/tiny2d.txt)."""
    x, cases = _read_tiny()
    assert len(cases) == 3
    for eps, expected in cases.items():
        assert _pairs(orc, x, eps) == expected, eps


@pytest.mark.parametrize("d", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("seed", [0, 1])
def test_dyadic_lattice_exact(orc, d, seed):
    """Coordinates k / 2^6 with small integers k make every binary64 operation of
    the sum exact, so the oracle must equal exact integer arithmetic, ties at
    exactly eps included (eps = r / 2^6, eps^2 exact)."""
    g = np.random.Generator(np.random.PCG64(100 + seed))
    n = 300
    k = g.integers(0, 40, size=(n, d))
    k[1] = k[0]  # a duplicate
    x = k.astype(np.float64) / 64.0
    for r in (0, 1, 5, 9, 17):
        eps = r / 64.0
        ki = k.astype(object)
        exp = set()
        for i in range(n):
            diff = ki - ki[i]
            s = (diff * diff).sum(axis=1)
            for j in np.nonzero(s <= r * r)[0]:
                exp.add((i, int(j)))
        assert _pairs(orc, x, eps) == exp, (d, r)


@pytest.mark.parametrize("d", [2, 4, 7])
def test_matches_scipy_kdtree(orc, d):
    """An independent implementation (scipy.spatial.cKDTree.query_pairs, which
    keeps pairs with distance <= r) gives the same set, up to pairs whose exact
    distance lies within 1e-9 of eps."""
    spatial = pytest.importorskip("scipy.spatial")
    g = np.random.Generator(np.random.PCG64(7))
    n = 2000
    x = g.random((n, d))
    eps = workloads.ball_eps(n, d, 20.0)
    tree = spatial.cKDTree(x)
    up = tree.query_pairs(eps, p=2.0, output_type="ndarray")
    keys = set((int(a) << 32) | int(b) for a, b in up)
    keys |= set((int(b) << 32) | int(a) for a, b in up)
    keys |= set((i << 32) | i for i in range(n))
    ref = np.array(sorted(keys), dtype=np.int64)
    got = orc.join(x, eps)
    only_ref, only_got, bad = orc.compare_pair_sets(x, eps, ref, got)
    assert bad == 0
    assert only_ref + only_got <= 2


def test_invariants(orc):
    """Symmetry, self pairs, eps below the smallest gap, eps above the diameter,
    dyadic translation and input permutation."""
    g = np.random.Generator(np.random.PCG64(3))
    n, d = 400, 3
    k = g.integers(0, 1000, size=(n, d))
    k[5] = k[6]
    x = k / 1024.0
    eps = 0.09
    keys = orc.join(x, eps)
    p = orc.keys_to_pairs(keys)
    sym = np.sort((p[:, 1] << 32) | p[:, 0])
    assert np.array_equal(sym, keys)
    selfk = (np.arange(n, dtype=np.int64) << 32) | np.arange(n, dtype=np.int64)
    assert np.isin(selfk, keys).all()
    # eps below the smallest non-zero gap: only self pairs and the duplicates
    diffs = x[:, None, :] - x[None, :, :]
    dd = np.sqrt((diffs ** 2).sum(-1))
    gap = dd[dd > 0].min()
    small = orc.join(x, gap * 0.5)
    assert small.size == n + 2
    # eps at least the diameter: all n^2 pairs
    assert orc.join(x, float(dd.max()) * 1.0001).size == n * n
    # translation by a dyadic shift keeps every operation exact
    shifted = x + np.array([0.25, -0.5, 3.0])
    assert np.array_equal(orc.join(shifted, eps), keys)
    # permutation: pairs map through the permutation
    perm = g.permutation(n)
    xp = x[perm]
    kp = orc.keys_to_pairs(orc.join(xp, eps))
    back = np.sort((perm[kp[:, 0]].astype(np.int64) << 32) | perm[kp[:, 1]].astype(np.int64))
    assert np.array_equal(back, keys)


def test_unit_square_closed_form(orc):
    """For n uniform points in the unit square and eps <= 1, a pair is within eps
    with probability pi eps^2 - 8 eps^3 / 3 + eps^4 / 2 (square line picking), so
    the mean count of other points within eps is (n - 1) times that.  The
    realised mean of one seeded draw lies within 5 sigma (sigma ~ 0.093 for the
    16384-point workload, from the U-statistic variance)."""
    w = workloads.uniform2d()
    e = w.eps
    expect = (w.n - 1) * (math.pi * e * e - 8.0 * e ** 3 / 3.0 + e ** 4 / 2.0)
    _, tot = orc.count(w.points, w.eps)
    got = (tot - w.n) / w.n
    assert abs(expect - 31.32) < 0.01
    assert abs(got - expect) < 5 * 0.093, (got, expect)


def test_distances_exact_on_lattice(orc):
    """Emitted distances are sqrt(s) correctly rounded: on a dyadic lattice with
    3-4-5 right triangles they are exact multiples of 1/64."""
    x = np.array([[0, 0], [3, 4], [6, 8], [0, 5]], dtype=np.float64) / 64.0
    keys, dist = orc.join(x, 10 / 64.0, with_dist=True)
    p = orc.keys_to_pairs(keys)
    exact = {(0, 1): 5, (1, 2): 5, (0, 2): 10, (0, 3): 5, (1, 3): math.sqrt(10), (2, 3): math.sqrt(45)}
    for (i, j), dv in zip(p, dist):
        if i == j:
            assert dv == 0.0
            continue
        a, b = min(i, j), max(i, j)
        want = exact[(a, b)] / 64.0
        assert dv == want if float(want * 64).is_integer() else abs(dv - want) <= 1e-16


def test_double_double_against_rationals(orc):
    """The double-double squared distance equals the exact rational one within
    a relative 2^-100 (checked with fractions.Fraction)."""
    g = np.random.Generator(np.random.PCG64(11))
    x = g.random((50, 9)) * g.choice([1.0, 1e-3, 1e3], size=(50, 1))
    for _ in range(200):
        i, j = (int(v) for v in g.integers(0, 50, size=2))
        hi, lo = orc.sqdist_dd(x, i, j)
        exact = sum((Fraction(float(a)) - Fraction(float(b))) ** 2 for a, b in zip(x[i], x[j]))
        err = abs(Fraction(hi) + Fraction(lo) - exact)
        assert err <= exact * Fraction(1, 2 ** 100) + Fraction(1, 2 ** 1000)


def test_borderline_classifier(orc):
    """Points at distance eps (1 + r) are borderline for |r| < 1e-9 and not for
    |r| > 1e-9 (1-D, exact differences)."""
    eps = 0.75
    for r, want in [(0.0, True), (4e-10, True), (-4e-10, True), (3e-9, False), (-3e-9, False), (0.1, False)]:
        x = np.array([[0.0], [eps * (1.0 + r)]])
        assert orc.is_borderline(x, 0, 1, eps) == want, r


def _lattice_rows():
    g = np.random.Generator(np.random.PCG64(77))
    k = g.integers(-50, 50, size=(300, 5))
    return k, k / 32.0


def lattice_row_ok(sqdist_row) -> bool:
    """Squared distances of one point to all points on a dyadic lattice: every
    binary64 operation is exact there, so each value must equal exact integer
    arithmetic, (sum of squared integer differences) / 2^10."""
    k, x = _lattice_rows()
    for q in (0, 17, 299):
        want = ((k - k[q]) ** 2).sum(1) / 1024.0
        if not np.array_equal(sqdist_row(x, q), want):
            return False
    return True


def test_sqdist_row_exact_on_lattice(orc):
    """The rows the GPU certification and kNN tests compare with (Eq. 1 squared,
    the decision rule's operation order) against exact integer arithmetic."""
    assert lattice_row_ok(orc.sqdist_row)


def test_rows_match_join(orc):
    """Per-query rows equal the corresponding slice of the full result."""
    w = workloads.uniform2d(n=3000, seed=4)
    keys = orc.join(w.points, w.eps)
    qs = np.array([0, 17, 2999, 1500])
    rk, rc = orc.rows(w.points, w.eps, qs)
    want = np.concatenate([keys[(keys >> 32) == q] for q in qs])
    assert np.array_equal(rk, want)
    assert rc.sum() == rk.size


def test_grid_is_lossless(orc):
    """Sec. III-B: with cells of side w >= eps, every pair within eps lies in
    adjacent cells, so the grid candidates contain the result and |R| <= the
    candidate count; with one cell the candidate count is n^2."""
    w = workloads.uniform2d(n=4000, seed=5)
    cells = orc.grid_cells(w.points, w.eps)
    keys = orc.join(w.points, w.eps)
    p = orc.keys_to_pairs(keys)
    assert np.abs(cells[p[:, 0]] - cells[p[:, 1]]).max() <= 1
    cand = orc.grid_candidate_count(w.points, w.eps)
    assert keys.size <= cand < w.n * w.n
    assert orc.grid_candidate_count(w.points, 10.0) == w.n * w.n
    assert orc.grid_candidate_count_fast(w.points, w.eps) == cand
    assert orc.grid_candidate_count_fast(w.points, 10.0) == w.n * w.n
    w3 = workloads.uniform4d(n=3000, seed=1)
    assert orc.grid_candidate_count_fast(w3.points, w3.eps) == orc.grid_candidate_count(w3.points, w3.eps)


def test_calibrated_eps_reaches_target(orc):
    """The calibrated eps gives the requested mean selectivity on the sample."""
    w = workloads.uniform2d(n=5000, seed=6)
    eps = orc.calibrate_eps(w.points, 20.0, n_queries=500)
    c, _ = orc.count(w.points, eps)
    assert abs((c.mean() - 1) - 20.0) < 2.0


def near_tie_points(seed: int = 21, npairs: int = 400, d: int = 4, eps: float = 0.05, delta: float = 1e-10):
    """Point pairs whose exact distance is eps (1 + r) with |r| about delta:
    far enough from eps that binary64 rounding (~1e-16) cannot flip the
    decision, close enough that any arithmetic coarser than ~1e-11 can."""
    g = np.random.Generator(np.random.PCG64(seed))
    a = g.random((npairs, d))
    u = g.standard_normal((npairs, d))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    r = delta * g.choice([-1.0, 1.0], size=npairs) * (1 + g.random(npairs))
    b = a + (eps * (1 + r))[:, None] * u
    x = np.empty((2 * npairs, d))
    x[0::2] = a
    x[1::2] = b
    return x, eps


def exact_in(x, i, j, eps):
    s = sum((Fraction(float(p)) - Fraction(float(q))) ** 2 for p, q in zip(x[i], x[j]))
    return s <= Fraction(eps * eps)


def test_near_ties_decided_exactly(orc):
    """Pairs within a relative 1e-10 .. 2e-10 of eps (but not within 1e-15) are
    decided as exact rational arithmetic decides them."""
    x, eps = near_tie_points()
    keys = set(int(k) for k in orc.join(x, eps))
    for p in range(x.shape[0] // 2):
        i, j = 2 * p, 2 * p + 1
        assert (((i << 32) | j) in keys) == exact_in(x, i, j, eps), p


def test_stored_brute_force_eps_is_the_oracle_calibration(orc):
    """The stored eps of the brute-force 16-D workload is what the oracle's
    calibration rule gives (mean selectivity 50 over 2000 seeded queries):
    the value was written by oracle/calibrate_eps.py, not by the GPU path."""
    from paper_2209_11287_gb300 import workloads
    w = workloads.brute16d(eps=1.0)
    assert orc.calibrate_eps(w.points, 50.0) == workloads._stored_eps("brute16d")
