"""Pins of the oracle's DBSCAN on the join (oracle.dbscan) against an
independent implementation, scikit-learn's DBSCAN (radius neighbourhoods,
dist <= eps, the point itself counted): the core points and their
partition into clusters must be the same up to renaming, the noise the same,
and every border point must carry the cluster of one of its core
neighbours (scikit-learn assigns border points by expansion order; the
oracle takes the smallest identifier).  Plus a hand-built case.  CPU only."""
import numpy as np
import pytest

import oracle

sk = pytest.importorskip("sklearn.cluster")


def _partition(labels, mask):
    """Canonical form of the clusters of the points in mask: each cluster as
    the sorted tuple of its members."""
    out = {}
    for p in np.nonzero(mask)[0].tolist():
        out.setdefault(int(labels[p]), []).append(p)
    return sorted(tuple(v) for v in out.values())


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("min_pts", [1, 4, 9])
def test_matches_scikit_learn(seed, min_pts):
    g = np.random.Generator(np.random.PCG64(50 + seed))
    centres = g.random((8, 2)) * 10
    x = np.concatenate([centres[g.integers(0, 8, 600)] + 0.25 * g.standard_normal((600, 2)),
                        g.random((150, 2)) * 10])
    eps = 0.35
    ours, k = oracle.dbscan(x, eps, min_pts)
    ref = sk.DBSCAN(eps=eps, min_samples=min_pts).fit(x)
    core = np.zeros(len(x), dtype=bool)
    core[ref.core_sample_indices_] = True
    keys = oracle.join(x, eps)
    deg = np.bincount(keys >> 32, minlength=len(x))
    assert np.array_equal(deg >= min_pts, core)
    assert _partition(ours, core) == _partition(ref.labels_, core)
    assert np.array_equal(ours == -1, ref.labels_ == -1)
    assert k == len(set(ref.labels_[core].tolist()))
    # border points: a cluster of one of their core neighbours
    i, j = keys >> 32, keys & 0xFFFFFFFF
    for p in np.nonzero((~core) & (ours != -1))[0].tolist():
        nb = j[(i == p)]
        assert ours[p] in set(ours[nb[core[nb]]].tolist())
    # identifiers: ranks of the clusters' smallest core points
    firsts = sorted(min(c) for c in _partition(ours, core))
    assert [int(ours[f]) for f in firsts] == list(range(k))


def test_hand_built():
    # a chain of 4 points 1 apart (core with min_pts 2), a border point 1
    # from the chain's end (its only neighbour), an isolated point
    x = np.array([[0.0], [1.0], [2.0], [3.0], [10.0], [11.0], [20.0]])
    labels, k = oracle.dbscan(x, 1.0, 3)
    # degrees (self included): 2, 3, 3, 2, 2, 2, 1 -> core 1, 2 (one
    # cluster); 0 and 3 are border points of it; 4, 5, 6 noise
    assert k == 1
    assert labels.tolist() == [0, 0, 0, 0, -1, -1, -1]
    labels, k = oracle.dbscan(x, 1.0, 2)
    assert k == 2 and labels.tolist() == [0, 0, 0, 0, 1, 1, -1]
