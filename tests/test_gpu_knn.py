"""The distance tile as an operation of its own (sj_sqdist_tile: the
brute-force tile of the Fig. 3 experiment, Sec. IV) and kNN from the join's
result (sj_knn_from_join, the reuse the paper names as future work, Sec. V),
both against the oracle exactly: the tile's values are the decision rule's
s (binary64, each operation rounded), so bit-identical to the oracle's; the
k nearest other eps-neighbours by (distance, index) are the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2209_11287_gb300 import binding, workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_11287_gb300 import build
    build.build()
    binding.load()


@pytest.mark.parametrize("m,nb,d", [(300, 1000, 5), (1, 1, 1), (130, 67, 37), (64, 64, 16), (2000, 300, 64)])
def test_sqdist_tile_bit_identical(m, nb, d):
    g = np.random.Generator(np.random.PCG64(m * 7 + nb + d))
    a = g.standard_normal((m, d)) * 3 + 1
    b = g.standard_normal((nb, d)) * 3 - 1
    got = binding.sj_sqdist_tile(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    x = np.concatenate([a, b])
    for i in np.unique(np.linspace(0, m - 1, min(m, 40)).astype(int)):
        assert np.array_equal(got[i], oracle.sqdist_row(x, int(i))[m:]), i


def _oracle_knn(x, eps, k):
    keys, dist = oracle.join(x, eps, with_dist=True)
    i, j = keys >> 32, keys & 0xFFFFFFFF
    keep = i != j
    i, j, dist = i[keep], j[keep], dist[keep]
    order = np.lexsort((j, dist, i))
    i, j, dist = i[order], j[order], dist[order]
    n = x.shape[0]
    idx = np.full((n, k), -1, dtype=np.int64)
    dd = np.full((n, k), np.inf)
    start = np.searchsorted(i, np.arange(n + 1))
    found = np.minimum(np.diff(start), k)
    for p in range(n):
        c = found[p]
        idx[p, :c] = j[start[p]:start[p] + c]
        dd[p, :c] = dist[start[p]:start[p] + c]
    return idx, dd, found


@pytest.mark.parametrize("kernel", ["filter_f32", "fp64_fma"])
@pytest.mark.parametrize("k", [1, 8, 40])
def test_knn_from_join_matches_oracle(kernel, k):
    w = workloads.uniform2d(n=8000, seed=17)
    ref_idx, ref_d, ref_f = _oracle_knn(w.points, w.eps, k)
    h = binding.sj_build_index(torch.from_numpy(w.points).cuda(), w.eps,
                               binding.sj_default_options(kernel=kernel, emit_distances=1))
    try:
        r = binding.sj_self_join(h)
        try:
            idx, dist, found = binding.sj_knn_from_join(r, w.n, k)
        finally:
            binding.sj_result_free(r)
    finally:
        binding.sj_destroy(h)
    assert np.array_equal(found, ref_f)
    assert np.array_equal(idx.astype(np.int64), ref_idx)
    assert np.array_equal(dist, ref_d)
    if k == 40:
        assert (found < k).any() and (found == k).any()  # both cases exercised


def test_knn_needs_distances():
    w = workloads.uniform2d(n=2000, seed=3)
    h = binding.sj_build_index(torch.from_numpy(w.points).cuda(), w.eps, binding.sj_default_options())
    try:
        r = binding.sj_self_join(h)
        try:
            with pytest.raises(binding.SimJoinError) as e:
                binding.sj_knn_from_join(r, w.n, 4)
            assert e.value.status == binding.SJ_ERR_ARG
        finally:
            binding.sj_result_free(r)
    finally:
        binding.sj_destroy(h)
