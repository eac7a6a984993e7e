"""Sharding one join over several GPUs (Sec. III-B: the queries of one cell
with their candidate runs are an independent unit), run here as the shards
one after another on one GPU: every shard builds its own index from the same
points (the order of the points inside a cell differs between builds),
runs its contiguous range of whole cells, and the disjoint union of the
shards' pair sets must be the oracle's set."""
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


@pytest.mark.parametrize("kernel", ["filter_f32", "fp64_fma", "filter_bf16x2"])
@pytest.mark.parametrize("n_shards", [2, 3, 8])
def test_shards_union_is_the_join(kernel, n_shards):
    # dense enough that many cells hold more than one work item (16 queries)
    w = workloads.uniform4d(n=60000, seed=21)
    w.eps *= 1.25
    ref = oracle.join(w.points, w.eps)
    pts = torch.from_numpy(w.points).cuda()
    parts, works = [], []
    for k in range(n_shards):
        h = binding.sj_build_index(pts, w.eps, binding.sj_default_options(kernel=kernel))
        try:
            work = binding.sj_index_item_work(h)
            bounds = binding.sj_shard_bounds(work, n_shards)
            r = binding.sj_self_join_range(h, int(bounds[k]), int(bounds[k + 1]))
            try:
                pairs, _ = binding.sj_result_copy(r)
            finally:
                binding.sj_result_free(r)
            info = binding.sj_index_info(h)
        finally:
            binding.sj_destroy(h)
        assert work.sum() == info["n_evaluated"]  # the cells' work is the join's
        if kernel != "filter_bf16x2":  # (its work items hold up to 248 queries)
            assert (work == 0).any()  # some cells span several work items
        assert all(work[b] > 0 for b in bounds[1:-1] if b < work.size)  # boundaries at cell starts
        works.append(int(work[bounds[k]:bounds[k + 1]].sum()))
        parts.append(binding.pairs_to_keys(pairs))
    got = np.sort(np.concatenate(parts))
    assert np.all(np.diff(got) > 0), "a pair came from two shards"
    assert np.array_equal(got, ref)
    # balanced: every shard within one cell's work of an equal share
    total = sum(works)
    assert max(abs(x - total / n_shards) for x in works) <= work.max()
