"""Batched self-joins (sj_join_batch) against the CPU oracle, per instance.

Every instance of a batch must give exactly the pair set (instance-local
indices) and distances the oracle gives for that instance alone; the batch
shares indexes, launches and the result pool, never decisions.
"""
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
    oracle.build()


def _keys(pairs):
    return binding.pairs_to_keys(pairs) if len(pairs) else np.zeros(0, dtype=np.int64)


def _mixed_batch(seed=0):
    """Small instances of every padded dimension, uneven n, and the
    degenerate ones: one point, all points equal, duplicates, a line, large
    offsets and negative coordinates."""
    g = np.random.default_rng(seed)
    pts, eps = [], []
    for d in (1, 2, 3, 4, 5, 8, 12, 16, 32):
        for n in (1, 7, 300, 1500):
            x = g.random((n, d))
            pts.append(x)
            eps.append(workloads.ball_eps(n, d, 16.0) if n > 1 else 0.1)
    pts.append(np.full((50, 3), 0.25))                 # one cell, all pairs
    eps.append(0.01)
    x = g.random((400, 4))
    pts.append(np.concatenate([x, x[:100]]))          # duplicates
    eps.append(0.05)
    pts.append(np.stack([np.linspace(0, 1, 500), np.zeros(500)], axis=1))  # a line
    eps.append(0.003)
    pts.append(1e6 + g.random((600, 2)))              # large offset
    eps.append(0.03)
    pts.append(-5.0 + 10.0 * g.random((800, 8)))      # negative coordinates, wide extent
    eps.append(4.0)
    pts.append(g.random((200, 2)))                    # eps above the diameter: n^2 pairs
    eps.append(2.0)
    pts.append(g.random((300, 16)))                   # eps below every gap: the diagonal
    eps.append(1e-9)
    # shuffle so groups and instance numbers interleave
    order = g.permutation(len(pts))
    return [np.ascontiguousarray(pts[i]) for i in order], [eps[i] for i in order]


def _check(pts, eps, out, with_dist):
    assert len(out) == len(pts)
    for k, (x, e, (pairs, dists, st)) in enumerate(zip(pts, eps, out)):
        if with_dist:
            ref, rd = oracle.join(x, e, with_dist=True)
        else:
            ref, rd = oracle.join(x, e), None
        got = _keys(pairs)
        assert st["count"] == ref.size, (k, x.shape, e, st["count"], ref.size)
        assert np.all(np.diff(got) > 0), f"instance {k}: duplicate pairs"
        assert np.array_equal(got, ref), f"instance {k} ({x.shape}, eps {e}) differs"
        if with_dist:
            p = pairs.astype(np.int64)
            order = np.argsort((p[:, 0] << 32) | p[:, 1], kind="stable")
            assert np.array_equal(dists[order], rd), f"instance {k}: distances differ"


@pytest.mark.parametrize("kernel", ["filter_f32", "fp64_fma", "filter_bf16x3", "filter_bf16x2", "filter_fp16x2",
                                    "auto"])
@pytest.mark.parametrize("symmetric", [1, 0])
def test_mixed_batch(kernel, symmetric):
    pts, eps = _mixed_batch()
    out = binding.join_batch([torch.from_numpy(x).cuda() for x in pts], eps, kernel=kernel, symmetric=symmetric)
    _check(pts, eps, out, with_dist=False)


@pytest.mark.parametrize("indexed_dims", [1, 3, 6])
def test_mixed_batch_indexed_dims(indexed_dims):
    """Any choice of indexed dims gives the same pairs."""
    pts, eps = _mixed_batch(seed=3)
    out = binding.join_batch(pts, eps, kernel="auto", indexed_dims=indexed_dims)
    _check(pts, eps, out, with_dist=False)


@pytest.mark.parametrize("kernel", ["filter_f32", "fp64_fma", "filter_bf16x3", "filter_bf16x2", "filter_fp16x2"])
def test_mixed_batch_distances_host_input(kernel):
    pts, eps = _mixed_batch(seed=1)
    out = binding.join_batch(pts, eps, kernel=kernel, emit_distances=True)
    _check(pts, eps, out, with_dist=True)


@pytest.mark.parametrize("kernel", ["filter_f32", "auto"])
def test_pool_regrow(kernel):
    """A pool far too small (64-pair pages, a 1-pair hint) is regrown from the
    exact counts and the joins rerun; the result is unchanged."""
    pts, eps = _mixed_batch(seed=2)
    out = binding.join_batch(pts, eps, kernel=kernel, page_pairs=64, max_pairs_hint=1,
                             emit_distances=True)
    assert max(st["reruns"] for _, _, st in out) >= 1
    _check(pts, eps, out, with_dist=True)


def test_candidate_counts_per_instance():
    """Each instance's canonical candidate count is that of its own grid
    (cells of side eps (1 + 2^-20) over its own extent, every dim indexed)."""
    g = np.random.default_rng(5)
    pts = [g.random((2000, 2)), g.random((3000, 2)), g.random((1000, 2))]
    eps = [0.02, 0.05, 0.04]
    out = binding.join_batch(pts, eps, kernel="fp64_fma", indexed_dims=2)
    for x, e, (_, _, st) in zip(pts, eps, out):
        assert st["n_candidates"] == oracle.grid_candidate_count(x, e * (1.0 + 2.0 ** -20))


@pytest.mark.parametrize("kernel", ["filter_f32", "filter_bf16x2", "filter_fp16x2", "auto"])
def test_extreme_coordinate_scales(kernel):
    """Instances whose coordinate spread underflows (1e-30) or overflows (1e25)
    binary32, beside an ordinary one: each instance's coordinates are scaled
    by its own power of two, and every instance's set is the oracle's."""
    g = np.random.Generator(np.random.PCG64(78))
    pts, eps = [], []
    for scale in (1e-30, 1.0, 1e25, 1e-100):
        c = g.random((10, 8))
        pts.append((c[g.integers(0, 10, 1500)] + 0.03 * g.standard_normal((1500, 8))) * scale)
        eps.append(0.1 * scale)
    out = binding.join_batch(pts, eps, kernel=kernel)
    _check(pts, eps, out, with_dist=False)


def test_unsupported_kernel_rejected():
    with pytest.raises(RuntimeError):
        binding.join_batch([np.random.default_rng(0).random((10, 4))], [0.1], kernel="fp64_dmma")
    with pytest.raises(RuntimeError):  # the tensor-core filter stops at d = 64
        binding.join_batch([np.random.default_rng(0).random((10, 65))], [0.1], kernel="filter_bf16x3")


def test_bad_instance_rejected():
    x = np.random.default_rng(0).random((10, 2))
    y = x.copy()
    y[3, 1] = np.nan
    with pytest.raises(RuntimeError):
        binding.join_batch([x, y], [0.1, 0.1])
    with pytest.raises(RuntimeError):
        binding.join_batch([x, x], [0.1, -1.0])


def test_workload_sample_rows():
    """The first 256 instances of the batched workload (n log-uniform in
    [256, 65536], d in {2, 4, 8, 16, 32}) in one batch: sampled instances give
    a symmetric pair set holding the diagonal, and sampled query rows match
    the oracle exactly."""
    insts = [workloads.batch_instance(i) for i in range(256)]
    pts = [w.points for w in insts]
    eps = [w.eps for w in insts]
    out = binding.join_batch([torch.from_numpy(x).cuda() for x in pts], eps, kernel="auto")
    g = np.random.default_rng(11)
    for k in range(0, 256, 8):
        x, e = pts[k], eps[k]
        pairs, _, st = out[k]
        p = pairs.astype(np.int64)
        keys = np.sort((p[:, 0] << 32) | p[:, 1])
        assert np.all(np.diff(keys) > 0)
        # symmetry and the diagonal
        mirror = np.sort((p[:, 1] << 32) | p[:, 0])
        assert np.array_equal(keys, mirror)
        assert np.count_nonzero(p[:, 0] == p[:, 1]) == len(x)
        rows = g.choice(len(x), size=min(24, len(x)), replace=False)
        for r in rows:
            ref = np.sort(oracle.rows(x, e, np.array([r]))[0])
            lo = np.searchsorted(keys, np.int64(r) << 32)
            hi = np.searchsorted(keys, np.int64(r + 1) << 32)
            assert np.array_equal(keys[lo:hi], ref), (k, r)
