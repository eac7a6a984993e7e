"""The autotuner (sj_autotune, sj_autotune_batch), joins that follow its
tuning cache, and batched joins whose join phase runs as a CUDA graph: every
tuned or graph-run join must still give exactly the oracle's pair set."""
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


TUNABLE = {binding.SJ_KERNEL_FILTER_F32, binding.SJ_KERNEL_FILTER_BF16X2, binding.SJ_KERNEL_FILTER_FP16X2,
           binding.SJ_KERNEL_FILTER_BF16X3}


@pytest.mark.parametrize("make", [lambda: workloads.uniform4d(n=20000, seed=5),
                                  lambda: workloads.mixture16d(n=6000, seed=6)], ids=["uniform4d", "mixture16d"])
def test_autotune_single_then_cached_join(tmp_path, make):
    w = make()
    cache = str(tmp_path / "tune.txt")
    pts = torch.from_numpy(w.points).cuda()
    best, ms = binding.sj_autotune(pts, w.eps, reps=2, cache_path=cache)
    assert best.kernel in TUNABLE and ms > 0
    assert best.queries_per_item >= 0 and best.indexed_dims >= 0
    entry = binding.sj_tune_lookup(cache, 0, w.d, w.n)
    assert entry == {"kernel": best.kernel, "qpi": best.queries_per_item, "m": best.indexed_dims}
    ref = oracle.join(w.points, w.eps)
    pairs, _, st = binding.self_join(pts, w.eps, tune_cache=cache)
    assert st["kernel"] == best.kernel
    if best.indexed_dims:
        assert st["m"] == best.indexed_dims
    assert np.array_equal(_keys(pairs), ref)
    # the winner's options used directly give the same set
    h = binding.sj_build_index(pts, w.eps, best)
    try:
        r = binding.sj_self_join(h)
        try:
            got, _ = binding.sj_result_copy(r)
        finally:
            binding.sj_result_free(r)
    finally:
        binding.sj_destroy(h)
    assert np.array_equal(_keys(got), ref)


@pytest.mark.parametrize("kernel,qpi", [("filter_f32", 4), ("filter_f32", 9), ("filter_bf16x2", 24),
                                        ("filter_bf16x3", 40)])
def test_queries_per_item_keeps_the_set(kernel, qpi):
    """Every item size the tuner may pick gives the oracle's set (items of
    a cell split at qpi queries; the self-cell triangle spans items)."""
    w = workloads.mixture16d(n=4000, seed=9) if "bf16" in kernel else workloads.uniform2d(n=6000, seed=9)
    pairs, _, st = binding.self_join(torch.from_numpy(w.points).cuda(), w.eps, kernel=kernel, queries_per_item=qpi)
    assert np.array_equal(_keys(pairs), oracle.join(w.points, w.eps))


def _batch(seed):
    g = np.random.default_rng(seed)
    pts, eps = [], []
    for d in (2, 3, 4, 8, 16, 32):
        for n in (5, 400, 2500):
            pts.append(g.random((n, d)))
            eps.append(workloads.ball_eps(n, d, 16.0) if d <= 4 else 0.25 * np.sqrt(d / 8.0))
    order = g.permutation(len(pts))
    return [np.ascontiguousarray(pts[i]) for i in order], [eps[i] for i in order]


def _check_batch(pts, eps, out):
    for k, (x, e, (pairs, _, st)) in enumerate(zip(pts, eps, out)):
        ref = oracle.join(x, e)
        assert st["count"] == ref.size, (k, x.shape)
        assert np.array_equal(_keys(pairs), ref), f"instance {k} ({x.shape}) differs"


def test_autotune_batch_then_graph_join(tmp_path):
    pts, eps = _batch(3)
    cache = str(tmp_path / "tune.txt")
    dev = [torch.from_numpy(x).cuda() for x in pts]
    inp = binding.BatchInputs(dev, eps)
    groups = binding.sj_autotune_batch(inp, reps=1, cache_path=cache)
    assert sorted(g["dp"] for g in groups) == [2, 4, 8, 16, 32]
    for g in groups:
        assert g["kernel"] in TUNABLE and g["qpi"] >= 0
        assert binding.sj_tune_lookup(cache, 1, g["dp"]) == {"kernel": g["kernel"], "qpi": g["qpi"], "m": 0}
    for graph in (0, 1):
        out = binding.join_batch(dev, eps, graph=graph, tune_cache=cache)
        _check_batch(pts, eps, out)
        by_dp = {g["dp"]: g["kernel"] for g in groups}
        for x, (_, _, st) in zip(pts, out):
            dp = 2
            while dp < x.shape[1]:
                dp *= 2
            assert st["kernel"] == by_dp[dp]


@pytest.mark.parametrize("kernel", ["auto", "filter_f32", "filter_bf16x2", "fp64_fma"])
def test_graph_join_phase_matches_oracle(kernel):
    """The graph-run join phase (two branches, groups concurrent) with
    distances, and twice in a row on the same inputs."""
    pts, eps = _batch(4)
    for _ in range(2):
        out = binding.join_batch(pts, eps, kernel=kernel, graph=1, emit_distances=True)
        assert all(st["ms_tile"] > 0 for _, _, st in out), "graph-run groups report their tile time"
        for k, (x, e, (pairs, dists, st)) in enumerate(zip(pts, eps, out)):
            ref, rd = oracle.join(x, e, with_dist=True)
            got = _keys(pairs)
            assert np.array_equal(got, ref), f"instance {k} differs"
            p = pairs.astype(np.int64)
            order = np.argsort((p[:, 0] << 32) | p[:, 1], kind="stable")
            assert np.array_equal(dists[order], rd)


def test_graph_join_phase_overflow_rerun():
    """A page pool too small for the result: the graph-run phase is
    recaptured with the exact pool and the sets stay exact."""
    pts, eps = _batch(5)
    out = binding.join_batch(pts, eps, graph=1, page_pairs=64, max_pairs_hint=64)
    _check_batch(pts, eps, out)
    assert any(st["reruns"] > 0 for _, _, st in out)
