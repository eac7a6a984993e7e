"""Host-side fault injection and independent checks of the index build.

* Allocation failures: the library's allocator is made to fail at every
  allocation of a build + join in turn (sj_debug_fail_allocations); each
  attempt must end with SJ_ERR_OOM and release every device block it took
  (sj_debug_live_allocations back to its value before), and once the
  injection no longer triggers the join returns the oracle's set.  No GPU
  fault is involved: the failure is made on the host.
* The sort by cell key (Sec. III-B: points grouped by grid cell) against an
  independent sort: the cell order of a built index, read back with
  sj_index_perm, must list the points by non-decreasing cell key, where the
  keys are computed on the host from the oracle's grid coordinates and sorted
  by torch.sort.
* Tracing of the build phases (sj_set_tracing / sj_index_phase_ms).
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
    yield
    binding.sj_debug_fail_allocations(-1)


def _single(x, eps, kernel):
    pts = torch.from_numpy(x).cuda()
    h = binding.sj_build_index(pts, eps, binding.sj_default_options(kernel=kernel))
    try:
        r = binding.sj_self_join(h)
        try:
            pairs, _ = binding.sj_result_copy(r)
        finally:
            binding.sj_result_free(r)
    finally:
        binding.sj_destroy(h)
    return binding.pairs_to_keys(pairs)


def _batch(insts, epss):
    return [binding.pairs_to_keys(p) for p, _, _ in binding.join_batch(insts, epss)]


def _sweep(run, check):
    """Fail allocation k for k = 0, 1, ... until the call succeeds; every
    failing attempt must leave the live block count unchanged."""
    run()  # warm: pools, events, caches
    torch.cuda.synchronize()
    base = binding.sj_debug_live_allocations()
    k = 0
    while True:
        binding.sj_debug_fail_allocations(k)
        ok = True
        try:
            out = run()
        except binding.SimJoinError as e:
            assert e.status == binding.SJ_ERR_OOM, (k, e)
            ok = False
        finally:
            binding.sj_debug_fail_allocations(-1)
        torch.cuda.synchronize()
        assert binding.sj_debug_live_allocations() == base, (k, binding.sj_debug_live_allocations(), base)
        if ok:
            check(out)
            return k
        k += 1
        assert k < 400


@pytest.mark.parametrize("kernel", ["filter_f32", "fp64_fma", "filter_bf16x2", "fp64_dmma"])
@pytest.mark.parametrize("eps_scale", [1.0, 0.01], ids=["dense_keys", "sparse_keys"])
def test_allocation_failure_single_join(kernel, eps_scale):
    w = workloads.uniform2d(n=3000, seed=5)
    eps = w.eps * eps_scale
    ref = oracle.join(w.points, eps)
    k = _sweep(lambda: _single(w.points, eps, kernel), lambda got: np.testing.assert_array_equal(got, ref))
    assert k >= 5  # the build and the join allocate at several points, each failed once


def test_allocation_failure_batched_join():
    insts = [workloads.uniform2d(n=1500, seed=1).points, workloads.mixture16d(n=1200, seed=2, eps=0.25).points,
             workloads.uniform4d(n=2000, seed=3).points]
    epss = [workloads.uniform2d(n=1500, seed=1).eps, 0.25, workloads.uniform4d(n=2000, seed=3).eps]
    refs = [oracle.join(x, e) for x, e in zip(insts, epss)]

    def check(out):
        for got, ref in zip(out, refs):
            np.testing.assert_array_equal(got, ref)

    assert _sweep(lambda: _batch(insts, epss), check) >= 5


def test_allocation_failure_join_to_host():
    w = workloads.uniform2d(n=4000, seed=6)
    ref = oracle.join(w.points, w.eps)

    def run():
        h = binding.sj_build_index(torch.from_numpy(w.points).cuda(), w.eps, binding.sj_default_options())
        try:
            out = np.empty((ref.size + 16, 2), dtype=np.int32)
            cnt, _ = binding.sj_self_join_to_host(h, out, 4096)
            return binding.pairs_to_keys(out[:cnt])
        finally:
            binding.sj_destroy(h)

    _sweep(run, lambda got: np.testing.assert_array_equal(got, ref))


def _host_keys(x, w, dims):
    """Row-major cell keys over `dims` from the oracle's grid coordinates
    (cells of side w from the per-dim minimum)."""
    c = oracle.grid_cells(x, w, dims)
    ext = c.max(axis=0) + 1
    key = np.zeros(x.shape[0], dtype=np.int64)
    for k in range(c.shape[1]):
        key = key * int(ext[k]) + c[:, k]
    return key


@pytest.mark.parametrize("eps_scale", [1.0, 0.01], ids=["counting_sort", "radix_sort"])
@pytest.mark.parametrize("d", [2, 3])
def test_cell_order_matches_independent_sort(d, eps_scale):
    g = np.random.Generator(np.random.PCG64(600 + d))
    x = g.random((20000, d))
    eps = 0.02 * eps_scale
    h = binding.sj_build_index(torch.from_numpy(x).cuda(), eps, binding.sj_default_options(kernel="filter_f32"))
    try:
        info = binding.sj_index_info(h)
        perm = binding.sj_index_perm(h, x.shape[0])
    finally:
        binding.sj_destroy(h)
    assert info["m"] == d  # every dim is indexed here
    assert np.array_equal(np.sort(perm), np.arange(x.shape[0]))  # a permutation
    key = _host_keys(x, eps * (1.0 + 2.0 ** -20), list(range(d)))
    got = torch.from_numpy(key[perm])
    want = torch.sort(torch.from_numpy(key)).values
    assert torch.equal(got, want)  # same multiset, non-decreasing
    # cells are the runs of equal keys: as many as the independent count
    assert info["n_cells"] == np.unique(key).size


def test_phase_tracing():
    """Tracing on: the four build phases get device and host times (the
    device times sum to at most the build's device time); off: -1."""
    w = workloads.uniform4d(n=200000, seed=8)
    pts = torch.from_numpy(w.points).cuda()
    binding.sj_set_tracing(True)
    try:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        h = binding.sj_build_index(pts, w.eps, binding.sj_default_options(kernel="filter_f32"))
        e1.record()
        torch.cuda.synchronize()
        try:
            dev, host = binding.sj_index_phase_ms(h)
        finally:
            binding.sj_destroy(h)
    finally:
        binding.sj_set_tracing(False)
    assert np.all(dev >= 0) and np.all(host >= 0)
    assert dev.sum() <= e0.elapsed_time(e1) * 1.05 + 0.05
    h = binding.sj_build_index(pts, w.eps, binding.sj_default_options(kernel="filter_f32"))
    try:
        dev, host = binding.sj_index_phase_ms(h)
    finally:
        binding.sj_destroy(h)
    assert np.all(dev == -1) and np.all(host == -1)
