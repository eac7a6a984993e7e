"""Parity of the CUDA self-join with the CPU oracle, through the C ABI.

The decision rule (s <= fl(eps^2), binary64 direct form) is fixed and every
kernel certifies its decisions and re-decides the pairs inside its error bound
with that rule, so the pair sets must be identical to the oracle's and the
emitted distances bit-identical (the tolerance the workload allows, pairs
within 1e-9 eps of eps and 1e-12 relative distance error, is not needed).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2209_11287_gb300 import binding, workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KERNELS = ["fp64_fma", "fp64_dmma", "filter_f32", "filter_bf16x3", "filter_bf16x2", "filter_fp16x2"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_11287_gb300 import build
    build.build()
    binding.load()
    oracle.build()


def gpu_join(x, eps, kernel, device_input=True, **kw):
    pts = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    if device_input:
        pts = pts.cuda()
    pairs, dists, stats = binding.self_join(pts, eps, kernel=kernel, **kw)
    torch.cuda.synchronize()
    keys = (pairs[:, 0].astype(np.int64) << 32) | pairs[:, 1].astype(np.int64)
    order = np.argsort(keys, kind="stable")
    keys = keys[order]
    if dists is not None:
        dists = dists[order]
    return keys, dists, stats


def assert_same_set(x, eps, ref, got):
    assert np.all(np.diff(got) > 0), "duplicate pairs emitted"
    only_ref, only_got, bad = oracle.compare_pair_sets(x, eps, ref, got)
    assert bad == 0, (only_ref, only_got)
    assert only_ref == 0 and only_got == 0, (only_ref, only_got)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("symmetric", [1, 0])
def test_uniform2d_full(kernel, symmetric):
    w = workloads.uniform2d()
    ref = oracle.join(w.points, w.eps)
    got, _, st = gpu_join(w.points, w.eps, kernel, symmetric=symmetric)
    assert_same_set(w.points, w.eps, ref, got)
    assert st["count"] == ref.size


@pytest.mark.parametrize("kernel", ["fp64_fma", "filter_f32"])
def test_evaluated_count_triangle(kernel):
    """Symmetric joins on the CUDA-core kernels evaluate the half
    neighbourhood with only the triangle of each self cell: item t of a cell
    (16 queries each) starts its self-cell candidates at its own first query,
    so the evaluations are (candidates + sum |c|^2) / 2 minus, per cell of q
    points, the sum over items of 16 t Q_t."""
    w = workloads.uniform2d()
    _, _, st = gpu_join(w.points, w.eps, kernel)
    cells = oracle.grid_cells(w.points, w.eps * (1.0 + 2.0 ** -20))
    _, cnt = np.unique(cells, axis=0, return_counts=True)
    skip = 0
    for q in cnt.tolist():
        skip += sum(16 * t * min(16, q - 16 * t) for t in range((q + 15) // 16))
    full = (st["n_candidates"] + int((cnt.astype(np.int64) ** 2).sum())) // 2
    assert st["n_evaluated"] == full - skip


def test_bbox_prune_counts():
    """The FP32 filter (padded d <= 8, no distances) drops candidates farther
    than eps from the bounding box of an item's queries before evaluating
    them: it performs fewer evaluations than the grid schedules (about half
    on uniform 4-D points) with the same pair set; the FP64 tile performs
    every scheduled one."""
    w = workloads.uniform4d(n=40000, seed=21)
    ref = oracle.join(w.points, w.eps)
    got, _, st = gpu_join(w.points, w.eps, "filter_f32")
    assert_same_set(w.points, w.eps, ref, got)
    assert 0.35 * st["n_evaluated"] < st["n_performed"] < 0.7 * st["n_evaluated"]
    _, _, st64 = gpu_join(w.points, w.eps, "fp64_fma")
    assert st64["n_performed"] == st64["n_evaluated"] == st["n_evaluated"]


@pytest.mark.parametrize("kernel", KERNELS)
def test_distances_bit_identical(kernel):
    w = workloads.uniform2d(n=6000, seed=3)
    ref, rd = oracle.join(w.points, w.eps, with_dist=True)
    got, gd, _ = gpu_join(w.points, w.eps, kernel, emit_distances=True)
    assert_same_set(w.points, w.eps, ref, got)
    assert np.array_equal(gd, rd)


def test_canonical_candidate_count():
    """The index's candidate count (full 3^m neighbourhoods, cells of side
    w = eps (1 + 2^-20)) equals the oracle's count on the same grid."""
    w = workloads.uniform2d()
    _, _, st = gpu_join(w.points, w.eps, "fp64_fma")
    assert st["m"] == 2
    assert st["n_candidates"] == oracle.grid_candidate_count(w.points, w.eps * (1.0 + 2.0 ** -20))
    assert st["n_evaluated"] < st["n_candidates"]


def _cases():
    g = np.random.Generator(np.random.PCG64(77))
    out = []
    out.append(("single_point", np.array([[0.5, 0.25]]), 0.1))
    out.append(("two_duplicates", np.array([[1.0, 2.0, 3.0]] * 2), 1e-3))
    out.append(("all_identical", np.full((300, 3), 0.125), 1e-6))
    out.append(("d1", g.random((3000, 1)), 1e-3))
    out.append(("d3", g.random((4000, 3)), 0.03))
    out.append(("d5", g.random((3000, 5)), 0.12))
    out.append(("d8", g.random((2500, 8)), 0.3))
    out.append(("d33", g.random((800, 33)), 1.0))
    k = g.integers(0, 24, size=(2000, 2))
    out.append(("lattice_ties", k / 8.0, 2.0 / 8.0))          # many pairs at exactly eps
    out.append(("lattice_cell_edges", k / 8.0, 1.0 / 8.0))    # points on cell boundaries
    out.append(("eps_above_diameter", g.random((500, 2)), 2.0))
    out.append(("eps_below_gaps", g.random((500, 4)), 1e-9))
    far = g.random((700, 2))
    far[0] = [1e6, -1e6]
    out.append(("one_far_point", far, 0.05))
    out.append(("negative_coords", g.standard_normal((3000, 3)) * 5.0, 0.4))
    clustered = np.repeat(g.random((20, 2)), 60, axis=0) + 1e-7 * g.standard_normal((1200, 2))
    out.append(("dense_cells", clustered, 0.01))
    return out


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_edge_cases(kernel, case):
    _, x, eps = case
    ref = oracle.join(x, eps)
    for sym in (1, 0):
        got, _, _ = gpu_join(x, eps, kernel, symmetric=sym)
        assert_same_set(x, eps, ref, got)


@pytest.mark.parametrize("kernel", KERNELS)
def test_mixture16d_small(kernel):
    w = workloads.mixture16d(n=12000, eps=0.25)
    ref = oracle.join(w.points, w.eps)
    got, _, _ = gpu_join(w.points, w.eps, kernel)
    assert_same_set(w.points, w.eps, ref, got)


@pytest.mark.parametrize("kernel", KERNELS)
def test_expo64d_small(kernel):
    w = workloads.expo64d(n=3000, eps=0.19)
    ref = oracle.join(w.points, w.eps)
    got, _, _ = gpu_join(w.points, w.eps, kernel)
    assert_same_set(w.points, w.eps, ref, got)


@pytest.mark.parametrize("kernel", KERNELS)
def test_near_ties(kernel):
    """Pairs at a relative 1e-10 from eps are decided exactly."""
    from tests.test_oracle_pins import near_tie_points
    x, eps = near_tie_points(npairs=3000)
    ref = oracle.join(x, eps)
    got, _, _ = gpu_join(x, eps, kernel)
    assert_same_set(x, eps, ref, got)


def test_host_input_matches_device_input():
    w = workloads.uniform2d(n=5000, seed=9)
    a, _, _ = gpu_join(w.points, w.eps, "filter_f32", device_input=True)
    b, _, _ = gpu_join(w.points, w.eps, "filter_f32", device_input=False)
    assert np.array_equal(a, b)


def test_overflow_regrows_and_reruns():
    """A page pool smaller than the result: the count stays exact, the pool
    grows to the exact size and the join runs once more."""
    w = workloads.uniform2d(n=8000, seed=2)
    ref = oracle.join(w.points, w.eps)
    opt = binding.sj_default_options(kernel="filter_f32", page_pairs=1024, max_pairs_hint=100)
    h = binding.sj_build_index(torch.from_numpy(w.points).cuda(), w.eps, opt)
    r = binding.sj_self_join(h)
    assert r.reruns == 1 and r.count == ref.size
    pairs, _ = binding.sj_result_copy(r)
    binding.sj_result_free(r)
    binding.sj_destroy(h)
    assert_same_set(w.points, w.eps, ref, binding.pairs_to_keys(pairs))


def test_small_pages():
    """Results spanning many pages (1024 pairs each) are assembled correctly."""
    w = workloads.uniform2d(n=8000, seed=8)
    ref = oracle.join(w.points, w.eps)
    opt = binding.sj_default_options(kernel="fp64_fma", page_pairs=1024)
    h = binding.sj_build_index(torch.from_numpy(w.points).cuda(), w.eps, opt)
    r = binding.sj_self_join(h)
    assert r.n_pages > 100
    pairs, _ = binding.sj_result_copy(r)
    binding.sj_result_free(r)
    binding.sj_destroy(h)
    got = binding.pairs_to_keys(pairs)
    assert_same_set(w.points, w.eps, ref, got)


def test_copy_to_device_tensor():
    w = workloads.uniform2d(n=5000, seed=10)
    h = binding.sj_build_index(torch.from_numpy(w.points).cuda(), w.eps, binding.sj_default_options())
    r = binding.sj_self_join(h)
    dev = torch.empty((r.count, 2), dtype=torch.int32, device="cuda")
    binding.sj_result_copy(r, dev)
    host, _ = binding.sj_result_copy(r)
    binding.sj_result_free(r)
    binding.sj_destroy(h)
    assert np.array_equal(dev.cpu().numpy(), host)


def test_non_finite_coordinate_rejected():
    x = np.random.default_rng(0).random((100, 3))
    x[17, 1] = np.nan
    with pytest.raises(binding.SimJoinError) as e:
        binding.sj_build_index(torch.from_numpy(x).cuda(), 0.1)
    assert e.value.status == binding.SJ_ERR_ARG


def _rows_from_gpu(pairs_dev, n, sample):
    sel = torch.zeros(n, dtype=torch.bool, device="cuda")
    sel[torch.from_numpy(sample).cuda()] = True
    p = pairs_dev[sel[pairs_dev[:, 0].long()]]
    keys = (p[:, 0].long() << 32) | p[:, 1].long()
    return torch.sort(keys).values.cpu().numpy()


@pytest.mark.parametrize("kernel", KERNELS)
def test_uniform4d_full_size_sampled_rows(kernel):
    """The 2M-point 4-D workload at full size, in the launch configuration the
    benchmark times: sampled query rows equal the oracle's rows, and the set is
    symmetric with every self pair."""
    w = workloads.uniform4d()
    pts = torch.from_numpy(w.points).cuda()
    opt = binding.sj_default_options(kernel=kernel)
    h = binding.sj_build_index(pts, w.eps, opt)
    r = binding.sj_self_join(h)
    pairs = torch.empty((r.count, 2), dtype=torch.int32, device="cuda")
    binding.sj_result_copy(r, pairs)
    count = int(r.count)
    binding.sj_result_free(r)
    binding.sj_destroy(h)
    sample = np.random.default_rng(1).choice(w.n, size=200, replace=False)
    got = _rows_from_gpu(pairs, w.n, sample)
    ref, _ = oracle.rows(w.points, w.eps, np.sort(sample))
    assert np.array_equal(got, np.sort(ref))
    # symmetric, self pairs, no duplicates
    keys = (pairs[:, 0].long() << 32) | pairs[:, 1].long()
    rev = (pairs[:, 1].long() << 32) | pairs[:, 0].long()
    ks = torch.sort(keys).values
    assert torch.equal(ks, torch.sort(rev).values)
    assert bool((ks[1:] > ks[:-1]).all())
    selfc = int((pairs[:, 0] == pairs[:, 1]).sum())
    assert selfc == w.n
    assert count > 1.0e8


def test_bounded_wait_gives_up():
    """A kernel waiting on an mbarrier that nothing arrives on gives up after
    its bound and reports it; the context stays usable for the next join."""
    st = binding.sj_selftest_bounded_wait()
    assert st == binding.SJ_ERR_TIMEOUT, (st, binding.sj_last_error_message())
    w = workloads.uniform2d(n=3000, seed=9)
    ref = oracle.join(w.points, w.eps)
    got, _, _ = gpu_join(w.points, w.eps, "filter_bf16x3")
    assert_same_set(w.points, w.eps, ref, got)


@pytest.mark.parametrize("kernel", ["filter_f32", "fp64_fma", "filter_bf16x2"])
@pytest.mark.parametrize("eps", [2e-4, 0.02], ids=["sparse_keys_radix_sort", "dense_keys_counting_sort"])
def test_key_space_paths(kernel, eps):
    """The index sorts by cell key with an LSD radix sort when the key space
    is large (2e-4: 5000^2 keys for 3000 points) and with a counting sort
    plus a dense key table when it is small (0.02: 51^2 keys); both give the
    oracle's set."""
    x = np.random.Generator(np.random.PCG64(123)).random((3000, 2))
    ref = oracle.join(x, eps)
    got, _, st = gpu_join(x, eps, kernel)
    assert_same_set(x, eps, ref, got)
    assert st["n_candidates"] == oracle.grid_candidate_count(x, eps * (1.0 + 2.0 ** -20))


@pytest.mark.parametrize("kernel", KERNELS)
def test_no_index_brute_force(kernel):
    """indexed_dims = SJ_NO_INDEX: one cell, every pair evaluated (the
    brute-force comparison of Sec. IV); the set is the oracle's, the
    candidate count n^2 and the evaluations those of one triangle (or all
    n^2 where a kernel evaluates the full self cell)."""
    w = workloads.brute16d(n=3000, seed=4)
    ref = oracle.join(w.points, w.eps)
    got, _, st = gpu_join(w.points, w.eps, kernel, indexed_dims=binding.SJ_NO_INDEX)
    assert_same_set(w.points, w.eps, ref, got)
    assert st["m"] == 0 and st["n_cells"] == 1
    assert st["n_candidates"] == w.n * w.n
    assert w.n * (w.n + 1) // 2 <= st["n_evaluated"] <= w.n * w.n


@pytest.mark.parametrize("kernel", ["filter_f32", "filter_bf16x2", "filter_fp16x2"])
@pytest.mark.parametrize("emit", [False, True], ids=["pairs", "distances"])
def test_recheck_queue_overflow(kernel, emit):
    """One point far from the rest makes the kernel coordinates' norms huge,
    so the certified bound covers every evaluated pair: all of them go to the
    recheck queue, more than it holds (2^20 entries or 1/64 of the
    evaluations), and the overflow is re-decided inside the tile kernel."""
    g = np.random.Generator(np.random.PCG64(31))
    x = np.concatenate([g.random((20000, 2)), [[1.0e4, 1.0e4]]])
    eps = 0.04
    ref, rd = oracle.join(x, eps, with_dist=True)
    got, dists, st = gpu_join(x, eps, kernel, emit_distances=emit)
    assert_same_set(x, eps, ref, got)
    assert st["n_rechecked"] > (1 << 20)
    if emit:
        assert np.array_equal(dists, rd)


@pytest.mark.parametrize("kernel", KERNELS)
def test_join_to_host_in_rounds(kernel):
    """Results larger than the device buffers: the join runs in rounds of
    work items through two buffers of 20000 pairs (the result holds 5.3e5)
    and the host gets exactly the oracle's set; a host array too small gets
    the exact count, an overflow status and a prefix of valid pairs."""
    w = workloads.uniform2d(n=16384, seed=7)
    ref = oracle.join(w.points, w.eps)
    pts = torch.from_numpy(w.points).cuda()
    h = binding.sj_build_index(pts, w.eps, binding.sj_default_options(kernel=kernel))
    try:
        out = torch.empty((ref.size + 64, 2), dtype=torch.int32).pin_memory()
        cnt, rounds = binding.sj_self_join_to_host(h, out, 20000)
        assert cnt == ref.size and rounds >= ref.size // 20000
        got = binding.pairs_to_keys(out[:cnt].numpy())
        assert np.array_equal(got, ref)
        small = np.empty((1000, 2), dtype=np.int32)  # pageable, too small
        with pytest.raises(binding.SimJoinError) as ei:
            binding.sj_self_join_to_host(h, small, 4096)
        assert ei.value.status == binding.SJ_ERR_RESULT_OVERFLOW
        assert str(ref.size) in str(ei.value)
        part = binding.pairs_to_keys(small)
        assert np.all(np.isin(part, ref)) and np.unique(part).size == 1000
    finally:
        binding.sj_destroy(h)


@pytest.mark.parametrize("kernel", KERNELS + ["auto"])
@pytest.mark.parametrize("scale", [1e-100, 1e-30, 1e25, 1e100], ids=lambda s: f"{s:g}")
def test_extreme_coordinate_scales(kernel, scale):
    """Coordinates whose spread underflows binary32 (1e-30: squared
    distances near 1e-60) or overflows it (1e25: squares near 1e50), and far
    beyond (1e-100, 1e100): the binary32 filters scale their coordinates by a
    power of two into range, so every kernel returns the oracle's set."""
    g = np.random.Generator(np.random.PCG64(77))
    d = 16 if kernel in ("filter_bf16x3", "filter_bf16x2", "filter_fp16x2", "auto") else 3
    centres = g.random((20, d))
    x = (centres[g.integers(0, 20, 3000)] + 0.03 * g.standard_normal((3000, d))) * scale
    eps = (0.15 if d == 16 else 0.05) * scale
    ref = oracle.join(x, eps)
    assert ref.size > 30 * 3000  # about 45 neighbours a point
    got, _, _ = gpu_join(x, eps, kernel)
    assert_same_set(x, eps, ref, got)
