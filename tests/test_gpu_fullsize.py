"""Parity at the full benchmark sizes of the 16-D, 64-D and batched workloads,
in the launch configuration bench.py times (default options per kernel).

The oracle cannot enumerate these joins whole, so each test compares sampled
query rows with the oracle's rows (Sec. II-A, Eq. 1; the grid of Sec. III-B
must prune nothing), and checks on the whole result what holds at any size:
the set is symmetric, holds every self pair (i, i) and no pair twice.
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


def _device_join(x, eps, kernel):
    """The join of the benchmark (default options for `kernel`), pairs left
    on the device as an (count, 2) int32 tensor."""
    pts = torch.from_numpy(x).cuda()
    h = binding.sj_build_index(pts, eps, binding.sj_default_options(kernel=kernel))
    try:
        r = binding.sj_self_join(h)
        try:
            pairs = torch.empty((int(r.count), 2), dtype=torch.int32, device="cuda")
            binding.sj_result_copy(r, pairs)
            assert r.reruns == 0 or r.count > 0
        finally:
            binding.sj_result_free(r)
    finally:
        binding.sj_destroy(h)
    return pairs


def _check_rows(x, eps, pairs, n_rows, seed):
    n = x.shape[0]
    sample = np.sort(np.random.default_rng(seed).choice(n, size=n_rows, replace=False))
    sel = torch.zeros(n, dtype=torch.bool, device="cuda")
    sel[torch.from_numpy(sample).cuda()] = True
    p = pairs[sel[pairs[:, 0].long()]]
    got = torch.sort((p[:, 0].long() << 32) | p[:, 1].long()).values.cpu().numpy()
    ref, _ = oracle.rows(x, eps, sample)
    assert np.array_equal(got, np.sort(ref))


def _check_whole(pairs, n):
    keys = (pairs[:, 0].long() << 32) | pairs[:, 1].long()
    rev = (pairs[:, 1].long() << 32) | pairs[:, 0].long()
    ks = torch.sort(keys).values
    assert bool((ks[1:] > ks[:-1]).all()), "a pair is emitted twice"
    assert torch.equal(ks, torch.sort(rev).values), "the set is not symmetric"
    del keys, rev
    diag = pairs[pairs[:, 0] == pairs[:, 1]][:, 0]
    assert diag.numel() == n and torch.equal(torch.sort(diag).values.cpu(), torch.arange(n, dtype=torch.int32))


@pytest.mark.parametrize("kernel", ["filter_bf16x2", "filter_bf16x3", "filter_fp16x2", "filter_f32"])
def test_mixture16d_full_size(kernel):
    """1M points in 16-D (32 Gaussians), the calibrated eps of the benchmark."""
    w = workloads.mixture16d()
    pairs = _device_join(w.points, w.eps, kernel)
    _check_rows(w.points, w.eps, pairs, 200, seed=16)
    _check_whole(pairs, w.n)
    assert pairs.shape[0] > 5e7


@pytest.mark.parametrize("kernel", ["filter_bf16x2", "filter_bf16x3", "filter_fp16x2"])
def test_expo64d_full_size(kernel):
    """500k points in 64-D (clipped exponential), the calibrated eps."""
    w = workloads.expo64d()
    pairs = _device_join(w.points, w.eps, kernel)
    _check_rows(w.points, w.eps, pairs, 200, seed=64)
    _check_whole(pairs, w.n)
    assert pairs.shape[0] > 1e7


def test_batched_full_size():
    """All 4096 instances in one batched join with the benchmark's default
    options (AUTO per dimension group); rows sampled from every 16th
    instance, and every sampled instance's whole set symmetric with its
    diagonal."""
    insts = workloads.batched(4096)
    pts = [torch.from_numpy(w.points).cuda() for w in insts]
    inputs = binding.BatchInputs(pts, [w.eps for w in insts])
    res = binding.sj_join_batch_raw(inputs, binding.sj_default_options())
    try:
        rng = np.random.default_rng(4096)
        for i in range(0, 4096, 16):
            w = insts[i]
            r = res[i]
            pairs = torch.empty((int(r.count), 2), dtype=torch.int32, device="cuda")
            binding.sj_result_copy(r, pairs)
            rows = int(min(w.n, 8))
            sample = np.sort(rng.choice(w.n, size=rows, replace=False))
            sel = torch.zeros(w.n, dtype=torch.bool, device="cuda")
            sel[torch.from_numpy(sample).cuda()] = True
            p = pairs[sel[pairs[:, 0].long()]]
            got = torch.sort((p[:, 0].long() << 32) | p[:, 1].long()).values.cpu().numpy()
            ref, _ = oracle.rows(w.points, w.eps, sample)
            assert np.array_equal(got, np.sort(ref)), i
            _check_whole(pairs, w.n)
    finally:
        binding.sj_results_free(res)
