"""The allocation-free entry point sj_self_join_noalloc, for callers that
cannot allocate device memory while they run (a device memory budget that
another allocator reserved up front, a runtime that forbids cudaMalloc after
start-up): it must return exactly the oracle's pair set (Sec. II-A, Eq. 1), and
the regular entry point's with the plain FP64 kernel, call after call,
although every call reuses the same static scratch.

This file is collected last so that a run stopping at its first failure has
already run every other test.
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


def _keys(pairs):
    p = np.asarray(pairs, dtype=np.int64)
    return np.sort((p[:, 0] << 32) | p[:, 1])


def _regular(x, eps):
    pairs, _, _ = binding.self_join(torch.from_numpy(x).cuda(), eps, kernel="fp64_fma")
    return _keys(pairs)


def _noalloc(x, eps, capacity):
    out = torch.empty((capacity, 2), dtype=torch.int32, device="cuda")
    cnt = binding.sj_self_join_noalloc(torch.from_numpy(x).cuda(), eps, out)
    torch.cuda.synchronize()
    return cnt, _keys(out[:cnt].cpu().numpy())


def test_two_calls_match_oracle_and_regular_entry_point():
    # first call: a larger 4-D set; second call: a smaller 2-D set, so any
    # state the first call left in the shared scratch would show
    a = workloads.uniform4d(n=30000, seed=5)
    b = workloads.uniform2d(n=9000, seed=6)
    for w in (a, b):
        ref = oracle.join(w.points, w.eps)
        cnt, got = _noalloc(w.points, w.eps, capacity=ref.size + 1024)
        assert cnt == ref.size
        assert np.array_equal(got, ref)
        assert np.array_equal(_regular(w.points, w.eps), ref)


def test_largest_accepted_size():
    """n = SJ_NOALLOC_MAX_N points of d = SJ_NOALLOC_MAX_D dims fill every
    region of the scratch (packed rows of all padded columns, perm, items);
    uniform in [0,1]^8 with eps for about 32 neighbours.  Run twice so the
    second call starts from the first call's leftovers."""
    n, d = 32768, 8
    x = np.random.Generator(np.random.PCG64(2024)).random((n, d))
    eps = workloads.ball_eps(n, d, 32.0)
    ref = oracle.join(x, eps)
    for _ in range(2):
        cnt, got = _noalloc(x, eps, capacity=ref.size + 64)
        assert cnt == ref.size
        assert np.array_equal(got, ref)


def test_limits_are_enforced():
    x = torch.zeros((40000, 2), dtype=torch.float64, device="cuda")
    out = torch.empty((16, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(binding.SimJoinError) as e:
        binding.sj_self_join_noalloc(x, 0.1, out)
    assert e.value.status == binding.SJ_ERR_ARG
    y = torch.zeros((100, 9), dtype=torch.float64, device="cuda")
    with pytest.raises(binding.SimJoinError) as e:
        binding.sj_self_join_noalloc(y, 0.1, out)
    assert e.value.status == binding.SJ_ERR_ARG


def test_overflow_reports_exact_count():
    w = workloads.uniform2d(n=5000, seed=7)
    ref = _regular(w.points, w.eps)
    out = torch.empty((100, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(binding.SimJoinError) as e:
        binding.sj_self_join_noalloc(torch.from_numpy(w.points).cuda(), w.eps, out)
    assert e.value.status == binding.SJ_ERR_RESULT_OVERFLOW
    assert str(ref.size) in str(e.value)
