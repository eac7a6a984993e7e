"""DBSCAN on the join's result (sj_dbscan), the reuse of the self-join the
paper names as future work (Sec. V): labels must equal the oracle's
(oracle.dbscan: the same definition on the oracle's own pair set, pinned
against scikit-learn in test_oracle_dbscan.py), for joins by every kernel."""
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


def _gpu_dbscan(x, eps, min_pts, kernel):
    h = binding.sj_build_index(torch.from_numpy(np.ascontiguousarray(x)).cuda(), eps,
                               binding.sj_default_options(kernel=kernel))
    try:
        r = binding.sj_self_join(h)
        try:
            return binding.sj_dbscan(r, x.shape[0], min_pts)
        finally:
            binding.sj_result_free(r)
    finally:
        binding.sj_destroy(h)


def _clusters(seed, n=20000, d=2):
    g = np.random.Generator(np.random.PCG64(seed))
    centres = g.random((40, d))
    x = np.concatenate([centres[g.integers(0, 40, n)] + 0.01 * g.standard_normal((n, d)),
                        g.random((n // 10, d))])
    return x


@pytest.mark.parametrize("kernel", ["filter_f32", "fp64_fma", "filter_bf16x2"])
@pytest.mark.parametrize("min_pts", [1, 5, 20])
def test_dbscan_matches_oracle(kernel, min_pts):
    x = _clusters(3)
    eps = 0.006
    ref, k_ref = oracle.dbscan(x, eps, min_pts)
    got, k = _gpu_dbscan(x, eps, min_pts, kernel)
    assert k == k_ref
    assert np.array_equal(got.astype(np.int64), ref)


def test_dbscan_4d_uniform_and_all_noise():
    w = workloads.uniform4d(n=100000, seed=4)
    ref, k_ref = oracle.dbscan(w.points, w.eps, 40)
    got, k = _gpu_dbscan(w.points, w.eps, 40, "filter_f32")
    assert k == k_ref and np.array_equal(got.astype(np.int64), ref)
    # min_pts above every degree: no core point, all noise
    got, k = _gpu_dbscan(w.points, w.eps, 10 ** 6, "filter_f32")
    assert k == 0 and np.all(got == -1)
