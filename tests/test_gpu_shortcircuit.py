"""The variance-ordered dims and the certified short-circuit of the FP64
CUDA-core tile (Sec. II-D orders dims by variance; Sec. III-B stops a tile
once every distance in it exceeds eps).  The short-circuit only skips tiles
whose every pair the full filter would also declare out, so the pair set
must stay the oracle's, with symmetric joins and without, on data where
the partial sums cross eps early (clustered, exponential, a far outlier)."""
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


def _join(x, eps, short_circuit, symmetric=1, emit=False):
    pairs, dists, st = binding.self_join(torch.from_numpy(np.ascontiguousarray(x)).cuda(), eps, kernel="fp64_fma",
                                         symmetric=symmetric, emit_distances=emit, short_circuit=short_circuit)
    keys = (pairs[:, 0].astype(np.int64) << 32) | pairs[:, 1].astype(np.int64)
    order = np.argsort(keys)
    return keys[order], (dists[order] if dists is not None else None), st


def _cases():
    g = np.random.Generator(np.random.PCG64(808))
    out = [("mixture16d", workloads.mixture16d(n=12000, seed=3, eps=0.25).points, 0.25),
           ("expo64d", workloads.expo64d(n=3000, seed=4, eps=0.19).points, 0.19),
           ("brute16d", workloads.brute16d(n=5000, seed=5).points, workloads.brute16d(n=5000, seed=5).eps)]
    # dims of very different spread: the variance order puts the wide ones first
    x = g.random((4000, 24)) * np.geomspace(4.0, 0.01, 24)
    out.append(("graded_spread24d", x, 0.08))
    far = g.random((3000, 17))
    far[0] = 50.0
    out.append(("far_point17d", far, 0.5))
    return out


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
@pytest.mark.parametrize("symmetric", [1, 0])
def test_short_circuit_keeps_the_set(case, symmetric):
    _, x, eps = case
    ref = oracle.join(x, eps)
    got, _, _ = _join(x, eps, 1, symmetric)
    assert np.array_equal(got, ref)


def test_short_circuit_distances_bit_identical():
    w = workloads.mixture16d(n=6000, seed=9, eps=0.25)
    ref, rd = oracle.join(w.points, w.eps, with_dist=True)
    got, gd, _ = _join(w.points, w.eps, 1, emit=True)
    assert np.array_equal(got, ref) and np.array_equal(gd, rd)


def test_brute_force_no_index_with_short_circuit():
    w = workloads.brute16d(n=4000, seed=6)
    ref = oracle.join(w.points, w.eps)
    pairs, _, st = binding.self_join(torch.from_numpy(w.points).cuda(), w.eps, kernel="fp64_fma",
                                     indexed_dims=binding.SJ_NO_INDEX, short_circuit=1)
    assert np.array_equal(binding.pairs_to_keys(pairs), ref)
    assert st["n_cells"] == 1
