"""The bounds-checking build (-DSJ_DEBUG_BOUNDS): its tile kernels check
every candidate, query and stage index before using it and report the first
failing site (SJ_ERR_CUDA) instead of touching memory.  Joins of every kernel,
symmetric and not, on workloads with ragged and dense cells, must pass all
checks and still return the oracle's set.  Run in a subprocess that loads the
debug library."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import sys
    import numpy as np
    import torch
    sys.path.insert(0, {root!r})
    import oracle
    from paper_2209_11287_gb300 import binding, workloads
    cases = [workloads.uniform2d(n=5000, seed=2), workloads.uniform4d(n=20000, seed=3),
             workloads.mixture16d(n=4000, seed=4, eps=0.25)]
    g = np.random.Generator(np.random.PCG64(9))
    dense = np.repeat(g.random((10, 3)), 300, axis=0) + 1e-6 * g.standard_normal((3000, 3))
    for w in cases + [(dense, 0.01)]:
        x, eps = (w.points, w.eps) if hasattr(w, "points") else w
        ref = oracle.join(x, eps)
        for kernel in ("fp64_fma", "fp64_dmma", "filter_f32", "filter_bf16x3", "filter_bf16x2", "filter_fp16x2"):
            for sym in (1, 0):
                pairs, _, _ = binding.self_join(torch.from_numpy(x).cuda(), eps, kernel=kernel, symmetric=sym)
                assert np.array_equal(binding.pairs_to_keys(pairs), ref), (kernel, sym)
    print("debug-bounds ok")
""")


def test_debug_bounds_build_passes_every_check():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_11287_gb300 import build
    lib = build.build(debug_bounds=True)
    env = dict(os.environ, SJ_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT)], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "debug-bounds ok" in r.stdout
