"""Certification of the low-precision filters, pair by pair.

Every filter kernel decides a pair with its own arithmetic (FP32 fma chains on
CUDA cores, or bf16 split products accumulated in FP32 by tcgen05 MMAs) and
trusts a certified bound E = c1 (P + pc) on the error of s~ = pc - 2 a against
the exact squared distance s_y of the stored kernel coordinates.  These tests
read the kernel's own value a of every evaluated pair (sj_debug_filter_dump)
and check, for every pair:

  * |s_y - s~| <= E, with s_y in double-double (error-free transformations:
    TwoSum, Knuth; TwoProduct by Dekker's split), so the bound itself holds on
    random, Gaussian-clustered, near-tie and cancellation-heavy data;
  * a >= thr_in  =>  the decision rule says in, a < thr_out => it says out,
    the rule being the oracle's binary64 direct form (Sec. II-A, Eq. 1);
  * every pair the FP32 filter's bounding-box prune dropped unevaluated has
    s_y above the prune radius^2 and is out under the decision rule.

The largest observed |s_y - s~| / E of each case is printed (pytest -s).
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


# ---- double-double arithmetic (numpy, elementwise) --------------------------

def _two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def _split(a):
    c = 134217729.0 * a  # 2^27 + 1
    hi = c - (c - a)
    return hi, a - hi


def _two_prod(a, b):
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


def _sqdist_dd(yq, yc):
    """||yq - yc||^2 of float32 rows as double-double (hi, lo), per row."""
    hi = np.zeros(yq.shape[0])
    lo = np.zeros(yq.shape[0])
    for k in range(yq.shape[1]):
        d, dl = _two_sum(yq[:, k].astype(np.float64), -yc[:, k].astype(np.float64))
        p, pl = _two_prod(d, d)
        pl = pl + 2.0 * d * dl + dl * dl
        hi, e = _two_sum(hi, p)
        lo = lo + e + pl
    return _two_sum(hi, lo)


def _cases():
    g = np.random.Generator(np.random.PCG64(4040))
    out = []
    w = workloads.uniform4d(n=6000, seed=11)
    out.append(("uniform4d", w.points, w.eps))
    w = workloads.uniform2d(n=6000, seed=12)
    out.append(("uniform2d", w.points, w.eps))
    # Gaussian clusters in 8-D: dense cells, many pairs near eps
    c = g.random((12, 8))
    x = c[g.integers(0, 12, size=5000)] + 0.02 * g.standard_normal((5000, 8))
    out.append(("clusters8d", x, 0.05))
    # 16-D Gaussian mixture (the tensor-core workload's distribution)
    w = workloads.mixture16d(n=4000, seed=13, eps=0.25)
    out.append(("mixture16d", w.points, w.eps))
    # near ties: pairs at a relative 1e-10 from eps
    from tests.test_oracle_pins import near_tie_points
    xt, et = near_tie_points(npairs=1500)
    out.append(("near_ties", xt, et))
    # cancellation: a tight cluster far from the centre of the extent (large
    # norms against tiny differences), the far corner holding one point
    x = 700.0 + 1e-3 * g.random((3000, 3))
    x = np.concatenate([x, [[-700.0, -700.0, -700.0]]])
    out.append(("cancellation", x, 2e-4))
    return out


CASES = _cases()
REPORT = {}


def _dump(x, eps, kernel):
    pts = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    h = binding.sj_build_index(pts, eps, binding.sj_default_options(kernel=kernel))
    try:
        ev = binding.sj_index_info(h)["n_evaluated"]
        cap = 2 * ev + 200000
        info, rec, arr = binding.sj_debug_filter_dump(h, cap)
    finally:
        binding.sj_destroy(h)
    assert 0 < info.records <= cap
    assert rec.shape[0] == info.records
    return info, rec, arr


def _rule_in(x, eps, perm, qs, cs):
    """The decision rule (oracle, input points) for pairs of cell positions."""
    e2 = eps * eps
    order = np.argsort(qs, kind="stable")
    qs_s, cs_s = qs[order], cs[order]
    bounds = np.flatnonzero(np.diff(qs_s)) + 1
    starts = np.concatenate([[0], bounds])
    ends = np.concatenate([bounds, [qs_s.size]])
    out = np.empty(qs.size, dtype=bool)
    for s0, s1 in zip(starts, ends):
        q = int(perm[qs_s[s0]])
        row = oracle.sqdist_row(x, q)
        out[order[s0:s1]] = row[perm[cs_s[s0:s1]]] <= e2
    return out


def _check(name, x, eps, kernel):
    info, rec, arr = _dump(x, eps, kernel)
    y = arr["y"]
    perm = arr["perm"]
    pruned = rec[:, 3] == 1
    if pruned.any():
        # the prune: s_y of each dropped pair is above the radius^2, and the
        # decision rule says out
        pq, pcs = rec[pruned, 0], rec[pruned, 1]
        sy_hi, sy_lo = _sqdist_dd(y[pq], y[pcs])
        assert np.all((sy_hi - info.prune_r2) + sy_lo > 0), f"{name}/{kernel}: a pruned pair within the radius"
        assert not np.any(_rule_in(x, eps, perm, pq, pcs)), f"{name}/{kernel}: a pruned pair is in"
    REPORT[(name, kernel, "pruned")] = int(pruned.sum())
    if kernel == "filter_f32" and name in ("uniform4d", "uniform2d"):
        # about 46% (4-D) and 20% (2-D) of the scheduled evaluations
        floor = 0.3 if name == "uniform4d" else 0.1
        assert pruned.sum() > floor * rec.shape[0], "the bounding-box prune removed almost nothing"
    rec = rec[~pruned]
    qs, cs = rec[:, 0], rec[:, 1]
    a = rec[:, 2].astype(np.int32).view(np.float32).astype(np.float64)
    pc = -2.0 * arr["h"].astype(np.float64)[cs]  # h = -pc / 2 exactly
    # s~ = pc - 2 a (both exact in binary64 as float values; the sum as
    # double-double), against s_y
    st_hi, st_lo = _two_sum(pc, -2.0 * a)
    sy_hi, sy_lo = _sqdist_dd(y[qs], y[cs])
    err = np.abs((st_hi - sy_hi) + (st_lo - sy_lo))
    E = info.c1 * (info.pbound + pc)
    ratio = err / E
    worst = float(ratio.max())
    REPORT[(name, kernel)] = worst
    print(f"\n{kernel:14s} {name:12s} pairs {rec.shape[0]:9d}  max |s_y - s~| / E = {worst:.3e}"
          f"  pruned {int(pruned.sum())}")
    assert worst < 1.0, (name, kernel, worst)
    # certified decisions against the decision rule (oracle, input points)
    tin = arr["thr_in"].astype(np.float64)[cs]
    tout = arr["thr_out"].astype(np.float64)[cs]
    cert_in = a >= tin
    cert_out = a < tout
    assert not np.any(cert_in & cert_out)
    rule_in = _rule_in(x, eps, perm, qs, cs)
    assert not np.any(cert_in & ~rule_in), f"{name}/{kernel}: a certified-in pair is out"
    assert not np.any(cert_out & rule_in), f"{name}/{kernel}: a certified-out pair is in"
    # the classes are not vacuous: most pairs are certified one way or the other
    assert cert_out.sum() + cert_in.sum() > 0.5 * qs.size or name == "cancellation"


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
@pytest.mark.parametrize("kernel", ["filter_f32", "filter_bf16x2", "filter_bf16x3", "filter_fp16x2"])
def test_certified_bound_per_pair(kernel, case):
    name, x, eps = case
    dp = 1 << max(1, (x.shape[1] - 1).bit_length())
    if kernel == "filter_f32" and dp > 8:
        pytest.skip("the FP32 filter's dump covers padded d <= 8")
    _check(name, x, eps, kernel)
