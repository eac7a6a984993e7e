"""Seeded synthetic inputs for the similarity self-join.

This module only draws points (numpy ``Generator(PCG64(seed))``, the same bit
stream on x86-64 and aarch64) and states each workload's eps.  It holds none
of the join's arithmetic; the CUDA library and the CPU oracle both read the
arrays it returns.

The paper evaluates on uniform and exponential synthetic sets of 2M/10M points
in 2-8 dims and on real sets that are not available here (Sec. IV-A, Tables 1
and 2); the workloads below are synthetic stand-ins of the same kinds:

* ``uniform2d``   n=16384 in [0,1]^2, eps = sqrt(32 / (pi n)) (mean ~32
                  neighbours from the disk area, boundary ignored).
* ``uniform4d``   n=2,000,000 in [0,1]^4, eps from the 4-ball volume for a
                  mean of 64 neighbours: eps^4 = 64 Gamma(3) / (n pi^2).
* ``mixture16d``  n=1,000,000 in d=16, 32 isotropic Gaussians (centres uniform
                  in [0,1]^16, sigma 0.04, equal weights), eps for a mean
                  selectivity of 100 (stored; calibrated with the oracle).
* ``expo64d``     n=500,000 in d=64, coordinates exponential(lambda=40)
                  clipped to [0,1], eps for a mean selectivity of 50 (stored;
                  calibrated with the oracle).
* ``brute16d``    n=2^17 in d=16, coordinates exponential(lambda=40) clipped
                  to [0,1], eps for a mean selectivity of 50 (stored;
                  calibrated with the oracle): the brute-force comparison of
                  Sec. IV (Fig. 3), joined without an index.
* ``batched``     4096 independent uniform instances: n log-uniform in
                  [256, 65536], d from {2,4,8,16,32}, eps per instance for a
                  mean of 32 neighbours.

Every generator takes ``n`` so tests can draw a smaller set of the same
distribution; eps then follows the same rule for that n (the stored,
calibrated values apply to the full sizes only, and smaller draws of the
calibrated workloads scale eps by (n_full / n)^(1/d)).
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
EPS_TABLE = os.path.join(_HERE, "workload_eps.json")


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Workload:
    name: str
    points: np.ndarray  # n x d binary64, row-major
    eps: float
    seed: int

    @property
    def n(self) -> int:
        return int(self.points.shape[0])

    @property
    def d(self) -> int:
        return int(self.points.shape[1])


def ball_eps(n: int, d: int, k: float) -> float:
    """Radius whose d-ball holds k points of a unit-density set of n points:
    k = n * pi^(d/2) eps^d / Gamma(d/2 + 1)."""
    return (k * math.gamma(d / 2 + 1) / (n * math.pi ** (d / 2))) ** (1.0 / d)


def _stored_eps(name: str):
    if not os.path.exists(EPS_TABLE):
        return None
    with open(EPS_TABLE) as f:
        return json.load(f).get(name)


def uniform2d(n: int = 16384, seed: int = 0) -> Workload:
    x = _rng(seed).random((n, 2))
    return Workload("uniform2d", x, math.sqrt(32.0 / (math.pi * n)), seed)


def uniform4d(n: int = 2_000_000, seed: int = 0) -> Workload:
    x = _rng(seed).random((n, 4))
    return Workload("uniform4d", x, ball_eps(n, 4, 64.0), seed)


def mixture16d(n: int = 1_000_000, seed: int = 0, eps: float | None = None) -> Workload:
    g = _rng(seed)
    centres = g.random((32, 16))
    labels = g.integers(0, 32, size=n)
    x = centres[labels] + 0.04 * g.standard_normal((n, 16))
    return Workload("mixture16d", np.ascontiguousarray(x), _eps_for("mixture16d", n, 16, 1_000_000, eps), seed)


def expo64d(n: int = 500_000, seed: int = 0, eps: float | None = None) -> Workload:
    x = np.minimum(_rng(seed).exponential(1.0 / 40.0, size=(n, 64)), 1.0)
    return Workload("expo64d", x, _eps_for("expo64d", n, 64, 500_000, eps), seed)


def brute16d(n: int = 1 << 17, seed: int = 0, eps: float | None = None) -> Workload:
    x = np.minimum(_rng(seed).exponential(1.0 / 40.0, size=(n, 16)), 1.0)
    return Workload("brute16d", x, _eps_for("brute16d", n, 16, 1 << 17, eps), seed)


def _eps_for(name: str, n: int, d: int, n_full: int, eps):
    if eps is not None:
        return float(eps)
    e = _stored_eps(name)
    if e is None:
        raise RuntimeError(f"no stored eps for {name}; run oracle/calibrate_eps.py")
    return float(e) * (n_full / n) ** (1.0 / d)


# ---- batched instances ---------------------------------------------------

BATCH_DIMS = (2, 4, 8, 16, 32)


def batch_instance_params(i: int):
    """(n, d) of instance i: n = floor(exp(U[ln 256, ln 65536])), d uniform
    over {2, 4, 8, 16, 32}; both drawn first from Generator(PCG64(i))."""
    g = _rng(i)
    n = int(math.floor(math.exp(g.uniform(math.log(256.0), math.log(65536.0)))))
    d = BATCH_DIMS[int(g.integers(0, len(BATCH_DIMS)))]
    return n, d, g


def batch_instance(i: int, eps: float | None = None) -> Workload:
    """Instance i of the batched workload: points uniform in [0,1]^d drawn
    after (n, d) from the same generator.  eps: the stored per-instance value
    (mean 32 neighbours), else the ball formula."""
    n, d, g = batch_instance_params(i)
    x = g.random((n, d))
    if eps is None:
        tab = _stored_eps("batched")
        if tab is not None and str(i) in tab:
            eps = float(tab[str(i)])
        else:
            eps = ball_eps(n, d, 32.0)
    return Workload(f"batched[{i}]", x, float(eps), i)


def batched(count: int = 4096):
    return [batch_instance(i) for i in range(count)]


CONFIGS = {
    "uniform2d": uniform2d,
    "uniform4d": uniform4d,
    "mixture16d": mixture16d,
    "expo64d": expo64d,
    "brute16d": brute16d,
}
