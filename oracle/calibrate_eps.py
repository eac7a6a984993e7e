"""Writes the stored eps of the calibrated workloads (test infrastructure).

For the 16-D Gaussian mixture (mean selectivity 100), the 64-D clipped
exponential set (mean selectivity 50), the 16-D clipped exponential set of the
brute-force workload (mean selectivity 50) and the batched instances of dimension
8 and more (mean 32 neighbours each; in a unit cube the d-ball formula is far
off there) no closed form gives eps, so it is calibrated with the oracle:
squared distances from seeded sample queries (2000, or 500 per batched
instance) to all points (oracle order, the query itself excluded), eps^2 =
the (target x queries)-th smallest of the pooled values.  The result goes to
paper_2209_11287_gb300/workload_eps.json, which the workload generators read.

Run: python oracle/calibrate_eps.py [--batched-only | --brute16d-only]
"""
import json
import os
import sys
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2209_11287_gb300 import workloads  # noqa: E402


def calibrate(x, target, n_queries=2000, seed=12345):
    """Same rule as oracle.calibrate_eps, with the rows computed in parallel."""
    n = x.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    qs = rng.choice(n, size=min(n_queries, n), replace=False)
    k = int(round(target * qs.size))
    kk = min(k, n - 1)

    def row(q):
        r = oracle.sqdist_row(x, int(q))
        r[q] = np.inf
        return np.partition(r, kk - 1)[:kk]

    with ThreadPoolExecutor(max_workers=os.cpu_count()) as ex:
        pooled = np.concatenate(list(ex.map(row, qs)))
    return float(np.sqrt(np.partition(pooled, k - 1)[k - 1]))


def main():
    oracle.build()
    out = {}
    if os.path.exists(workloads.EPS_TABLE):
        out = json.load(open(workloads.EPS_TABLE))
    if "--brute16d-only" in sys.argv:
        b = workloads.brute16d(eps=1.0)
        out["brute16d"] = calibrate(b.points, 50.0)
        print("brute16d", out["brute16d"], flush=True)
        with open(workloads.EPS_TABLE, "w") as f:
            json.dump(out, f, indent=1, sort_keys=True)
            f.write("\n")
        return
    batched = {}
    for i in range(4096):
        n, d, _ = workloads.batch_instance_params(i)
        if d >= 8:
            w = workloads.batch_instance(i, eps=1.0)
            batched[str(i)] = calibrate(w.points, 32.0, n_queries=500, seed=1000 + i)
    out["batched"] = batched
    print("batched", len(batched), "instances calibrated", flush=True)
    if "--batched-only" in sys.argv:
        with open(workloads.EPS_TABLE, "w") as f:
            json.dump(out, f, indent=1, sort_keys=True)
            f.write("\n")
        return
    m = workloads.mixture16d(eps=1.0)
    out["mixture16d"] = calibrate(m.points, 100.0)
    print("mixture16d", out["mixture16d"], flush=True)
    e = workloads.expo64d(eps=1.0)
    out["expo64d"] = calibrate(e.points, 50.0)
    print("expo64d", out["expo64d"], flush=True)
    b = workloads.brute16d(eps=1.0)
    out["brute16d"] = calibrate(b.points, 50.0)
    print("brute16d", out["brute16d"], flush=True)
    with open(workloads.EPS_TABLE, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
