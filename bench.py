"""Benchmark of the similarity self-join on the 2M-point 4-D uniform workload.

One step = the whole hot path on one batch: build the grid index of the
points already resident on the GPU (extent, cell keys, radix sort, cell table,
packing, neighbour runs, work items) and run the join (distance tiles, eps
threshold, compaction into result pages) until the result count is known.

Prints ONE JSON line (rank 0).  ``value`` is candidate pairs per second for the
headline kernel: the candidate pairs of the full 3^4 grid neighbourhoods
(ordered, self pairs included) divided by the step time, summed over ranks.
The plain FP64 kernels are timed in the same run under ``variants``.

--impl reference runs the CPU oracle instead (brute force, all host cores, a
bounded sample of queries per step, scaled to the whole workload).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import shutil
import statistics
import subprocess
import tempfile
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "self-join candidate pairs/s and join time, n=2M d=4: FP64 plain vs low-prec filter"
UNIT = "candidate pairs/s"
HEADLINE = "filter_f32"
VARIANTS = ["filter_f32", "fp64_fma", "fp64_dmma"]
L2_FLUSH_BYTES = 256 << 20
FP32_FMA_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x 2 flop x max clock
FP64_DFMA_TFLOPS = 1.255                                  # measured, profiles/fp64_peaks_gb300.txt
FP64_DMMA_TFLOPS = 1.102                                  # measured, profiles/fp64_peaks_gb300.txt
KERNEL_NAMES = {"filter_f32": "k_join_f32s (d <= 8) | k_join_cc<float>", "fp64_fma": "k_join_cc<double>",
                "fp64_fma_sc": "k_join_cc<double> (short-circuit)", "fp64_dmma": "k_join_dmma",
                "filter_bf16x3": "k_join_tc", "filter_bf16x2": "k_join_tc", "filter_fp16x2": "k_join_tc"}
DTYPES = {"auto": "fp16x2|bf16x2|f32+f64", "filter_f32": "f32+f64", "filter_bf16x3": "bf16x3+f64",
          "filter_bf16x2": "bf16x2+f64", "filter_fp16x2": "fp16x2+f64", "fp64_fma": "f64",
          "fp64_dmma": "f64", "fp64_fma_sc": "f64", "tuned": "fp16x2|bf16x2|bf16x3|f32+f64", "tuned_graph": "fp16x2|bf16x2|bf16x3|f32+f64",
          "auto_graph": "fp16x2|bf16x2|f32+f64"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n", type=int, default=0, help="points (0 = the workload's full size)")
    ap.add_argument("--variants", default=",".join(VARIANTS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-queries", type=int, default=0, help="oracle sample size (0 = sized for ~15 s)")
    ap.add_argument("--hint", type=int, default=0, help="expected result pairs (0 = the library's automatic pool)")
    ap.add_argument("--workload", default="uniform4d",
                    choices=["uniform4d", "uniform2d", "mixture16d", "expo64d", "brute16d", "batched"],
                    help="uniform4d: the 2M-point 4-D self-join (the headline); uniform2d: 16384 x 2; mixture16d: "
                         "1M x 16 Gaussian mixture; expo64d: 500k x 64 clipped exponential; batched: 4096 "
                         "independent joins")
    ap.add_argument("--batch-count", type=int, default=4096)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(v: float, world: int, dev) -> float:
    """The maximum of v over all ranks (the slowest replica's time); v itself
    on one rank.  dev: the device of the process group's tensors."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_of(item_work, rank: int, world: int):
    """The contiguous range of work items rank `rank` runs: shards of about
    equal pair evaluations (the library's host-side partition, the same on
    every rank)."""
    from paper_2209_11287_gb300 import binding
    b = binding.sj_shard_bounds(item_work, world)
    return int(b[rank]), int(b[rank + 1])


def instance_shard(sizes, rank: int, world: int):
    """The contiguous range of batch instances rank `rank` joins: shards of
    about equal sum of n_i^2 (the grid-independent work of an instance), by
    the library's host-side partition, the same on every rank."""
    import numpy as np
    return shard_of(np.asarray(sizes, dtype=np.int64) ** 2, rank, world)


def gather_sums(values, world: int, dev) -> list:
    """Element-wise sums over the ranks of a few int64 values (counts of a
    sharded batch), on every rank."""
    if world == 1:
        return [int(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([int(v) for v in values], dtype=torch.int64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [int(v) for v in t.tolist()]


def gather_counts(count: int, world: int, dev) -> list:
    """Every rank's result count (int64), gathered on every rank: the one
    exchange of a sharded join (|R| is their sum)."""
    if world == 1:
        return [int(count)]
    import torch
    import torch.distributed as dist
    t = torch.tensor([int(count)], dtype=torch.int64, device=dev)
    out = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(out, t)
    return [int(o.item()) for o in out]


WORKLOAD_TEXT = {
    "uniform4d": "points i.i.d. uniform in [0,1]^4, eps from the 4-ball volume for a mean of 64 neighbours",
    "uniform2d": "points i.i.d. uniform in [0,1]^2, eps = sqrt(32 / (pi n))",
    "mixture16d": "32 isotropic Gaussians in 16-D (centres uniform in [0,1]^16, sigma 0.04, equal weights), "
                  "eps calibrated on the oracle for a mean of 100 neighbours",
    "expo64d": "64-D coordinates i.i.d. exponential(40) clipped to [0,1], eps calibrated on the oracle for a "
               "mean of 50 neighbours",
    "brute16d": "16-D coordinates i.i.d. exponential(40) clipped to [0,1], eps calibrated on the oracle for a "
                "mean of 50 neighbours, joined without an index (brute force: every pair evaluated)",
}
METRICS = {
    "uniform4d": METRIC,
    "uniform2d": "self-join candidate pairs/s and join time, n=16384 d=2: FP64 plain vs low-prec filter",
    "mixture16d": "self-join candidate pairs/s and join time, n=1M d=16 Gaussian mixture: FP64 plain vs low-prec filter",
    "brute16d": "brute-force self-join (no index) pairs/s and join time, n=2^17 d=16 clipped exponential: FP64 "
                "CUDA cores vs FP64 tensor cores vs low-prec filter",
    "expo64d": "self-join candidate pairs/s and join time, n=500k d=64 clipped exponential: FP64 plain vs "
               "low-prec filter",
}
DEFAULT_VARIANTS = {
    "uniform4d": ["filter_f32", "tuned", "fp64_fma", "fp64_dmma", "filter_fp16x2", "filter_bf16x2", "filter_bf16x3"],
    "uniform2d": ["filter_f32", "fp64_fma", "fp64_dmma", "filter_bf16x2"],
    "mixture16d": ["filter_fp16x2", "tuned", "filter_bf16x2", "filter_bf16x3", "filter_f32", "fp64_fma",
                   "fp64_fma_sc"],
    "expo64d": ["filter_fp16x2", "filter_bf16x2", "filter_bf16x3", "filter_f32"],
    "brute16d": ["filter_fp16x2", "filter_bf16x2", "filter_bf16x3", "filter_f32", "fp64_fma", "fp64_fma_sc",
                 "fp64_dmma"],
}


def workload_config(w, extra=None):
    cfg = {"workload": f"{w.name}: n={w.n} {WORKLOAD_TEXT.get(w.name, '')} (seed {w.seed}), eps={w.eps:.7g}",
           "n": w.n, "d": w.d, "eps": w.eps}
    if extra:
        cfg.update(extra)
    return cfg


def make_workload(args):
    from paper_2209_11287_gb300 import workloads
    make = workloads.CONFIGS[args.workload]
    return make(n=args.n) if args.n > 0 else make()


# ---- clocks sampled during the timed region -----------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---- native arm -------------------------------------------------------------------

def run_native(args):
    import torch

    from paper_2209_11287_gb300 import binding, build, workloads

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    binding.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    w = make_workload(args)
    pts = torch.from_numpy(w.points).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    def slowest(v: float) -> float:
        return max_over_ranks(v, world, dev)

    def one_step(opt, host=None, host_out=None):
        """Build + join (+ copy out).  With several ranks every rank builds the
        same index, runs its shard of the work items and the counts are
        gathered; the step's count is the whole join's.  End to end on one
        GPU (host points, host_out given) the join runs in rounds whose pairs
        are copied to host_out while the next round runs."""
        h = binding.sj_build_index(pts if host is None else host, w.eps, opt, stream)
        if world == 1 and host_out is not None:
            count, _ = binding.sj_self_join_to_host(h, host_out, e2e_device_pairs)
            info = binding.sj_index_info(h)
            binding.sj_destroy(h)
            return (count, info["n_candidates"], info["n_evaluated"], 0, 0, 0.0, -1)
        if world > 1:
            i0, i1 = shard_of(binding.sj_index_item_work(h), rank, world)
            r = binding.sj_self_join_range(h, i0, i1)
        else:
            r = binding.sj_self_join(h)
        if host_out is not None:
            binding.sj_result_copy(r, host_out)
        count = sum(gather_counts(int(r.count), world, dev))
        info = (count, int(r.n_candidates), int(r.n_evaluated), int(r.n_rechecked), int(r.reruns),
                float(r.ms_tile), int(r.kernel))
        binding.sj_result_free(r)
        binding.sj_destroy(h)
        return info

    knames = {v: k for k, v in binding.KERNELS.items()}
    tuned = {}

    def make_opt(kname):
        """Options of a variant: a kernel name, or "tuned" (the autotuner's
        pick for this workload, tuned once before the variant's warm-up)."""
        if kname != "tuned":
            sc = kname.endswith("_sc")  # FP64 tile with the variance order and short-circuit
            return binding.sj_default_options(kernel=kname[:-3] if sc else kname, max_pairs_hint=args.hint,
                                              short_circuit=int(sc),
                                              indexed_dims=binding.SJ_NO_INDEX if w.name == "brute16d" else 0)
        if not tuned:
            t0 = time.perf_counter()
            best, ms = binding.sj_autotune(pts, w.eps, binding.sj_default_options(max_pairs_hint=args.hint), stream,
                                           reps=3)
            tuned.update(opt=best, ms=ms, seconds=round(time.perf_counter() - t0, 1))
        return tuned["opt"]

    results = {}
    sampler = ClockSampler(local)
    variants = [v for v in args.variants.split(",") if v]
    if args.variants == ",".join(VARIANTS):
        variants = DEFAULT_VARIANTS[args.workload]
    # the clock sampler (an nvidia-smi process) starts before the first
    # warm-up and settles, so its start-up does not fall into timed steps
    sampler.start()
    time.sleep(1.0)
    for vi, kname in enumerate(variants):
        opt = make_opt(kname)
        for _ in range(args.warmup):
            one_step(opt)
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        launches0 = binding.sj_kernel_launches()
        info = None
        tile_ms = []
        for k in range(args.steps):
            flush.fill_(float(k))  # evict the inputs from L2 between steps
            ev[k][0].record(stream)
            info = one_step(opt)
            ev[k][1].record(stream)
            tile_ms.append(info[5])
        barrier()
        launches = binding.sj_kernel_launches() - launches0
        clocks = sampler.stop() if vi == len(variants) - 1 else None
        times = [a.elapsed_time(b) for a, b in ev]
        ms = slowest(sum(times) / len(times))
        count, cand, evald, rech, reruns, _, kused = info
        results[kname] = {"kernel": knames.get(kused, kname), "ms_per_step": ms, "count": count,
                          "n_candidates": cand, "n_evaluated": evald,
                          "n_rechecked": rech, "reruns": reruns, "launches": launches, "clocks": clocks,
                          "ms_min": min(times), "ms_max": max(times),
                          "tile_ms": slowest(statistics.mean(tile_ms))}

    # the distance-tile kernel's duration: CUDA events the library records on
    # its stream around the launch, averaged over the timed steps
    head = results[variants[0]]
    kern_ms = head["tile_ms"]

    # end to end through the C ABI with host buffers (pinned), copies inside
    # the timed region; the pairs reach host memory in rounds of work items
    # (two device buffers of about an eighth of the result each), each
    # round's copy overlapping the next round's tiles
    host_pts = torch.from_numpy(w.points).pin_memory()
    host_out = torch.empty((head["count"] + 16, 2), dtype=torch.int32).pin_memory()
    e2e_device_pairs = max(1 << 20, head["count"] // 8)
    link = link_bandwidth(host_pts, host_out, dev)
    opt = make_opt(variants[0])
    one_step(opt, host_pts, host_out)
    barrier()
    t_e2e = []
    for k in range(max(3, min(args.steps, 10))):
        flush.fill_(float(k))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        one_step(opt, host_pts, host_out)
        torch.cuda.synchronize(dev)
        t_e2e.append(time.perf_counter() - t0)
    e2e_s = slowest(statistics.mean(t_e2e))

    if rank == 0:
        line = make_line(args, w, results, variants, world, kern_ms, e2e_s, head)
        line["e2e"].update(link)
        line["e2e"]["ms_min"] = round(min(t_e2e) * 1e3, 3)
        line["e2e"]["ms_max"] = round(max(t_e2e) * 1e3, 3)
        line["e2e"]["d2h_floor_ms"] = round(head["count"] * 8 / (link["d2h_gbs"] * 1e9) * 1e3, 3)
        line["e2e"]["path"] = ("sj_build_index on pinned host points, sj_self_join_to_host into pinned host memory "
                               "(rounds of work items, copies overlapping the next round)" if world == 1 else
                               "sj_build_index on pinned host points, sj_self_join_range, sj_result_copy")
        if tuned:
            o = tuned["opt"]
            line["autotune"] = {"kernel": knames.get(o.kernel, "?"), "queries_per_item": o.queries_per_item,
                                "indexed_dims": o.indexed_dims, "tuned_ms": round(tuned["ms"], 4),
                                "seconds": tuned["seconds"]}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w, head["n_candidates"], args.cpu_queries)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def link_bandwidth(host_pts, host_out, dev):
    """Host-link copy rates with the step's own pinned buffers: the points
    host to device, the first 256 MB of the result buffer device to host."""
    import torch
    d_pts = torch.empty_like(host_pts, device=dev)
    nb = min(host_out.numel() * 4, 256 << 20) // 4
    h_out = host_out.view(-1)[:nb]
    d_out = torch.empty(nb, dtype=torch.int32, device=dev)
    out = {}
    for name, dst, src, nbytes in (("h2d_gbs", d_pts, host_pts, host_pts.numel() * 8),
                                   ("d2h_gbs", h_out, d_out, nb * 4)):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(5):
            dst.copy_(src, non_blocking=True)
        b.record()
        torch.cuda.synchronize(dev)
        out[name] = round(5 * nbytes / (a.elapsed_time(b) * 1e-3) / 1e9, 1)
    return out


def kernel_source_sha(kname):
    """Short hash of the sources of a distance kernel (its file and the shared
    tile header), to tie committed counters to the code they were taken on."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2209_11287_gb300", "csrc")
    main = {"fp64_dmma": "sj_join_dmma.cu", "filter_bf16x3": "sj_join_tc.cu", "filter_bf16x2": "sj_join_tc.cu",
            "filter_fp16x2": "sj_join_tc.cu", "filter_f32": "sj_join_f32s.cu"}.get(kname, "sj_join_cc.cuh")
    files = [main, "sj_join_common.cuh"]
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def read_traffic(kname, workload="uniform4d"):
    """DRAM bytes per launch of the distance kernel from the committed ncu
    summary (a line 'dram_bytes_per_launch: <int>' and 'kernel_source_sha:
    <sha>'), or None when absent or taken on different kernel sources."""
    path = os.path.join(ROOT, "profiles", f"join_{kname}_{workload}.txt")
    if not os.path.exists(path):
        return None
    sha = kernel_source_sha(kname)
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha") != sha:
        return None
    try:
        return int(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def roofline(kname, w, r, kern_ms):
    """Roofline of one distance-tile kernel launch.  Arithmetic: d fused
    multiply-adds (2d flop) per evaluated (query, candidate) pair, in FP32 for
    the CUDA-core filter (peak from the SM count, FP32 lanes and maximum
    clock) and in FP64 for the plain kernels (peaks of the committed
    micro-benchmark, profiles/fp64_peaks_gb300.txt); for the tensor-core
    filter 2 K flop per evaluated pair (K the padded split-row length, 6
    products per dim plus the norm slots) against the measured burst bf16
    peak (K = 6 dp + 3 for BF16x3, 3 dp + 3 for BF16x2, padded to 16).  Bytes:
    every packed point read once (coordinates, norm, two thresholds, input
    index) plus 8 bytes per emitted pair, against the measured HBM copy
    bandwidth.  The larger fraction is the binding one."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    elt = 4 if kname.startswith("filter") else 8
    dp = 2
    while dp < w.d:
        dp *= 2
    if kname in ("filter_bf16x3", "filter_bf16x2", "filter_fp16x2"):
        kp = ((6 if kname == "filter_bf16x3" else 3) * dp + 3 + 15) // 16 * 16
        flops = 2.0 * kp * r["n_evaluated"]
        # (fp16 and bf16 have the same dense tensor rate: the bf16 peak serves both)
        fp_peak, unit_bound = float(peaks.get("bf16_tflops", 1900.0)), "tensor"
        fp_source = ("MEASURED_PEAKS.json bf16_tflops (cuBLAS bf16 burst, measured on this pool)"
                     if "bf16_tflops" in peaks else "fallback 1900 TFLOP/s bf16")
    else:
        flops = 2.0 * w.d * r["n_evaluated"]
        fp_peak = {"fp64_fma": FP64_DFMA_TFLOPS, "fp64_dmma": FP64_DMMA_TFLOPS}.get(kname, FP32_FMA_PEAK_TFLOPS)
        fp_source = ("profiles/fp64_peaks_gb300.txt (this repository's FP64 micro-benchmark)"
                     if kname in ("fp64_fma", "fp64_dmma", "fp64_fma_sc") else
                     "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (formula)")
        unit_bound = "alu"
    tfl = flops / (kern_ms * 1e-3) / 1e12
    bytes_alg = w.n * (elt * (dp + 3) + 4) + 8 * r["count"]
    gbs = bytes_alg / (kern_ms * 1e-3) / 1e9
    frac_alu, frac_hbm = tfl / fp_peak, gbs / hbm_peak
    hbm_source = ("MEASURED_PEAKS.json hbm_gbs (copy bandwidth, measured on this pool)" if "hbm_gbs" in peaks
                  else "fallback 6800 GB/s")
    # flop convention: d fused multiply-adds (2 d flop) per evaluated pair
    common = {"traffic": read_traffic(kname, w.name), "kernel": KERNEL_NAMES.get(kname, kname),
              "kernel_ms": round(kern_ms, 4), "flop_per_launch": flops, "bytes_per_launch": bytes_alg}
    if frac_alu >= frac_hbm:
        return {"bound": unit_bound, "achieved": round(tfl, 3), "peak": round(fp_peak, 3), "unit": "TFLOP/s",
                "frac": round(frac_alu, 4), "peak_source": fp_source, "hbm_frac": round(frac_hbm, 4), **common}
    return {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(frac_hbm, 4), "peak_source": hbm_source, "alu_frac": round(frac_alu, 4),
            "alu_peak_source": fp_source, **common}


def make_line(args, w, results, variants, world, kern_ms, e2e_s, head):
    kname = variants[0]
    cand = head["n_candidates"]
    # every rank runs a shard of the same join: the whole join's candidates
    # over the slowest rank's step time (strong scaling)
    value = cand / (head["ms_per_step"] * 1e-3)
    roof = roofline(head.get("kernel", kname), w, head, kern_ms)
    var = {}
    for k in variants:
        r = results[k]
        rk = roofline(r.get("kernel", k), w, r, r["tile_ms"])
        var[k] = {"ms_per_step": round(r["ms_per_step"], 4),
                  "candidate_pairs_per_s": r["n_candidates"] / (r["ms_per_step"] * 1e-3),
                  "result_pairs_per_s": r["count"] / (r["ms_per_step"] * 1e-3), "result_pairs": r["count"],
                  "evaluated_pairs": r["n_evaluated"], "rechecked_pairs": r["n_rechecked"], "reruns": r["reruns"],
                  "tile_kernel_ms": round(r["tile_ms"], 4), "kernel": r.get("kernel", k),
                  "tile_roofline": {key: rk[key] for key in ("bound", "achieved", "peak", "unit", "frac",
                                                             "peak_source")}}
    e2e_val = cand / e2e_s
    line = {
        "metric": METRICS[args.workload], "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(head["ms_per_step"], 4), "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": DTYPES.get(kname, "f64"), "data": "synthetic",
        "config": workload_config(w, {"kernel": kname, "symmetric": 1, "parallelism": f"work-item shards x{world}" if world > 1 else "1 GPU",
                                      "l2": "flushed between steps (256 MB write)",
                                      "candidate_pairs": cand, "result_pairs": head["count"]}),
        "variants": var,
        "roofline": roof,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": world * w.n * w.d * 8,
                "d2h_bytes_per_step": head["count"] * 8, "ms_per_step": round(e2e_s * 1e3, 3)},
        "gpu_launches": int(head["launches"]),
        "clocks": results[variants[-1]]["clocks"],
    }
    return line


# ---- CPU oracle ----------------------------------------------------------------------

def cpu_baseline(w, n_candidates, n_queries=0):
    """The oracle (brute force, every query against all n points) on the host
    cores for a sample of queries, scaled to the whole workload."""
    import oracle
    oracle.build()
    cores = oracle.threads(0)
    rng = np.random.Generator(np.random.PCG64(4242))
    if n_queries <= 0:
        # size the sample for ~15 s: probe with a small one first
        probe = np.sort(rng.choice(w.n, size=max(64, 4 * cores), replace=False))
        t0 = time.perf_counter()
        oracle.rows(w.points, w.eps, probe)
        dt = time.perf_counter() - t0
        n_queries = int(min(w.n, max(probe.size, probe.size * 15.0 / max(dt, 1e-3))))
    sample = np.sort(rng.choice(w.n, size=n_queries, replace=False))
    t0 = time.perf_counter()
    oracle.rows(w.points, w.eps, sample)
    dt = time.perf_counter() - t0
    full_s = dt * w.n / n_queries
    return {"value": n_candidates / full_s, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_queries} of {w.n} queries, each against all {w.n} points, scaled by n / sample",
            "sample_seconds": round(dt, 2), "full_join_seconds_est": round(full_s, 1)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    if args.workload != "uniform4d":
        print(json.dumps({"impl": "reference", "unavailable": "the CPU oracle arm is defined for the uniform4d "
                          "headline workload only (its canonical 3^d grid candidate count)"}), flush=True)
        return
    from paper_2209_11287_gb300 import workloads
    import oracle
    oracle.build()
    w = make_workload(args)
    cand = canonical_candidates_host(w)
    cores = oracle.threads(0)
    rng = np.random.Generator(np.random.PCG64(99))
    # per step: a bounded sample of queries sized so all steps end in a few minutes
    per_step = max(64, int(args.cpu_queries) if args.cpu_queries else 2000)
    times = []
    for k in range(args.warmup + args.steps):
        sample = np.sort(rng.choice(w.n, size=per_step, replace=False))
        t0 = time.perf_counter()
        oracle.rows(w.points, w.eps, sample)
        dt = (time.perf_counter() - t0) * w.n / per_step
        if k >= args.warmup:
            times.append(dt)
    s = statistics.mean(times)
    value = cand / s
    line = {"metric": METRICS[args.workload], "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": s * 1e3, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(w, {"kernel": "oracle brute force (CPU)"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} of {w.n} queries per step against all points, scaled by n / sample"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- batched workload ------------------------------------------------------------------

BATCH_METRIC = ("batched self-joins: brute-force pair equivalents/s (sum of n_i^2 / step time) and join time, 4096 "
                "instances, n log-uniform [256, 65536], d in {2,4,8,16,32}")
BATCH_UNIT = "pair equivalents/s"


def batch_config(count, total_n, extra=None):
    cfg = {"workload": f"batched: {count} independent self-joins, instance i drawn from PCG64(i): n = "
                       f"floor(exp(U[ln 256, ln 65536])), d uniform over {{2,4,8,16,32}}, points uniform in "
                       f"[0,1]^d, per-instance eps for a mean of 32 neighbours; {total_n} points in all",
           "instances": count, "points": total_n}
    if extra:
        cfg.update(extra)
    return cfg


def run_batched(args):
    """One step = sj_join_batch over all instances (segmented index builds,
    one distance-tile launch per dimension group, results in device pages)
    until every instance's count is known; results are released after the
    step."""
    from paper_2209_11287_gb300 import workloads
    rank, world, local = dist_env()
    sizes = [workloads.batch_instance_params(i)[0] for i in range(args.batch_count)]
    total_n = sum(sizes)
    nsq = float(sum(n * n for n in sizes))  # the grid-independent unit of work of the whole batch
    # several ranks: each joins a contiguous range of instances of about equal
    # sum of n^2 (the batch shards by instance, no data-path exchange)
    i0, i1 = (0, args.batch_count) if world == 1 else instance_shard(sizes, rank, world)
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps({"impl": "reference", "unavailable": "the CPU oracle arm is defined for the uniform4d "
                          "headline workload only (its canonical grid candidate count); batched runs report the "
                          "oracle in cpu_baseline of the native line"}), flush=True)
        return

    import torch
    from paper_2209_11287_gb300 import binding, build
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    binding.load()
    insts = [workloads.batch_instance(i) for i in range(i0, i1)]
    eps = [w.eps for w in insts]
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    pts = [torch.from_numpy(w.points).to(dev) for w in insts]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def sync_all():
        torch.cuda.synchronize(dev)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    dims = [w.d for w in insts]
    knames = {v: k for k, v in binding.KERNELS.items()}

    dp_of = np.array([1 << max(1, (dd - 1).bit_length()) for dd in dims])
    dims_np = np.array(dims, dtype=np.float64)
    prepared = binding.BatchInputs(pts, eps)  # pointer arrays marshalled once

    def one_step(opt, inputs, host_out=None):
        res = binding.sj_join_batch_raw(inputs, opt, stream)
        if host_out is not None:
            for r in res:
                binding.sj_result_copy(r, host_out[: int(r.count)])
        t = binding.results_table(res)
        groups = {}  # padded dim -> tile time, kernel, evaluated pairs and 2 d per pair
        for dp in np.unique(dp_of):
            sel = dp_of == dp
            first = int(np.argmax(sel))
            ev = t["n_evaluated"][sel]
            groups[int(dp)] = {"ms": float(t["ms_tile"][first]), "kernel": knames.get(int(t["kernel"][first]), "?"),
                               "evaluated": int(ev.sum()), "flops_2d": float((2.0 * dims_np[sel] * ev).sum()),
                               "instances": int(sel.sum()), "points": int(sum(len(pts[i]) for i in np.nonzero(sel)[0]))}
        out = (int(t["count"].sum()), int(t["n_candidates"].sum()), int(t["n_evaluated"].sum()),
               int(t["reruns"].max()), sum(g["ms"] for g in groups.values()), groups, int(t["count"].max()))
        binding.sj_results_free(res)
        return out

    # variants: a kernel name; "tuned" = AUTO with the tuning cache the
    # autotuner writes before the variant's warm-up (untimed); "*_graph" = the
    # join phase as one CUDA graph
    allowed = ("tuned_graph", "tuned", "auto_graph", "auto", "filter_f32", "filter_bf16x3", "filter_bf16x2", "filter_fp16x2",
               "fp64_fma")
    asked = (args.variants.split(",") if args.variants != ",".join(VARIANTS)
             else ["tuned_graph", "tuned", "auto", "filter_f32", "fp64_fma"])
    variants = [v for v in asked if v in allowed] or ["auto"]
    tune_dir = tempfile.mkdtemp(prefix="sj_tune_")
    tune_path = os.path.join(tune_dir, "batch.txt")
    tuned = {}

    def make_opt(kname):
        cache = tune_path if kname.startswith("tuned") else None
        if cache and not tuned:
            t0 = time.perf_counter()
            tuned["groups"] = binding.sj_autotune_batch(
                prepared, binding.sj_default_options(max_pairs_hint=args.hint), stream, reps=1, cache_path=cache)
            tuned["seconds"] = round(time.perf_counter() - t0, 1)
        base = kname.replace("tuned", "auto").replace("_graph", "")
        return binding.sj_default_options(kernel=base, max_pairs_hint=args.hint, graph=int(kname.endswith("_graph")),
                                          tune_cache=cache)

    sampler = ClockSampler(local)
    results = {}
    sampler.start()  # before the first warm-up, so its start-up is not timed
    time.sleep(1.0)
    for vi, kname in enumerate(variants):
        opt = make_opt(kname)
        for _ in range(args.warmup):
            one_step(opt, prepared)
        sync_all()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        l0 = binding.sj_kernel_launches()
        tiles = []
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            info = one_step(opt, prepared)
            ev[k][1].record(stream)
            tiles.append(info[4])
        sync_all()
        launches = (binding.sj_kernel_launches() - l0) // args.steps
        clocks = sampler.stop() if vi == len(variants) - 1 else None
        times = [a.elapsed_time(b) for a, b in ev]
        # the whole batch: the slowest rank's time, the sums of the ranks' counts
        count, n_cand, n_eval = gather_sums(info[:3], world, dev)
        results[kname] = {"ms_per_step": max_over_ranks(statistics.mean(times), world, dev), "count": count,
                          "n_candidates": n_cand, "n_evaluated": n_eval, "reruns": info[3],
                          "tile_ms": max_over_ranks(statistics.mean(tiles), world, dev),
                          "groups": info[5], "max_count": info[6], "launches": launches, "clocks": clocks,
                          "local_count": info[0]}
    head = results[variants[0]]
    # end to end: host inputs (pinned), every instance's pairs copied back to pinned host memory
    host_pts = binding.BatchInputs([torch.from_numpy(w.points).pin_memory() for w in insts], eps)
    host_out = torch.empty((head["max_count"] + 16, 2), dtype=torch.int32).pin_memory()
    sync_all()
    opt = make_opt(variants[0])
    t_e2e = []
    for k in range(max(2, min(args.steps, 4))):
        flush.fill_(float(k))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        one_step(opt, host_pts, host_out)
        torch.cuda.synchronize(dev)
        t_e2e.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(statistics.mean(t_e2e), world, dev)
    shutil.rmtree(tune_dir, ignore_errors=True)
    if rank != 0:
        return
    var = {}
    for k in variants:
        r = results[k]
        var[k] = {"ms_per_step": round(r["ms_per_step"], 3),
                  "pair_equivalents_per_s": nsq / (r["ms_per_step"] * 1e-3),
                  "candidate_pairs": r["n_candidates"],
                  "instances_per_s": args.batch_count / (r["ms_per_step"] * 1e-3),
                  "result_pairs": r["count"], "evaluated_pairs": r["n_evaluated"], "reruns": r["reruns"],
                  "tile_kernel_ms": round(r["tile_ms"], 3), "launches_per_step": r["launches"],
                  "groups": batch_rooflines(r)}
    line = {"metric": BATCH_METRIC, "value": nsq / (head["ms_per_step"] * 1e-3),
            "unit": BATCH_UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(head["ms_per_step"], 3), "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": DTYPES.get(variants[0], "f64"),
            "data": "synthetic",
            "config": batch_config(args.batch_count, total_n, {"kernel": variants[0], "symmetric": 1,
                                                          "parallelism": "1 GPU" if world == 1 else
                                                          f"instance shards x{world} (equal sum of n^2)",
                                                          "l2": "inputs (4.7 GB) larger than L2; 256 MB flush too",
                                                          "candidate_pairs": head["n_candidates"],
                                                          "result_pairs": head["count"]}),
            "variants": var,
            "autotune": None if not tuned else {
                "seconds": tuned["seconds"],
                "groups": {str(g["dp"]): {"kernel": knames.get(g["kernel"], "?"), "queries_per_item": g["qpi"],
                                          "tile_ms": round(g["ms"], 3)} for g in tuned["groups"]}},
            "e2e": {"value": nsq / e2e_s, "unit": BATCH_UNIT,
                    "h2d_bytes_per_step": sum(n * workloads.batch_instance_params(i)[1] * 8
                                              for i, n in enumerate(sizes)),
                    "d2h_bytes_per_step": head["count"] * 8, "ms_per_step": round(e2e_s * 1e3, 1)},
            "roofline": max(batch_rooflines(head).values(), key=lambda g: g["kernel_ms"]),
            "cpu_baseline": None if (args.no_cpu_baseline or world > 1) else batch_cpu_baseline(insts, nsq),
            "gpu_launches": int(head["launches"]),
            "clocks": results[variants[-1]]["clocks"]}
    print(json.dumps(line), flush=True)


def batch_cpu_baseline(insts, nsq):
    """The oracle (brute force, every sampled query against all points of its
    instance) on the host cores for sampled queries of sampled instances,
    scaled by n / sample per instance and by instances / sampled instances."""
    import oracle
    oracle.build()
    cores = oracle.threads(0)
    rng = np.random.Generator(np.random.PCG64(77))
    pick = rng.choice(len(insts), size=64, replace=False)

    def run(q_per_inst):
        est, t_all = 0.0, 0.0
        for i in pick:
            w = insts[i]
            q = np.sort(rng.choice(w.n, size=min(q_per_inst, w.n), replace=False))
            t0 = time.perf_counter()
            oracle.rows(w.points, w.eps, q)
            dt = time.perf_counter() - t0
            t_all += dt
            est += dt * w.n / q.size
        return est * len(insts) / len(pick), t_all

    _, probe = run(16)
    qpi = int(max(16, min(4096, 16 * 10.0 / max(probe, 1e-3))))  # ~10 s of oracle work
    full_s, spent = run(qpi)
    return {"value": nsq / full_s, "unit": BATCH_UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{qpi} queries of each of 64 sampled instances (seeded), each against all points of its "
                      f"instance, scaled by n / sample and 4096 / 64",
            "sample_seconds": round(spent, 2), "full_batch_seconds_est": round(full_s, 1)}


def batch_rooflines(r):
    """Roofline of each dimension group's distance-tile launch (event-timed by
    the library): the tensor-core filter against the measured sustained bf16
    peak with 2 K flop per evaluated pair (K the padded split-row length,
    6 products per dim plus the norm slots); the FP32 filter and the FP64
    kernel with 2 d flop per evaluated pair against the FP32 peak and the
    measured DFMA peak."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    bf16 = float(peaks.get("bf16_tflops_sustained", 1700.0))
    out = {}
    for dp, g in sorted(r["groups"].items()):
        sec = max(g["ms"], 1e-6) * 1e-3
        if g["kernel"] in ("filter_bf16x3", "filter_bf16x2", "filter_fp16x2"):
            kp = ((6 if g["kernel"] == "filter_bf16x3" else 3) * dp + 3 + 15) // 16 * 16
            flops, peak, kern = 2.0 * kp * g["evaluated"], bf16, "k_join_tc<" + g["kernel"][7:] + ">"
            bound = "tensor"
            source = ("MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS bf16 under the power cap, measured on "
                      "this pool)" if "bf16_tflops_sustained" in peaks else "fallback 1700 TFLOP/s bf16")
        else:
            flops = g["flops_2d"]
            peak = FP64_DFMA_TFLOPS if g["kernel"] == "fp64_fma" else FP32_FMA_PEAK_TFLOPS
            kern, bound = KERNEL_NAMES.get(g["kernel"], g["kernel"]), "alu"
            source = ("profiles/fp64_peaks_gb300.txt (this repository's FP64 micro-benchmark)"
                      if g["kernel"] == "fp64_fma" else "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (formula)")
        tfl = flops / sec / 1e12
        out[f"d{dp}"] = {"bound": bound, "achieved": round(tfl, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
                         "frac": round(tfl / peak, 4), "peak_source": source, "traffic": None, "kernel": kern,
                         "kernel_ms": round(g["ms"], 3), "instances": g["instances"],
                         "evaluated_pairs": g["evaluated"]}
    return out


def canonical_candidates_host(w):
    """Candidate pairs of the full 3^d neighbourhoods on the grid of side
    eps (1 + 2^-20), counted with the oracle's grid helper."""
    import oracle
    return oracle.grid_candidate_count_fast(w.points, w.eps * (1.0 + 2.0 ** -20))


def main():
    args = parse()
    if args.workload == "batched":
        run_batched(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
