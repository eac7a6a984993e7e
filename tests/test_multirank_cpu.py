"""The multi-process path of bench.py on CPU: two gloo ranks, launched the
way torchrun launches the bench (RANK / WORLD_SIZE / LOCAL_RANK and a
127.0.0.1 rendezvous), agree on the slowest rank's time, partition the work
items of one join into contiguous shards of equal work (the library's host
side partition, no GPU needed) and gather their result counts, the one
exchange of a sharded join (Sec. III-B: the work items are independent)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    slowest = bench.max_over_ranks(1.5 + rank, w, torch.device("cpu"))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, r, w, local, slowest))


def test_two_gloo_ranks_agree_on_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[:4] for o in out] == [(0, 0, 2, 0), (1, 1, 2, 1)]
    assert all(o[4] == 2.5 for o in out)  # max(1.5, 2.5) on every rank


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1, torch.device("cpu")) == 3.25


def _shard_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # the per-item work of an index: every rank holds the same array (the
    # build is deterministic); heavy-tailed like dense cells
    g = np.random.Generator(np.random.PCG64(77))
    work = (g.pareto(1.5, size=50000) * 1000).astype(np.int64) + 1
    work[g.random(50000) < 0.2] = 0  # items that continue their cell
    i0, i1 = bench.shard_of(work, rank, world)
    mine = int(work[i0:i1].sum())
    counts = bench.gather_counts(mine, world, torch.device("cpu"))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, i0, i1, mine, counts, int(work.sum()), int(work.max()), i0 == 50000 or work[i0] > 0))


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_shard_the_items_and_gather_counts(world):
    from paper_2209_11287_gb300 import binding, build
    build.build()
    binding.load()
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    total, wmax = out[0][5], out[0][6]
    # contiguous, disjoint, covering [0, n_items)
    assert out[0][1] == 0 and out[-1][2] == 50000
    assert all(out[k][2] == out[k + 1][1] for k in range(world - 1))
    # balanced to within one item's work of an equal share, never starting
    # inside a cell (an item of no work)
    assert all(abs(o[3] - total / world) <= wmax for o in out)
    assert all(o[7] for o in out)
    # every rank gathered the same counts, rank order, summing to the whole
    for o in out:
        assert o[4] == [x[3] for x in out]
        assert sum(o[4]) == total


def _batch_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from paper_2209_11287_gb300 import workloads
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = [workloads.batch_instance_params(i)[0] for i in range(4096)]
    i0, i1 = bench.instance_shard(sizes, rank, world)
    mine = sum(n * n for n in sizes[i0:i1])
    sums = bench.gather_sums([i1 - i0, mine], world, torch.device("cpu"))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, i0, i1, mine, sums))


@pytest.mark.parametrize("world", [2, 3])
def test_batch_shards_by_instance(world):
    """The batched workload on several ranks: contiguous ranges of instances
    covering the batch once, of about equal sum of n^2, the same partition on
    every rank, and the ranks' counts summed by the one exchange."""
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    from paper_2209_11287_gb300 import workloads
    sizes = [workloads.batch_instance_params(i)[0] for i in range(4096)]
    total = sum(n * n for n in sizes)
    biggest = max(n * n for n in sizes)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batch_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][1] == 0 and out[-1][2] == 4096
    for a, b in zip(out, out[1:]):
        assert a[2] == b[1]  # contiguous, disjoint
    for o in out:
        assert abs(o[3] - total / world) <= biggest  # balanced to within one instance
        assert o[4] == [4096, total]  # every rank holds the sums
