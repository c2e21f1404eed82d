"""Multi-rank host logic on CPU (gloo, world size 2): sample sharding and the
whole-job throughput reduction the benchmark uses for N > 1."""
import os
import socket

import pytest

from paper_1804_02418_gb300 import parallel, workloads as W


def test_sharding_is_a_balanced_partition():
    samples = W.ensemble(37, w_lo=16, w_hi=64)
    sites = [s.sites for s in samples]
    for world in (1, 2, 3, 8):
        parts = [parallel.shard_samples(sites, r, world) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(samples)))
        loads = [sum(sites[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sites)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r processed 100 (r + 1) units in 2 (r + 1) seconds
        thr = parallel.job_throughput(100.0 * (rank + 1), 2.0 * (rank + 1))
        mx = parallel.max_over_ranks(float(rank))
        sites = [s.sites for s in W.ensemble(11, w_lo=16, w_hi=64)]
        mine = parallel.shard_samples(sites, rank, world)
        total = parallel.sum_over_ranks(float(len(mine)))
        out.put((rank, thr, mx, total))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_reduce_like_the_benchmark():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, thr, mx, total in res:
        assert thr == pytest.approx(300.0 / 4.0)     # (100 + 200) units over max(2, 4) s
        assert mx == 1.0
        assert total == 11.0
