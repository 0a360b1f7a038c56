"""Multi-rank host logic on CPU: two gloo ranks shard a scan, reduce the step
time and gather per-pair results; a rank that fails is seen by the other."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1907_05993_gb300.shard import gather_results, max_over_ranks, shard_range


def test_shard_ranges_partition_the_scan():
    for n in (0, 1, 7, 10_000, 10_001):
        for world in (1, 2, 3, 8):
            rs = [shard_range(n, r, world) for r in range(world)]
            assert [i for r in rs for i in r] == list(range(n))
            assert max(map(len, rs)) - min(map(len, rs)) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n_total, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    shard = shard_range(n_total, rank, world)
    # stand-in per-pair results: the pair index in F[.., 0], a status bit
    F = torch.zeros((len(shard), 9), dtype=torch.float64)
    F[:, 0] = torch.tensor(list(shard), dtype=torch.float64)
    st = torch.full((len(shard),), rank, dtype=torch.int32)
    t = max_over_ranks(1.5 + rank)
    res = gather_results({"F": F, "status": st}, n_total)
    if rank == 0:
        q.put((t, res["F"][:, 0].tolist(), res["status"].tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    n = 11
    port = _port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n, q)) for r in range(2)]
    for p in procs:
        p.start()
    t, idx, st = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert t == 2.5
    assert idx == list(range(n))
    assert st == [0] * 6 + [1] * 5


def _failing_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import datetime
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        raise SystemExit(3)   # this rank leaves between steps, before the collective
    try:
        max_over_ranks(1.0)
        q.put("no error")
    except Exception as e:   # the survivor learns of it through the failed collective
        q.put(type(e).__name__)


def test_a_failed_rank_is_detected_by_the_other():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    msg = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert msg != "no error"
    assert procs[1].exitcode == 3
