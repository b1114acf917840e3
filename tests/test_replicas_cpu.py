"""The N>1 layout (independent replicas) on CPU ranks: gloo, world size 2.

Checks the pieces that bench.py and a served mix use across ranks: the round-robin
shard of independent units partitions the list, the timed region's duration is the
maximum over ranks, and the whole-job rate counts every rank's units."""
import os
import socket

import pytest

from paper_2301_05844_gb300 import replicas as R


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, lr, w = R.rank_info()
        mine = R.shard(list(range(11)), r, w)
        dur = 1.0 + 0.5 * r  # rank 1 is the slowest
        dist.barrier()
        slowest = R.max_over_ranks(dur)
        rate = R.whole_job_rate(7, w, slowest)
        gathered = [None] * w
        dist.all_gather_object(gathered, mine)
        q.put((r, lr, w, slowest, rate, gathered))
    finally:
        dist.destroy_process_group()


def test_replicas_on_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, lr, w, slowest, rate, gathered in out:
        assert w == 2 and lr == r
        assert slowest == 1.5
        assert rate == pytest.approx(7 * 2 / 1.5)
        flat = sorted(x for part in gathered for x in part)
        assert flat == list(range(11))
        assert not set(gathered[0]) & set(gathered[1])


def test_single_process_defaults():
    assert R.max_over_ranks(2.5) == 2.5
    assert R.shard([1, 2, 3], 0, 1) == [1, 2, 3]
    with pytest.raises(ValueError):
        R.shard([1], 2, 2)
    with pytest.raises(ValueError):
        R.whole_job_rate(1, 1, 0.0)
