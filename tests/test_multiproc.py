"""The multi-process path of bench.py on CPU (gloo, world size 2): each rank runs its own
replica; the job's time is the slowest rank's, and the throughput counts every rank's solve."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, times, out):
    import torch.distributed as tdist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, _ = bench.dist()
    t = bench.job_seconds(times[rank], w, device="cpu")
    tdist.barrier()
    out.put((r, w, t, bench.replica_throughput(t, w)))
    tdist.destroy_process_group()


def test_two_rank_replicas_time_is_max_over_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [0.25, 0.40]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, *_ in res] == [0, 1]
    for _, w, t, thr in res:
        assert w == 2
        assert t == pytest.approx(0.40)            # the slowest rank
        assert thr == pytest.approx(2 / 0.40)      # both replicas' solves


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_seconds(0.3, 1) == 0.3
    assert bench.replica_throughput(0.5, 1) == 2.0
