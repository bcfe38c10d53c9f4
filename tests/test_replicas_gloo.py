"""The N-rank (replicas) host logic on CPU ranks: world_size 2, gloo.

Each rank reports its own step time; the job's time is the slowest rank's
(MAX all-reduce) and its throughput is all ranks' units over that time.
"""
import os

import pytest

torch = pytest.importorskip("torch")


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1505_04650_gb300 import replicas
    w, rk, lr = replicas.world()
    ms = 10.0 + 5.0 * rank                     # rank 1 is the slower one
    dist.barrier()
    slow = replicas.slowest_ms(ms)
    rate = replicas.job_rate(3, slow, w)
    out.put((rk, lr, w, slow, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_gloo():
    import socket
    mp = torch.multiprocessing.get_context("spawn")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = mp.Queue()
    procs = [mp.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (rk, lr, w, slow, rate) in enumerate(res):
        assert (rk, lr, w) == (rank, rank, 2)
        assert slow == 15.0                     # the slowest rank's time
        assert rate == pytest.approx(2 * 3 * 1000.0 / 15.0)


def test_single_process_passthrough():
    from paper_1505_04650_gb300 import replicas
    assert replicas.slowest_ms(7.5) == 7.5
    assert replicas.job_rate(1, 12.5, 1) == pytest.approx(80.0)
