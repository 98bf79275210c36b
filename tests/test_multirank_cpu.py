"""The multi-GPU bench path's host logic on CPU: two gloo ranks (one process each) reduce
their timed regions to the slowest rank, count the whole job's samples, and draw
independent chain seeds.  Replicas only: there is no data-path collective to test."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    ms = bench.max_over_ranks(100.0 + 50.0 * rank, device="cpu")
    out.put((r, ws, ms, bench.job_throughput(1000, ws, ms), bench.rank_seed(7, r)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, *_ in res] == [0, 1]
    assert all(ws == 2 for _, ws, *_ in res)
    assert all(ms == 150.0 for _, _, ms, *_ in res)          # max over ranks
    assert all(abs(v - 2 * 1000 / 0.150) < 1e-6 for *_, v, _ in res)   # whole-job samples/s
    assert res[0][4] != res[1][4]                             # independent chains per rank


def test_single_process_is_unchanged():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, device="cpu") == 42.0
    assert bench.job_throughput(8192, 1, 1000.0) == 8192.0
