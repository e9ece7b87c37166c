"""The multi-rank bookkeeping of bench.py on CPU: two gloo ranks, each timing
its own replica; the job is timed by the slowest rank and its throughput counts
both replicas."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    ms = 10.0 + 5.0 * rank                        # rank 1 is the slower one
    m = bench.max_over_ranks(ms, dist, device="cpu")
    out.put((r, w, m, bench.whole_job_mlups(1000, 20, w, m), bench.THETA_SWEEP[r % len(bench.THETA_SWEEP)]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[2] == 15.0 for r in res)                           # max over ranks
    assert all(r[3] == pytest.approx(1000 * 20 * 2 / 15e-3 / 1e6) for r in res)
    assert res[0][4] != res[1][4]                                   # each replica its own angle


def test_single_process_is_its_own_max():
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.whole_job_mlups(100, 10, 1, 1.0) == pytest.approx(1.0)
