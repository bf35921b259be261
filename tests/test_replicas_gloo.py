"""The multi-GPU path of bench.py runs independent replicas (one box per rank, no
collective on the data path): its host logic -- the whole-job time is the slowest rank's,
the throughput counts every rank's units, the reference arm runs on rank 0 only -- on
two gloo ranks over 127.0.0.1, no GPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, ms_by_rank, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench.dist_setup() == (ws, rank, rank)
    ms = bench.job_ms(ms_by_rank[rank], ws, "cpu")
    out.put((rank, ms, bench.job_value(1000, ws, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ms_by_rank = [2.0, 3.5]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, ms_by_rank, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [3.5, 3.5]
    assert all(r[2] == pytest.approx(2 * 1000 / 3.5e-3) for r in res)


def test_reference_arm_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup = 1, 0

    assert bench.run_reference(A(), 2, 1) == 0
    assert capsys.readouterr().out == ""
