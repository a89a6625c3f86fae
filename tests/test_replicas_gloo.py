"""Multi-rank host logic of the replica mode, on CPU with the gloo backend (world size 2)."""
import math
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1104_4263_gb300 import replicas  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        units = 100.0 * (rank + 1)          # ranks did different amounts of work
        secs = 1.0 + rank                   # and took different times
        total, tmax = replicas.combine(units, secs, dist)
        thr = replicas.throughput(units, secs, dist)
        out.put((rank, total, tmax, thr, replicas.angle_for_rank(rank)))
    finally:
        dist.destroy_process_group()


def test_combine_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, tmax, thr, psi in res:
        assert total == 300.0 and tmax == 2.0 and thr == 150.0
        assert psi == pytest.approx(2 * math.pi * rank / 8)
    assert res[0][4] != res[1][4]          # each rank solves its own incidence angle


def test_single_process_is_identity():
    assert replicas.combine(7.0, 2.0) == (7.0, 2.0)
    assert replicas.throughput(10.0, 4.0) == 2.5
    assert replicas.angle_for_rank(9) == replicas.angle_for_rank(1)
