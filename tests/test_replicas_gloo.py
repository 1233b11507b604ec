"""Multi-rank host logic on CPU: two gloo ranks (world_size 2) exchange their
timings through replicas.max_over_ranks and get the element-wise maximum;
their refinement schedules are independent (replicas only, no data-path
collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    from paper_2108_07205_gb300 import replicas, inputs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = replicas.rank_info()
        replicas.barrier()
        mx = replicas.max_over_ranks([10.0 * (r + 1), 5.0 - r])
        sched = inputs.time_schedule(replicas.schedule_seed(r), 1024, 3)
        q.put((r, w, mx, sched[0][0][0]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for r, w, mx, _ in res:
        assert w == 2 and mx == [20.0, 5.0]
    from paper_2108_07205_gb300 import replicas
    assert replicas.schedule_seed(0) != replicas.schedule_seed(1)
