"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): every rank
runs an independent replica, timing is the maximum over ranks, and no
collective touches the data path.  Runs without a GPU."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        # each replica "measures" a different time; the job time is the slowest
        t = bench.allmax(world, 10.0 + 5.0 * rank, device="cpu")
        # replicas use different seeds: the workloads differ, the sizes do not
        c0 = bench.workload("cbl128", seed=1 + rank)
        q.put((rank, t, c0.seed, c0.n))
    finally:
        dist.destroy_process_group()


def test_two_replicas_on_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][2] != res[1][2] and res[0][3] == res[1][3]
