"""The multi-process path of the bench on CPU: two ranks over gloo.

The nodal solve has no exchange step (maps and batches are independent), so `--gpus N` runs N
replicas; the only cross-rank operations are a barrier around the timed region and max/sum
reductions of timing scalars, from which rank 0 reports the whole job's throughput (all ranks'
solves over the slowest rank's time).  Those operations are checked here with world size 2 on
gloo, as two spawned processes rendezvousing on 127.0.0.1.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    d = bench.Dist(backend="gloo")
    try:
        d.barrier()
        mx = d.max(float(rank + 1))
        sm = d.sum(10.0 * (rank + 1))
        # replicas: rank r solves 100 vectors in its own time; the job's value is total / slowest
        t_rank = (0.5, 0.8)[rank]
        value = d.sum(100.0) / d.max(t_rank)
        d.barrier()
        q.put((rank, d.world, mx, sm, value))
    finally:
        d.close()


def test_replica_reductions_two_ranks_gloo():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [p.exitcode for p in procs] == [0, 0]
    assert [r[0] for r in res] == [0, 1]
    for _, world, mx, sm, value in res:
        assert world == 2
        assert mx == 2.0 and sm == 30.0
        assert value == pytest.approx(200.0 / 0.8)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    env = {k: os.environ.get(k) for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    for k in env:
        os.environ.pop(k, None)
    try:
        d = bench.Dist(backend="gloo")
        assert d.world == 1 and d.pg is None
        assert d.max(3.5) == 3.5 and d.sum(2.0) == 2.0
        d.barrier()
        d.close()
    finally:
        for k, v in env.items():
            if v is not None:
                os.environ[k] = v
