"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

The workload shards into independent replicas (frequencies, right-hand sides,
meshes); the only collectives are the start barrier and the max over ranks of
the timed region, which this test exercises with the gloo backend.
"""

import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r = bench._dist()
    assert (ws, r) == (world, rank)
    dist.barrier()
    t = bench._barrier_max(10.0 * (rank + 1), ws, device="cpu")
    q.put((rank, t))
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=10) for _ in range(2))
    assert res == {0: 20.0, 1: 20.0}


def test_reference_arm_other_ranks_exit(monkeypatch, capsys):
    """Under torchrun only rank 0 runs the reference arm; other ranks return without work."""
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup, workload, cpu_rows = 1, 3, "pec_sphere_1920", 1

    bench.run_reference(A())
    assert capsys.readouterr().out == ""
