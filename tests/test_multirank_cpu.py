"""The multi-GPU path of bench.py is replicas only (each rank advances its
own copy of the workload; weak scaling, no collective on the data path).
Its host logic -- max-over-ranks timing and the whole-job value -- runs here
as two gloo ranks on CPU, as does the reference arm's exit on ranks > 0."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    t = bench.max_over_ranks(local_ms, world)
    v = bench.job_value(world, 1000, 10, t)
    dist.barrier()
    q.put((rank, t, v))
    dist.destroy_process_group()


def test_replicas_timing_and_value_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == 150.0                      # max over ranks
        assert v == pytest.approx(2 * 1000 * 10 / 0.150)


def test_reference_arm_exits_quietly_on_other_ranks(monkeypatch, capsys):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:
        gpus, steps, warmup, workload = 2, 1, 0, "tgv256"
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""
