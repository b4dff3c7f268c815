"""The N > 1 path of bench.py on CPU: world-size-2 gloo ranks (127.0.0.1).
Each GPU would run an independent replica; the whole-job number divides the
units of all ranks by the slowest rank's time."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took (r + 1) seconds for (r + 1) * 1000 units
    T, U = bench.aggregate_over_ranks(rank + 1.0, (rank + 1) * 1000, dist, device="cpu")
    dist.barrier()
    q.put((rank, T, U))
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, T, U in out:
        assert T == 2.0          # the slowest rank
        assert U == 3000.0       # all ranks' units


def test_single_process_is_identity():
    import bench
    assert bench.aggregate_over_ranks(1.5, 42) == (1.5, 42.0)


def test_reference_arm_is_rank0_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        config = "cfg1"
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""
