"""Host logic of the multi-rank benchmark path on CPU with gloo (world size 2):
each rank runs an independent replica, the time is the max over ranks and the
value the pixels of all ranks over it; the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    per_rank_ms = [100.0, 250.0][rank]
    mx = bench.barrier_max(world, per_rank_ms)
    value = bench.whole_job_value(world, 8 * 1352 * 1014, 10, mx)
    q.put((rank, mx, value))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value():
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
    assert [o[1] for o in out] == [250.0, 250.0]
    expected = 2 * 8 * 1352 * 1014 * 10 / 0.25 / 1e6
    assert all(abs(o[2] - expected) < 1e-9 * expected for o in out)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    called = []
    monkeypatch.setattr(bench, "oracle_step", lambda *a, **k: called.append(1))
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "3"]) == 0
    assert called == []
