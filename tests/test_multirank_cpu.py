"""The benchmark's multi-rank path on CPU (gloo, world size 2): replicas
only, so the one collective is the max over ranks of the timed region, and
the job's throughput counts every replica's bytes over the slowest time.
Rank 1 of the reference arm does no work and exits 0."""
import multiprocessing as mp
import os
import socket
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t = bench._max_over_ranks(10.0 + 5.0 * rank, ws, "cpu")
    g = bench._job_gbs(10 ** 9, 4, ws, t)
    dist.barrier()
    q.put((rank, t, g))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_with_two_gloo_ranks():
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
    for rank, t, g in out:
        assert t == 15.0                      # the slower rank's time on both
        assert g == pytest.approx(2 * 4 * 1e9 / 15e-3 / 1e9)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench._job_gbs(2 * 10 ** 9, 3, 1, 2.0) == pytest.approx(3000.0)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(SimpleNamespace(gpus=2, steps=1, warmup=0)) == 0
    assert capsys.readouterr().out == ""
