"""The multi-GPU path of the benchmark is replicas: one process per GPU, each stepping its own
lattice, joined only for barriers and the maximum of the timings.  Its host logic runs here with
two gloo ranks on the CPU: rank discovery from the launcher's environment, the max over ranks,
the whole-job aggregate, and the reference arm's rule that only rank 0 works."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w, local = bench.dist_setup(world, backend="gloo")
    ms = 10.0 + 5.0 * r                       # the ranks' own timings
    bench.barrier(w)
    ms_max = bench.barrier_max(ms, w)
    value = bench.aggregate_mlups(1000, 20, w, ms_max)
    out.put((r, w, local, ms_max, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[:3] for r in res] == [(0, 2, 0), (1, 2, 1)]
    assert all(r[3] == 15.0 for r in res)                                  # max over ranks
    assert all(r[4] == pytest.approx(1000 * 20 * 2 / 15e-3 / 1e6) for r in res)


def test_single_process_needs_no_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_setup(1) == (0, 1, 0)
    assert bench.barrier_max(3.5, 1) == 3.5
    assert bench.aggregate_mlups(2048 * 1024, 100, 1, 7.5) == pytest.approx(2048 * 1024 * 100 / 7.5e-3 / 1e6)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    args = bench.argparse.Namespace(gpus=2, steps=1, warmup=1)
    bench.run_reference(args)                  # returns at once: no oracle work, no output
    assert capsys.readouterr().out == ""
