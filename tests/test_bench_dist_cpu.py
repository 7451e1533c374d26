"""The multi-process path of bench.py (one process per GPU, replicas of the
solve, barrier and max-over-ranks timing) exercised with two gloo ranks on
the CPU: no GPU, no data-path collective."""
import importlib.util
import os
import socket
import tempfile

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _rank(rank, world, port, outdir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    b = _bench()
    r, w, local, pg = b.dist_setup(world, backend="gloo")
    b.barrier(pg)
    ms = 100.0 * (rank + 1)                       # the slower rank decides
    ms_max = b.max_over_ranks(pg, ms)
    value = b.replica_throughput(w, 4, ms_max)
    with open(os.path.join(outdir, f"r{rank}.txt"), "w") as f:
        f.write(f"{r} {w} {local} {ms_max} {value}\n")
    b.barrier(pg)
    pg.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_gloo_ranks_max_time_and_whole_job_throughput():
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank, args=(world, _free_port(), d), nprocs=world, join=True,
                           start_method="spawn")
        rows = [open(os.path.join(d, f"r{r}.txt")).read().split() for r in range(world)]
    for r, row in enumerate(rows):
        rank, w, local, ms_max, value = int(row[0]), int(row[1]), int(row[2]), float(row[3]), float(row[4])
        assert (rank, w, local) == (r, world, r)
        assert ms_max == 200.0                     # max over ranks, on every rank
        assert value == pytest.approx(world * 4 / 0.2)   # 2 replicas x 4 solves in 0.2 s


def test_single_process_needs_no_process_group():
    b = _bench()
    os.environ.pop("WORLD_SIZE", None)
    rank, world, local, pg = b.dist_setup(1)
    assert (rank, world, pg) == (0, 1, None)
    assert b.max_over_ranks(pg, 12.5) == 12.5
    assert b.replica_throughput(1, 2, 500.0) == pytest.approx(4.0)
