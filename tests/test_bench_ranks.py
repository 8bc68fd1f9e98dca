"""The multi-replica side of bench.py on CPU: two gloo ranks agree on the
slowest rank's time and report the whole-job rate; under --impl reference
only rank 0 works."""
import os
import socket
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world)  # rank 1 is the slow one
    rate = bench.job_rate(100.0, ms * 1e-3, world)
    q.put((rank, ms, rate))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in got:
        assert ms == 15.0
        assert rate == pytest.approx(2 * 100.0 / 0.015)


def test_single_rank_passes_through():
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_rate(7.0, 2.0, 1) == 3.5


def test_reference_arm_only_on_rank_zero(monkeypatch, capsys):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1"])
    bench.main()
    assert capsys.readouterr().out == ""
