"""The multi-rank logic of bench.py on CPU: world size 2 over gloo (127.0.0.1).

Each rank fits its own replica (no data-path collective), so the only
exchange is the timing: the job's time is the slowest rank's, and the value
counts the units of every rank. The reference arm runs on rank 0 alone."""
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


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)
        slowest = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")    # rank times 10 ms and 15 ms
        value = bench.whole_job_rate(4.0e6, ws, slowest / 1e3)
        out.put((rank, slowest, value))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_rank_and_count_all_units():
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
    for rank, slowest, value in res:
        assert slowest == 15.0
        assert value == pytest.approx(2 * 4.0e6 / 0.015)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    import synth
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class Args:
        seed = 0
        warmup = 3
        steps = 2
    # rank 1 returns at once (exit status 0) without building or timing anything
    assert bench.run_reference(Args(), synth.WORKLOADS["nb_medium"]) == 0
