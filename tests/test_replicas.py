"""The N-process bench path on CPU (gloo, world size 2): the renders shard as independent
replicas with no data-path collective, so the only cross-rank steps are the barrier around the
timed region and the MAX reduction of the elapsed time; the whole-job value is N x units of one
replica over the slowest rank's time.  The reference arm runs on rank 0 only."""
import argparse
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    reps = bench.Replicas(world, rank, "gloo")
    reps.barrier()
    t = reps.max(times[rank])
    rate = reps.job_rate(1000.0, t)
    reps.close()
    q.put((rank, t, rate))


def test_two_gloo_replicas_take_the_slowest_rank_and_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [1.5, 4.0]
    ps = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [4.0, 4.0]          # every rank sees the slowest time
    assert all(abs(o[2] - 2 * 1000.0 / 4.0) < 1e-9 for o in out)  # N x units / slowest time


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    reps = bench.Replicas(1, 0)
    reps.barrier()
    assert reps.max(2.5) == 2.5 and reps.job_rate(10.0, 2.0) == 5.0
    reps.close()


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(steps=1, warmup=1, gpus=2, impl="reference")
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""  # no work and no line on the other ranks
