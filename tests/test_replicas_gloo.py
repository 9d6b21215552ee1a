"""Multi-rank host logic of `bench.py` on the CPU: two gloo ranks.

Each rank runs an independent replica (its own seeded shots), the timed
region is bracketed by barriers, the reported time is the maximum over ranks
and the whole-job rate is all ranks' work over that time; rank 0 alone
prints.  The GPU runs the same code with NCCL.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2104_00794_gb300.replicas import Replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    env = {"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)}
    os.environ.update(env, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    reps = Replicas(env).init("gloo")
    reps.barrier()
    ms = [120.0, 150.0][rank]  # rank 1 is the slowest
    ms_max = reps.max_over_ranks(ms)
    rate = reps.whole_job_rate(1e9, ms_max)
    reps.barrier()
    out.put((rank, reps.printer, reps.seed_offset(), ms_max, rate))
    reps.close()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_max_time_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=90) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    assert [r[1] for r in res] == [True, False]     # rank 0 alone prints
    assert [r[2] for r in res] == [0, 1]            # each rank its own shots
    for _, _, _, ms_max, rate in res:
        assert ms_max == 150.0                      # the slowest rank's time
        assert rate == pytest.approx(2 * 1e9 / 0.150)


def test_single_rank_needs_no_process_group():
    reps = Replicas({}).init("gloo")
    assert reps.world == 1 and reps.printer
    assert reps.max_over_ranks(3.5) == 3.5
    assert reps.whole_job_rate(10.0, 1000.0) == 10.0
    reps.close()


def test_bad_rank_rejected():
    with pytest.raises(ValueError):
        Replicas({"RANK": "2", "WORLD_SIZE": "2"})


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    assert bench.run_reference(None, rank=1) is None  # no work, no line
    assert capsys.readouterr().out == ""
