"""The multi-GPU path of bench.py on CPU: two gloo ranks.

The simulation shards by independent problems (each rank simulates its own
replica; there is no collective on the data path), so what the N-rank run
adds is host logic: per-rank seeds, the slowest rank's time as the job time,
the whole-job throughput, and the reference arm running on rank 0 only.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    from paper_2604_23305_b300 import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, loc = bench.dist_env()
        seeds = bench.replica_seeds(r)
        sc = W.scenario("single_pixel_small", nt_total=64, **seeds)
        screen_sum = float(np.asarray(sc["atmosphere"]["screen"], dtype=np.float64).sum())
        elapsed = bench.max_over_ranks(1.0 + r, dist, "cpu")           # rank r "took" 1 + r seconds
        value = bench.job_value(w, 1000.0, 5, elapsed)
        gathered = [None] * world
        dist.all_gather_object(gathered, (r, seeds, screen_sum, elapsed, value))
        out_q.put((rank, w, loc, gathered))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_run_independent_replicas_and_report_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, w, loc, gathered in results:
        assert w == world and loc == rank
        by_rank = {g[0]: g for g in gathered}
        assert by_rank[0][1] != by_rank[1][1]                    # different seeds per replica
        assert by_rank[0][2] != by_rank[1][2]                    # hence different screens
        assert all(g[3] == 2.0 for g in gathered)                # job time = slowest rank
        assert all(g[4] == pytest.approx(2 * 1000.0 * 5 / 2.0) for g in gathered)


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        workload, ref_samples, warmup, steps = "ifu25", 4, 0, 1

    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""
