"""The N > 1 path of bench.py, on CPU with world_size 2 over gloo.

Each rank matches an independent replica (weak scaling, no data-path
collective); the only cross-rank steps are the barrier and the reduction of
the timings: the slowest rank's time and the pairs of all ranks.
"""
import argparse
import json
import os
import socket

import numpy as np
import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_ms = (10.0, 30.0)[rank]     # device time of this rank's timed steps
    K = (100, 300)[rank]          # pairs of this rank's replica
    e2e_s = (1.0, 2.0)[rank]
    tot = bench.job_totals(t_ms, K, 5, e2e_s, 3, world, torch.device("cpu"))
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
        json.dump(tot, fh)
    dist.barrier()
    dist.destroy_process_group()


def test_job_totals_two_ranks(tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for rank in range(2):
        tot = json.loads((tmp_path / f"rank{rank}.json").read_text())
        assert tot["t_max_s"] == pytest.approx(0.030)          # the slowest rank
        assert tot["pairs_all_ranks"] == 400                     # every rank's pairs
        assert tot["value"] == pytest.approx(400 * 5 / 0.030)
        assert tot["ms_per_step"] == pytest.approx(6.0)
        assert tot["e2e_value"] == pytest.approx(400 * 3 / 2.0)


def test_job_totals_single_rank_needs_no_process_group():
    import torch
    import bench
    tot = bench.job_totals(20.0, 50, 4, 0.5, 2, 1, torch.device("cpu"))
    assert tot["value"] == pytest.approx(50 * 4 / 0.020)
    assert tot["e2e_value"] == pytest.approx(50 * 2 / 0.5)


def test_ranks_match_different_replicas():
    import bench
    for d in (1, 3):
        args = argparse.Namespace(alpha=1.0, N=2000, d=d)
        a, b = bench.workload(args, 0), bench.workload(args, 1)
        assert a.sub_lo.shape == b.sub_lo.shape == (d, 1000)
        assert not np.array_equal(a.sub_lo, b.sub_lo)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(argparse.Namespace(alpha=1.0, N=2000, d=1, steps=1, warmup=0, gpus=2))
    assert capsys.readouterr().out == ""
