"""The benchmark's multi-rank logic on CPU (gloo, world size 2): each rank
draws its own events, the job time is the slowest rank's, and the job rate
counts every rank's events.  No GPU and no collective on the data path."""
import json
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import bench
    import synth.workloads
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.workloads.get("sipm8x8_xy")
    ev = w.events(64, seed=bench.rank_seed(w.event_seed, rank))
    local_time = 1.5 + rank  # rank 1 is the slow one
    t = bench.max_over_ranks(local_time, device="cpu")
    rate = bench.job_rate(64, world, 3, t)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"t": t, "rate": rate, "first": ev.signals[0].tolist(), "xyz0": ev.xyz[0].tolist()}, f)


def test_two_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r = [json.load(open(tmp_path / f"r{k}.json")) for k in range(2)]
    assert r[0]["t"] == r[1]["t"] == 2.5  # max over ranks, seen by every rank
    assert r[0]["rate"] == pytest.approx(64 * 2 * 3 / 2.5)
    assert r[0]["first"] != r[1]["first"] and r[0]["xyz0"] != r[1]["xyz0"]  # independent events per rank
    import bench
    import synth.workloads
    w = synth.workloads.get("sipm8x8_xy")
    again = w.events(64, seed=bench.rank_seed(w.event_seed, 1))
    assert np.allclose(again.signals[0], r[1]["first"])  # a rank's events are reproducible


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.job_rate(10, 1, 2, 4.0) == 5.0
