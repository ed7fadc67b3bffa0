"""The multi-rank bench path on CPU: two gloo ranks take the slowest rank's
time, draw rank-dependent workloads (independent replicas, no data-path
collective) and count the whole job's throughput."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    slowest = bench.max_over_ranks(10.0 * (rank + 1), world, "cpu")
    params, _ = bench.workload("cfg2", rank)
    seeds = sorted(p["seed"] for p in params)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as fh:
        fh.write("%r\n%r\n" % (slowest, seeds))


def test_two_gloo_ranks_agree_on_the_slowest_time(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = []
    for r in range(world):
        lines = (tmp_path / ("rank%d.txt" % r)).read_text().splitlines()
        res.append((eval(lines[0]), eval(lines[1])))
    assert res[0][0] == res[1][0] == 20.0
    # replicas: every rank draws its own lattices
    assert set(res[0][1]).isdisjoint(res[1][1])


def test_job_throughput_counts_every_rank():
    import bench
    assert bench.job_mlups(1e6, 100, 1, 1.0) == pytest.approx(100.0)
    assert bench.job_mlups(1e6, 100, 4, 2.0) == pytest.approx(200.0)
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
