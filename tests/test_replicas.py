"""Host logic of `bench.py --gpus N` (replicas only: every rank runs its own copy of the
workload with its own data seed; the only exchange is the max of the step times) on two gloo
ranks on the CPU."""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        class A:
            workload = "tiny_plain"
            rows = 1000
        w = bench.workload(A, rank)
        # rank-dependent "step time": the slowest rank decides
        got = bench.replica_max(10.0 + 5.0 * rank, dist, "cpu")
        env = bench.dist_env()
        dist.barrier()
        with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
            json.dump({"seed": w.data.seed, "n_rows": w.data.n_rows, "max": got, "env": list(env),
                       "params": [w.params.K, w.params.L, w.params.R, w.params.range_bits, w.params.seed]}, f)
    finally:
        dist.destroy_process_group()


def test_two_replicas_seed_apart_and_take_the_slowest_time(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    r = [json.load(open(tmp_path / ("rank%d.json" % i))) for i in range(world)]
    assert r[0]["max"] == r[1]["max"] == 15.0
    assert r[0]["env"] == [0, 2, 0] and r[1]["env"] == [1, 2, 1]
    # each replica hashes its own rows (data seed apart), with the same method parameters
    assert r[0]["seed"] != r[1]["seed"]
    assert r[0]["n_rows"] == r[1]["n_rows"] == 1000
    assert r[0]["params"] == r[1]["params"]


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        workload = "tiny_plain"
        rows = 1000
        steps = 1
        warmup = 0
        gpus = 2
    bench.run_reference(A)  # returns at once on a rank other than 0: no work, no line
    assert capsys.readouterr().out == ""

