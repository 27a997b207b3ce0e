"""Host logic of bench.py's multi-GPU mode on CPU: world_size 2 over gloo.  The path does
not shard (replicas only): each rank solves its own problem, the job's step time is the
slowest rank's, the whole-job value counts every rank's units, and the reference arm
runs on rank 0 alone."""
import json
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


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms, value = bench.job_time_and_value(100.0 + 50.0 * rank, 1.0e9, world, device="cpu")
        w, r, lr = bench.dist_env()
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
            json.dump({"ms": ms, "value": value, "env": [w, r, lr]}, fh)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_count_both(tmp_path):
    world = 2
    out = str(tmp_path)
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    res = [json.load(open(os.path.join(out, f"rank{r}.json"))) for r in range(world)]
    for r, d in enumerate(res):
        assert d["env"] == [world, r, r]
        assert d["ms"] == 150.0                      # MAX over ranks, seen by every rank
        assert abs(d["value"] - 2 * 1.0e9 / 0.150) < 1e-3 * d["value"]


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.job_time_and_value(200.0, 5.0e8, 1, device="cpu") == (200.0, 5.0e8 / 0.2)


def test_reference_arm_prints_nothing_on_other_ranks(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:
        workload, steps, warmup, ref_slices = "heat3d", 1, 0, 1
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
