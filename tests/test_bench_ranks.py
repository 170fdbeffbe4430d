"""The multi-GPU path of bench.py on the CPU: every rank runs an independent replica of the chain (the
path has no data-path collective), and the job's time is the slowest rank's. Two gloo ranks check the
max-over-ranks reduction and the whole-job line rate computed from it, and the self-launch that
`bench.py --gpus N` uses without torchrun gives each rank the rendezvous environment torchrun would."""

from __future__ import annotations

import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out_dir: str) -> None:
    import json

    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took 10 (r + 1) ms for its steps and 12 (r + 1) ms end to end
    total, e2e = bench.max_over_ranks([10.0 * (rank + 1), 12.0 * (rank + 1)], dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    value = bench.replica_line_rate(world, bits_per_step=8 << 20, steps=5, total_ms=total)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"total": total, "e2e": e2e, "value": value}, f)


def test_two_ranks_take_the_slowest_replica(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    import json
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for r in res:
        assert r["total"] == 20.0 and r["e2e"] == 24.0
        # 2 replicas x 8 Mi bits x 5 steps in 20 ms
        assert abs(r["value"] - 2 * (8 << 20) * 5 / 0.020 / 1e9) < 1e-9


def test_single_process_is_unchanged():
    import bench
    assert bench.max_over_ranks([3.5, float("inf")]) == [3.5, float("inf")]
    assert abs(bench.replica_line_rate(1, 1 << 23, 20, 14.4) - (1 << 23) * 20 / 0.0144 / 1e9) < 1e-12


def _env_rank(out_dir: str) -> None:
    import json

    import torch
    import torch.distributed as dist

    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    dist.init_process_group("gloo")                       # env:// rendezvous from the spawned environment
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"env{rank}.json"), "w") as f:
        json.dump({"rank": rank, "world": world, "local": int(os.environ["LOCAL_RANK"]),
                   "addr": os.environ["MASTER_ADDR"], "sum": float(t[0])}, f)


def test_self_launch_gives_each_rank_the_torchrun_environment(tmp_path):
    pytest.importorskip("torch.multiprocessing")
    import json

    import bench
    world = 2
    bench.spawn_ranks(world, _env_rank, str(tmp_path))
    res = sorted((json.load(open(tmp_path / f"env{r}.json")) for r in range(world)), key=lambda d: d["rank"])
    assert [d["rank"] for d in res] == [0, 1] and all(d["world"] == world for d in res)
    assert [d["local"] for d in res] == [0, 1] and all(d["addr"] == "127.0.0.1" for d in res)
    assert all(d["sum"] == 3.0 for d in res)
