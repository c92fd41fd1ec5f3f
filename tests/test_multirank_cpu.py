"""The N>1 host path of bench.py on CPU: two ranks over gloo (no GPU).

With more than one GPU the bench runs one independent replica of the step per
rank (each rank its own seeded scene); the only exchanges are the timing max and
the sum of the pixels the replicas processed, and under the reference arm only
rank 0 runs the oracle.  These tests run those pieces in two spawned processes.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    import json
    import types

    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = bench.dist_info()
    ms = bench.max_over_ranks(10.0 + rank, world)
    pix = bench.sum_over_ranks(1000 * (rank + 1), world)
    # the reference arm: ranks other than 0 return at once without work
    t = None
    if rank != 0:
        import time
        t0 = time.perf_counter()
        a = types.SimpleNamespace(n=500_000, views=16, warmup=3, steps=10, cpu_sample=384, gpus=world)
        bench.run_reference(a, rank, world)
        t = time.perf_counter() - t0
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"info": got, "ms": ms, "pix": pix, "ref_s": t}, f)


def test_two_gloo_ranks_agree_on_max_time_and_total_pixels(tmp_path):
    import json
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, d in enumerate(res):
        assert d["info"] == [r, world, r]
        assert d["ms"] == pytest.approx(11.0)      # the slowest rank's time, on every rank
        assert d["pix"] == pytest.approx(3000.0)   # 1000 + 2000 pixels over the replicas
    assert res[1]["ref_s"] is not None and res[1]["ref_s"] < 5.0  # rank 1 builds no scene, runs no oracle


def test_single_rank_reductions_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.sum_over_ranks(7.0, 1) == 7.0
