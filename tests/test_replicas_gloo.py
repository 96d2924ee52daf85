"""The N > 1 path of bench.py on CPU: two gloo ranks.

The minor cycle does not shard (each iteration depends on the residual the
previous one left), so N GPUs run N independent replicas of the workload,
one image per rank, with no collective on the data path.  What crosses ranks
is the bookkeeping: the whole-job time is the slowest rank's, the work is the
sum over ranks.  These tests run that host logic as two gloo processes and
check that the replicas really are different images.
"""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, outdir: str):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: 100 ms * (r + 1) for 10 * (r + 1) iterations
        t, n, pe = bench.aggregate(100.0 * (rank + 1), 10 * (rank + 1), 1000 * (rank + 1), "cpu")
        w, r, _ = bench._dist()
        with open(os.path.join(outdir, f"r{rank}.json"), "w") as f:
            json.dump({"t": t, "n": n, "pe": pe, "world": w, "rank": r}, f)
    finally:
        dist.destroy_process_group()


def test_aggregate_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    for r, x in enumerate(res):
        assert x["rank"] == r and x["world"] == 2
        assert x["t"] == 200.0            # the slowest rank's time
        assert x["n"] == 30               # 10 + 20 iterations
        assert x["pe"] == 3000
    # whole-job throughput = sum of work / slowest time
    assert res[0]["n"] / (res[0]["t"] / 1e3) == pytest.approx(150.0)


def test_aggregate_single_process_is_identity():
    import bench
    assert bench.aggregate(12.5, 7, 99, "cpu") == (12.5, 7, 99)


def test_replicas_are_distinct_images():
    import bench
    a = bench._workload(2, 64, 0)
    b = bench._workload(2, 64, 1)
    assert a.dirty.shape == b.dirty.shape
    assert abs(a.dirty - b.dirty).max() > 0.0
    # same seed, same image: a rank's workload is reproducible
    c = bench._workload(2, 64, 0)
    assert (a.dirty == c.dirty).all() and (a.psf == c.psf).all()


def test_reference_arm_other_ranks_exit_quietly(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = type("A", (), dict(gpus=2, steps=1, warmup=0, size=64, cpu_budget=1.0))()
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
