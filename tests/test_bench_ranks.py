"""The benchmark's multi-rank host logic on CPU: two gloo ranks run as replicas (no
data-path collective), the timed region is bracketed by barriers, and the whole-job rate
is all ranks' work over the slowest rank's time."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_init()
    bench.barrier(w)
    # rank r processed 1000 units in 1 + r seconds: the job processed 2000 units, and the
    # slowest rank took 2 s
    rate = bench.aggregate_rate(1000.0, 1.0 + r, w)
    slowest = bench.max_over_ranks(1.0 + r, w)
    bench.barrier(w)
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"world": w, "rank": r, "rate": rate, "slowest": slowest}, f)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_replicas(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r, d in enumerate(res):
        assert d["world"] == 2 and d["rank"] == r
        assert d["slowest"] == 2.0
        assert d["rate"] == pytest.approx(2 * 1000.0 / 2.0)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.aggregate_rate(10.0, 2.0, 1) == 5.0
    bench.barrier(1)  # no process group: a no-op
