"""The bench's multi-rank path on CPU: two gloo ranks reduce their step times to the slowest one and
report the whole job's throughput; under a launcher only rank 0 of the reference arm does any work.
(Every rank runs the same replica: the path has no exchange step.)"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch

    sys.path.insert(0, ROOT)
    import bench

    torch.distributed.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                                         world_size=world)
    ms = [2.0, 3.5][rank]  # rank 1 is the slowest
    slowest = bench.max_over_ranks(ms, world, "cpu")
    value = bench.whole_job_value(1000.0, world, slowest)
    torch.distributed.barrier()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"slowest": slowest, "value": value}, f)
    torch.distributed.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step(tmp_path):
    torch = pytest.importorskip("torch")
    port = _free_port()
    torch.multiprocessing.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        d = json.load(open(tmp_path / f"rank{r}.json"))
        assert d["slowest"] == 3.5
        assert d["value"] == pytest.approx(1000.0 * 2 / 3.5e-3)


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(1.25, 1) == 1.25
    assert bench.whole_job_value(10.0, 1, 2.0) == pytest.approx(5000.0)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
