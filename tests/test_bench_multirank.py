"""The benchmark's multi-rank logic on CPU with the gloo backend (world size 2):
independent replicas are timed by the slowest rank and counted by all ranks,
and the reference arm runs on rank 0 only."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, ws, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    # rank r measured 10 (r + 1) ms over 2 steps, 1e9 flop per rank and step
    ms_step, gflops = bench.combine_ranks(10.0 * (rank + 1), 2, 1e9, ws, torch.device("cpu"))
    out.put((rank, ms_step, gflops))
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_takes_the_slowest_rank_and_all_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_step, gflops in res:
        assert ms_step == pytest.approx(10.0)               # max(10, 20) ms / 2 steps
        assert gflops == pytest.approx(2 * 1e9 / 0.010 / 1e9)  # both ranks' flops over the slowest time


def test_single_rank_is_the_local_measurement():
    import torch
    sys.path.insert(0, ROOT)
    import bench
    ms_step, gflops = bench.combine_ranks(30.0, 3, 2e9, 1, torch.device("cpu"))
    assert ms_step == pytest.approx(10.0) and gflops == pytest.approx(200.0)


def test_reference_arm_prints_only_on_rank_0():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--ref-n", "64"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line_on_rank_0():
    import json
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--ref-n", "64"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GFLOP/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
