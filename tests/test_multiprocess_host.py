"""Host logic of the multi-GPU path (replicas only: every rank advances its own
copy of the workload, no exchange on the data path), run as world-size-2
gloo process groups on the CPU.

* bench.job_time_max gives every rank the slowest rank's time and
  bench.whole_job_rate turns it into the whole job's rate.
* The reference arm under torchrun: rank 0 alone runs and prints the JSON
  line, the other ranks exit 0 without output.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.job_time_max(times[rank], dist, "cpu")
    rate = bench.whole_job_rate(100.0, world, t)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t, rate))


def test_slowest_rank_time_and_whole_job_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [1.25, 3.5]
    procs = [ctx.Process(target=_worker, args=(r, world, port, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate in res:
        assert t == 3.5
        assert abs(rate - 2 * 100.0 / 3.5) < 1e-12


def _run_reference(rank):
    env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--gpus", "2", "--steps", "1", "--warmup", "3", "--ref-hex", "1"],
                          env=env, capture_output=True, text=True, timeout=600, cwd=ROOT)


def test_reference_arm_prints_on_rank_zero_only():
    r1 = _run_reference(1)
    assert r1.returncode == 0, r1.stderr
    assert r1.stdout.strip() == ""
    r0 = _run_reference(0)
    assert r0.returncode == 0, r0.stderr
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
