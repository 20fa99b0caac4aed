"""The N > 1 bench path on CPU: two ranks over gloo (no GPU).

Every rank runs its own replica (weak scaling, no collective on the data
path); the only cross-rank steps are the barrier and the reduction of the
timed region, which must give the slowest rank's time and the sum of all
ranks' particle updates.  The reference arm under torchrun prints one line
from rank 0 and lets the other ranks exit without work.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r was timed at 10 (r + 1) ms over 1000 (r + 1) updates
    ms, units = bench.aggregate_over_ranks(10.0 * (rank + 1), 1000 * (rank + 1), dist, "cpu")
    out.put((rank, ms, units))
    dist.destroy_process_group()


def test_timing_reduction_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest time and the total work
    assert got == [(0, 20.0, 3000), (1, 20.0, 3000)]


def test_single_rank_reduction_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(12.5, 77, None) == (12.5, 77)


def test_reference_arm_under_torchrun_two_ranks():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--workload", "plain_32", "--cpu-sample", "2048", "--steps", "1",
           "--warmup", "0", "--gpus", "2"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout           # rank 0 alone prints
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2
    assert out["value"] > 0 and out["cpu_baseline"]["kind"] == "oracle"
    assert out["e2e"]["h2d_bytes_per_step"] == 0
