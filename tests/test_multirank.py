"""The bench's multi-rank logic on CPU: two gloo ranks, the barrier, the maximum of the
per-rank times, whole-job throughput, and the reference arm doing no work on rank 1.

Replicas only: each rank solves the whole workload on its own GPU, so the only
cross-rank operations are the barrier around the timed region and the max-reduction
of the times; both run here through torch.distributed on the gloo backend.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.environ["PBS_ROOT"])
import torch
import torch.distributed as dist
import bench
rank, ws = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=ws)
r = bench.Ranks(ws, torch.device("cpu"))
r.barrier()
ms = r.max(10.0 * (rank + 1))
r.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "ms_max": ms, "value": bench.job_throughput(ws, 31, ms)}))
"""


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank: int, ws: int, port: int) -> dict:
    env = dict(os.environ)
    env.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(port), PBS_ROOT=ROOT)
    return env


def test_two_gloo_ranks_barrier_and_max():
    port = _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", RANK_SCRIPT], env=_env(r, 2, port), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["ms_max"] == 20.0  # the slower rank's time
        assert o["value"] == pytest.approx(2 * 31 / 0.020)  # both ranks' k-points over the max time


def test_reference_arm_runs_on_rank_zero_only():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=_env(1, 2, _free_port()), capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
