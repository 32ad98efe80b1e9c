"""The bench's multi-rank logic on CPU ranks (gloo, world size 2): the job's
time is the slowest rank's, its rate counts every rank's frames, and the
reference arm runs on rank 0 only (other ranks exit without work)."""
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


WORKER = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
mine = [12.5, 31.0][rank]
t = bench.max_over_ranks(mine, world)
print(json.dumps({{"rank": rank, "max": t, "rate": bench.job_rate(world, 100, t)}}), flush=True)
dist.destroy_process_group()
"""


def test_max_over_ranks_and_job_rate_with_two_gloo_ranks(tmp_path):
    script = tmp_path / "worker.py"
    script.write_text(WORKER.format(root=ROOT))
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(free_port()), WORLD_SIZE="2")
    procs = []
    for r in range(2):
        e = dict(env, RANK=str(r), LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, str(script)], env=e, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for o in outs:
        assert o["max"] == 31.0
        assert abs(o["rate"] - 2 * 100 / 0.031) < 1e-6


def test_single_rank_is_its_own_maximum():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.25, 1) == 7.25
    assert bench.job_rate(1, 300, 150.0) == 2000.0


def test_reference_arm_runs_on_rank_zero_only(tmp_path):
    """Two gloo ranks under the torchrun launcher: rank 0 prints the
    reference line, rank 1 exits 0 without output."""
    pytest.importorskip("torch")
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1 and lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2
    assert lines[0]["cpu_baseline"]["cores"] >= 1 and lines[0]["value"] > 0
