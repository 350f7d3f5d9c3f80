"""The benchmark's multi-process plumbing on CPU (gloo, world size 2): the
rank-0-only reference arm under torchrun, and the barrier / max-over-ranks
helpers that the GPU arm uses to time N replicas."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def torchrun(args, timeout=240):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={free_port()}"] + args
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=timeout)


def test_reference_arm_prints_one_line_from_rank_zero():
    r = torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "2",
                  "--warmup", "1", "--side", "12"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 2
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_on_the_pcg_workload():
    r = torchrun(["bench.py", "--impl", "reference", "--workload", "pcg", "--gpus", "2",
                  "--steps", "2", "--warmup", "1", "--side", "10"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "iterations/s" and d["value"] > 0
    assert d["metric"].startswith("PCG") and "pcg_stencil3d_10" in d["config"]["workload"]


HELPER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import bench
class A: pass
world, rank, local = bench.dist_setup(A())
assert world == 2
v = bench.max_over_ranks(world, 10.0 + rank)
bench.barrier(world)
with open(os.path.join({out!r}, f"rank{{rank}}.json"), "w") as fh:
    json.dump({{"rank": rank, "max": v}}, fh)
import torch.distributed as dist
dist.destroy_process_group()
"""


def test_barrier_and_max_over_ranks(tmp_path):
    script = tmp_path / "helper.py"
    script.write_text(HELPER.format(root=ROOT, out=str(tmp_path)))
    r = torchrun([str(script)])
    assert r.returncode == 0, r.stderr[-2000:]
    out = [json.loads((tmp_path / f"rank{k}.json").read_text()) for k in range(2)]
    assert sorted(o["rank"] for o in out) == [0, 1]
    assert all(o["max"] == 11.0 for o in out)
