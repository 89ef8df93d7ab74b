"""The benchmark's multi-rank path on CPU: two gloo ranks (as torchrun would
launch them) exchange only the timing and point counts -- there is no
collective on the data path -- and only rank 0 prints.  The reference arm
(the FP64 oracle on the host cores) runs on rank 0 alone."""
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


WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank = dist.get_rank(); world = dist.get_world_size()
# rank r timed 100*(r+1) ms for 1000*(r+1) points
t, total, value = bench.weak_scaling_value(world, 100.0 * (rank + 1), 1000.0 * (rank + 1))
bench.barrier(world)
with open(os.path.join({out!r}, "rank%d.json" % rank), "w") as fh:
    json.dump({{"rank": rank, "t": t, "total": total, "value": value}}, fh)
dist.destroy_process_group()
"""


def _torchrun(script_args, env_extra=None, nproc=2, timeout=240):
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", PYTHONPATH=ROOT)
    env.update(env_extra or {})
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
           "--nproc-per-node", str(nproc), "--master-addr", "127.0.0.1",
           "--master-port", str(_free_port())] + script_args
    return subprocess.run(cmd, capture_output=True, text=True, timeout=timeout, env=env,
                          cwd=ROOT)


def test_weak_scaling_aggregation_two_gloo_ranks(tmp_path):
    pytest.importorskip("torch")
    script = tmp_path / "worker.py"
    script.write_text(WORKER.format(root=ROOT, out=str(tmp_path)))
    r = _torchrun([str(script)])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads((tmp_path / ("rank%d.json" % k)).read_text()) for k in range(2)]
    for x in lines:
        # slowest rank 200 ms; 3000 points in total
        assert x["t"] == 200.0 and x["total"] == 3000.0
        assert x["value"] == pytest.approx(3000.0 / 0.2 / 1e9)


def test_reference_arm_rank0_only_two_ranks():
    pytest.importorskip("torch")
    r = _torchrun([os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                   "--steps", "1", "--warmup", "0", "--workload", "sin3d"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1                     # rank 1 prints nothing
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
