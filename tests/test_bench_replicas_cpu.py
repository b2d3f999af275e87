"""The replica aggregation of bench.py over two gloo ranks on the CPU.

bench.py on N GPUs advances N independent chains, one per rank (replicas:
no data-path collective; whole-job throughput = all ranks' pairs / the
slowest rank's time).  The sharded evaluation, which splits one chain's pass
over ranks with an exchange of partial sums, is tested in test_shard_cpu.py
and test_shard_gpu.py.  This checks the max-over-ranks reduction and the
aggregate with unequal per-rank times, and that the reference arm's ranks
other than 0 exit without work.
"""
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


_WORKER = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
rank, world, _ = bench.dist_env()
dist.init_process_group("gloo")
secs = 2.0 + rank            # rank 1 is the slower one
units = 1000.0
out = dict(rank=rank, max=bench.reduce_max(secs, world), rate=bench.replica_rate(units, secs, world))
bench.barrier(world)
print("OUT " + json.dumps(out), flush=True)
dist.destroy_process_group()
"""


def _launch(code, world, extra_env=None, args=()):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        env.update(extra_env or {})
        cmd = [sys.executable, "-c", code] if code else [sys.executable, os.path.join(ROOT, "bench.py"), *args]
        procs.append(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env,
                                      cwd=ROOT))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=240)
        assert p.returncode == 0, e[-2000:]
        outs.append(o)
    return outs


def test_replicas_max_over_ranks_and_aggregate():
    outs = _launch(_WORKER.format(root=ROOT), 2)
    res = [json.loads(ln[4:]) for o in outs for ln in o.splitlines() if ln.startswith("OUT ")]
    assert sorted(r["rank"] for r in res) == [0, 1]
    for r in res:
        assert r["max"] == 3.0                       # the slowest rank's time on every rank
        assert r["rate"] == pytest.approx(2 * 1000.0 / 3.0)


def test_reference_arm_nonzero_ranks_exit_without_work():
    # rank 1 of the reference arm prints nothing and exits 0 at once
    port = _free_port()
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True, env=env, cwd=ROOT,
                       timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
