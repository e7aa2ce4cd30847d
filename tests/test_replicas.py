"""Multi-rank path of bench.py on CPU (gloo, world size 2): replicas do not
exchange data; the job rate is all ranks' work over the slowest rank's time,
and the reference arm prints from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


WORKER = r'''
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
dist.init_process_group("gloo")
import bench
rank = int(os.environ["RANK"]); ws = int(os.environ["WORLD_SIZE"])
ms_local = 10.0 + 5.0 * rank            # rank 1 is the slow replica
value, ms = bench.job_throughput(1000.0, ms_local, ws)
print(json.dumps({{"rank": rank, "value": value, "ms": ms}}))
dist.destroy_process_group()
'''


def _launch(code, ws=2, extra_env=None):
    port = _free_port()
    procs = []
    for r in range(ws):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(ws),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=180)
        assert p.returncode == 0, e[-2000:]
        outs.append(o)
    return outs


def test_replica_throughput_uses_slowest_rank():
    outs = _launch(WORKER.format(root=ROOT))
    rows = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    for r in rows:
        assert r["ms"] == pytest.approx(15.0)
        assert r["value"] == pytest.approx(2 * 1000.0 / 0.015)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    import bench

    class Args:
        gpus, steps, warmup = 2, 1, 0

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    called = []
    monkeypatch.setattr(bench, "oracle_timing", lambda *a: called.append(a))
    assert bench.run_reference(Args()) == 0
    assert called == []
