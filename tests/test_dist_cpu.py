"""The multi-process path of the benchmark on the host: two ranks over gloo
(127.0.0.1) take the world size and ranks from the torchrun environment,
reduce their timings (max over ranks) and work (sum over ranks), meet at
the barrier, and under `--impl reference` only rank 0 runs the oracle while
the other ranks exit 0 without work.  Every rank on the GPU runs its own
trench replica (seed 3 + rank); there is no collective on the data path."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import bench
dist, rank, ws = bench._dist()
mx = bench._reduce_max(dist, float(rank + 1))
sm = bench._reduce_sum(dist, 10.0 * (rank + 1))
bench._barrier(dist)
print(json.dumps({"rank": rank, "ws": ws, "max": mx, "sum": sm, "backend": dist.get_backend()}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, ws, port):
    env = dict(os.environ)
    env.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(ws),
                "RANK": str(rank), "LOCAL_RANK": str(rank), "CUDA_VISIBLE_DEVICES": ""})
    return env


def _run_ranks(args, ws=2, timeout=300):
    pytest.importorskip("torch")
    port = _free_port()
    procs = [subprocess.Popen(args, env=_env(r, ws, port), cwd=ROOT, stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(ws)]
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=timeout)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        outs.append((p.returncode, out, err))
    return outs


def test_two_ranks_reduce_and_meet_over_gloo():
    outs = _run_ranks([sys.executable, "-c", WORKER, ROOT])
    for rc, out, err in outs:
        assert rc == 0, err
    lines = [json.loads(o.strip().splitlines()[-1]) for _, o, _ in outs]
    assert sorted(l["rank"] for l in lines) == [0, 1]
    for l in lines:
        assert l["ws"] == 2 and l["backend"] == "gloo"
        assert l["max"] == 2.0 and l["sum"] == 30.0


def test_reference_arm_runs_on_rank_zero_only():
    outs = _run_ranks([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2",
                       "--steps", "1", "--warmup", "0"], timeout=600)
    (rc0, out0, err0), (rc1, out1, err1) = outs
    assert rc0 == 0, err0
    assert rc1 == 0, err1
    assert out1.strip() == ""
    line = json.loads(out0.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
