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


DECOMP_WORKER = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import torch
import bench
import synth
from paper_1610_03918_gb300 import distributed as pd

dist, rank, ws = bench._dist()

# exact integer sums over the ranks, beyond 2^53 and negative
big = torch.tensor([2 ** 62 + rank, -(2 ** 60) - 7 * rank, 3], dtype=torch.int64)
pd.allreduce_sum_int64(big)


class HostRank:
    # Stands in for one rank's context on the host: its particle phase
    # deposits its particles' cells as integer counts of 2^20 units into the
    # exchange buffer [nodes | bottom counts]; its field phase reads rho from
    # the (summed) buffer and moves the particles by a fixed step.
    def __init__(self, w, parts):
        self.w, self.p = w, parts
        self.nn = (w.nx + 1) * w.ny
        self.buf = torch.zeros(self.nn + w.ny, dtype=torch.int64)
        self.bottom = np.zeros(w.ny, np.int64)
        self.torch_stream = None
        self.rho = None

    def exchange_buffer(self):
        return self.buf

    def step_particles(self):
        i = np.floor(self.p.x).astype(np.int64)
        j = np.floor(self.p.y).astype(np.int64)
        acc = np.zeros(self.nn, np.int64)
        np.add.at(acc, i * self.w.ny + j, 1 << 20)
        hit = i >= self.w.nx - 2
        np.add.at(self.bottom, j[hit], 1)
        self.buf[:] = torch.from_numpy(np.concatenate([acc, self.bottom]))

    def step_fields(self):
        self.rho = self.buf.numpy()[: self.nn].astype(np.float64) / (1 << 20)
        self.bot = self.buf.numpy()[self.nn:].copy()
        self.p.x = np.mod(self.p.x + 0.37 * self.p.vx, self.w.nx - 1)

    def counts(self):
        return np.zeros((2, 8), np.int64) + len(self.p), np.array([len(self.p), 0])


w = synth.small_trench(nx=40, ny=32, depth=10, width=6, ppc=4, seed=3)
full = synth.maxwellian_load(w, 1)
lo, hi = pd.shard_bounds(len(full), rank, ws)
mine = pd.DistributedSim(HostRank(w, pd.shard(full, rank, ws)))
mine.step(3)
walls, live = mine.counts()
one = HostRank(w, synth.maxwellian_load(w, 1))
for _ in range(3):
    one.step_particles()
    one.step_fields()
print(json.dumps({"rank": rank, "lo": lo, "hi": hi, "n": len(full), "big": big.tolist(),
                  "rho_equal": bool(np.array_equal(mine.sim.rho, one.rho)),
                  "bottom_equal": bool(np.array_equal(mine.sim.bot, one.bot)),
                  "live": int(live[0])}))
dist.destroy_process_group()
"""


def test_particle_decomposition_driver_over_gloo():
    # two gloo ranks on the host: contiguous shards cover the particles once,
    # the int64 all-reduce is exact, and a two-rank run of the decomposed
    # step driver gives the one-rank run's summed deposit bit for bit
    outs = _run_ranks([sys.executable, "-c", DECOMP_WORKER, ROOT])
    for rc, out, err in outs:
        assert rc == 0, err
    lines = sorted((json.loads(o.strip().splitlines()[-1]) for _, o, _ in outs), key=lambda l: l["rank"])
    assert lines[0]["lo"] == 0 and lines[0]["hi"] == lines[1]["lo"] and lines[1]["hi"] == lines[0]["n"]
    for l in lines:
        assert l["big"] == [2 ** 63 + 1, -(2 ** 61) - 7, 6] or l["big"] == [-(2 ** 63) + 1, -(2 ** 61) - 7, 6]
        assert l["rho_equal"] and l["bottom_equal"]
        assert l["live"] == l["n"]
