"""Benchmark of the PIC step loop on the 512 (y, periodic) x 1024 (x) trench
workload: particle-steps/s, the HBM roofline fraction of the fused particle
kernel, Poisson milliseconds to a 1e-6 relative residual, end-to-end
throughput through the C ABI from pinned host buffers, and the FP64 oracle
timed on the host cores.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun (N > 1) every rank advances its own trench run (a different
seed) with no data-path exchange; the aggregate is the sum of the ranks'
particle-steps over the slowest rank's time (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "particle-steps/s & %HBM roofline (trench cfg); Poisson ms to 1e-6 residual"
UNIT = "particle-steps/s"
# Algorithmic bytes of the fused particle kernel per particle-step: the
# 20-byte state (int32 cell, FP32 fx, fy, vx, vy) read once and written once.
BYTES_PER_PARTICLE_STEP = 40
# DRAM bytes per live particle of the fused particle kernel from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum over the launch),
# valid for the kernel source whose hash is recorded with it.
NCU_TRAFFIC = {
    # k_particles<0, 0>, 512x1024 trench at 20 ppc (16.96M particles, 0.4 GB of
    # state, larger than L2), launches 3 and 4: 354.4 MB read + 287.4 / 284.2
    # MB written
    "source_sha256": "15dc1fe1b005f98e3c89cc6f7b48311bb7e7475cd7c9646380bd9e7e747d9204",
    "bytes_per_particle": 37.76,
}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _poisson_method(pg, args):
    return pg.POISSON_MULTIGRID if args.poisson_method == "multigrid" else pg.POISSON_AUTO


def _kernel_sha():
    src = os.path.join(ROOT, "paper_1610_03918_gb300", "csrc", "particles.cu")
    return hashlib.sha256(open(src, "rb").read()).hexdigest()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    """(process group or None, rank, world size) from the torchrun environment;
    NCCL when a GPU is visible, gloo otherwise (the host-side tests)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1
    import torch
    import torch.distributed as dist
    dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return dist, dist.get_rank(), ws


def _reduce(dist, v, op):
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def _reduce_max(dist, v):
    return v if dist is None else _reduce(dist, v, dist.ReduceOp.MAX)


def _reduce_sum(dist, v):
    return v if dist is None else _reduce(dist, v, dist.ReduceOp.SUM)


def _barrier(dist):
    if dist is not None:
        import torch
        if torch.cuda.is_available():
            torch.cuda.synchronize()
        dist.barrier()


# The oracle's timed sample of the trench workload, shared by the CPU-baseline
# leg and the reference arm: the full 512 x 1024 grid (its sparse LU
# factorised once, untimed) with ORACLE_SAMPLE particles per species drawn
# uniformly over the plasma cells, advanced by whole oracle steps.
ORACLE_SAMPLE = 100_000


def _oracle_sample(w, seed_shift=0):
    from oracle.sim import Sim as OracleSim
    from oracle import poisson
    os_ = OracleSim(w)
    for s in (0, 1):
        os_.load_particles(s, synth.random_state(w, s, ORACLE_SAMPLE, seed=w.seed + 17 + seed_shift))
    poisson.solve_direct(os_.geom, np.zeros((os_.geom.nxn, os_.geom.nyn)))   # factorise once
    os_.prepare()
    return os_


def _oracle_timed(w, steps, seed_shift=0, solves=0):
    """(particle-steps, seconds) of `steps` oracle steps on the sample; with
    solves > 0 also the seconds of one field solve (the oracle's own
    solve_fields, repeated `solves` times on the final state)."""
    os_ = _oracle_sample(w, seed_shift)
    done = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        done += int(os_.live().sum())
        os_.step(1)
    t = time.perf_counter() - t0
    if solves <= 0:
        return done, t
    t1 = time.perf_counter()
    for _ in range(solves):
        os_.solve_fields()
    return done, t, (time.perf_counter() - t1) / solves


def _oracle_replica(a):
    w, steps, k = a
    return _oracle_timed(w, steps, seed_shift=k)


def _host_info():
    info = {"nproc": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        keep = ("Architecture", "Model name", "CPU(s)", "Thread(s) per core", "Core(s) per socket",
                "Socket(s)", "CPU max MHz")
        info["lscpu"] = {k.strip(): v.strip() for k, v in
                         (l.split(":", 1) for l in out.splitlines() if ":" in l) if k.strip() in keep}
    except (OSError, subprocess.SubprocessError):
        info["lscpu"] = None
    return info


def oracle_baseline(w, steps=40):
    """The FP64 oracle as it stands on the shared sample: one process (numpy
    and scipy run it on one core), and one independent replica per core at
    once (different particle draws), all started by spawn."""
    import multiprocessing as mp
    n1, t1, t_solve = _oracle_timed(w, steps, solves=5)
    cores = min(os.cpu_count() or 1, 16)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        t0 = time.perf_counter()
        res = pool.map(_oracle_replica, [(w, steps, 1 + k) for k in range(cores)])
        wall = time.perf_counter() - t0
    # the replicas' factorisations overlap their timed steps only partly:
    # the all-core figure uses each replica's own timed seconds, the slowest
    nall = sum(r[0] for r in res)
    tall = max(r[1] for r in res)
    sample = (f"{w.name}: full 512x1024 grid (sparse LU factorised once, untimed), "
              f"{ORACLE_SAMPLE} particles/species of {int(synth.plasma_cells(w).sum()) * w.ppc}, "
              f"{steps} oracle steps")
    # the step split into its field solve and its particle phase (one core)
    t_part = max(t1 / steps - t_solve, 1e-12)
    phases = {"poisson_ms_per_solve": 1e3 * t_solve,
              "particle_phase_particle_steps_per_s": n1 / steps / t_part,
              "note": "the oracle's solve_fields (rho from the particles, sparse LU solve, E) "
                      "timed 5 times on the final state; the particle phase is the rest of a step"}
    return {"value": n1 / t1, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
            "phases_one_core": phases,
            "all_cores": {"value": nall / tall, "unit": UNIT, "cores": cores,
                          "sample": f"{cores} independent replicas of the sample at once "
                                    f"(spawned processes, {wall:.1f} s wall with their set-up)"},
            "host": _host_info()}


def errors_vs_oracle(pg):
    """The CUDA path against the FP64 oracle on a small seeded trench state
    (72 x 40 cells, 12 ppc/species, solves to 1e-10): the largest error of
    every quantity after the first solve and after one step."""
    from oracle.sim import Sim as OracleSim
    w = synth.small_trench(nx=72, ny=40, depth=20, width=6, ppc=12, seed=11).replace(poisson_rtol=1e-10)
    gs = pg.Sim(w)
    os_ = OracleSim(w)
    for s in (0, 1):
        p = synth.maxwellian_load(w, s)
        gs.load_particles(s, p)
        os_.load_particles(s, p)
    gs.step(0)
    os_.prepare()
    out = {"workload": w.name}
    rmax = np.abs(os_.rho).max()
    out["rho_rel_max"] = float(np.abs(gs.rho() - os_.rho).max() / rmax)
    ex, ey = gs.efield()
    emax = max(np.abs(os_.Ex).max(), np.abs(os_.Ey).max())
    out["E_rel_max"] = float(max(np.abs(ex - os_.Ex).max(), np.abs(ey - os_.Ey).max()) / emax)
    out["phi_rel_max"] = float(np.abs(gs.phi() - os_.phi).max() / np.abs(os_.phi).max())
    gs.step(1)
    os_.step(1)
    dx = dv = 0.0
    for s in (0, 1):
        g = gs.state(s)
        g = g[:, np.argsort(g[4], kind="stable")]
        ps = os_.p[s]
        o = np.argsort(ps["ids"], kind="stable")
        common, ig, io = np.intersect1d(g[4].astype(np.int64), ps["ids"][o].astype(np.int64),
                                        return_indices=True)
        dx = max(dx, np.abs(g[0, ig] - ps["x"][o][io]).max(), np.abs(g[1, ig] - ps["y"][o][io]).max())
        vs = np.maximum(np.maximum(np.abs(ps["vx"][o][io]), np.abs(ps["vy"][o][io])), w.vth[s])
        dv = max(dv, (np.abs(g[2, ig] - ps["vx"][o][io]) / vs).max(), (np.abs(g[3, ig] - ps["vy"][o][io]) / vs).max())
    out["x_abs_max_cells"] = float(dx)
    out["v_rel_max"] = float(dv)
    e = gs.energy()
    out["KE_rel"] = [float(abs(e[s] - os_.ke[s]) / os_.ke[s]) for s in (0, 1)]
    out["FE_rel"] = float(abs(e[2] - os_.fe) / os_.fe)
    walls, live = gs.counts()
    out["wall_tallies_equal"] = bool(np.array_equal(walls, os_.counts))
    out["live_counts_equal"] = bool(np.array_equal(live, os_.live()))
    out["bottom_counts_equal"] = bool(np.array_equal(gs.surface(), os_.bottom))
    gs.close()
    return out


def run_reference(args):
    """The oracle as it stands on the host cores, on the trench workload's
    full grid with the shared particle sample, one oracle step per step."""
    dist, rank, ws = _dist()
    if rank != 0:
        return 0
    w = synth.trench_512x1024()
    t_start = time.perf_counter()
    os_ = _oracle_sample(w)
    os_.step(max(args.warmup, 0))
    live = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        live.append(int(os_.live().sum()))
        os_.step(1)
    dt = time.perf_counter() - t0
    v = float(np.sum(live)) / dt
    sample = (f"{w.name}: full 512x1024 grid (sparse LU factorised once, untimed), "
              f"{ORACLE_SAMPLE} particles/species of {int(synth.plasma_cells(w).sum()) * w.ppc}, "
              f"{args.steps} oracle steps in {dt:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_start}
    print(json.dumps(line), flush=True)
    return 0


def ensemble_cut(pg, device, members, steps):
    """A cut of the trench-width ensemble: members k = 0 .. members-1 of the
    48-member recipe, one captured graph per ensemble step; particle-steps
    per second over `steps` steps after 10 warm-up steps (CUDA events)."""
    import torch
    wl = [synth.ensemble_member(k).replace(sort_every=24) for k in range(members)]
    batch = pg.Batch(wl, capacities=[int(synth.plasma_cells(w).sum()) * w.ppc for w in wl],
                     device=device, timing=True)
    for m, w in zip(batch.members, wl):
        for s in (0, 1):
            m.load_particles(s, synth.maxwellian_load(w, s), v_at_t0=True)
    batch.step(10)
    batch.timing()
    live0 = sum(int(m.counts()[1].sum()) for m in batch.members)
    batch.step(steps)
    t = batch.timing()
    live1 = sum(int(m.counts()[1].sum()) for m in batch.members)
    batch.close()
    torch.cuda.synchronize()
    v = 0.5 * (live0 + live1) * steps / (t["ms"] * 1e-3)
    return {"members": members, "live_particles": 0.5 * (live0 + live1), "steps": steps,
            "ms_per_step": t["ms"] / max(t["steps"], 1), "particle_steps_per_s": v,
            "hbm_frac_at_40B": BYTES_PER_PARTICLE_STEP * v / 1e9 / _peaks()[0],
            "note": "members 0.. of the 48-member width sweep (widths 1 + round(39k/47), grids "
                    "128x256 .. 512x512, 64 ppc); bench.py --workload ensemble runs all 48"}


def run_ensemble(args):
    """The trench-width sweep: members k = 0..M-1 of the recipe (widths
    1..40, grids 128x256 .. 512x512, 64 ppc), one graph launch per step."""
    dist, rank, ws = _dist()
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    import __graft_entry__
    if rank == 0 or dist is None:
        __graft_entry__.build()
    _barrier(dist)
    import paper_1610_03918_gb300 as pg
    wl = [synth.ensemble_member(k) for k in range(args.members)]
    if args.ppc:
        wl = [w.replace(ppc=args.ppc) for w in wl]
    # an ensemble takes one fixed interval (the tuned one is per context)
    wl = [w.replace(sort_every=args.sort_every or 24) for w in wl]
    batch = pg.Batch(wl, capacities=[int(synth.plasma_cells(w).sum()) * w.ppc for w in wl],
                     device=local, timing=True, poisson_method=_poisson_method(pg, args))
    n0 = 0
    for m, w in zip(batch.members, wl):
        for s in (0, 1):
            p = synth.maxwellian_load(w, s)
            n0 += len(p)
            m.load_particles(s, p, v_at_t0=True)
            del p
    batch.step(args.warmup)
    batch.timing()
    live0 = sum(int(m.counts()[1].sum()) for m in batch.members)
    clocks = ClockSampler(local)
    clocks.start()
    _barrier(dist)
    batch.step(args.steps)
    t = batch.timing()
    _barrier(dist)
    clk = clocks.stop()
    live1 = sum(int(m.counts()[1].sum()) for m in batch.members)
    ms = _reduce_max(dist, t["ms"])
    ps_total = _reduce_sum(dist, 0.5 * (live0 + live1) * args.steps)
    value = ps_total / (ms * 1e-3)
    peak, peak_kind = _peaks()
    achieved = BYTES_PER_PARTICLE_STEP * value / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"trench_width_ensemble_{args.members}", "members": args.members,
                       "ppc": wl[0].ppc, "particles_loaded": n0, "sort_every": wl[0].sort_every,
                       "tile": ("16x16 for every member (timed one by one, most members "
                                "prefer 32x32 or 16x32, which share the GPU worse)"),
                       "l2": "inputs larger than L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "note": "whole ensemble step (all phases) at 40 B per particle-step"},
            "clocks": clk}), flush=True)
    batch.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_warmstart(args):
    """Poisson time to a 1e-6 relative residual on the trench geometry with
    the learned initial guess against the zero, lift (empty-box potential)
    and previous-step starts, on
    held-out trench widths, timed inside the captured step graph with CUDA
    events (the learned guess -- network input, inference, guess -- is part of
    the solve phase).  The network is initialised by the library and trained
    by its kernels on (rho, phi) pairs dumped by the library from runs at
    other widths; pairs stream through a shuffled ring buffer, so any number
    of them fits in memory."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_03918_gb300 as pg
    from paper_1610_03918_gb300 import warmstart as ws
    t0 = time.perf_counter()

    def trench(width, seed):
        return synth.trench_512x1024(trench_width=width, trench_y0=(512 - width) // 2, seed=seed)

    net = pg.Unet(args.batch, ws.padded_rows(1025), 512)
    net.init(seed=0)
    widths = [int(v) for v in args.train_widths.split(",")]
    rng = np.random.default_rng(0)
    ring, n_pairs, n_steps = [], 0, 0
    t_data = t_train = 0.0
    per_run = max(1, args.pairs // max(args.runs, 1))
    for r in range(args.runs):
        td = time.perf_counter()
        w = trench(widths[r % len(widths)], 200 + r)
        sim = pg.Sim(w, capacity=int(synth.plasma_cells(w).sum()) * w.ppc)
        for s in (0, 1):
            sim.load_particles(s, synth.maxwellian_load(w, s), v_at_t0=True)
        sim.step(args.settle)
        t_data += time.perf_counter() - td
        for k in range(per_run):
            td = time.perf_counter()
            pair = ws.dump_pairs(sim, steps=args.dump_every, every=args.dump_every)[0]
            n_pairs += 1
            if len(ring) < args.ring:
                ring.append(pair)
            else:
                ring[int(rng.integers(len(ring)))] = pair
            t1 = time.perf_counter()
            t_data += t1 - td
            # one Adam step per `batch` new pairs, on a minibatch drawn from the ring
            if len(ring) >= args.batch and n_pairs % args.batch == 0:
                idx = rng.choice(len(ring), args.batch, replace=False)
                x = torch.stack([ring[i][0] for i in idx])
                t = torch.stack([ring[i][1] for i in idx])
                frac = n_pairs / max(args.pairs, 1)
                net.train_step(x, t, args.lr * (1.0 - 0.9 * min(frac, 1.0)))
                n_steps += 1
            torch.cuda.synchronize()
            t_train += time.perf_counter() - t1
        sim.close()
    # the network's error on pairs from the ring (training) and on held-out widths
    def rel_mse(pairs_):
        out = []
        for x, t in pairs_:
            loss, _ = probe.gradients(x[None], t[None])
            out.append(loss / float((t * t).mean()))
        return float(np.mean(out))
    probe = pg.Unet(1, ws.padded_rows(1025), 512)
    probe.set_params(net.get_params())
    train_err = rel_mse(ring[:8]) if ring else None
    held = []
    for k, width in enumerate(int(v) for v in args.eval_widths.split(",")):
        w = trench(width, 950 + k)
        sim = pg.Sim(w, capacity=int(synth.plasma_cells(w).sum()) * w.ppc)
        for s in (0, 1):
            sim.load_particles(s, synth.maxwellian_load(w, s), v_at_t0=True)
        sim.step(args.settle)
        held += ws.dump_pairs(sim, steps=20, every=10)
        sim.close()
    held_err = rel_mse(held)
    probe.close()
    del held, ring
    eval_net = pg.Unet(1, ws.padded_rows(1025), 512)
    eval_net.set_params(net.get_params())
    res, its, rel0 = {}, {}, {}
    for name, mode in (("zero", 0), ("lift", 4), ("previous", 1), ("learned", 3)):
        ms, it = [], []
        for k, width in enumerate(int(v) for v in args.eval_widths.split(",")):
            w = trench(width, 900 + k)
            sim = pg.Sim(w, capacity=int(synth.plasma_cells(w).sum()) * w.ppc,
                         poisson_method=pg.POISSON_MULTIGRID, warm_start=1 if mode == 3 else mode,
                         timing=True)
            if mode == 3:
                sim.set_learned_start(eval_net)
            for s in (0, 1):
                sim.load_particles(s, synth.maxwellian_load(w, s), v_at_t0=True)
            sim.step(args.settle)
            sim.timing()
            r0 = []
            for _ in range(args.steps):
                sim.step(1)
                st = sim.poisson_stats()
                it.append(st[0])
                r0.append(st[4])
            tm = sim.timing()
            ms.append(tm["ms_poisson"] / max(tm["steps"], 1))
            sim.close()
        res[name] = float(np.mean(ms))
        its[name] = float(np.mean(it))
        rel0[name] = float(np.exp(np.mean(np.log(np.maximum(r0, 1e-30)))))
    line = {
        "metric": "Poisson ms to 1e-6 residual (learned warm start)",
        "value": res["learned"], "unit": "ms", "higher_is_better": False, "n_gpus": 1,
        "steps": args.steps, "warmup": args.settle, "dtype": "bf16 net / f32+f64 solver",
        "data": "synthetic", "vs_baseline": None,
        "config": {"workload": "trench_512x1024 geometry, held-out widths " + args.eval_widths,
                   "inner_solver": "multigrid PCG (the warm starts serve the iterative solver)",
                   "timing": "CUDA events around the solve phase of each captured step "
                             "(the learned guess included)",
                   "train_widths": args.train_widths, "train_pairs": n_pairs, "runs": args.runs,
                   "train_steps": n_steps, "batch": args.batch, "data_s": t_data,
                   "train_s": t_train, "init": "library He initialisation (pic_unet_init)"},
        "ms_per_solve": res,
        "pcg_iterations_per_solve": its,
        "initial_rel_residual_geomean": rel0,
        "network_relative_mse": {"training_pairs": train_err, "held_out_pairs": held_err},
        "speedup_vs_zero": res["zero"] / res["learned"],
        "speedup_vs_lift": res["lift"] / res["learned"],
        "speedup_vs_previous": res["previous"] / res["learned"],
        "wall_s": time.perf_counter() - t0,
    }
    print(json.dumps(line), flush=True)
    net.close()
    eval_net.close()
    return 0


def unet_flops(H, W, B=1):
    """FLOPs of one forward pass of the warm-start U-Net at H x W: the 3x3
    convolutions (2 x 9 x cin x cout per output pixel), the transposed 2x2
    convolutions (2 x cin x cout per output pixel) and the head."""
    C = (32, 64, 128, 256)
    f = 0.0
    cin = 2                         # the input's two channels (rho / s and the mask)
    for l in range(4):
        px = B * (H >> l) * (W >> l)
        f += 2 * 9 * px * (cin * C[l] + C[l] * C[l])
        cin = C[l]
    for l in (2, 1, 0):
        px = B * (H >> l) * (W >> l)
        f += 2 * px * C[l + 1] * C[l] + 2 * 9 * px * (2 * C[l] * C[l] + C[l] * C[l])
    return f + 2 * B * H * W * C[0]


def run_unet(args):
    """Forward and training-step time of the warm-start U-Net at the trench
    grid (1032 x 512, batch 1 for inference), on the tcgen05 convolutions and
    on the mma.sync ones, CUDA events over repeated calls on the net's stream."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_03918_gb300 as pg
    H, W = 1032, 512
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"] \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1900.0
    out = {}
    for name, impl in (("tcgen05", 0), ("mma_sync", 1)):
        res = {}
        for B, what in ((1, "forward"), (args.batch, "train_step")):
            net = pg.Unet(B, H, W)
            net.set_conv_impl(impl)
            net.init(seed=0)
            x = torch.randn((B, H, W, 2), device="cuda")
            t = torch.randn((B, H, W), device="cuda")
            fn = (lambda: net.forward(x)) if what == "forward" else (lambda: net.train_step(x, t, 1e-4))
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(net.stream)
            for _ in range(args.steps):
                fn()
            e1.record(net.stream)
            torch.cuda.synchronize()
            assert net.status() == pg.PIC_OK
            ms = e0.elapsed_time(e1) / args.steps
            fl = unet_flops(H, W, B) * (1 if what == "forward" else 3)
            res[what] = {"ms": ms, "batch": B, "tflops": fl / (ms * 1e-3) / 1e12,
                         "frac_of_bf16_peak": fl / (ms * 1e-3) / 1e12 / peak}
            net.close()
        out[name] = res
    line = {"metric": "warm-start U-Net forward ms (1032 x 512 trench grid)",
            "value": out["tcgen05"]["forward"]["ms"], "unit": "ms", "higher_is_better": False,
            "n_gpus": 1, "steps": args.steps, "warmup": 3, "dtype": "bf16 (fp32 accumulate)",
            "data": "synthetic", "vs_baseline": None,
            "config": {"workload": "unet_4level_32ch_1032x512", "forward_flop": unet_flops(H, W),
                       "train_step_flop": "3 x forward per sample (forward, data and weight gradients)"},
            "roofline": {"bound": "tensor", "achieved": out["tcgen05"]["forward"]["tflops"],
                         "peak": peak, "unit": "TFLOP/s",
                         "frac": out["tcgen05"]["forward"]["tflops"] / peak, "traffic": None,
                         "peak_kind": "measured bf16 burst"},
            "by_kernel": out}
    print(json.dumps(line), flush=True)
    return 0


# The paper's tallies (Sec. III-C, III-D): ions reaching the trench bottom and
# the two sidewalls in the window, and their ratio sidewalls / bottom (the
# paper's printed ratios 2.31, 1.85 and 3.49; the printed counts give 2.30,
# 1.87 and 3.49).
PAPER_TALLIES = {"w15": (2137, 4920, 6000), "w4": (831, 1558, 6000), "w15_buildup": (1094, 3820, 7000)}


def run_paper(args):
    """The paper's own trench runs (80 x 30, widths 15 and 4, and width 15
    with the fixed test-ion density n_i = 5 on the row above the bottom; RF
    electrode, m_i / m_e = 3672, T_i = T_e, ions recycled in the bulk,
    t <= 1000), several seeds each, as one ensemble; the bottom and
    sidewall ion tallies in the paper's windows (600 <= t <= 1000, and
    700 <= t <= 1000 for the build-up run) beside the paper's counts."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_03918_gb300 as pg
    t0 = time.perf_counter()
    cases = list(PAPER_TALLIES)
    ws_, tags = [], []
    for case in cases:
        for seed in range(1, args.paper_seeds + 1):
            ws_.append(synth.paper_trench(4 if case == "w4" else 15, seed=seed, sort_every=8))
            tags.append(case)
    caps = [int(synth.plasma_cells(w).sum()) * w.ppc + 64 for w in ws_]
    batch = pg.Batch(ws_, capacities=caps, hit_capacity=16)
    for m, w, tag in zip(batch.members, ws_, tags):
        for s in (0, 1):
            m.load_particles(s, synth.maxwellian_load(w, s), v_at_t0=True)
        if tag == "w15_buildup":
            m.set_rho_ext(synth.paper_buildup_density(w))
    marks = {}
    done = 0
    for at in sorted({v[2] for v in PAPER_TALLIES.values()} | {10000}):
        batch.step(at - done)
        done = at
        marks[at] = [m.counts()[0][1].copy() for m in batch.members]
    wall_s = time.perf_counter() - t0
    out = {}
    for case in cases:
        start = PAPER_TALLIES[case][2]
        ks = [k for k, t in enumerate(tags) if t == case]
        d = sum(marks[10000][k] - marks[start][k] for k in ks)
        bottom = int(d[pg.WALL_XMAX])
        side = int(d[pg.WALL_COND_PY] + d[pg.WALL_COND_MY])
        pb, ps, _ = PAPER_TALLIES[case]
        out[case] = {"bottom_per_run": bottom / len(ks), "sidewalls_per_run": side / len(ks),
                     "ratio_sidewalls_to_bottom": side / max(bottom, 1),
                     "paper": {"bottom": pb, "sidewalls": ps, "ratio": ps / pb},
                     "window_t": [start * 0.1, 1000.0], "seeds": len(ks)}
    line = {"metric": "ions reaching the trench bottom and sidewalls (paper Sec. III-C, III-D)",
            "value": out["w15"]["ratio_sidewalls_to_bottom"], "unit": "sidewalls / bottom",
            "higher_is_better": False, "n_gpus": 1, "steps": 10000, "warmup": 0, "dtype": "f32",
            "data": "synthetic", "vs_baseline": None,
            "config": {"workload": "paper_trench_80x30 (w15, w4, w15 + n_i = 5 build-up)",
                       "members": len(ws_), "ppc": 100, "mass_ratio": 3672, "tau": 1.0,
                       "rf": "5 sin(0.01 t)", "recycling": "ions, bulk rows 0 <= x < 60"},
            "tallies": out, "wall_s": wall_s}
    print(json.dumps(line), flush=True)
    batch.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 1000 for the trench step, 100 otherwise)")
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="trench",
                    choices=["trench", "ensemble", "warmstart", "paper", "unet"],
                    help="trench: the 512x1024 trench run; ensemble: the 48-run width sweep; "
                         "warmstart: Poisson time to 1e-6 with the learned initial guess")
    ap.add_argument("--train-widths", default="2,4,5,6,7,8,9,10,12,13,14,15,16,17,18,20")
    ap.add_argument("--eval-widths", default="3,11,19")
    ap.add_argument("--pairs", type=int, default=2000, help="training pairs (warmstart)")
    ap.add_argument("--runs", type=int, default=10, help="training runs the pairs come from")
    ap.add_argument("--dump-every", type=int, default=10, help="steps between dumped pairs")
    ap.add_argument("--settle", type=int, default=100, help="steps before dumping / timing")
    ap.add_argument("--ring", type=int, default=256, help="pairs held for shuffled minibatches")
    ap.add_argument("--batch", type=int, default=4, help="training minibatch")
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--members", type=int, default=48, help="ensemble members")
    ap.add_argument("--paper-seeds", type=int, default=4, help="seeds per case (paper workload)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cold-steps", type=int, default=50, help="captured steps timed with a cold start")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the U-Net forward and the ensemble cut in the trench line")
    ap.add_argument("--ensemble-members", type=int, default=16)
    ap.add_argument("--ensemble-steps", type=int, default=100)
    ap.add_argument("--ppc", type=int, default=None, help="override particles per cell")
    ap.add_argument("--poisson-method", default="auto", choices=["auto", "multigrid"],
                    help="inner Poisson solver: auto (direct where the box allows) or multigrid PCG")
    ap.add_argument("--sort-every", type=int, default=0,
                    help="steps between tile sorts; 0 (default): the library times and picks it "
                         "during the warm-up")
    ap.add_argument("--warm-start", type=int, default=1,
                    help="Poisson initial guess: 0 zero, 1 previous, 2 extrapolated, 4 lift")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the 16x16 tile variant instead of the library's autotuner's choice")
    ap.add_argument("--autotune-steps", type=int, default=16,
                    help="particle steps timed per tile variant by the autotuner")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch the step's kernels from the host loop (for kernel profilers)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 1000 if (args.workload == "trench" and args.impl == "ours") else 100
    if args.impl == "reference":
        return run_reference(args)
    args.warmup = max(args.warmup, 3)
    if args.workload == "ensemble":
        return run_ensemble(args)
    if args.workload == "warmstart":
        return run_warmstart(args)
    if args.workload == "paper":
        return run_paper(args)
    if args.workload == "unet":
        return run_unet(args)

    dist, rank, ws = _dist()
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    import __graft_entry__
    if rank == 0 or dist is None:
        __graft_entry__.build()
    _barrier(dist)
    import paper_1610_03918_gb300 as pg

    w = synth.trench_512x1024(seed=3 + rank)
    if args.ppc:
        w = w.replace(ppc=args.ppc)
    if args.sort_every is not None:
        w = w.replace(sort_every=args.sort_every)
    parts = [synth.maxwellian_load(w, s) for s in (0, 1)]
    n0 = sum(len(p) for p in parts)
    sim = pg.Sim(w, capacity=len(parts[0]), device=local, timing=False, graphs=not args.no_graphs,
                 warm_start=args.warm_start, poisson_method=_poisson_method(pg, args))
    for s in (0, 1):
        sim.load_particles(s, parts[s], v_at_t0=True)
    sim.step(args.warmup)
    warm = args.warmup
    # the tile variant chosen by the library's autotuner on this run (each
    # variant's particle kernel timed right after a sort into its tiles)
    tile_tune = None
    if not args.no_autotune:
        import shutil
        import tempfile
        tdir = tempfile.mkdtemp(prefix="picgb_tiles_")
        try:
            cache = os.path.join(tdir, "tiles.json")
            chosen = sim.autotune(steps=args.autotune_steps, cache=cache)
            with open(cache) as f:
                entry = json.load(f)[0]
            tile_tune = {"particle_ms_per_variant": entry["particle_ms"], "chosen": chosen,
                         "steps_per_variant": args.autotune_steps}
        finally:
            shutil.rmtree(tdir, ignore_errors=True)
        warm += 4 * (args.autotune_steps + 1)
    tile = sim.tile()
    while sim.sort_interval()[0] == 0:    # a tuned sort interval is chosen before timing starts
        sim.step(8)
        warm += 8
    sort_interval, sort_tuned = sim.sort_interval()
    sim.timing()
    live0 = int(sim.counts()[1].sum())

    clocks = ClockSampler(local)
    clocks.start()
    _barrier(dist)
    stream = sim.torch_stream
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if stream is not None:
        ev0.record(stream)
    else:
        ev0.record()
    sim.step(args.steps)
    if stream is not None:
        ev1.record(stream)
    else:
        ev1.record()
    torch.cuda.synchronize()
    _barrier(dist)
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    launches = int(sim.timing()["launches"])
    live1 = int(sim.counts()[1].sum())
    pstats = sim.poisson_stats()

    # phase pass: the same number of steps again with event nodes between the
    # phases (they end the programmatic overlap across each phase boundary,
    # so the headline steps above run without them); the particle kernel's
    # live duration for the roofline comes from its events here
    sim.set_timing(True)
    sim.step(args.warmup)
    sim.timing()
    livep0 = int(sim.counts()[1].sum())
    e0p = torch.cuda.Event(enable_timing=True)
    e1p = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0p.record(stream) if stream is not None else e0p.record()
    sim.step(args.steps)
    e1p.record(stream) if stream is not None else e1p.record()
    torch.cuda.synchronize()
    tm_ms = e0p.elapsed_time(e1p) / args.steps
    tm = sim.timing()
    livep1 = int(sim.counts()[1].sum())

    # Poisson time to 1e-6 from the zero guess (cold start), in the captured
    # step on the same run: the solve phase's CUDA events, direct inner solve
    sim.set_warm_start(0)
    sim.step(3)
    sim.timing()
    sim.step(args.cold_steps)
    tcold = sim.timing()
    cold_direct = tcold["ms_poisson"] / max(tcold["steps"], 1)
    sim.set_warm_start(args.warm_start)
    sim.set_timing(False)
    # ... and with the multigrid-preconditioned CG inner solve: a context of
    # the same geometry holding this run's charge density as a fixed external
    # density (no particles), each captured step solving from zero
    rho_now = sim.rho()
    mg = pg.Sim(w, capacity=16, device=local, timing=True, warm_start=0,
                poisson_method=pg.POISSON_MULTIGRID, graphs=not args.no_graphs)
    mg.set_rho_ext(rho_now)
    mg.step(3)
    mg.timing()
    mg.step(args.cold_steps)
    tmg = mg.timing()
    cold_mg = tmg["ms_poisson"] / max(tmg["steps"], 1)
    mg_iters = mg.poisson_stats()[0]
    mg.close()

    live_mean = 0.5 * (live0 + live1)
    ps_local = live_mean * args.steps
    ms_max = _reduce_max(dist, ms)
    ps_total = _reduce_sum(dist, ps_local)
    value = ps_total / (ms_max * 1e-3)

    # roofline of the dominant kernel (fused gather/push/absorb/deposit)
    peak, peak_kind = _peaks()
    part_ms = tm["ms_particles"] / max(tm["steps"], 1)
    achieved = BYTES_PER_PARTICLE_STEP * 0.5 * (livep0 + livep1) / (part_ms * 1e-3) / 1e9
    traffic = None   # captured for the 16x16 variant's kernel
    if (NCU_TRAFFIC["source_sha256"] == _kernel_sha() and NCU_TRAFFIC["bytes_per_particle"]
            and tile[0] == 0):
        traffic = NCU_TRAFFIC["bytes_per_particle"] * live_mean

    # end to end through the C ABI with pinned host buffers: every step loads
    # the full state from the host, advances one step, reads the energies back
    e2e = None
    if args.e2e_steps > 0:
        st = [sim.state(s) for s in (0, 1)]
        pinned = []
        h2d = 0
        for s in (0, 1):
            n = st[s].shape[1]
            bufs = [torch.empty(n, dtype=torch.float64, pin_memory=True).numpy() for _ in range(4)]
            for k in range(4):
                bufs[k][:] = st[s][k]
            ids = torch.empty(n, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
            ids[:] = st[s][4].astype(np.uint32)
            pinned.append((bufs, ids))
            h2d += n * (4 * 8 + 4)
        out = torch.empty(4, dtype=torch.float64, pin_memory=True).numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            for s in (0, 1):
                bufs, ids = pinned[s]
                sim.load(s, bufs[0], bufs[1], bufs[2], bufs[3], ids)
            sim.step(1)
            sim.diag(pg.PIC_DIAG_ENERGY, out)
        t_e2e = time.perf_counter() - t0
        n_state = sum(p[0][0].size for p in pinned)
        e2e_val = _reduce_sum(dist, n_state * args.e2e_steps) / _reduce_max(dist, t_e2e)
        e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": 32,
               "note": "per step: pic_load of the full state from pinned host memory "
                       "(which re-deposits and re-solves), pic_step(1), pic_diag(ENERGY)"}
        # the same with the whole particle state read back to the host every
        # step, into pinned buffers the export kernel writes directly
        outs = [torch.empty(5 * p[0][0].size, dtype=torch.float64, pin_memory=True).numpy()
                for p in pinned]
        d2h = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            for s in (0, 1):
                bufs, ids = pinned[s]
                sim.load(s, bufs[0], bufs[1], bufs[2], bufs[3], ids)
            sim.step(1)
            d2h = 0
            for s in (0, 1):
                d2h += sim.state(s, out=outs[s]).nbytes
        t_full = time.perf_counter() - t0
        e2e_full = {"value": _reduce_sum(dist, n_state * args.e2e_steps) / _reduce_max(dist, t_full),
                    "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "note": "per step: pic_load of the full state from pinned host memory, "
                            "pic_step(1), pic_diag(STATE) of both species (x, y, vx, vy, id as FP64) "
                            "into pinned host buffers"}

    # the warm-start network's forward pass at this grid (tcgen05 convolutions)
    # and a cut of the trench-width ensemble, measured in the same run
    unet = ens = None
    if rank == 0 and not args.no_extras:
        net = pg.Unet(1, 1032, 512)
        net.init(seed=0)
        xin = torch.randn((1, 1032, 512, 2), device="cuda")
        for _ in range(3):
            net.forward(xin)
        torch.cuda.synchronize()
        e0u = torch.cuda.Event(enable_timing=True)
        e1u = torch.cuda.Event(enable_timing=True)
        e0u.record(net.stream)
        for _ in range(20):
            net.forward(xin)
        e1u.record(net.stream)
        torch.cuda.synchronize()
        ums = e0u.elapsed_time(e1u) / 20
        bf16_peak = 1900.0
        pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
        if os.path.exists(pp):
            bf16_peak = float(json.load(open(pp))["bf16_tflops"])
        ufl = unet_flops(1032, 512)
        unet = {"forward_ms": ums, "tflops": ufl / (ums * 1e-3) / 1e12,
                "frac_of_bf16_peak": ufl / (ums * 1e-3) / 1e12 / bf16_peak,
                "note": "4-level BF16 U-Net at 1032 x 512, tcgen05 convolutions, CUDA events; "
                        "bench.py --workload unet / warmstart for the full figures"}
        net.close()
        del xin
        ens = ensemble_cut(pg, local, args.ensemble_members, args.ensemble_steps)

    cpu = errs = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = oracle_baseline(synth.trench_512x1024())
        errs = errors_vs_oracle(pg)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "ppc": w.ppc,
                       "particles_loaded": n0, "live_particles": live_mean,
                       "sort_every": (f"tuned by the library: {sort_interval}" if sort_tuned
                                      else sort_interval),
                       "tile": {"variant": tile[0], "cells": [tile[1], tile[2]], "halo": tile[3],
                                "threads": tile[4],
                                "chosen_by": ("pic_autotune" if tile_tune else "fixed (--no-autotune)"),
                                "autotune": tile_tune},
                       "warmup_steps_run": warm, "poisson_rtol": w.poisson_rtol,
                       "warm_start": {0: "zero", 1: "previous", 2: "extrapolated",
                                      4: "lift"}[args.warm_start],
                       "poisson_inner_solver": "direct" if sim.solver() == pg.POISSON_AUTO else "multigrid PCG",
                       "l2": "inputs larger than L2 (particle state %.1f GB)" % (n0 * 24 / 1e9),
                       "timing": "value: the timed steps run without phase events; phases and the "
                                 "roofline's kernel time: CUDA events between the phases over a "
                                 "second pass of the same number of steps",
                       "parallelism": f"replicas{ws}" if ws > 1 else "single"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": f"k_particles<0, {tile[0]}> (gather+push+absorb+deposit)",
                         "peak_kind": peak_kind, "bytes_per_particle_step": BYTES_PER_PARTICLE_STEP},
            "phases_ms_per_step": {
                "particles": part_ms,
                "sort": tm["ms_sort"] / max(tm["steps"], 1),
                "poisson": tm["ms_poisson"] / max(tm["steps"], 1),
                "rho": tm["ms_rho"] / max(tm["steps"], 1),
            },
            "poisson_ms_to_1e-6": tm["ms_poisson"] / max(tm["steps"], 1),
            "poisson_ms_to_1e-6_by_start": {
                "previous_step": tm["ms_poisson"] / max(tm["steps"], 1),
                "zero_direct": cold_direct,
                "zero_multigrid_pcg": cold_mg,
                "multigrid_pcg_iterations_from_zero": mg_iters,
                "note": "CUDA events around the solve phase of captured steps (E included); "
                        "zero: cold start each step"},
            "poisson_last": {"iterations": pstats[0], "outer": pstats[1], "rel_residual": pstats[2]},
            "gpu_launches": launches,
            "ms_per_step_with_phase_events": tm_ms,
            "clocks": clk,
            "e2e": e2e,
            "e2e_full_state": e2e_full if args.e2e_steps > 0 else None,
            "cpu_baseline": cpu,
            "errors_vs_oracle": errs,
            "unet_forward": unet,
            "ensemble": ens,
        }
        print(json.dumps(line), flush=True)
    sim.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
