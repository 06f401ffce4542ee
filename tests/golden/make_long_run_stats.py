"""Writes the oracle side of the long-run statistical parity tests
(tests/test_gpu_long_run.py).  Calls only oracle/ and synth/.

  python tests/golden/make_long_run_stats.py [--procs N]

1. Ion impact angles on the trench bottom (the paper's Sec. III-C, Fig. 5b:
   velocity distribution of the ions reaching the bottom).  Reduced trench
   (48 y-cells periodic x 64 x-cells, electrode slab 16 cells deep at -20
   T_e/e, trench 10 cells wide), 32 particles per cell per species, ions
   recycled into the bulk rows (Sec. III-A), no surface-charge feedback,
   16 seeds x 3000 steps.  For every ion absorbed on the bottom face (wall 1)
   at step >= 500 the angle theta = atan(|v_y| / v_x) of its velocity is
   binned into 2000 equal bins on [0, pi/2].  Output: ion_bottom_angles.txt.
2. Field-energy history of the 64 x 64 doubly periodic box (50 particles
   per cell per species, 500 steps) for 4 seeds: FE after each step.
   Output: field_energy_periodic64.txt.
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

ANGLE_BINS = 2000
ANGLE_SETTLE = 500
ANGLE_STEPS = 3000
ANGLE_SEEDS = list(range(101, 117))
FE_SEEDS = [1, 2, 3, 4]
FE_STEPS = 500


def angle_workload(seed):
    import synth
    return synth.small_trench(nx=64, ny=48, depth=16, width=10, ppc=32, seed=seed).replace(
        surface_charge=False, recycle=True, recycle_seed=seed, name="angle_trench_48x64_w10_d16_ppc32")


def fe_workload(seed):
    import synth
    return synth.periodic_square_64(seed=seed)


def run_angles(seed):
    import synth
    from oracle.sim import Sim
    w = angle_workload(seed)
    s = Sim(w)
    for sp in (0, 1):
        s.load_particles(sp, synth.maxwellian_load(w, sp), v_at_t0=True)
    s.step(ANGLE_STEPS)
    h = s.hit_table()
    m = (h["species"] == 1) & (h["wall"] == 1) & (h["step"] >= ANGLE_SETTLE)
    theta = np.arctan2(np.abs(h["vy"][m]), h["vx"][m])
    return np.histogram(theta, bins=ANGLE_BINS, range=(0.0, np.pi / 2))[0]


def run_fe(seed):
    import synth
    from oracle.sim import Sim
    w = fe_workload(seed)
    s = Sim(w)
    for sp in (0, 1):
        s.load_particles(sp, synth.maxwellian_load(w, sp), v_at_t0=True)
    fe = []
    for _ in range(FE_STEPS):
        s.step(1)
        fe.append(s.fe)
    return np.array(fe)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=os.cpu_count())
    args = ap.parse_args()
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.procs) as pool:
        fe_async = pool.map_async(run_fe, FE_SEEDS)
        hists = pool.map(run_angles, ANGLE_SEEDS)
        fes = fe_async.get()
    hist = np.sum(hists, axis=0)
    with open(os.path.join(HERE, "ion_bottom_angles.txt"), "w") as f:
        f.write("# Oracle: angles theta = atan(|v_y| / v_x) of ions absorbed on the trench bottom\n")
        f.write("# (Sec. III-C, Fig. 5b), written by tests/golden/make_long_run_stats.py\n")
        f.write(f"# workload {angle_workload(0).name}: 64 x-cells x 48 y-cells (periodic), slab 16 deep,\n")
        f.write("# trench 10 wide, -20 T_e/e, 32 ppc/species, ions recycled, no surface charge\n")
        f.write(f"# seeds {ANGLE_SEEDS[0]}..{ANGLE_SEEDS[-1]}, {ANGLE_STEPS} steps, hits at step >= {ANGLE_SETTLE}\n")
        f.write(f"# {ANGLE_BINS} equal bins on [0, pi/2]; total {int(hist.sum())} hits\n")
        for c in hist:
            f.write(f"{int(c)}\n")
    with open(os.path.join(HERE, "field_energy_periodic64.txt"), "w") as f:
        f.write("# Oracle: field energy FE = 1/2 sum |E|^2 after each step, 64 x 64 doubly periodic box,\n")
        f.write("# 50 ppc/species, Maxwellian load (v_e = 1, T_i / T_e = 0.1, m_i / m_e = 1836),\n")
        f.write(f"# written by tests/golden/make_long_run_stats.py; one column per seed {FE_SEEDS}\n")
        for k in range(FE_STEPS):
            f.write(" ".join(f"{fe[k]:.10e}" for fe in fes) + "\n")
    print("ion bottom hits:", int(hist.sum()))


if __name__ == "__main__":
    main()
