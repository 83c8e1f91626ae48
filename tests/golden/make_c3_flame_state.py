"""Writes c3_flame_n64_20steps.txt: the FP64 oracle's state after 20 SDC
steps (Sec. 3.1, eq. expsdc: 3 Gauss-Lobatto nodes, 4 sweeps) of the planar
flame configuration (9 species / 21 reactions, tanh temperature profile
300-2000 K, 3% velocity perturbations) on a 64^3 periodic box with the
256^3 configuration's spacing (h = 1/256 cm) and time step, at 160 seeded
sample cells, with each component's maxima over the whole box.

Calls only the oracle (and the seeded input generators).  Run from the
repository root:  python tests/golden/make_c3_flame_state.py
(about 20 minutes on one host core).
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import rhs as orhs  # noqa: E402
from oracle import sdc as osdc  # noqa: E402
from oracle import thermo  # noqa: E402
from paper_1309_7327_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c3_flame_n64_20steps.txt")
SEED, N, STEPS, NCELLS = 1, 64, 20, 160


def main():
    wl = synth.workload("c3", seed=SEED, n=N)
    g = wl.grid
    prim = synth.boxes_to_global(g, wl.prim)
    U0 = thermo.conserved(prim, wl.mech.nasa7, wl.mech.W)

    def f(u, t=0.0):
        return orhs.rhs_periodic(u, wl.mech, g.dx)

    t0 = time.time()
    u, F = U0, None
    for s in range(STEPS):
        u, F, _ = osdc.sdc_step(u, f, wl.dt, nodes=wl.nodes, sweeps=wl.sweeps, F0=F)
        print(f"step {s + 1}/{STEPS} {time.time() - t0:.0f} s", flush=True)
    rng = np.random.default_rng(2024)
    cells = np.stack([rng.integers(0, N, NCELLS) for _ in range(3)], axis=1)   # z, y, x
    nv = U0.shape[0]
    inc_max = np.abs(u - U0).reshape(nv, -1).max(axis=1)
    u_max = np.abs(u).reshape(nv, -1).max(axis=1)
    with open(OUT, "w") as fh:
        fh.write("# FP64 oracle state after 20 SDC steps (Sec. 3.1, eq. expsdc; 3 Gauss-Lobatto\n")
        fh.write("# nodes, 4 sweeps) of the planar-flame configuration, 9 species / 21\n")
        fh.write(f"# reactions, seed {SEED}, {N}^3 periodic cells of h = 1/256 cm, dt = {wl.dt!r}.\n")
        fh.write("# Written by tests/golden/make_c3_flame_state.py (oracle only).\n")
        fh.write("# inc_max: per component max over all cells of |U_20 - U_0|\n")
        fh.write("inc_max " + " ".join(repr(float(v)) for v in inc_max) + "\n")
        fh.write("# u_max: per component max over all cells of |U_20|\n")
        fh.write("u_max " + " ".join(repr(float(v)) for v in u_max) + "\n")
        fh.write("# cell z y x, then U_20 at that cell (rho, rho u, rho v, rho w, rho E, rho Y_k)\n")
        for z, y, x in cells:
            fh.write(f"cell {z} {y} {x} " + " ".join(repr(float(v)) for v in u[:, z, y, x]) + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
