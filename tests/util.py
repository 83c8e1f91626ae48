"""Shared helpers of the test suite (inputs, oracle calls, error metrics)."""
import numpy as np

from oracle import rhs as orhs
from oracle import thermo
from paper_1309_7327_gb300 import synth


def state(name="c1", seed=1, n=None, p_amp=None):
    """(workload, U in box layout, U on the global grid) for a configuration."""
    wl = synth.workload(name, seed=seed, n=n)
    g = wl.grid
    prim_g = synth.boxes_to_global(g, wl.prim)
    if p_amp is not None:
        rng = np.random.default_rng(seed + 7)
        nx, ny, nz = g.domain
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        prim_g[4] *= 1.0 + p_amp * np.sin(2 * np.pi * x / nx + rng.uniform(0, 6)) \
            * np.cos(2 * np.pi * y / ny + rng.uniform(0, 6))
    U_g = thermo.conserved(prim_g, wl.mech.nasa7, wl.mech.W)
    return wl, synth.global_to_boxes(g, U_g), U_g


def oracle_rhs(wl, U_g, parts=False, **opt):
    o = orhs.Options(**opt)
    r = orhs.rhs_periodic(U_g, wl.mech, wl.grid.dx, o, parts=parts)
    if parts:
        return tuple(synth.global_to_boxes(wl.grid, x) for x in r)
    return synth.global_to_boxes(wl.grid, r)


def relerr(a, b):
    """Per-component max-norm relative error max|a - b| / max|b|."""
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    scale = np.abs(b).max(axis=1)
    scale = np.where(scale > 0, scale, 1.0)
    return np.abs(a - b).max(axis=1) / scale
