"""The appendix heat-equation problems T1 and T2 (App. A).  Oracle, test
infrastructure only.

u_t = (a u_x)_x + (b u_y)_y + g on the periodic square [0, 2 pi]^2, both
second-derivative terms by the narrow stencil (eqs. DaDu/H), time by SDC with
3 Gauss-Lobatto nodes and 4 sweeps (Sec. 3.1) to t = 1.

Readings (the paper is silent on them):
* grid points x_i = 2 pi i / N, i = 0..N-1;
* dt_0 = 0.4 / ((dx^-2 + dy^-2) max(a, b)) with the max over the grid, then
  n = ceil(1 / dt_0) steps of dt = 1/n so that t = 1 is hit exactly.
"""
from __future__ import annotations

import math

import numpy as np

from . import sdc, stencil

EPS_T1 = 0.1
EPS_T2 = 0.9


def _grid(N):
    x = 2.0 * math.pi * np.arange(N) / N
    Yg, Xg = np.meshgrid(x, x, indexing="ij")
    return Xg, Yg, 2.0 * math.pi / N


def t1_coeffs(N):
    X, Y, h = _grid(N)
    a = 1.0 + EPS_T1 * np.cos(X) * np.cos(Y)
    return X, Y, h, a, a.copy()


def t2_coeffs(N):
    X, Y, h = _grid(N)
    a = 1.0 + EPS_T2 * np.cos(2 * X) * np.sin(2 * Y + math.pi / 3)
    b = 1.0 + EPS_T2 * np.cos(2 * X + math.pi / 3) * np.sin(2 * Y)
    return X, Y, h, a, b


def operator(a, b, h, M):
    """u -> (a u_x)_x + (b u_y)_y on the periodic grid (axis 1 = x, axis 0 = y)."""
    ap = np.pad(a, 4, mode="wrap")
    bp = np.pad(b, 4, mode="wrap")

    def L(u):
        up = np.pad(u, 4, mode="wrap")
        lx = stencil.narrow(ap[4:-4, :], up[4:-4, :], 1, h, M)
        ly = stencil.narrow(bp[:, 4:-4], up[:, 4:-4], 0, h, M)
        return lx + ly
    return L


def time_step(a, b, h):
    dt0 = 0.4 / ((2.0 / h ** 2) * max(a.max(), b.max()))
    n = math.ceil(1.0 / dt0)
    return 1.0 / n, n


def solve(problem: str, N: int, m47=stencil.M47_SMC, m48=stencil.M48_SMC,
          t_end: float = 1.0, nsteps: int | None = None):
    """Integrate T1 or T2 to t_end; returns (u, exact-or-None, n_evals)."""
    M = stencil.to_float(stencil.narrow8_exact(m47, m48))
    if problem == "T1":
        X, Y, h, a, b = t1_coeffs(N)
        cc = np.cos(X) * np.cos(Y)
        ss = np.sin(X) * np.sin(Y)

        def g(t):
            return (1.0 + 4.0 * EPS_T1 * cc) * math.exp(-t) * ss
    else:
        X, Y, h, a, b = t2_coeffs(N)
        ss = np.sin(X) * np.sin(Y)

        def g(t):
            return 0.0
    L = operator(a, b, h, M)

    def f(u, t):
        return L(u) + g(t)

    dt, n = time_step(a, b, h)
    if nsteps is not None:
        n = nsteps
        dt = t_end / n
    u = ss.copy()
    F = None
    t = 0.0
    nev = 0
    for _ in range(n):
        u, F, k = sdc.sdc_step(u, f, dt, nodes=3, sweeps=4, F0=F, t0=t)
        nev += k
        t += dt
    exact = math.exp(-t) * ss if problem == "T1" else None
    return u, exact, nev


def errors(u, exact):
    d = u - exact
    return float(np.abs(d).max()), float(np.sqrt(np.mean(d ** 2)))
