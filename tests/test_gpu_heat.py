"""The appendix heat problems (App. A) through smc_heat2d: the GPU solution
equals the oracle's to rounding, and its T1 errors reproduce the paper's
Table stenciltest1."""
import math
import os

import numpy as np
import pytest

from oracle import heat2d, stencil
from paper_1309_7327_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
STENCILS = {"SMC": (stencil.M47_SMC, stencil.M48_SMC),
            "ZERO": (stencil.M47_ZERO, stencil.M48_ZERO),
            "OPTIMAL": (stencil.M47_OPT, stencil.M48_OPT)}


@pytest.fixture(scope="module")
def smc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1309_7327_gb300 import smc as S
    return S


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to("cuda:0")


def gpu_solve(S, problem, N, name="SMC", nsteps=None, t_end=1.0):
    f = synth.heat_fields(problem, N)
    dt, n = heat2d.time_step(f["a"], f["b"], f["h"])
    if nsteps is not None:
        n, dt = nsteps, t_end / nsteps
    u = dev(f["u0"])
    G = dev(f["G"]) if f["G"] is not None else None
    nev = S.smc_heat2d(N, f["h"], dev(f["a"]), dev(f["b"]), G, u, 0.0, dt, n, *STENCILS[name])
    return u.cpu().numpy(), nev, n


def golden():
    out = {}
    for l in open(os.path.join(GOLDEN, "stenciltest1.txt")):
        if l.strip() and not l.startswith("#"):
            s, n, li, l2 = l.split()
            out[(s, int(n))] = (float(li), float(l2))
    return out


@pytest.mark.parametrize("name", ["SMC", "ZERO", "OPTIMAL"])
@pytest.mark.parametrize("N", [20, 40])
def test_heat_T1_matches_oracle_and_paper(smc, name, N):
    u, nev, n = gpu_solve(smc, "T1", N, name)
    ref, exact, nev_o = heat2d.solve("T1", N, *STENCILS[name])
    assert nev == nev_o == 1 + 8 * n
    assert np.abs(u - ref).max() <= 1e-12 * np.abs(ref).max()
    g = golden()[(name, N)]
    linf, l2 = heat2d.errors(u, exact)
    assert abs(linf / g[0] - 1) < 0.01 and abs(l2 / g[1] - 1) < 0.01, (linf, l2, g)


def test_heat_T1_80_eighth_order(smc):
    u, _, _ = gpu_solve(smc, "T1", 80)
    exact = math.exp(-1.0) * synth.heat_fields("T1", 80)["u0"]
    linf = np.abs(u - exact).max()
    g = golden()
    assert abs(linf / g[("SMC", 80)][0] - 1) < 0.05
    assert 7.8 < math.log2(g[("SMC", 40)][0] / linf) < 8.2


def test_heat_T2_matches_oracle(smc):
    """T2 (strongly varying a, b) to t = 0.2 at the stable step of the
    paper's rule."""
    f = synth.heat_fields("T2", 32)
    dt, _ = heat2d.time_step(f["a"], f["b"], f["h"])
    n = math.ceil(0.2 / dt)
    u, nev, _ = gpu_solve(smc, "T2", 32, nsteps=n, t_end=0.2)
    ref, _, nev_o = heat2d.solve("T2", 32, t_end=0.2, nsteps=n)
    assert np.abs(ref).max() < 1.0
    assert nev == nev_o
    assert np.abs(u - ref).max() <= 1e-12 * np.abs(ref).max()


def test_heat_rejects_bad_arguments(smc):
    f = synth.heat_fields("T2", 16)
    a, u = dev(f["a"]), dev(f["u0"])
    a4, u4 = a.flatten()[:16].contiguous(), u.flatten()[:16].contiguous()
    with pytest.raises(smc.SmcError):
        smc.smc_heat2d(4, f["h"], a4, a4, None, u4, 0.0, 0.1, 1)       # N < 8
    with pytest.raises(ValueError):
        smc.smc_heat2d(8, f["h"], a, a, None, u, 0.0, 0.1, 1)          # arrays of another size
    with pytest.raises(smc.SmcError):
        smc.smc_heat2d(16, f["h"], a.cpu(), a, None, u, 0.0, 0.1, 1)   # host array
    assert smc.smc_heat2d(16, f["h"], a, a, None, u, 0.0, 0.1, 0) == 1  # no steps: F(U_0) only
