"""Full-size configurations in the launch configuration the benchmark uses,
checked at sampled cells that the oracle evaluates one by one in extended
precision (np.longdouble): FP64 to 1e-12 or three times the FP64
conditioning floor of the component (see test_gpu_rhs), mixed precision to
1e-5.  Covers the 256^3 flame (c3), the 64-box 21-species batch (c4) in
mixed precision, and the 512x256x256 box with non-periodic x ends (c5),
including cells next to both x ends.  Also the state error of the mixed
path after 20 SDC steps of the flame configuration on a 16^3 box."""
import numpy as np
import pytest

from oracle import rhs as orhs
from oracle import sdc as osdc
from oracle import thermo
from paper_1309_7327_gb300 import synth

from util import relerr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12
TOL_MIXED = 1e-5


@pytest.fixture(scope="module")
def smc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1309_7327_gb300 import smc as S
    return S


def conserved(wl):
    prim_g = synth.boxes_to_global(wl.grid, wl.prim)
    return thermo.conserved(prim_g, wl.mech.nasa7, wl.mech.W)


def gpu_rhs(S, wl, U, precision):
    with S.Smc(wl.grid, wl.mech, {"precision": precision}, x_outflow=wl.x_outflow) as h:
        Ud = torch.from_numpy(U).to("cuda:0")
        Fd = torch.empty_like(Ud)
        h.rhs(Ud, Fd)
        h.synchronize()
        return Fd.cpu().numpy()


def patch_at(U, z, y, x, outflow):
    """The ghosted neighbourhood that determines dU/dt at (z, y, x), the
    oracle options for it, and the cell's x index inside the patch.  Next to
    a non-periodic x end the patch spans the 16 cells of that end (the
    lowered stencils read no farther; the patch's other end is never read)."""
    nz, ny, nx = U.shape[1:]
    iz = np.arange(z - 4, z + 5) % nz
    iy = np.arange(y - 4, y + 5) % ny
    if outflow and x < 4:
        ix, xi = np.arange(-4, 20) % nx, x
    elif outflow and x >= nx - 4:
        ix, xi = np.arange(nx - 20, nx + 4) % nx, x - (nx - 16)
    else:
        ix, xi = np.arange(x - 4, x + 5) % nx, 0
    opt = orhs.Options(x_outflow=bool(outflow and (x < 4 or x >= nx - 4)))
    return U[:, iz][:, :, iy][:, :, :, ix], opt, xi


def oracle_cells(U_g, cells, mech, dx, outflow, trials=4):
    """Extended-precision RHS at the cells and the FP64 floor there: the
    larger of (a) its largest change over `trials` perturbations that move
    every input by one ulp (random signs) and (b) the FP64 oracle's own
    distance from it -- the rounding inside an FP64 evaluation (the Newton
    residual, p from T) moves the pressure at several ulps, which the
    one-sided stencils next to the x ends amplify in the momentum."""
    rng = np.random.default_rng(5)
    ref = np.empty((U_g.shape[0], len(cells)))
    dev = np.zeros_like(ref)
    for i, (z, y, x) in enumerate(cells):
        P, opt, xi = patch_at(U_g, z, y, x, outflow)
        r = orhs.rhs_ghosted(P.astype(np.longdouble), mech, dx, opt)[:, 0, 0, xi]
        ref[:, i] = r.astype(np.float64)
        r64 = orhs.rhs_ghosted(P, mech, dx, opt)[:, 0, 0, xi]
        dev[:, i] = np.abs(r64 - r.astype(np.float64))
        for _ in range(trials):
            s = rng.choice([-1.0, 1.0], size=P.shape)
            rp = orhs.rhs_ghosted((P * (1.0 + s * 2.0 ** -53)).astype(np.longdouble), mech, dx,
                                  opt)[:, 0, 0, xi]
            dev[:, i] = np.maximum(dev[:, i], np.abs((rp - r).astype(np.float64)))
    return ref, dev.max(axis=1)


def sample_cells(rng, grid, k, outflow):
    nx, ny, nz = grid.domain
    cells = [(0, 0, 0), (nz - 1, ny - 1, nx - 1)]
    if outflow:
        cells += [(3, 5, 2), (7, 1, 3), (nz - 2, 4, nx - 3), (1, ny - 3, nx - 4)]
    for _ in range(k):
        cells.append((int(rng.integers(nz)), int(rng.integers(ny)), int(rng.integers(nx))))
    return cells


@pytest.mark.parametrize("name,precisions", [("c2", (1,)), ("c3", (0, 1)), ("c4", (1,)),
                                              ("c5", (0, 1))])
def test_full_size_sampled_cells(smc, name, precisions):
    wl = synth.workload(name, seed=1)
    g = wl.grid
    U_g = conserved(wl)
    U = synth.global_to_boxes(g, U_g)
    cells = sample_cells(np.random.default_rng(0), g, 8, wl.x_outflow)
    ref, floor_abs = oracle_cells(U_g, cells, wl.mech, g.dx, wl.x_outflow)
    for prec in precisions:
        F = synth.boxes_to_global(g, gpu_rhs(smc, wl, U, prec))
        scale = np.abs(F).reshape(F.shape[0], -1).max(axis=1)
        got = np.stack([F[:, z, y, x] for z, y, x in cells], axis=1)
        err = np.abs(got - ref).max(axis=1) / scale
        print(f"{name} precision {prec}: max error {err.max():.2e}")
        if prec == 0:
            bar = np.maximum(TOL, 3.0 * floor_abs / scale)
            assert (err <= bar).all(), (err, floor_abs / scale)
        else:
            assert err.max() < TOL_MIXED, err


def test_mixed_state_after_20_steps_of_the_flame(smc):
    """The precision configuration (tanh flame, 9 species) on a 16^3 box:
    20 SDC steps (3 nodes, 4 sweeps) in mixed precision against the FP64
    oracle: the state and its increment over the 20 steps, per field, within
    the mixed tolerance (measured: increments <= 5.4e-7, states <= 4e-7 --
    the transverse momenta are small, so their state error is of the size of
    their increment error)."""
    wl = synth.workload("c3", seed=2, n=16)
    U_g = conserved(wl)
    U = synth.global_to_boxes(wl.grid, U_g)
    with smc.Smc(wl.grid, wl.mech, {"precision": 1}) as h:
        Ud = torch.from_numpy(U).to("cuda:0")
        for _ in range(20):
            h.sdc_step(Ud, wl.dt)
        h.synchronize()
        U20 = Ud.cpu().numpy()

    def f(u, t=0.0):
        return orhs.rhs_periodic(u, wl.mech, wl.grid.dx)
    u, F = U_g, None
    for _ in range(20):
        u, F, _ = osdc.sdc_step(u, f, wl.dt, F0=F)
    ref = synth.global_to_boxes(wl.grid, u)
    inc = relerr(U20 - U, ref - U)
    state = relerr(U20, ref)
    print("mixed 20-step increment error", np.array2string(inc, precision=2))
    print("mixed 20-step state error", np.array2string(state, precision=2))
    assert inc.max() < TOL_MIXED, inc
    assert state.max() < TOL_MIXED, state


def _golden_c3():
    """The oracle's state after 20 SDC steps of the flame configuration on a
    64^3 box (tests/golden/c3_flame_n64_20steps.txt, written by
    tests/golden/make_c3_flame_state.py from the oracle alone)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "c3_flame_n64_20steps.txt")
    cells, vals, inc_max, u_max = [], [], None, None
    for line in open(path):
        if line.startswith("inc_max "):
            inc_max = np.array([float(v) for v in line.split()[1:]])
        elif line.startswith("u_max "):
            u_max = np.array([float(v) for v in line.split()[1:]])
        elif line.startswith("cell "):
            parts = line.split()
            cells.append(tuple(int(v) for v in parts[1:4]))
            vals.append([float(v) for v in parts[4:]])
    return cells, np.array(vals).T, inc_max, u_max


@pytest.mark.parametrize("precision", [0, 1])
def test_flame_state_after_20_steps_on_64_cubed(smc, precision):
    """The precision configuration (planar tanh flame, 9 species / 21
    reactions, 3% velocity perturbations) on a 64^3 box of the 256^3 run's
    spacing and time step: 20 SDC steps (3 Gauss-Lobatto nodes, 4 sweeps)
    on the GPU against the FP64 oracle's 20-step state at 160 sampled cells.
    Errors per field relative to the field's largest 20-step change and to
    its largest value over the box.  FP64: within 1e-9 of the change (the
    single-step bar is 1e-10; twenty steps accumulate it).  Mixed: within
    1e-5 of the change."""
    cells, ref, inc_max, u_max = _golden_c3()
    wl = synth.workload("c3", seed=1, n=64)
    U_g = conserved(wl)
    U = synth.global_to_boxes(wl.grid, U_g)
    with smc.Smc(wl.grid, wl.mech, {"precision": precision}) as h:
        Ud = torch.from_numpy(U).to("cuda:0")
        for _ in range(20):
            h.sdc_step(Ud, wl.dt, wl.nodes, wl.sweeps, 0)
        h.synchronize()
        U20 = synth.boxes_to_global(wl.grid, Ud.cpu().numpy())
    got = np.stack([U20[:, z, y, x] for z, y, x in cells], axis=1)
    e_inc = np.abs(got - ref).max(axis=1) / inc_max
    e_state = np.abs(got - ref).max(axis=1) / u_max
    print(f"precision {precision}: 20-step error / change", np.array2string(e_inc, precision=2))
    print(f"precision {precision}: 20-step error / state", np.array2string(e_state, precision=2))
    if precision == 0:
        assert e_inc.max() < 1e-9, e_inc
    else:
        assert e_inc.max() < TOL_MIXED, e_inc
        assert e_state.max() < TOL_MIXED, e_state


def test_mixed_rhs_of_the_bump_at_full_size_every_cell(smc):
    """The 64^3 bump configuration (9 species), where one species' gradient
    and pressure-gradient diffusion fluxes are each several times its net flux
    and its face fluxes tens of times their divergence: the mixed right-hand
    side at every cell within 1e-5 of the FP64 one (itself held to the oracle
    at sampled cells by test_full_size_sampled_cells)."""
    wl = synth.workload("c2", seed=1)
    U = synth.global_to_boxes(wl.grid, conserved(wl))
    F64 = gpu_rhs(smc, wl, U, 0)
    Fm = gpu_rhs(smc, wl, U, 1)
    err = relerr(Fm, F64)
    print("c2 mixed vs FP64, every cell:", np.array2string(err, precision=2))
    assert err.max() < TOL_MIXED, err
