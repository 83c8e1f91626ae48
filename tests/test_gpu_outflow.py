"""Non-periodic x ends (boundary-lowered stencils, Sec. 2.2 boundary
paragraph) through the C ABI against the oracle's x_outflow right-hand
side: FP64 to 1e-12, mixed precision to 1e-5, single and multiple boxes,
both diffusion modes, and an SDC step."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def flame_box(n=(24, 12, 12), ns=9, nr=21, seed=3):
    """A hot slab across x (two tanh fronts) on one box, 9 species."""
    grid = synth.single_box(n, 1.0 / 256)
    mech = synth.make_mechanism(ns, nr, seed)
    prim = synth.flame_fields(grid, ns, seed + 100)
    U_g = thermo.conserved(prim, mech.nasa7, mech.W)
    return grid, mech, U_g


def oracle(grid, mech, U_g, **opt):
    return synth.global_to_boxes(grid, orhs.rhs_periodic(U_g, mech, grid.dx,
                                                         orhs.Options(x_outflow=True, **opt)))


def oracle_ld(grid, mech, U_g, **opt):
    """The x_outflow oracle in extended precision, and its FP64 conditioning
    floor: the change of the extended-precision RHS when every input moves
    by one unit in the last place (random sign), relative to the component's
    maximum.  The one-sided stencils at the end cells weigh values by up to
    18/6 and cancel them (their weights sum to zero), so an FP64 evaluation
    of the pressure gradient there rounds at ~1e-11 of the momentum RHS."""
    o = orhs.Options(x_outflow=True, **opt)
    ref = orhs.rhs_periodic(U_g.astype(np.longdouble), mech, grid.dx, o)
    r = np.random.default_rng(5).choice([-1.0, 1.0], size=U_g.shape)
    pert = orhs.rhs_periodic((U_g * (1.0 + r * 2.0 ** -53)).astype(np.longdouble), mech, grid.dx, o)
    scale = np.abs(ref).reshape(ref.shape[0], -1).max(axis=1).astype(np.float64)
    floor = np.abs((pert - ref).astype(np.float64)).reshape(ref.shape[0], -1).max(axis=1) / scale
    return synth.global_to_boxes(grid, ref.astype(np.float64)), floor


def gpu_rhs(S, grid, mech, U, **options):
    with S.Smc(grid, mech, options, x_outflow=True) as h:
        Ud = dev(U)
        F = torch.empty_like(Ud)
        h.rhs(Ud, F)
        h.synchronize()
        return F.cpu().numpy()


@pytest.mark.parametrize("mode", [0, 1])
def test_outflow_rhs_single_box_fp64(smc, mode):
    grid, mech, U_g = flame_box()
    U = synth.global_to_boxes(grid, U_g)
    got = gpu_rhs(smc, grid, mech, U, diffusion_mode=mode)
    ref, floor = oracle_ld(grid, mech, U_g, mode="vc" if mode == 0 else "ref")
    err = relerr(got, ref)
    print("outflow FP64 error", np.array2string(err, precision=2), "floor",
          np.array2string(floor, precision=2))
    assert (err <= np.maximum(TOL, 3.0 * floor)).all(), (err, floor)


def test_outflow_rhs_multibox_21_species_fp64_and_mixed(smc):
    """8 uneven boxes; the boxes at both x ends carry the lowered cells."""
    wl = synth.workload("c4", seed=3, n=12)
    prim_g = synth.boxes_to_global(wl.grid, wl.prim)
    U_g = thermo.conserved(prim_g, wl.mech.nasa7, wl.mech.W)
    U = synth.global_to_boxes(wl.grid, U_g)
    ref = oracle(wl.grid, wl.mech, U_g)
    for march in (0, 1):
        err = relerr(gpu_rhs(smc, wl.grid, wl.mech, U, march=march), ref)
        assert err.max() < TOL, (march, err)
    errm = relerr(gpu_rhs(smc, wl.grid, wl.mech, U, precision=1), ref)
    print("outflow mixed error", np.array2string(errm, precision=2))
    assert errm.max() < TOL_MIXED, errm


@pytest.mark.parametrize("march", [0, 1])
def test_outflow_rhs_mixed_single_box(smc, march):
    grid, mech, U_g = flame_box()
    U = synth.global_to_boxes(grid, U_g)
    err = relerr(gpu_rhs(smc, grid, mech, U, precision=1, march=march), oracle(grid, mech, U_g))
    assert err.max() < TOL_MIXED, err


def test_outflow_differs_from_periodic_only_near_the_x_ends(smc):
    grid, mech, U_g = flame_box()
    U = synth.global_to_boxes(grid, U_g)
    out = gpu_rhs(smc, grid, mech, U)
    with smc.Smc(grid, mech) as h:
        Ud = dev(U)
        F = torch.empty_like(Ud)
        h.rhs(Ud, F)
        h.synchronize()
        per = F.cpu().numpy()
    nx = grid.domain[0]
    o = out.reshape(out.shape[0], grid.domain[2], grid.domain[1], nx)
    p = per.reshape(o.shape)
    assert np.array_equal(o[..., 4:nx - 4], p[..., 4:nx - 4])
    assert np.abs(o[..., :4] - p[..., :4]).max() > 0


def test_outflow_sdc_step(smc):
    grid, mech, U_g = flame_box(n=(16, 8, 8), ns=3, nr=2, seed=5)
    U = synth.global_to_boxes(grid, U_g)
    dt = 2e-9
    with smc.Smc(grid, mech, x_outflow=True) as h:
        Ud = dev(U)
        h.sdc_step(Ud, dt)
        h.synchronize()
        U1 = Ud.cpu().numpy()
    f = lambda u, t=0.0: orhs.rhs_periodic(u, mech, grid.dx, orhs.Options(x_outflow=True))  # noqa: E731
    ref, _, _ = osdc.sdc_step(U_g, f, dt)
    ref = synth.global_to_boxes(grid, ref)
    err = relerr(U1 - U, ref - U)
    assert err.max() < 1e-10, err


def test_mode2_step_with_outflow_x_ends(smc):
    """MRSDC mode 2 (eq. mrupdate2) on a box with non-periodic x ends: the
    advection-diffusion evaluations use the lowered stencils, the implicit
    reaction integration is pointwise; against the oracle's mode-2 step."""
    from oracle import react
    grid, mech, U_g = flame_box(n=(16, 8, 8), ns=3, nr=2, seed=4)
    U = synth.global_to_boxes(grid, U_g)
    dt = 2e-9
    rtol, atol = 1e-10, 1e-14
    with smc.Smc(grid, mech, {"mr_mode": 2, "bdf_rtol": rtol, "bdf_atol": atol},
                 x_outflow=True) as h:
        Ud = dev(U)
        h.sdc_step(Ud, dt, nodes=3, sweeps=2, reaction_substeps=3)
        h.synchronize()
        got = Ud.cpu().numpy()
    o = orhs.Options(x_outflow=True)

    def fA(u):
        return orhs.rhs_periodic(u, mech, grid.dx, o, parts=True)[0]

    def fR(u):
        return orhs.rhs_periodic(u, mech, grid.dx, o, parts=True)[1]

    def integ(Up, G, dtp):
        return react.integrate(Up, G, dtp, mech, rtol=rtol, atol=atol)

    ref, _, _, _, _ = osdc.mrsdc2_step(U_g, fA, fR, integ, dt, coarse=3, fine=3, sweeps=2,
                                       species=slice(5, 5 + mech.ns))
    ref = synth.global_to_boxes(grid, ref)
    ratio = np.max(np.abs(got[5:] - ref[5:]) / (rtol * np.abs(ref[5:]) + atol * U[0][None]))
    assert ratio < 1e-2, ratio
    err = relerr(got[:5] - U[:5], ref[:5] - U[:5])
    assert err.max() < 1e-6, err
