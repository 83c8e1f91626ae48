"""Mixed precision (SMC_OPT_PRECISION = 1): FP32 stencils and transport on
float-pair fields, FP64 temperature, Gibbs energies, exponentials, rates and
SDC accumulation.  Target: at most 1e-5 relative (max-norm per component)
against the FP64 oracle, and eighth-order spatial convergence retained down
to the FP32 floor."""
import numpy as np
import pytest

from oracle import sdc as osdc
from oracle import thermo
from paper_1309_7327_gb300 import synth

from util import oracle_rhs, relerr, state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def smc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1309_7327_gb300 import smc as S
    return S


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def gpu_rhs(S, grid, mech, U, **options):
    options.setdefault("precision", 1)
    with S.Smc(grid, mech, options) as h:
        Ud = dev(U)
        F = torch.empty_like(Ud)
        h.rhs(Ud, F)
        h.synchronize()
        return F.cpu().numpy()


@pytest.mark.parametrize("march", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_mixed_rhs_c1(smc, mode, march):
    """Both line kernels (per-face windows, sliding register windows)."""
    wl, U, U_g = state("c1", seed=1, p_amp=0.03)
    got = gpu_rhs(smc, wl.grid, wl.mech, U, diffusion_mode=mode, march=march)
    err = relerr(got, oracle_rhs(wl, U_g, mode="vc" if mode == 0 else "ref"))
    print("mixed c1 per-component error", np.array2string(err, precision=2))
    assert err.max() < TOL, err


def test_mixed_rhs_bump_nine_species(smc):
    wl, U, U_g = state("c2", seed=1, n=24)
    err = relerr(gpu_rhs(smc, wl.grid, wl.mech, U), oracle_rhs(wl, U_g))
    print("mixed c2(24^3) per-component error", np.array2string(err, precision=2))
    assert err.max() < TOL, err


def test_mixed_rhs_flame(smc):
    """Planar hot slab 300-2000 K with a 1000 cm/s base flow (the c3 field on
    a 32^3 box)."""
    wl, U, U_g = state("c3", seed=1, n=32)
    err = relerr(gpu_rhs(smc, wl.grid, wl.mech, U), oracle_rhs(wl, U_g))
    print("mixed c3(32^3) per-component error", np.array2string(err, precision=2))
    assert err.max() < TOL, err


@pytest.mark.parametrize("march", [0, 1])
def test_mixed_rhs_multibox_21_species(smc, march):
    wl = synth.workload("c4", seed=3, n=12)
    prim_g = synth.boxes_to_global(wl.grid, wl.prim)
    U_g = thermo.conserved(prim_g, wl.mech.nasa7, wl.mech.W)
    U = synth.global_to_boxes(wl.grid, U_g)
    err = relerr(gpu_rhs(smc, wl.grid, wl.mech, U, march=march), oracle_rhs(wl, U_g))
    print("mixed c4(8 boxes) per-component error", np.array2string(err, precision=2))
    assert err.max() < TOL, err


def test_mixed_sdc_step(smc):
    """State error after one 3-node / 4-sweep step: the increment U_new - U_0
    within the RHS tolerance."""
    wl, U, U_g = state("c1", seed=2, p_amp=0.03)
    with smc.Smc(wl.grid, wl.mech, {"precision": 1}) as h:
        Ud = dev(U)
        h.sdc_step(Ud, wl.dt)
        h.synchronize()
        U1 = Ud.cpu().numpy()
    from oracle import rhs as orhs

    def f(u, t):
        return orhs.rhs_periodic(u, wl.mech, wl.grid.dx)
    ref, _, _ = osdc.sdc_step(U_g, f, wl.dt)
    ref = synth.global_to_boxes(wl.grid, ref)
    err = relerr(U1 - U, ref - U)
    assert err.max() < TOL, err
    # the state itself is far more accurate
    assert relerr(U1, ref).max() < 1e-8


@pytest.mark.parametrize("rates", [0, 1])
def test_mixed_mrsdc_step_multibox(smc, rates):
    """Mode-1 multirate step (3 coarse / 5 fine nodes, 4 sweeps) on 8 uneven
    boxes with 21 species, FP64 rates or FP32-mantissa rates in the reaction
    substeps: the increment within the mixed tolerance of the FP64 oracle."""
    wl = synth.workload("c4", seed=2, n=10)
    prim_g = synth.boxes_to_global(wl.grid, wl.prim)
    U_g = thermo.conserved(prim_g, wl.mech.nasa7, wl.mech.W)
    U = synth.global_to_boxes(wl.grid, U_g)
    with smc.Smc(wl.grid, wl.mech, {"precision": 1, "rates": rates}) as h:
        Ud = dev(U)
        h.sdc_step(Ud, wl.dt, nodes=3, sweeps=4, reaction_substeps=5)
        h.synchronize()
        U1 = Ud.cpu().numpy()
    from oracle import rhs as orhs

    def part(which):
        def f(u, t=0.0):
            tr, ch = orhs.rhs_periodic(u, wl.mech, wl.grid.dx, parts=True)
            return tr if which == "transport" else ch
        return f
    ref, _, _, _, _ = osdc.mrsdc_step(U_g, part("transport"), part("chem"), wl.dt,
                                      coarse=3, fine=5, sweeps=4)
    ref = synth.global_to_boxes(wl.grid, ref)
    err = relerr(U1 - U, ref - U)
    print("mixed MRSDC increment error", np.array2string(err, precision=2))
    assert err.max() < TOL, err


@pytest.mark.parametrize("rates", [0, 1])
@pytest.mark.parametrize("name,n", [("c3", 16), ("c4", 10)])
def test_mixed_rates_match_fp64_rates(smc, name, n, rates):
    """The mixed path's production rates alone (its full right-hand side
    minus its reaction-free one, which share every transport operation),
    FP64 or with FP32 mantissas: against the oracle's rates, per species, on
    the 300-2000 K flame field and on the 21-species mechanism.  FP64 rates
    at the temperature of the float-pair primitives agree to ~1e-12; FP32
    mantissas within the mixed tolerance."""
    if name == "c4":
        wl = synth.workload("c4", seed=4, n=n)
        prim_g = synth.boxes_to_global(wl.grid, wl.prim)
        U_g = thermo.conserved(prim_g, wl.mech.nasa7, wl.mech.W)
        U = synth.global_to_boxes(wl.grid, U_g)
    else:
        wl, U, U_g = state(name, seed=2, n=n)
    full = gpu_rhs(smc, wl.grid, wl.mech, U, rates=rates)
    noreact = gpu_rhs(smc, wl.grid, wl.mech, U, reactions=0, rates=rates)
    from oracle import rhs as orhs
    _, ch = orhs.rhs_periodic(U_g, wl.mech, wl.grid.dx, parts=True)
    ch = synth.global_to_boxes(wl.grid, ch)
    assert np.array_equal(full[:5], noreact[:5])
    err = relerr(full[5:] - noreact[5:], ch[5:])
    print(f"mixed rates error ({name}, rates={rates})", np.array2string(err, precision=2))
    assert err.max() < (TOL if rates else 1e-9), err


def test_mixed_keeps_eighth_order_to_the_fp32_floor(smc):
    """Self-convergence of the mixed RHS on a smooth quasi-2-D field: the
    32/64/128 differences fall by ~2^8 until the FP32 floor is reached."""
    from test_oracle_physics import _manufactured
    mech = synth.make_mechanism(3, 2, 1)
    vals = {}
    for N in (16, 32, 64):
        prim, dx = _manufactured(N, mech)
        Ug = thermo.conserved(prim, mech.nasa7, mech.W)
        grid = synth.single_box((N, N, 4), dx)
        F = gpu_rhs(smc, grid, mech, synth.global_to_boxes(grid, Ug), reactions=0)
        vals[N] = synth.boxes_to_global(grid, F)
    e1 = np.abs(vals[16][:, 0] - vals[32][:, 0, ::2, ::2]).max(axis=(1, 2))
    e2 = np.abs(vals[32][:, 0] - vals[64][:, 0, ::2, ::2]).max(axis=(1, 2))
    scale = np.abs(vals[64]).reshape(vals[64].shape[0], -1).max(axis=1)
    rates = np.log2(e1 / e2)
    print("mixed self-convergence rates", np.array2string(rates, precision=2))
    # components whose difference is still above the FP32 floor converge at ~8
    live = e2 / scale > 1e-5
    assert (rates[live] > 6.5).all(), (rates, e2 / scale)
