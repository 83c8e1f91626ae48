"""The largest mechanism the kernels are built for (64 species), on a small
ragged box: the FP64 and mixed right-hand sides and one multirate step
against the oracle.  Every per-species array of the kernels is at its full
length here."""
import numpy as np
import pytest

from oracle import rhs as orhs
from oracle import sdc as osdc
from oracle import thermo
from paper_1309_7327_gb300 import synth

from util import relerr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def smc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1309_7327_gb300 import smc as S
    return S


@pytest.fixture(scope="module")
def case():
    mech = synth.make_mechanism(64, 160, 3)
    grid = synth.single_box((6, 7, 9), (0.01, 0.011, 0.012))
    prim = synth.smooth_fields(grid, 64, 5, T0=1250.0, T1=250.0, umax=5000.0, p_amp=0.03)
    U_g = thermo.conserved(prim, mech.nasa7, mech.W)
    return mech, grid, U_g


def _rhs(smc, mech, grid, U, **opts):
    with smc.Smc(grid, mech, opts) as h:
        Ud = torch.from_numpy(U).to("cuda:0")
        F = torch.empty_like(Ud)
        h.rhs(Ud, F)
        h.synchronize()
        return F.cpu().numpy()


def test_rhs_64_species_fp64_and_mixed(smc, case):
    mech, grid, U_g = case
    U = synth.global_to_boxes(grid, U_g)
    ref = synth.global_to_boxes(grid, orhs.rhs_periodic(U_g, mech, grid.dx))
    for march in (0, 3):
        err = relerr(_rhs(smc, mech, grid, U, march=march), ref)
        assert err.max() < 1e-12, (march, err.max())
    errm = relerr(_rhs(smc, mech, grid, U, precision=1), ref)
    print("64 species: mixed error", errm.max())
    assert errm.max() < 1e-5, errm.max()


def test_multirate_step_64_species(smc, case):
    """One MRSDC step (3 coarse, 3 fine nodes per coarse interval, 2
    sweeps): the reaction chain with 64 species per cell."""
    mech, grid, U_g = case
    U = synth.global_to_boxes(grid, U_g)
    dt = 2e-9
    with smc.Smc(grid, mech) as h:
        Ud = torch.from_numpy(U).to("cuda:0")
        h.sdc_step(Ud, dt, nodes=3, sweeps=2, reaction_substeps=3)
        h.synchronize()
        got = Ud.cpu().numpy()

    def part(which):
        def f(u):
            tr, ch = orhs.rhs_periodic(u, mech, grid.dx, parts=True)
            return tr if which == 0 else ch
        return f
    ref, _, _, _, _ = osdc.mrsdc_step(U_g, part(0), part(1), dt, coarse=3, fine=3, sweeps=2)
    ref = synth.global_to_boxes(grid, ref)
    err = relerr(got - U, ref - U)
    assert err.max() < 1e-10, err.max()
