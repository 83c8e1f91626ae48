"""Degenerate grids of eq. cns on the periodic domain.

* A domain one cell thick along an axis: every difference along that axis is
  of equal values, so that direction contributes nothing and the RHS is the
  one of the remaining directions; compared with the oracle, FP64 and mixed.
* A single-cell domain: the state is uniform, every transport term vanishes
  exactly (differences of equal values), and the RHS is the chemistry alone.
"""
import numpy as np
import pytest

from oracle import thermo
from paper_1309_7327_gb300 import synth

from util import oracle_rhs, relerr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def smc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1309_7327_gb300 import smc as S
    return S


class _Workload:
    def __init__(self, grid, mech):
        self.grid, self.mech = grid, mech


def _case(shape, ns, nr, seed):
    mech = synth.make_mechanism(ns, nr, seed)
    grid = synth.single_box(shape, (0.01, 0.011, 0.012))
    prim = synth.smooth_fields(grid, ns, seed, p_amp=0.03)
    U_g = thermo.conserved(prim, mech.nasa7, mech.W)
    return _Workload(grid, mech), U_g


def _gpu(smc, wl, U, **opts):
    with smc.Smc(wl.grid, wl.mech, opts) as h:
        Ud = torch.from_numpy(U).to("cuda:0")
        F = torch.full_like(Ud, float("nan"))
        h.rhs(Ud, F)
        h.synchronize()
        return F.cpu().numpy()


@pytest.mark.parametrize("shape", [(12, 10, 1), (12, 1, 9), (1, 10, 9), (1, 1, 11)])
@pytest.mark.parametrize("precision,march", [(0, 0), (0, 1), (1, 1)])
def test_rhs_domain_one_cell_thick(smc, shape, precision, march):
    wl, U_g = _case(shape, 9, 21, 5)
    U = synth.global_to_boxes(wl.grid, U_g)
    got = _gpu(smc, wl, U, precision=precision, march=march)
    err = relerr(got, oracle_rhs(wl, U_g))
    assert np.isfinite(got).all()
    assert err.max() < (1e-12 if precision == 0 else 1e-5), (shape, err)


@pytest.mark.parametrize("precision", [0, 1])
def test_rhs_single_cell_domain_is_the_chemistry(smc, precision):
    wl, U_g = _case((1, 1, 1), 9, 21, 6)
    U = synth.global_to_boxes(wl.grid, U_g)
    got = _gpu(smc, wl, U, precision=precision)
    # mass, momentum and energy: no transport, no chemical source
    assert (got[:5] == 0.0).all(), got[:5]
    ref = oracle_rhs(wl, U_g)
    assert (ref[:5] == 0.0).all()
    # the species: the production rates at the cell's temperature
    scale = np.abs(ref[5:]).max()
    assert scale > 0.0
    assert np.abs(got[5:] - ref[5:]).max() <= 1e-12 * scale
