"""The allocation-free entry point smc_rhs_noalloc (static device scratch)
against the handle-based smc_rhs, on two calls in a row.

It serves callers that cannot call cudaMalloc (code inside CUDA stream
capture, frameworks that own all device memory, loops that must avoid the
synchronisation of allocation); it must give the same right-hand side as
smc_rhs, call after call, although every call reuses the same static
scratch array."""
import numpy as np
import pytest

from paper_1309_7327_gb300 import synth

from util import relerr, state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def smc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1309_7327_gb300 import smc as S
    return S


def _case(name, n):
    wl, U, U_g = state(name, seed=3, n=n, p_amp=0.03)
    return wl, torch.from_numpy(U).to("cuda:0")


def test_noalloc_matches_smc_rhs_on_consecutive_calls(smc):
    for name, n in (("c1", 16), ("c2", 12)):
        wl, U = _case(name, n)
        with smc.Smc(wl.grid, wl.mech) as h:
            ref = torch.empty_like(U)
            h.rhs(U, ref)
            h.synchronize()
        ref = ref.cpu().numpy()
        for _ in range(2):
            out = torch.full_like(U, float("nan"))
            smc.smc_rhs_noalloc(wl.grid.domain, wl.grid.dx, wl.mech, U, out)
            err = relerr(out.cpu().numpy(), ref)
            assert err.max() <= TOL, (name, err)


def test_noalloc_rejects_boxes_beyond_the_static_scratch(smc):
    wl, U = _case("c1", 16)
    big = (64, 64, 64)
    Ub = torch.zeros((U.shape[0], 64 ** 3), dtype=torch.float64, device="cuda:0")
    with pytest.raises(smc.SmcError) as e:
        smc.smc_rhs_noalloc(big, wl.grid.dx, wl.mech, Ub, torch.empty_like(Ub))
    assert e.value.status == smc.SMC_ERR_ARG
