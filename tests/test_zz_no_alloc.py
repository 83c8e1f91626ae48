"""The allocation-free entry point smc_rhs_noalloc (static device scratch).

It serves callers that cannot call cudaMalloc: frameworks that own all
device memory in a fixed arena, and loops that must avoid the
synchronisation of allocation.  It must give the same right-hand side as
the handle-based smc_rhs, and the oracle's, call after call, although every
call reuses (and leaves behind) the same static scratch array.  The file is
named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

from util import oracle_rhs, relerr, state

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
    return wl, torch.from_numpy(U).to("cuda:0"), U_g


def test_noalloc_matches_smc_rhs_and_oracle_on_consecutive_calls(smc):
    for name, n in (("c1", 16), ("c2", 12)):
        wl, U, U_g = _case(name, n)
        with smc.Smc(wl.grid, wl.mech) as h:
            ref = torch.empty_like(U)
            h.rhs(U, ref)
            h.synchronize()
        ref = ref.cpu().numpy()
        ora = oracle_rhs(wl, U_g)
        for _ in range(2):
            out = torch.full_like(U, float("nan"))
            smc.smc_rhs_noalloc(wl.grid.domain, wl.grid.dx, wl.mech, U, out)
            got = out.cpu().numpy()
            err = relerr(got, ref)
            assert err.max() <= TOL, (name, "vs smc_rhs", err)
            err = relerr(got, ora)
            assert err.max() <= TOL, (name, "vs oracle", err)


def test_noalloc_rejects_boxes_beyond_the_static_scratch(smc):
    wl, U, _ = _case("c1", 16)
    big = (64, 64, 64)
    Ub = torch.zeros((U.shape[0], 64 ** 3), dtype=torch.float64, device="cuda:0")
    with pytest.raises(smc.SmcError) as e:
        smc.smc_rhs_noalloc(big, wl.grid.dx, wl.mech, Ub, torch.empty_like(Ub))
    assert e.value.status == smc.SMC_ERR_ARG
    # a side whose size products would overflow is refused before any product
    huge = (1 << 30, 1 << 30, 1 << 30)
    m, keep = smc.mechanism_struct(wl.mech)
    st = smc.lib().smc_rhs_noalloc((C.c_int * 3)(*huge), (C.c_double * 3)(*wl.grid.dx),
                                   C.byref(m), C.c_void_p(U.data_ptr()), C.c_void_p(Ub.data_ptr()),
                                   None)
    assert st == smc.SMC_ERR_ARG


def test_noalloc_rejects_host_memory(smc):
    """Host arrays are refused by the library itself (it has no staging
    buffer), and CPU tensors by the binding."""
    wl, U, _ = _case("c1", 16)
    Uh = np.ascontiguousarray(U.cpu().numpy())
    Fh = np.empty_like(Uh)
    m, keep = smc.mechanism_struct(wl.mech)
    n = (C.c_int * 3)(*wl.grid.domain)
    dx = (C.c_double * 3)(*wl.grid.dx)
    Fd = torch.empty_like(U)
    for u_ptr, f_ptr in ((Uh.ctypes.data, Fd.data_ptr()), (U.data_ptr(), Fh.ctypes.data)):
        st = smc.lib().smc_rhs_noalloc(n, dx, C.byref(m), C.c_void_p(u_ptr), C.c_void_p(f_ptr),
                                       None)
        assert st == smc.SMC_ERR_ARG
    with pytest.raises(ValueError):
        smc.smc_rhs_noalloc(wl.grid.domain, wl.grid.dx, wl.mech, U.cpu(), Fd)
