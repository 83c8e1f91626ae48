"""Parity of the CUDA implicit reaction integrator (smc_react_integrate) and
of the mode-2 multirate step (Sec. 3.2, eq. mrupdate2) with the oracle.

Both sides run the same variable-order BDF algorithm; the CUDA one factors
its Newton matrix in FP32 (the oracle in FP64), so their Newton iterates
stop at slightly different points inside the Newton tolerance, which is
1e-4 of the local error tolerance.  The bar is therefore the integrator's
own tolerance: per element |y_gpu - y_oracle| <= C (rtol |y| + atol rho).
Measured: C ~ 1e-5 (the two sides take the same step and order decisions,
and the Newton iterates converge well inside their stopping test); the
small-grid bars allow 1e-2, the full-size sampled one 10 (one cell whose
accept/reject decision flipped would differ by about the tolerance)."""
import numpy as np
import pytest

from oracle import react, rhs as orhs, sdc as osdc, thermo
from paper_1309_7327_gb300 import synth

from util import relerr, state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-10, 1e-14


@pytest.fixture(scope="module")
def smc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1309_7327_gb300 import smc as S
    return S


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def tol_ratio(y, ref, rho, rtol=RTOL, atol=ATOL):
    """max over elements of |y - ref| / (rtol |ref| + atol rho)."""
    return float(np.max(np.abs(y - ref) / (rtol * np.abs(ref) + atol * rho)))


def _opts(**kw):
    o = {"bdf_rtol": RTOL, "bdf_atol": ATOL}
    o.update(kw)
    return o


def test_react_integrate_matches_oracle_every_cell(smc):
    """8^3 cells, 3 species, with the advection-diffusion RHS as forcing and
    20 acoustic time steps of integration."""
    wl, U, U_g = state("c1", seed=1, n=8)
    ns = wl.mech.ns
    G_g = orhs.rhs_periodic(U_g, wl.mech, wl.grid.dx, parts=True)[0]
    G = synth.global_to_boxes(wl.grid, G_g)
    dt = 20 * wl.dt
    with smc.Smc(wl.grid, wl.mech, _opts()) as h:
        Ud, Gd = dev(U), dev(G)
        out = torch.empty_like(Ud)
        h.react_integrate(Ud, Gd, dt, out)
        h.synchronize()
        st = h.stats()
        got = out.cpu().numpy()
    ref = react.integrate(U, G, dt, wl.mech, rtol=RTOL, atol=ATOL)
    assert np.allclose(got[:5], U[:5] + dt * G[:5], rtol=1e-15, atol=0)
    r = tol_ratio(got[5:], ref[5:], U[0][None])
    assert r < 1e-2, r
    # the composition moved by far more than the tolerance
    assert np.abs(ref[5:] - U[5:]).max() > 1e4 * RTOL * np.abs(U[5:]).max()
    assert st["bdf_steps"] >= U.shape[1] and st["bdf_evals"] > st["bdf_steps"]


def test_react_integrate_in_place_and_without_forcing(smc):
    wl, U, _ = state("c2", seed=2, n=6)
    dt = 50 * wl.dt
    with smc.Smc(wl.grid, wl.mech, _opts()) as h:
        Ud = dev(U)
        h.react_integrate(Ud, None, dt, Ud)
        h.synchronize()
        got = Ud.cpu().numpy()
    cells = list(range(0, U.shape[1], 7))
    ref = react.integrate(U, None, dt, wl.mech, rtol=RTOL, atol=ATOL, cells=cells)
    assert np.array_equal(got[:5], U[:5])
    assert tol_ratio(got[5:, cells], ref[5:], U[0][None, cells]) < 1e-2
    # mass: sum_k rho Y_k = rho at every cell
    assert np.abs(got[5:].sum(0) - got[0]).max() <= 1e-12 * got[0].max()


def test_react_integrate_full_size_sampled(smc):
    """The 64-box, 4.7M-cell, 21-species configuration: every cell on the
    GPU, sampled cells against the oracle, mass at every cell."""
    wl = synth.workload("c4")
    U = thermo.conserved(wl.prim, wl.mech.nasa7, wl.mech.W)
    dt = 10 * wl.dt
    with smc.Smc(wl.grid, wl.mech, _opts()) as h:
        Ud = dev(U)
        out = torch.empty_like(Ud)
        h.react_integrate(Ud, None, dt, out)
        h.synchronize()
        got = out.cpu().numpy()
        del Ud, out
    rng = np.random.default_rng(4)
    cells = sorted(rng.choice(U.shape[1], 10, replace=False).tolist()) + [0, U.shape[1] - 1]
    ref = react.integrate(U, None, dt, wl.mech, rtol=RTOL, atol=ATOL, cells=cells)
    assert tol_ratio(got[5:, cells], ref[5:], U[0][None, cells]) < 10.0
    assert np.abs(got[5:].sum(0) - got[0]).max() <= 1e-12 * got[0].max()
    assert np.isfinite(got).all()


def _mode2_oracle(wl, U_g, dt, coarse, fine, sweeps, repeat=1, eps=0.0, history=None):
    ns = wl.mech.ns

    def fA(u):
        return orhs.rhs_periodic(u, wl.mech, wl.grid.dx, parts=True)[0]

    def fR(u):
        return orhs.rhs_periodic(u, wl.mech, wl.grid.dx, parts=True)[1]

    def integ(Up, G, dtp):
        return react.integrate(Up, G, dtp, wl.mech, rtol=RTOL, atol=ATOL)

    return osdc.mrsdc2_step(U_g, fA, fR, integ, dt, coarse=coarse, fine=fine, sweeps=sweeps,
                            repeat=repeat, species=slice(5, 5 + ns), eps=eps, history=history)


@pytest.mark.parametrize("nodes,fine,sweeps", [(3, 3, 2), (3, 2, 3), (5, 2, 2)])
def test_mode2_step_matches_oracle(smc, nodes, fine, sweeps):
    wl, U, U_g = state("c1", seed=3, n=8, p_amp=0.03)
    dt = wl.dt
    with smc.Smc(wl.grid, wl.mech, _opts(mr_mode=2)) as h:
        Ud = dev(U)
        h.sdc_step(Ud, dt, nodes=nodes, sweeps=sweeps, reaction_substeps=fine)
        h.synchronize()
        st = h.stats()
        got = Ud.cpu().numpy()
    ref, _, _, nA, nR = _mode2_oracle(wl, U_g, dt, nodes, fine, sweeps)
    ref = synth.global_to_boxes(wl.grid, ref)
    M1 = nodes - 1
    M2 = M1 * (fine - 1)
    assert (st["n_rhs"], st["n_react"]) == (nA, nR) == (sweeps * M2 + 1, sweeps * M1 + 1)
    assert tol_ratio(got[5:], ref[5:], U[0][None]) < 1e-2
    err = relerr(got[:5] - U[:5], ref[:5] - U[:5])
    assert err.max() < 1e-7, err


def test_mode2_type_c_step_matches_oracle(smc):
    """Two groups of 3 fine Gauss-Lobatto nodes per coarse interval."""
    wl, U, U_g = state("c1", seed=6, n=8, p_amp=0.03)
    with smc.Smc(wl.grid, wl.mech, _opts(mr_mode=2, fine_repeat=2)) as h:
        Ud = dev(U)
        h.sdc_step(Ud, wl.dt, nodes=3, sweeps=2, reaction_substeps=3)
        h.synchronize()
        st = h.stats()
        got = Ud.cpu().numpy()
    ref, _, _, nA, nR = _mode2_oracle(wl, U_g, wl.dt, 3, 3, 2, repeat=2)
    ref = synth.global_to_boxes(wl.grid, ref)
    assert (st["n_rhs"], st["n_react"]) == (nA, nR) == (2 * 8 + 1, 2 * 2 + 1)
    assert tol_ratio(got[5:], ref[5:], U[0][None]) < 1e-2
    assert relerr(got[:5] - U[:5], ref[:5] - U[:5]).max() < 1e-7


def test_mode2_residual_exit_matches_oracle(smc):
    """The mode-2 residual (coarse quadrature of R, fine quadrature of A)
    after every sweep, and the stagnation exit, against the oracle."""
    wl, U, U_g = state("c1", seed=7, n=8, p_amp=0.03)
    with smc.Smc(wl.grid, wl.mech, _opts(mr_mode=2, sdc_exit=0.5)) as h:
        Ud = dev(U)
        h.sdc_step(Ud, wl.dt, nodes=3, sweeps=14, reaction_substeps=3)
        h.synchronize()
        st = h.stats()
        got = Ud.cpu().numpy()
    hist = []
    ref, _, _, _, _ = _mode2_oracle(wl, U_g, wl.dt, 3, 3, 14, eps=0.5, history=hist)
    res = st["residual"]
    # The exit compares successive residuals.  Once they reach the floor
    # set by the implicit integrations (their tolerance, 1e-10 here, not
    # FP64 rounding) the ratio is noise on either side, so the stop may come
    # up to two sweeps apart -- only there: every earlier sweep matches, and
    # the residual where they stop is at that floor.
    assert len(res) == st["sweeps_done"] < 14, res
    assert abs(st["sweeps_done"] - len(hist)) <= 2, (res, hist)
    if st["sweeps_done"] != len(hist):
        assert max(res[-1], hist[-1]) < 1e-9, (res, hist)
    for g, o in zip(res, hist):
        if o > 1e-9:
            assert abs(g - o) <= 1e-3 * o, (res, hist)
    ref = synth.global_to_boxes(wl.grid, ref)
    assert tol_ratio(got[5:], ref[5:], U[0][None]) < 10.0


def test_mode2_two_steps_graphs_and_eager_agree(smc):
    """The second (recycled) step is replayed as a CUDA graph; it gives the
    same state, bit for bit, as kernel-by-kernel launches."""
    wl, U, _ = state("c1", seed=4, n=8)
    outs = []
    for graphs in (0, 1):
        with smc.Smc(wl.grid, wl.mech, _opts(mr_mode=2, use_graphs=graphs)) as h:
            stream = torch.cuda.Stream()
            h.set_stream(stream)
            Ud = dev(U)
            torch.cuda.synchronize()
            for _ in range(3):
                h.sdc_step(Ud, wl.dt, nodes=3, sweeps=2, reaction_substeps=3)
            h.synchronize()
            outs.append(Ud.cpu().numpy())
            st = h.stats()
            assert st["n_rhs"] == 3 * 2 * 4 + 1
    assert np.array_equal(outs[0], outs[1])


def test_mode2_mixed_precision_within_1e5_of_fp64(smc):
    wl, U, _ = state("c1", seed=5, n=8, p_amp=0.03)
    got = {}
    for prec in (0, 1):
        with smc.Smc(wl.grid, wl.mech, _opts(mr_mode=2, precision=prec)) as h:
            Ud = dev(U)
            h.sdc_step(Ud, wl.dt, nodes=3, sweeps=3, reaction_substeps=3)
            h.synchronize()
            got[prec] = Ud.cpu().numpy()
    err = relerr(got[1] - U, got[0] - U)
    assert err.max() < 1e-5, err


def test_mode2_and_integrator_reject_more_than_32_species(smc):
    wl, U, _ = state("c1", seed=1, n=8)
    mech = synth.make_mechanism(40, 10, 3)
    nv = 5 + 40
    with smc.Smc(wl.grid, mech, {"mr_mode": 2}) as h:
        Z = torch.zeros((nv, U.shape[1]), dtype=torch.float64, device="cuda:0")
        with pytest.raises(smc.SmcError):
            h.react_integrate(Z, None, 1e-8, Z)
        with pytest.raises(smc.SmcError):
            h.sdc_step(Z, 1e-8, nodes=3, sweeps=1, reaction_substeps=3)


def test_react_integrate_30_species(smc):
    """The 25-32-species instance of the integrator (30 species, 60
    reactions) on a small box, sampled cells against the oracle."""
    grid = synth.single_box((8, 8, 4), 1.0 / 64)
    mech = synth.make_mechanism(30, 60, 5)
    prim = synth.global_to_boxes(grid, synth.smooth_fields(grid, 30, 105, T0=1400.0, T1=200.0,
                                                            umax=3000.0))
    U = thermo.conserved(prim, mech.nasa7, mech.W)
    dt = 2e-7
    with smc.Smc(grid, mech, _opts()) as h:
        Ud = dev(U)
        out = torch.empty_like(Ud)
        h.react_integrate(Ud, None, dt, out)
        h.synchronize()
        got = out.cpu().numpy()
    cells = [0, 37, 101, 200, 255]
    ref = react.integrate(U, None, dt, mech, rtol=RTOL, atol=ATOL, cells=cells)
    assert np.abs(ref[5:] - U[5:, cells]).max() > 1e4 * RTOL * np.abs(U[5:]).max()
    assert tol_ratio(got[5:, cells], ref[5:], U[0][None, cells]) < 1e-2
    assert np.abs(got[5:].sum(0) - got[0]).max() <= 1e-12 * got[0].max()
