"""Pins of the oracle's thermodynamics, chemistry and full right-hand side
against invariants the equations fix (Sec. 2.1, Sec. 2.4).  CPU only."""
import math

import numpy as np
import pytest

from oracle import chem, rhs, stencil, thermo
from paper_1309_7327_gb300 import synth


def periodic_state(name="c1", n=None, seed=1, **kw):
    wl = synth.workload(name, seed=seed, n=n)
    g = wl.grid
    nx, ny, nz = g.domain
    prim = synth.boxes_to_global(g, wl.prim)
    U = thermo.conserved(prim, wl.mech.nasa7, wl.mech.W)
    return wl, prim, U


def test_newton_recovers_temperature_and_ideal_gas():
    wl, prim, U = periodic_state("c2", n=12)
    P = thermo.primitives(U, wl.mech.nasa7, wl.mech.W)
    assert P["converged"].all()
    assert np.abs(P["T"] / prim[3] - 1).max() < 1e-13
    assert np.abs(P["p"] / prim[4] - 1).max() < 1e-13
    assert np.abs(P["X"].sum(0) - 1).max() < 1e-14


def test_thermo_polynomials_consistent():
    """dh/dT = cp and ds/dT = cp/T (checked by central differences)."""
    m = synth.make_mechanism(9, 21, 4)
    T = np.array([400.0, 1100.0, 1900.0])
    d = 1e-3
    dh = (thermo.h_RT(m.nasa7, T + d) * (T + d) - thermo.h_RT(m.nasa7, T - d) * (T - d)) / (2 * d)
    assert np.allclose(dh, thermo.cp_R(m.nasa7, T), rtol=1e-8)
    ds = (thermo.s_R(m.nasa7, T + d) - thermo.s_R(m.nasa7, T - d)) / (2 * d)
    assert np.allclose(ds, thermo.cp_R(m.nasa7, T) / T, rtol=1e-7)
    cp = thermo.cp_R(m.nasa7, np.linspace(200, 3500, 200))
    assert cp.min() >= 2.5 and cp.max() <= 8.0


@pytest.mark.parametrize("ns,nr", [(3, 2), (9, 21), (21, 84)])
def test_chemistry_conserves_mass(ns, nr):
    """sum_k W_k omega_k = 0 for element-balanced reactions."""
    m = synth.make_mechanism(ns, nr, 7)
    rng = np.random.default_rng(0)
    T = rng.uniform(400, 2000, 50)
    Y = rng.uniform(0.01, 1, (ns, 50))
    Y /= Y.sum(0)
    rho = rng.uniform(1e-4, 1e-3, 50)
    w = chem.production_rates(rho, T, Y, m)
    assert np.abs(w.sum(0)).max() <= 1e-13 * np.abs(w).max()
    assert np.abs(w).max() > 0


@pytest.mark.parametrize("ns,nr", [(3, 2), (9, 21), (21, 84)])
def test_chemistry_vanishes_at_constructed_equilibrium(ns, nr):
    """Shift each species' entropy constant so that the chemical potential
    mu_k = g_k/(R T*) + ln(c*_k R T*/p_atm) is zero at a chosen state; then
    every reaction has sum nu mu = 0 and its net rate vanishes, while the
    forward rates stay large."""
    m = synth.make_mechanism(ns, nr, 11)
    rng = np.random.default_rng(5)
    Tst = 1300.0
    Y = rng.uniform(0.05, 1, ns)
    Y /= Y.sum()
    rho = 3e-4
    c = rho * Y / m.W
    mu0 = (thermo.h_RT(m.nasa7, np.array([Tst]))[:, 0] - thermo.s_R(m.nasa7, np.array([Tst]))[:, 0]
           + np.log(c * thermo.R_U * Tst / thermo.P_ATM))
    m.nasa7 = m.nasa7.copy()
    m.nasa7[:, 6] += mu0          # g/RT = h/RT - s/R drops by mu0
    w = chem.production_rates(np.array([rho]), np.array([Tst]), Y[:, None], m)
    # the size of the cancelling terms
    kf = m.A * Tst ** m.b * np.exp(-m.Ea / (thermo.R_CAL * Tst))
    fwd = kf * np.prod(c[None, :] ** m.nu_f, axis=1)
    assert np.abs(w).max() < 1e-12 * np.max(fwd * m.W.max())
    # away from the equilibrium temperature the rates are not zero
    w2 = chem.production_rates(np.array([rho]), np.array([Tst * 1.2]), Y[:, None], m)
    assert np.abs(w2).max() > 1e-6 * np.max(fwd * m.W.max())


def test_chemistry_single_reaction_closed_form():
    """A + A2 <=> A3 with hand-picked constants: forward and reverse rates by
    the law of mass action with K_c from the Gibbs energies."""
    m = synth.make_mechanism(3, 2, 1)
    m.nu_f = np.array([[1, 1, 0]], dtype=np.int32)
    m.nu_r = np.array([[0, 0, 1]], dtype=np.int32)
    m.A = np.array([2.0e12])
    m.b = np.array([0.5])
    m.Ea = np.array([12000.0])
    T = 1500.0
    Y = np.array([0.2, 0.3, 0.5])
    rho = 2.0e-4
    c = rho * Y / m.W
    kf = 2.0e12 * math.sqrt(T) * math.exp(-12000.0 / (1.98720425864083 * T))
    g = [float(thermo.h_RT(m.nasa7[k:k + 1], np.array([T]))[0, 0]
               - thermo.s_R(m.nasa7[k:k + 1], np.array([T]))[0, 0]) for k in range(3)]
    dg = g[2] - g[0] - g[1]
    Kc = math.exp(-dg) * (1.01325e6 / (8.31446261815324e7 * T)) ** (-1)
    q = kf * c[0] * c[1] - kf / Kc * c[2]
    w = chem.production_rates(np.array([rho]), np.array([T]), Y[:, None], m)[:, 0]
    assert np.allclose(w, [-m.W[0] * q, -m.W[1] * q, m.W[2] * q], rtol=1e-13)


def test_rhs_species_sum_equals_density_rhs():
    wl, prim, U = periodic_state("c1")
    F = rhs.rhs_periodic(U, wl.mech, wl.grid.dx)
    assert np.abs(F[5:].sum(0) - F[0]).max() < 1e-13 * np.abs(F[0]).max()


def test_rhs_uniform_state_has_only_chemistry():
    wl, prim, U = periodic_state("c1")
    Uc = np.broadcast_to(U[:, :1, :1, :1], U.shape).copy()
    tr, ch = rhs.rhs_periodic(Uc, wl.mech, wl.grid.dx, parts=True)
    assert np.abs(tr).max() < 1e-6 * np.abs(ch).max()
    assert np.abs(tr[:5]).max() == 0.0


@pytest.mark.parametrize("mode", ["vc", "ref"])
def test_rhs_periodic_telescoping(mode):
    """Flux-form terms telescope over a periodic domain: mass and momentum in
    both modes; every component in reference-species mode (Sec. 2.1, 2.4)."""
    wl, prim, U = periodic_state("c1", p_amp=0.0)
    opt = rhs.Options(mode=mode, reactions=False)
    F = rhs.rhs_periodic(U, wl.mech, wl.grid.dx, opt)
    comps = range(F.shape[0]) if mode == "ref" else range(4)
    for c in comps:
        assert abs(F[c].sum()) <= 1e-12 * np.abs(F[c]).max() * F[c].size, c
    if mode == "vc":
        # the chain-rule correction terms are not in flux form
        assert abs(F[4].sum()) > 1e-8 * np.abs(F[4]).max() * F[4].size


def test_rhs_pointwise_patch_equals_full():
    wl, prim, U = periodic_state("c1")
    F = rhs.rhs_periodic(U, wl.mech, wl.grid.dx)
    cells = [(0, 0, 0), (5, 15, 2), (15, 8, 9)]
    S = rhs.rhs_at(U, cells, wl.mech, wl.grid.dx)
    for i, (z, y, x) in enumerate(cells):
        assert np.allclose(S[:, i], F[:, z, y, x], rtol=0, atol=1e-14 * np.abs(F).max())


def _manufactured(N, mech):
    """Smooth quasi-2-D periodic state on an N x N x 4 grid with nodes x = i h."""
    L = 1.0
    h = L / N
    x = h * np.arange(N)
    z = h * np.arange(4)
    Z, Yy, X = np.meshgrid(z, x, x, indexing="ij")
    k = 2 * np.pi / L
    ns = mech.W.shape[0]
    prim = np.empty((5 + ns,) + X.shape)
    prim[0] = 3000.0 * np.sin(k * X + 0.3) * np.cos(k * Yy)
    prim[1] = -2000.0 * np.cos(k * X) * np.sin(k * Yy + 0.5)
    prim[2] = 500.0 * np.sin(k * X + k * Yy)
    prim[3] = 1200.0 + 200.0 * np.sin(k * X) * np.sin(k * Yy + 1.0)
    prim[4] = 1.01325e6 * (1 + 0.02 * np.cos(k * X + 0.7))
    raw = np.stack([1.5 + 0.4 * np.sin(k * X + j) * np.cos(k * Yy - j) for j in range(ns)])
    prim[5:] = raw / raw.sum(0)
    return prim, (h, h, h)


@pytest.mark.slow
def test_rhs_spatial_order_eight():
    """Self-convergence of the whole spatial operator: the difference between
    the N- and 2N-grid right-hand sides at shared points falls by ~2^8 per
    doubling (Sec. 5.1: eighth order in space)."""
    mech = synth.make_mechanism(3, 2, 1)
    vals = {}
    for N in (32, 64, 128):
        prim, dx = _manufactured(N, mech)
        U = thermo.conserved(prim, mech.nasa7, mech.W)
        vals[N] = rhs.rhs_periodic(U, mech, dx, rhs.Options(reactions=False))
    e1 = np.abs(vals[32][:, 0] - vals[64][:, 0, ::2, ::2]).max(axis=(1, 2))
    e2 = np.abs(vals[64][:, 0] - vals[128][:, 0, ::2, ::2]).max(axis=(1, 2))
    rates = np.log2(e1 / e2)
    assert (rates > 7.5).all() and (rates < 8.5).all(), rates


def test_x_outflow_rhs_changes_only_the_cells_near_the_x_ends():
    """With non-periodic x ends the right-hand side equals the periodic one
    at every cell four or more cells from both x ends (same stencils, same
    data), differs next to the ends, and still vanishes (transport) on a
    uniform state."""
    from util import state
    wl, U, U_g = state("c1", seed=4, p_amp=0.03)
    opt = rhs.Options(x_outflow=True)
    per = rhs.rhs_periodic(U_g, wl.mech, wl.grid.dx)
    out = rhs.rhs_periodic(U_g, wl.mech, wl.grid.dx, opt)
    nx = U_g.shape[-1]
    assert np.array_equal(per[..., 4:nx - 4], out[..., 4:nx - 4])
    for c in (0, 3, nx - 4, nx - 1):
        assert np.abs(per[..., c] - out[..., c]).max() > 0
    uni = np.broadcast_to(U_g[:, :1, :1, :1], U_g.shape).copy()
    tr, _ = rhs.rhs_periodic(uni, wl.mech, wl.grid.dx, opt, parts=True)
    assert np.abs(tr).max() <= 1e-9 * np.abs(uni).max()


def test_spectral_velocity_is_solenoidal_with_the_requested_spectrum():
    """The scale configuration's velocity generator: divergence-free (in
    Fourier space), the requested rms, and an energy spectrum of slope
    -5/3 over the seeded band."""
    g = synth.single_box((48, 48, 48), 1.0 / 256)
    u = synth.spectral_velocity(g, 3, rms=1000.0, kmax=12)
    assert abs(np.sqrt(np.mean(u ** 2)) - 1000.0) < 1e-9 * 1000.0
    U = [np.fft.fftn(u[c]) for c in range(3)]
    k = np.fft.fftfreq(48, 1.0 / 48)
    KZ, KY, KX = np.meshgrid(k, k, k, indexing="ij")
    div = KX * U[0] + KY * U[1] + KZ * U[2]
    assert np.abs(div).max() < 1e-12 * np.abs(KX * U[0]).max()
    km = np.rint(np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)).astype(int)
    P = sum(np.abs(x) ** 2 for x in U)
    E = np.array([P[km == kk].sum() for kk in range(2, 12)])
    slope = np.polyfit(np.log(np.arange(2, 12)), np.log(E), 1)[0]
    assert -1.9 < slope < -1.45, slope
