"""Pins of the oracle's BDF integrator and of the reaction ODE it integrates
in MRSDC mode 2 (Sec. 3.2, eq. mrupdate2): closed-form solutions, a matrix
exponential, an independent library integrator, polynomial exactness of the
step-size change, and the invariants of the chemistry.  CPU only."""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.linalg as sla

from oracle import bdf, chem, react, thermo
from paper_1309_7327_gb300 import synth


def test_rescale_is_identity_at_unit_ratio():
    for k in range(1, 6):
        assert np.allclose(bdf.rescale_matrix(k, 1.0), np.eye(k + 1), atol=1e-14)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("rho", [0.3, 0.5, 1.7, 2.0])
def test_rescale_is_exact_for_polynomials_of_the_order(k, rho):
    """Backward differences of a degree-k polynomial sampled at spacing h,
    rescaled, equal its differences at spacing rho h."""
    rng = np.random.default_rng(k)
    coef = rng.normal(size=k + 1)
    p = np.polynomial.Polynomial(coef)
    h, tn = 0.37, 1.3

    def diffs(step):
        v = [p(tn - j * step) for j in range(k + 1)]
        return np.array([sum((-1) ** j * math.comb(m, j) * v[j] for j in range(m + 1))
                         for m in range(k + 1)])

    new = bdf.rescale_matrix(k, rho) @ diffs(h)
    assert np.allclose(new, diffs(rho * h), rtol=1e-12, atol=1e-12)


def test_bdf_stiff_scalar_with_known_solution():
    """y' = lam (y - cos t) - sin t, y(0) = 1: y = cos t for any lam."""
    lam = -1e4
    f = lambda t, y: lam * (y - np.cos(t)) - np.sin(t)          # noqa: E731
    jac = lambda t, y: (f(t, y), np.array([[lam]]))            # noqa: E731
    y, st = bdf.bdf_integrate(f, jac, 2.0, np.array([1.0]), np.array([1e-12]), 1e-8)
    assert abs(y[0] - math.cos(2.0)) < 1e-7
    assert st["steps"] < 400
    assert max(st["orders"]) >= 3


def test_bdf_linear_system_matches_matrix_exponential():
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.normal(size=(4, 4)))
    A = Q @ np.diag([-1.0, -30.0, -1e3, -1e5]) @ Q.T
    y0 = rng.normal(size=4)
    f = lambda t, y: A @ y                                     # noqa: E731
    jac = lambda t, y: (A @ y, A)                              # noqa: E731
    T = 1.5
    y, _ = bdf.bdf_integrate(f, jac, T, y0, np.full(4, 1e-12), 1e-9)
    exact = sla.expm(A * T) @ y0
    assert np.abs(y - exact).max() < 1e-7 * np.abs(y0).max()


def test_bdf_robertson_against_a_library_integrator():
    """The stiff Robertson kinetics, against scipy's Radau IIA at tight
    tolerances (an independent implicit Runge-Kutta method)."""
    def f(t, y):
        return np.array([-0.04 * y[0] + 1e4 * y[1] * y[2],
                         0.04 * y[0] - 1e4 * y[1] * y[2] - 3e7 * y[1] ** 2,
                         3e7 * y[1] ** 2])

    def jac(t, y):
        J = np.array([[-0.04, 1e4 * y[2], 1e4 * y[1]],
                      [0.04, -1e4 * y[2] - 6e7 * y[1], -1e4 * y[1]],
                      [0.0, 6e7 * y[1], 0.0]])
        return f(t, y), J

    y0 = np.array([1.0, 0.0, 0.0])
    y, st = bdf.bdf_integrate(f, jac, 40.0, y0, np.array([1e-10, 1e-14, 1e-10]), 1e-8)
    ref = si.solve_ivp(f, (0, 40.0), y0, method="Radau", rtol=1e-12, atol=[1e-16, 1e-20, 1e-16],
                       jac=lambda t, y: jac(t, y)[1]).y[:, -1]
    assert np.all(np.abs(y - ref) <= 1e-6 * np.abs(ref) + 1e-15)
    assert abs(y.sum() - 1.0) < 1e-12                 # linear invariant kept to rounding


def test_bdf_reaches_fifth_order_on_a_smooth_problem():
    f = lambda t, y: -y                                        # noqa: E731
    jac = lambda t, y: (-y, -np.eye(1))                        # noqa: E731
    y, st = bdf.bdf_integrate(f, jac, 10.0, np.array([1.0]), np.array([1e-16]), 1e-11)
    assert max(st["orders"]) == 5
    assert abs(y[0] - math.exp(-10.0)) < 1e-9 * math.exp(-10.0) * 100


def _cell(ns, nr, seed=2, T=1400.0):
    m = synth.make_mechanism(ns, nr, seed)
    rng = np.random.default_rng(seed)
    Y = rng.uniform(0.02, 1.0, ns)
    Y /= Y.sum()
    prim = np.concatenate([[300.0, -200.0, 150.0, T, thermo.P_ATM], Y])
    U = thermo.conserved(prim.reshape(-1, 1), m.nasa7, m.W)[:, 0]
    return m, U


@pytest.mark.parametrize("ns,nr", [(3, 2), (9, 21), (21, 84)])
def test_reaction_jacobian_matches_central_differences(ns, nr):
    """The analytic Jacobian (fixed rho and e: the temperature moves with
    the composition) against central differences of the cell ODE."""
    m, U = _cell(ns, nr)
    G = np.zeros_like(U)
    f, jac, y0, rho0 = react.cell_ode(U, G, m)
    _, J = jac(0.0, y0)
    Jfd = np.zeros_like(J)
    for j in range(ns):
        d = 1e-6 * max(abs(y0[j]), 1e-3 * rho0)
        yp, ym = y0.copy(), y0.copy()
        yp[j] += d
        ym[j] -= d
        Jfd[:, j] = (f(0.0, yp) - f(0.0, ym)) / (2 * d)
    scale = np.abs(Jfd).max()
    assert np.abs(J - Jfd).max() <= 1e-5 * scale
    # the temperature coupling is a real part of it
    w = chem.production_rates(np.asarray(rho0), np.asarray(1400.0), y0 / rho0, m)
    assert np.abs(J).max() > 0 and np.abs(w).max() > 0


def test_reaction_ode_keeps_mass_and_elements():
    """Sum_k rho Y_k = rho and the element totals are linear invariants of
    the reaction ODE; the BDF method keeps them to rounding."""
    m, U = _cell(9, 21, seed=4, T=1800.0)
    G = np.zeros_like(U)
    out, st = react.integrate_cell(U, G, 2e-6, m)
    y0, y = U[5:], out[5:]
    assert st["steps"] > 3
    assert np.abs(y - y0).max() > 1e-6 * U[0]          # the composition moved
    assert abs(y.sum() - U[0]) <= 1e-13 * U[0]
    el0 = m.composition.T @ (y0 / m.W)
    el = m.composition.T @ (y / m.W)
    assert np.abs(el - el0).max() <= 1e-12 * np.abs(el0).max()
    assert np.array_equal(out[:5], U[:5])


def test_reaction_ode_two_isomers_closed_form():
    """A <=> B with identical thermodynamics and molar mass: K_c = 1, T and
    rho fixed, so c_A - c_B decays as exp(-2 k t) exactly."""
    m = synth.make_mechanism(3, 2, 1)
    nasa = m.nasa7.copy()
    nasa[1] = nasa[0]
    W = m.W.copy()
    W[1] = W[0]
    m.nasa7, m.W = nasa, W
    m.nu_f = np.array([[1, 0, 0]], dtype=np.int32)
    m.nu_r = np.array([[0, 1, 0]], dtype=np.int32)
    m.A = np.array([3.0e5])
    m.b = np.array([0.0])
    m.Ea = np.array([0.0])
    Y = np.array([0.7, 0.1, 0.2])
    prim = np.concatenate([[0.0, 0.0, 0.0, 1200.0, thermo.P_ATM], Y]).reshape(-1, 1)
    U = thermo.conserved(prim, m.nasa7, m.W)[:, 0]
    t = 4e-6
    out, _ = react.integrate_cell(U, np.zeros_like(U), t, m, rtol=1e-10, atol=1e-14)
    cA0, cB0 = U[5] / W[0], U[6] / W[0]
    diff = (cA0 - cB0) * math.exp(-2 * 3.0e5 * t)
    tot = cA0 + cB0
    assert abs(out[5] / W[0] - 0.5 * (tot + diff)) <= 1e-8 * tot
    assert abs(out[6] / W[0] - 0.5 * (tot - diff)) <= 1e-8 * tot
    assert out[7] == U[7]


def test_reaction_ode_at_equilibrium_stays_put():
    """At a constructed chemical equilibrium (every reaction's net rate zero)
    with no forcing the integrator returns the initial state."""
    m = synth.make_mechanism(9, 21, 11)
    rng = np.random.default_rng(5)
    Tst = 1300.0
    Y = rng.uniform(0.05, 1, 9)
    Y /= Y.sum()
    prim = np.concatenate([[0.0, 0.0, 0.0, Tst, thermo.P_ATM], Y]).reshape(-1, 1)
    U = thermo.conserved(prim, m.nasa7, m.W)[:, 0]
    c = U[0] * Y / m.W
    mu0 = (thermo.h_RT(m.nasa7, np.array([Tst]))[:, 0] - thermo.s_R(m.nasa7, np.array([Tst]))[:, 0]
           + np.log(c * thermo.R_U * Tst / thermo.P_ATM))
    m.nasa7 = m.nasa7.copy()
    m.nasa7[:, 6] += mu0
    out, _ = react.integrate_cell(U, np.zeros_like(U), 1e-5, m)
    assert np.abs(out[5:] - U[5:]).max() <= 1e-12 * U[0]


def test_reaction_ode_with_forcing_moves_the_linear_components():
    m, U = _cell(3, 2)
    G = np.zeros_like(U)
    G[0] = 1e-3 * U[0]
    G[5:] = G[0] * U[5:] / U[0]              # consistent with the density forcing
    G[1] = 5.0 * U[0]
    G[4] = 1e-2 * U[4]
    dt = 1e-5
    out, _ = react.integrate_cell(U, G, dt, m)
    assert np.allclose(out[:5], U[:5] + dt * G[:5], rtol=1e-15, atol=0)
    assert abs(out[5:].sum() - out[0]) <= 1e-12 * out[0]


def test_mode2_fixed_point_on_a_chemistry_cell_is_lobatto_collocation():
    """With no advection-diffusion, the mode-2 sweeps (BDF integration of the
    reactions over each coarse interval) converge to the 3-node Lobatto IIIA
    collocation solution of the cell's reaction ODE, solved independently as
    one nonlinear system."""
    import scipy.optimize as so
    from oracle import sdc
    m = synth.make_mechanism(3, 2, 1, kmax=1e9)
    rng = np.random.default_rng(8)
    Y = rng.uniform(0.1, 1.0, 3)
    Y /= Y.sum()
    prim = np.concatenate([[100.0, 0.0, -50.0, 1450.0, thermo.P_ATM], Y]).reshape(-1, 1)
    u0 = thermo.conserved(prim, m.nasa7, m.W)[:, 0]
    f, jac, y0, rho0 = react.cell_ode(u0, np.zeros(8), m)
    dt = 2e-8

    def fR(u):
        fu, _, yu, _ = react.cell_ode(u, np.zeros(8), m)
        out = np.zeros(8)
        out[5:] = fu(0.0, yu)
        return out

    integ = lambda Up, G, dtp: react.integrate_cell(Up, G, dtp, m, rtol=1e-12,   # noqa: E731
                                                    atol=1e-18)[0]
    u2 = sdc.mrsdc2_step(u0, lambda u: np.zeros(8), fR, integ, dt, coarse=3, fine=3, sweeps=30,
                         species=slice(5, 8))[0]
    tau = sdc.gauss_lobatto(3)
    Q = sdc.q_matrix(tau)

    def resid(x):
        Yn = x.reshape(2, 3)
        F = [f(0.0, y0)] + [f(tau[k + 1] * dt, Yn[k]) for k in range(2)]
        return np.concatenate([Yn[k] - y0 - dt * sum(Q[k, j] * F[j] for j in range(3))
                               for k in range(2)]) / rho0

    yc = so.fsolve(resid, np.concatenate([y0, y0]), xtol=1e-14).reshape(2, 3)[1]
    change = np.abs(yc - y0).max()
    assert change > 1e-4 * rho0                       # the chemistry moved
    assert np.abs(u2[5:] - yc).max() < 1e-9 * change
