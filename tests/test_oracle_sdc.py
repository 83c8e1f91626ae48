"""Pins of the oracle's SDC / MRSDC integrators (Sec. 3) and of its
narrow-stencil + SDC heat-equation solver against the paper's App. A
Table stenciltest1.  CPU only."""
import math
import os

import numpy as np
import pytest

from oracle import heat2d, sdc, stencil

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_lobatto_nodes():
    assert np.allclose(sdc.gauss_lobatto(3), [0, 0.5, 1])
    r = math.sqrt(3.0 / 7.0)
    assert np.allclose(sdc.gauss_lobatto(5), [0, (1 - r) / 2, 0.5, (1 + r) / 2, 1])


def test_q_last_row_is_lobatto_quadrature():
    """Last row of Q = Simpson for 3 nodes, the 5-point Lobatto rule for 5."""
    assert np.allclose(sdc.q_matrix(sdc.gauss_lobatto(3))[-1], [1 / 6, 2 / 3, 1 / 6], atol=1e-15)
    assert np.allclose(sdc.q_matrix(sdc.gauss_lobatto(5))[-1],
                       [1 / 20, 49 / 180, 16 / 45, 49 / 180, 1 / 20], atol=1e-15)


def test_s_matrix_three_nodes():
    S = sdc.s_matrix(sdc.gauss_lobatto(3))
    assert np.allclose(S, [[5 / 24, 1 / 3, -1 / 24], [-1 / 24, 1 / 3, 5 / 24]], atol=1e-15)
    # node-to-node integrals sum to the Q rows
    Q = sdc.q_matrix(sdc.gauss_lobatto(5))
    S5 = sdc.s_matrix(sdc.gauss_lobatto(5))
    assert np.allclose(np.cumsum(S5, axis=0), Q, atol=1e-15)


def pade(z, n):
    """Diagonal Pade approximant of e^z of order (n, n)."""
    num = sum(math.factorial(2 * n - j) * math.factorial(n)
              / (math.factorial(2 * n) * math.factorial(j) * math.factorial(n - j)) * z ** j
              for j in range(n + 1))
    den = sum(math.factorial(2 * n - j) * math.factorial(n)
              / (math.factorial(2 * n) * math.factorial(j) * math.factorial(n - j)) * (-z) ** j
              for j in range(n + 1))
    return num / den


@pytest.mark.parametrize("nodes,n", [(3, 2), (5, 4)])
def test_sdc_fixed_point_is_lobatto_iiia(nodes, n):
    """Many sweeps converge to the collocation (Lobatto IIIA) solution whose
    stability function is the (M, M) Pade approximant (eq. compact)."""
    for z in (-0.3, 0.2, -1.0 + 0.5j):
        u, _, _ = sdc.sdc_step(np.array([1.0 + 0j]), lambda u, t: z * u, 1.0,
                               nodes=nodes, sweeps=60)
        assert abs(u[0] - pade(z, n)) < 1e-13


@pytest.mark.parametrize("nodes,sweeps", [(3, 2), (3, 4), (5, 6), (5, 8)])
def test_sdc_order_equals_sweeps(nodes, sweeps):
    """K sweeps give order K when the rule is at least order K (Sec. 3.1)."""
    def f(u, t):
        return np.array([-u[0] * u[1], u[0] ** 2 - 0.5 * u[1] + math.cos(t)])

    def run(n):
        dt = 3.0 / n
        u = np.array([1.0, 0.5])
        F = None
        t = 0.0
        for _ in range(n):
            u, F, _ = sdc.sdc_step(u, f, dt, nodes=nodes, sweeps=sweeps, F0=F, t0=t)
            t += dt
        return u
    ref = run(512)
    e1 = np.abs(run(8) - ref).max()
    e2 = np.abs(run(16) - ref).max()
    rate = math.log2(e1 / e2)
    assert sweeps - 0.5 < rate < sweeps + 1.0, rate


def test_eval_counts_table_mrsdc_runtime():
    """N_evals = steps K M (+1 for f(U_0)) reproduces Table mrsdc_runtime."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "mrsdc_runtime_evals.txt"))
            if l.strip() and not l.startswith("#")]
    for dt_ns, fine, repeat, n_ad, n_r in [tuple(int(v) for v in r) for r in rows]:
        steps = round(420 / dt_ns)
        u = np.array([1.0])
        if fine == 0:
            F, tot = None, 0
            for _ in range(steps):
                u, F, k = sdc.sdc_step(u, lambda u, t: -u, 0.01, nodes=3, sweeps=4, F0=F)
                tot += k
            assert (tot, tot) == (n_ad, n_r)
        else:
            F1 = F2 = None
            t1 = t2 = 0
            for _ in range(steps):
                u, F1, F2, a, b = sdc.mrsdc_step(u, lambda u: -u, lambda u: -2 * u, 0.01,
                                                 coarse=3, fine=fine, repeat=repeat,
                                                 sweeps=4, F10=F1, F20=F2)
                t1 += a
                t2 += b
            assert (t1, t2) == (n_ad, n_r)


@pytest.mark.parametrize("fine,repeat", [(5, 1), (3, 2), (9, 1)])
def test_mrsdc_fourth_order_for_any_fine_nodes(fine, repeat):
    """With 3 coarse Gauss-Lobatto nodes MRSDC is 4th order whatever the fine
    nodes (Sec. 5.1.2)."""
    def f1(u):
        return np.array([-0.5 * u[1], 0.5 * u[0]])

    def f2(u):
        return np.array([-3.0 * u[0] + u[1] ** 2, -2.0 * u[1]])

    def run(n):
        dt = 1.0 / n
        u = np.array([1.0, 0.7])
        F1 = F2 = None
        for _ in range(n):
            u, F1, F2, _, _ = sdc.mrsdc_step(u, f1, f2, dt, coarse=3, fine=fine,
                                             repeat=repeat, sweeps=4, F10=F1, F20=F2)
        return u
    ref = run(512)
    e1 = np.abs(run(8) - ref).max()
    e2 = np.abs(run(16) - ref).max()
    rate = math.log2(e1 / e2)
    assert 3.5 < rate < 5.0, rate


def test_mrsdc_single_fine_group_reduces_to_sdc():
    """With fine = 2 nodes per coarse interval (t2 = t1) and f2 = 0 the
    multirate sweep is the single-rate sweep."""
    def f(u, t=0.0):
        return np.array([-u[0] * u[1], u[0] - u[1]])
    u0 = np.array([1.0, 0.3])
    a, _, _ = sdc.sdc_step(u0, f, 0.3, nodes=3, sweeps=4)
    b, _, _, _, _ = sdc.mrsdc_step(u0, lambda u: f(u), lambda u: 0 * u, 0.3, coarse=3,
                                   fine=2, repeat=1, sweeps=4)
    assert np.allclose(a, b, rtol=1e-14, atol=1e-15)


def _golden_t1():
    out = {}
    for l in open(os.path.join(GOLDEN, "stenciltest1.txt")):
        if l.strip() and not l.startswith("#"):
            s, n, li, l2 = l.split()
            out[(s, int(n))] = (float(li), float(l2))
    return out


STENCILS = {"SMC": (stencil.M47_SMC, stencil.M48_SMC),
            "ZERO": (stencil.M47_ZERO, stencil.M48_ZERO),
            "OPTIMAL": (stencil.M47_OPT, stencil.M48_OPT)}


@pytest.mark.parametrize("name", ["SMC", "ZERO", "OPTIMAL"])
@pytest.mark.parametrize("N", [20, 40])
def test_heat_T1_matches_paper_table(name, N):
    """App. A, Table stenciltest1: narrow stencil + 3-node/4-sweep SDC on T1.
    The printed errors are reproduced to 1% (they agree to 4 digits)."""
    g = _golden_t1()[(name, N)]
    u, ex, _ = heat2d.solve("T1", N, *STENCILS[name])
    linf, l2 = heat2d.errors(u, ex)
    assert abs(linf / g[0] - 1) < 0.01, (linf, g[0])
    assert abs(l2 / g[1] - 1) < 0.01, (l2, g[1])


@pytest.mark.slow
def test_heat_T1_80_and_rate():
    g = _golden_t1()
    u, ex, _ = heat2d.solve("T1", 80, *STENCILS["SMC"])
    linf, l2 = heat2d.errors(u, ex)
    assert abs(linf / g[("SMC", 80)][0] - 1) < 0.05
    rate = math.log2(g[("SMC", 40)][0] / linf)
    assert 7.8 < rate < 8.2


def _collocation_linear(lam, dt, nodes):
    """Closed form of the Gauss-Lobatto collocation solution of u' = lam u,
    u(0) = 1, over one step: U = 1 + dt lam Q U at every node."""
    tau = sdc.gauss_lobatto(nodes)
    Q = np.vstack([np.zeros(nodes), sdc.q_matrix(tau)])      # row 0: U_0 itself
    return np.linalg.solve(np.eye(nodes) - dt * lam * Q, np.ones(nodes))


@pytest.mark.parametrize("nodes", [3, 5])
def test_residual_vanishes_at_the_collocation_solution(nodes):
    """eq. residual: the residual is zero at the collocation solution (in
    closed form for u' = lam u), the SDC sweeps drive it there, and the early
    exit stops once it stagnates, with U_M at the collocation value."""
    lam, dt = -3.0, 0.05
    Uc = _collocation_linear(lam, dt, nodes)
    tau = sdc.gauss_lobatto(nodes)
    F = [np.array([lam * u]) for u in Uc]
    R = sdc.sdc_residual(np.array([1.0]), np.array([Uc[-1]]), F, dt, nodes)
    assert abs(R[0]) < 1e-15
    U, _, nev, hist = sdc.sdc_step_exit(np.array([1.0]), lambda u, t: lam * u, dt, nodes=nodes,
                                        max_sweeps=40, eps=0.5)
    assert abs(U[0] - Uc[-1]) < 1e-15
    # geometric decrease, then the stop once the ratio falls below 1.5
    assert all(hist[i] > 2 * hist[i + 1] for i in range(len(hist) - 2) if hist[i + 1] > 1e-14)
    assert len(hist) < 40 and hist[-1] < 1e-14
    assert nev == 1 + len(hist) * (nodes - 1)


def test_residual_norm_is_per_component_relative():
    R = np.array([[1e-3, -2e-3], [5.0, 0.0]])
    U0 = np.array([[1.0, -4.0], [1e4, 2e4]])
    assert sdc.residual_norm(R, U0) == pytest.approx(max(2e-3 / 4.0, 5.0 / 2e4))
    assert sdc.stop_rule([1e-3, 9e-4], 0.5) and not sdc.stop_rule([1e-3, 1e-5], 0.5)
    assert sdc.stop_rule([1e-3, 0.0], 0.5)


def test_mrsdc_residual_exit_reaches_the_multirate_collocation_solution():
    """The multirate residual (coarse quadrature of f1 plus fine quadrature
    of f2) is driven to rounding level by repeated sweeps and the exit stops
    there; the state then agrees with a 60-sweep run."""
    f1 = lambda u: -1.0 * u
    f2 = lambda u: -4.0 * u
    hist = []
    U, _, _, _, _ = sdc.mrsdc_step(np.array([1.0]), f1, f2, 0.05, coarse=3, fine=5, repeat=1,
                                   sweeps=60, eps=0.5, history=hist)
    Uref, _, _, _, _ = sdc.mrsdc_step(np.array([1.0]), f1, f2, 0.05, coarse=3, fine=5,
                                      sweeps=60)
    assert len(hist) < 60 and hist[-1] < 1e-14
    assert abs(U[0] - Uref[0]) < 1e-15


# ------------------------------------------------------------ mode 2 (eq. mrupdate2)

def _linear_exact_integrate(r):
    """U(dt) of U' = r U + G (closed form)."""
    def integ(U, G, dt):
        return (U + G / r) * math.exp(r * dt) - G / r
    return integ


def _mr2_collocation(u0, a, r, dt, coarse, fine):
    """Mode-2 multirate collocation solution of u' = a u + r u: the
    advection-like term a u on the fine nodes (S22), r u on the coarse ones
    (S21), solved as one linear system."""
    t1, t2, S21, S22 = sdc.mr_matrices(coarse, fine)
    M1, M2 = coarse - 1, t2.shape[0] - 1
    per = M2 // M1
    A = np.zeros((M2 + 1, M2 + 1))
    b = np.zeros(M2 + 1)
    A[0, 0] = 1.0
    b[0] = u0
    for q in range(M2):
        A[q + 1, q + 1] += 1.0
        A[q + 1, q] -= 1.0
        for j in range(M1 + 1):
            A[q + 1, j * per] -= dt * S21[q, j] * r
        for t in range(M2 + 1):
            A[q + 1, t] -= dt * S22[q, t] * a
    return np.linalg.solve(A, b)[-1]


@pytest.mark.parametrize("coarse,fine", [(3, 3), (3, 5), (5, 3)])
def test_mrsdc2_fixed_point_is_the_multirate_collocation_solution(coarse, fine):
    """Iterated to convergence on u' = a u + r u (a on the fine nodes, r on
    the coarse ones, the coarse term integrated exactly over each interval)
    mode 2 reaches the multirate collocation solution."""
    a, r, dt, u0 = -1.3, -4.0, 0.3, 1.7
    ref = _mr2_collocation(u0, a, r, dt, coarse, fine)
    U, _, _, _, _ = sdc.mrsdc2_step(np.array([u0]), lambda u: a * u, lambda u: r * u,
                                    _linear_exact_integrate(r), dt, coarse=coarse, fine=fine,
                                    sweeps=60)
    assert abs(U[0] - ref) < 1e-13
    # and it is a 2 M1-order approximation of exp((a + r) dt), not that value
    assert abs(ref - u0 * math.exp((a + r) * dt)) < 1e-2 * u0


def test_mrsdc2_order_equals_sweeps():
    """u' = r u - u^2 (the logistic equation, closed form) with the linear
    term on the coarse nodes: 4 sweeps, 3 coarse nodes give 4th order, 2
    sweeps 2nd order."""
    r, u0, T = -3.0, 1.0, 1.0
    exact = r / (1.0 + (r / u0 - 1.0) * math.exp(-r * T))
    for sweeps, order in ((4, 4), (2, 2)):
        errs = []
        for n in (8, 16, 32):
            u = np.array([u0])
            dt = T / n
            for _ in range(n):
                u, _, _, _, _ = sdc.mrsdc2_step(u, lambda x: -x * x, lambda x: r * x,
                                                _linear_exact_integrate(r), dt, coarse=3,
                                                fine=3, sweeps=sweeps)
            errs.append(abs(u[0] - exact))
        rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
        assert min(rates) > order - 0.4, (sweeps, errs, rates)


def test_mrsdc2_is_stable_where_mode1_is_not():
    """A stiff coarse term, r dt_p = -100: mode 2 integrates it implicitly and
    its sweeps settle on the collocation solution; mode 1 (the same term
    explicit on the fine nodes) blows up."""
    r, dt, u0 = -2e3, 0.1, 1.0
    A = lambda x: -x * x + 1.0                                 # noqa: E731
    R = lambda x: r * x                                        # noqa: E731
    integ = _linear_exact_integrate(r)
    U = {}
    for sweeps in (12, 30, 60):
        U[sweeps], _, _, _, _ = sdc.mrsdc2_step(np.array([u0]), A, R, integ, dt, coarse=3,
                                                fine=3, sweeps=sweeps)
    assert np.isfinite(U[60][0]) and abs(U[60][0]) < 2.0
    assert abs(U[30][0] - U[60][0]) < 1e-9
    assert abs(U[12][0] - U[60][0]) < 1e-3
    with np.errstate(all="ignore"):
        U1, _, _, _, _ = sdc.mrsdc_step(np.array([u0]), A, R, dt, coarse=3, fine=3, sweeps=4)
    assert not np.isfinite(U1[0]) or abs(U1[0]) > 1e6


def test_mrsdc2_with_the_bdf_integrator_matches_exact_integration():
    """The BDF integrator in place of the closed form changes a mode-2 step
    by no more than its tolerance (stiff coarse term)."""
    from oracle import bdf
    r, dt, u0 = -2e3, 0.05, 1.0
    A = lambda x: -x * x + 1.0                                 # noqa: E731
    R = lambda x: r * x                                        # noqa: E731

    def integ_bdf(U, G, dtp):
        f = lambda t, y: r * y + G                             # noqa: E731
        jac = lambda t, y: (r * y + G, np.array([[r]]))        # noqa: E731
        y, _ = bdf.bdf_integrate(f, jac, dtp, U, np.array([1e-14]), 1e-10)
        return y

    ex, _, _, _, _ = sdc.mrsdc2_step(np.array([u0]), A, R, _linear_exact_integrate(r), dt,
                                     coarse=3, fine=3, sweeps=4)
    bd, _, _, _, _ = sdc.mrsdc2_step(np.array([u0]), A, R, integ_bdf, dt, coarse=3, fine=3,
                                     sweeps=4)
    assert abs(bd[0] - ex[0]) < 1e-8 * abs(ex[0]) + 1e-13


def test_mrsdc2_residual_vanishes_at_the_collocation_solution_and_exit_stops_there():
    """Mode 2's residual (coarse quadrature of the reactions, fine quadrature
    of A) is zero at the multirate collocation solution: the sweeps drive it
    to rounding, the exit stops at stagnation, and the state is the
    collocation value.  (Its sweeps contract more slowly than mode 1's, so
    the stagnation threshold is tighter.)"""
    a, r, dt, u0 = -1.3, -4.0, 0.3, 1.7
    hist = []
    U, _, _, _, _ = sdc.mrsdc2_step(np.array([u0]), lambda u: a * u, lambda u: r * u,
                                    _linear_exact_integrate(r), dt, coarse=3, fine=3, sweeps=60,
                                    eps=0.05, history=hist)
    assert 3 < len(hist) < 60 and hist[-1] < 1e-14
    assert all(hist[i + 1] < hist[i] for i in range(len(hist) - 3))
    assert abs(U[0] - _mr2_collocation(u0, a, r, dt, 3, 3)) < 1e-13
