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
