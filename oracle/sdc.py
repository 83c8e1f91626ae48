"""Spectral deferred corrections (Sec. 3.1) and mode-1 multirate SDC
(Sec. 3.2).  Oracle, test infrastructure only; plain NumPy FP64.

Nodes are on the unit interval; the integration matrices are per unit
time step and are multiplied by dt in the updates.

* Gauss-Lobatto nodes: 0, 1 and the roots of P'_{M}(2t - 1).
* Q (eq. gaussapp / compact): q_{mj} = integral over [0, tau_m] of the
  Lagrange polynomial L_j through all nodes, m = 1..M  (M x (M+1)).
* S (node-to-node): s_{mj} = integral over [tau_m, tau_{m+1}] of L_j,
  m = 0..M-1  (M x (M+1)).
  Integrals are exact: Gauss-Legendre quadrature with more points than the
  polynomial degree requires.
* SDC sweep (eq. expsdc), spread start U^0 = [U_0, ..., U_0]:
    U^{k+1}_{m+1} = U^{k+1}_m + dt_m [f(U^{k+1}_m) - f(U^k_m)] + dt (S F^k)_m.
  f(U_0) is evaluated once and recycled from the previous step's last node
  (so N_evals = K M per step, plus one for the very first step).
* MRSDC mode 1 (eq. mrupdate), type (b)/(c) fine nodes: each coarse
  interval holds R repetitions of a Y-point Gauss-Lobatto group; S21 uses the
  coarse Lagrange basis, S22 the piecewise (per group) Lagrange basis, and
  the coarse term f1 is frozen at the coarse node p to the left of the fine
  node q.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as L


def gauss_lobatto(n: int) -> np.ndarray:
    """n Gauss-Lobatto nodes on [0, 1]."""
    if n < 2:
        raise ValueError("at least two Lobatto nodes")
    c = np.zeros(n)
    c[-1] = 1.0                                   # P_{n-1}
    inner = L.legroots(L.legder(c)) if n > 2 else np.array([])
    x = np.concatenate([[-1.0], np.sort(inner.real), [1.0]])
    return 0.5 * (x + 1.0)


def _lagrange_integrals(nodes: np.ndarray, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """I[i, j] = integral_{a_i}^{b_i} L_j(t) dt, L_j the Lagrange basis on nodes."""
    n = nodes.shape[0]
    gx, gw = L.leggauss(n + 2)
    out = np.zeros((a.shape[0], n))
    for i in range(a.shape[0]):
        t = 0.5 * (b[i] - a[i]) * gx + 0.5 * (b[i] + a[i])
        w = 0.5 * (b[i] - a[i]) * gw
        for j in range(n):
            lj = np.ones_like(t)
            for m in range(n):
                if m != j:
                    lj = lj * (t - nodes[m]) / (nodes[j] - nodes[m])
            out[i, j] = np.sum(w * lj)
    return out


def q_matrix(nodes: np.ndarray) -> np.ndarray:
    M = nodes.shape[0] - 1
    return _lagrange_integrals(nodes, np.zeros(M), nodes[1:])


def s_matrix(nodes: np.ndarray) -> np.ndarray:
    return _lagrange_integrals(nodes, nodes[:-1], nodes[1:])


def sdc_step(U0, f, dt: float, nodes: int = 3, sweeps: int = 4, F0=None, t0: float = 0.0):
    """One SDC time step of eq. expsdc.

    f: callable (U, t) -> dU/dt.  F0: f(U0, t0) if already known (recycled).
    Returns (U_new, f(U_new), number of f evaluations made).
    """
    tau = gauss_lobatto(nodes)
    M = nodes - 1
    S = s_matrix(tau)
    dtm = dt * np.diff(tau)
    nev = 0
    if F0 is None:
        F0 = f(U0, t0)
        nev += 1
    tm = t0 + dt * tau
    Fold = [F0] * (M + 1)               # spread start: F^0 = f(U0) at every node
    U = U0
    for _ in range(sweeps):
        Fnew = [F0] + [None] * M
        U = U0
        for m in range(M):
            if m > 0:
                Fnew[m] = f(U, tm[m])
                nev += 1
            SF = sum(S[m, j] * Fold[j] for j in range(M + 1))
            U = U + dtm[m] * (Fnew[m] - Fold[m]) + dt * SF
        Fnew[M] = f(U, tm[M])
        nev += 1
        Fold = Fnew
    return U, Fold[M], nev


def sdc_residual(U0, Unodes_last, F, dt, nodes):
    """R^k = U_0 + dt q . F^k - U_M^k  (eq. residual), q the last row of Q."""
    q = q_matrix(gauss_lobatto(nodes))[-1]
    return U0 + dt * sum(q[j] * F[j] for j in range(nodes)) - Unodes_last


def residual_norm(R, U0) -> float:
    """|R| = max over components c of max|R_c| / max|U0_c| (the paper gives
    no norm; this reading is scale-free per component).  Arrays [nv, ...]."""
    R = np.abs(np.asarray(R)).reshape(np.shape(R)[0], -1).max(axis=1)
    S = np.abs(np.asarray(U0)).reshape(np.shape(U0)[0], -1).max(axis=1)
    return float(np.max(np.where(S > 0, R / np.where(S > 0, S, 1.0), R)))


def stop_rule(hist, eps: float) -> bool:
    """End the step once |R^(k-1)| / |R^k| < 1 + eps (the successive
    residuals no longer shrink) or |R^k| = 0."""
    if hist[-1] == 0.0:
        return True
    return len(hist) > 1 and hist[-2] / hist[-1] < 1.0 + eps


def sdc_step_exit(U0, f, dt: float, nodes: int = 3, max_sweeps: int = 8, eps: float = 0.5,
                  F0=None, t0: float = 0.0):
    """sdc_step with the residual early exit of Sec. 3.1: after every sweep
    compute |R^k| (eq. residual) and stop by stop_rule.  Returns (U_new,
    f(U_new), evaluations, residual history)."""
    tau = gauss_lobatto(nodes)
    M = nodes - 1
    S = s_matrix(tau)
    q = q_matrix(tau)[-1]
    dtm = dt * np.diff(tau)
    nev = 0
    if F0 is None:
        F0 = f(U0, t0)
        nev += 1
    tm = t0 + dt * tau
    Fold = [F0] * (M + 1)
    U = U0
    hist = []
    for _ in range(max_sweeps):
        Fnew = [F0] + [None] * M
        U = U0
        for m in range(M):
            if m > 0:
                Fnew[m] = f(U, tm[m])
                nev += 1
            SF = sum(S[m, j] * Fold[j] for j in range(M + 1))
            U = U + dtm[m] * (Fnew[m] - Fold[m]) + dt * SF
        Fnew[M] = f(U, tm[M])
        nev += 1
        Fold = Fnew
        R = U0 + dt * sum(q[j] * Fold[j] for j in range(M + 1)) - U
        hist.append(residual_norm(R, U0))
        if stop_rule(hist, eps):
            break
    return U, Fold[M], nev, hist


# ---------------------------------------------------------------- multirate

def mr_nodes(coarse: int, fine: int, repeat: int = 1):
    """Coarse Gauss-Lobatto nodes and the fine nodes: in every coarse interval
    ``repeat`` consecutive groups of ``fine`` Gauss-Lobatto nodes (type (b) for
    repeat = 1, type (c) otherwise).  Returns (t1, t2, group_of_fine_interval,
    group_node_indices)."""
    t1 = gauss_lobatto(coarse)
    g = gauss_lobatto(fine)
    t2 = [0.0]
    groups = []
    for p in range(coarse - 1):
        a, b = t1[p], t1[p + 1]
        for r in range(repeat):
            lo = a + (b - a) * r / repeat
            hi = a + (b - a) * (r + 1) / repeat
            start = len(t2) - 1
            t2.extend(list(lo + (hi - lo) * g[1:]))
            groups.append(list(range(start, start + fine)))
    t2 = np.array(t2)
    interval_group = []
    for gi, nodes in enumerate(groups):
        interval_group.extend([gi] * (fine - 1))
    return t1, t2, np.array(interval_group), groups


def mr_matrices(coarse: int, fine: int, repeat: int = 1):
    """S21 (M2 x (M1+1)) and S22 (M2 x (M2+1)) per unit time step."""
    t1, t2, ig, groups = mr_nodes(coarse, fine, repeat)
    M2 = t2.shape[0] - 1
    S21 = _lagrange_integrals(t1, t2[:-1], t2[1:])
    S22 = np.zeros((M2, M2 + 1))
    for q in range(M2):
        nodes = groups[ig[q]]
        blk = _lagrange_integrals(t2[nodes], t2[q:q + 1], t2[q + 1:q + 2])
        S22[q, nodes] = blk[0]
    return t1, t2, S21, S22


def mrsdc_step(U0, f1, f2, dt: float, coarse: int = 3, fine: int = 5, repeat: int = 1,
               sweeps: int = 4, F10=None, F20=None, eps: float = 0.0, history=None):
    """One mode-1 MRSDC step (eq. mrupdate).  f1: slow (advection-diffusion),
    f2: fast (reactions).  Returns (U_new, f1(U_new), f2(U_new), n_f1, n_f2).

    eps > 0: after every sweep the residual U_0 + dt (q1 . F1 + q2 . F2) - U_M
    (eq. residual with the coarse and the fine quadrature, q1 and q2 the
    column sums of S21 and S22) is appended to `history` (a list) and the
    step ends by stop_rule.  f2 returns full-size arrays (zero outside the
    species components)."""
    t1, t2, S21, S22 = mr_matrices(coarse, fine, repeat)
    M1, M2 = coarse - 1, t2.shape[0] - 1
    per = M2 // M1                       # fine intervals per coarse interval
    dtq = dt * np.diff(t2)
    n1 = n2 = 0
    if F10 is None:
        F10 = f1(U0)
        n1 += 1
    if F20 is None:
        F20 = f2(U0)
        n2 += 1
    F1old = [F10] * (M1 + 1)
    F2old = [F20] * (M2 + 1)
    U = U0
    for _ in range(sweeps):
        F1new = [F10] + [None] * M1
        F2new = [F20] + [None] * M2
        U = U0
        for q in range(M2):
            p = q // per
            if q % per == 0 and p > 0:
                F1new[p] = f1(U)
                n1 += 1
            if q > 0:
                F2new[q] = f2(U)
                n2 += 1
            S1 = sum(S21[q, j] * F1old[j] for j in range(M1 + 1))
            S2 = sum(S22[q, j] * F2old[j] for j in range(M2 + 1) if S22[q, j] != 0.0)
            U = (U + dtq[q] * (F1new[p] - F1old[p]) + dtq[q] * (F2new[q] - F2old[q])
                 + dt * S2 + dt * S1)
        F1new[M1] = f1(U)
        F2new[M2] = f2(U)
        n1 += 1
        n2 += 1
        F1old, F2old = F1new, F2new
        if eps > 0.0:
            q1 = S21.sum(axis=0)
            q2 = S22.sum(axis=0)
            R = (U0 + dt * sum(q1[j] * F1old[j] for j in range(M1 + 1))
                 + dt * sum(q2[t] * F2old[t] for t in range(M2 + 1)) - U)
            history.append(residual_norm(R, U0))
            if stop_rule(history, eps):
                break
    return U, F1old[M1], F2old[M2], n1, n2


def mrsdc2_step(U0, fA, fR, integrate, dt: float, coarse: int = 3, fine: int = 5,
                repeat: int = 1, sweeps: int = 4, FA0=None, FR0=None, species=None,
                eps: float = 0.0, history=None):
    """One mode-2 MRSDC step (eq. mrupdate2): the reactions R are the coarse
    component (nodes t1), advection-diffusion A the fine one (nodes t2,
    forward-Euler substeps).  Returns (U_new, A(U_new), R(U_new), n_A, n_R).

    The coarse term is held at the right coarse node p + 1 of the interval
    and is implicit.  Reading of "computed with VODE": the reaction ODE of
    the interval, dU/dtau = R(U) + G (`integrate(U_p, G, dt_p)`, G constant),
    is integrated from U^{k+1}_p with the BDF method, and its mean reaction
    rate Rt = (U*(dt_p) - U_p)/dt_p - G (species components) stands for
    f_slow(U^{k+1}_{p+1}); Rt^k (the previous sweep's) for f_slow(U^k_{p+1}).
    Per coarse interval p of a sweep:

    1. G1 = (dt/dt_p) sum_{q in p} [(S21 F1^k)_q + (S22 F2^k)_q] - Rt^k_{p+1}
       (the terms of the summed fine updates known before the interval's
       sweep); Rt' from integrate(U_p, G1, dt_p);
    2. the fine substeps of eq. mrupdate2 with f_slow(U^{k+1}_{p+1}) = Rt',
       which give A(U^{k+1}_q) at the interval's fine nodes;
    3. G2 = G1 + (1/dt_p) sum_q dt_q [A(U^{k+1}_q) - A^k_q];
       U^{k+1}_{p+1} = integrate(U_p, G2, dt_p) and Rt^{k+1}_{p+1} its mean
       rate: the end value satisfies eq. mrupdate2 summed over the interval
       with every term of this sweep, the stiff reaction term implicitly;
    4. F1^{k+1}_{p+1} = R(U^{k+1}_{p+1}) (true R at the coarse node, for the
       next sweep's quadrature S21 F1).

    At a fixed point Rt' = Rt^{k+1} = Rt^k, the substeps of 2 end where 3
    does, and U is the multirate collocation solution.  Spread start:
    Rt^0 = F1^0 = R(U_0), F2^0 = A(U_0).  Taking the end value from the
    fine substeps instead (one integration per interval) is not stable once
    the reaction time scale is far below dt_p: the advection corrections
    would then enter the end value explicitly, next to a stiff R.

    fR returns full-size arrays (zero outside the species components);
    `species` is the index (slice or mask) of those components, used to
    zero Rt outside them.  eps > 0: the residual of eq. residual (the
    coarse quadrature of R, the fine one of A) after every sweep goes to
    `history` and the step ends by stop_rule, as in mrsdc_step."""
    t1, t2, S21, S22 = mr_matrices(coarse, fine, repeat)
    M1, M2 = coarse - 1, t2.shape[0] - 1
    per = M2 // M1
    dtq = dt * np.diff(t2)
    nA = nR = 0
    if FA0 is None:
        FA0 = fA(U0)
        nA += 1
    if FR0 is None:
        FR0 = fR(U0)
        nR += 1
    F1old = [FR0] * (M1 + 1)             # true R at the coarse nodes
    Rtold = [FR0] * (M1 + 1)             # interval-mean R at the coarse nodes 1..M1
    F2old = [FA0] * (M2 + 1)             # A at the fine nodes

    def mean_rate(Up, G, dtp):
        Us = integrate(Up, G, dtp)
        Rt = (Us - Up) / dtp - G
        if species is not None:
            mask = np.zeros(Rt.shape[0], dtype=bool)
            mask[species] = True
            Rt[~mask] = 0.0
        return Us, Rt

    U = U0
    for _ in range(sweeps):
        F1new = [FR0] + [None] * M1
        Rtnew = [None] * (M1 + 1)
        F2new = [FA0] + [None] * M2
        U = U0
        for p in range(M1):
            qs = range(p * per, (p + 1) * per)
            dtp = dt * (t1[p + 1] - t1[p])
            S = {q: dt * sum(S21[q, j] * F1old[j] for j in range(M1 + 1))
                 + dt * sum(S22[q, j] * F2old[j] for j in range(M2 + 1) if S22[q, j] != 0.0)
                 for q in qs}
            G1 = sum(S[q] for q in qs) / dtp - Rtold[p + 1]
            _, Rt1 = mean_rate(U, G1, dtp)
            W = U
            for q in qs:
                if q > 0:
                    F2new[q] = fA(W)
                    nA += 1
                W = (W + dtq[q] * (Rt1 - Rtold[p + 1]) + dtq[q] * (F2new[q] - F2old[q]) + S[q])
            G2 = G1 + sum(dtq[q] * (F2new[q] - F2old[q]) for q in qs) / dtp
            U, Rtnew[p + 1] = mean_rate(U, G2, dtp)
            F1new[p + 1] = fR(U)
            nR += 1
        F2new[M2] = fA(U)
        nA += 1
        F1old, F2old, Rtold = F1new, F2new, Rtnew
        if eps > 0.0:
            q1 = S21.sum(axis=0)
            q2 = S22.sum(axis=0)
            R = (U0 + dt * sum(q1[j] * F1old[j] for j in range(M1 + 1))
                 + dt * sum(q2[t] * F2old[t] for t in range(M2 + 1)) - U)
            history.append(residual_norm(R, U0))
            if stop_rule(history, eps):
                break
    return U, F2old[M2], F1old[M1], nA, nR
