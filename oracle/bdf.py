"""Variable-order, variable-step BDF integrator for stiff ODE systems
(oracle; test infrastructure only, plain NumPy FP64).

The paper integrates the reaction terms of MRSDC mode 2 (Sec. 3.2, eq.
mrupdate2) with the variable-order BDF methods of VODE.  VODE is a separate
package that the paper only cites; what is restated here is the method
family it belongs to, written from the textbook form of the BDF methods:

* Order k = 1..5 backward differentiation formula in backward-difference
  form (Hairer & Wanner, Solving ODEs II, Sec. III.1 / IV.8):
      sum_{m=1}^{k} (1/m) nabla^m y_{n+1} = h f(t_{n+1}, y_{n+1}).
  With the predictor y^(0) = sum_{m=0}^{k} nabla^m y_n and
  d = y_{n+1} - y^(0) (= nabla^{k+1} y_{n+1}) this is
      gamma_k d + sum_{m=1}^{k} gamma_m nabla^m y_n = h f(y^(0) + d),
  gamma_m = sum_{j=1}^{m} 1/j, solved for d by Newton's method with the
  iteration matrix I - (h / gamma_k) J.
* Local error estimate d / (k + 1) (the leading error constant of the
  order-k formula times nabla^{k+1} y); weighted RMS norm with weights
  w_i = wabs_i + rtol |y_n,i| (VODE's error weights).
* Step changes keep the backward differences of the interpolating
  polynomial: the polynomial through y_n .. y_{n-k} at spacing h is
  resampled at spacing rho h (`rescale_matrix`) -- the quasi-constant
  step-size form (Shampine & Reichelt, SIAM J. Sci. Comput. 18, 1997).
* Order and step selection after k + 1 steps of equal size: the orders
  k - 1, k, k + 1 are compared by their predicted step factors
  err^(-1/(order+1)) (errors of k - 1 and k + 1 from nabla^k y and
  nabla^{k+2} y); rejected steps shrink by max(0.2, 0.9 err^(-1/(k+1))),
  Newton failures halve the step.
* Starting step: the algorithm of Hairer, Norsett & Wanner (Solving ODEs I,
  Sec. II.4) for a first-order start.

* The Newton matrix I - c J (c = h / gamma_k) is kept across steps, as in
  VODE: it is rebuilt (Jacobian at the predicted point, new factors) when
  there is none, after 20 steps, when c has moved by more than 30% since
  the factorisation, or when the Newton iteration failed with an old one
  (the step is then retried with the same h); with an old matrix the
  correction is scaled by 2 / (1 + c / c_lu).  A Newton failure with a new
  matrix halves the step.

The constants (NEWTON_MAXITER, the Newton tolerance, the factors, the
rebuild thresholds) are this restatement's choices; the CUDA integrator
uses the same ones.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

MAX_ORDER = 5
NEWTON_MAXITER = 4
SAFETY = 0.9
MIN_FACTOR = 0.2
MAX_FACTOR = 10.0
LU_MAX_STEPS = 20       # steps before the Newton matrix is rebuilt regardless
LU_MAX_CHANGE = 0.3     # |c / c_lu - 1| above which it is rebuilt
EPS = float(np.finfo(np.float64).eps)

GAMMA = np.array([0.0] + [sum(1.0 / j for j in range(1, m + 1)) for m in range(1, MAX_ORDER + 1)])


def newton_tol(rtol: float) -> float:
    """Newton stopping tolerance in units of the local error tolerance."""
    return max(10.0 * EPS / rtol, min(0.03, math.sqrt(rtol)))


def rescale_matrix(k: int, rho: float) -> np.ndarray:
    """(k+1) x (k+1) matrix T with nabla'(rows 0..k) = T @ nabla(rows 0..k)
    when the step changes from h to rho h.

    Newton's backward form of the interpolating polynomial,
        P(t_n + s h) = sum_m [s (s+1) .. (s+m-1) / m!] nabla^m y_n,
    is sampled at s = -j rho (j = 0..k) and differenced again:
        nabla'^m = sum_j (-1)^j C(m, j) P(t_n - j rho h)."""
    A = np.zeros((k + 1, k + 1))
    for j in range(k + 1):
        s = -j * rho
        for m in range(k + 1):
            v = 1.0
            for i in range(m):
                v *= (s + i) / (i + 1)
            A[j, m] = v
    B = np.zeros((k + 1, k + 1))
    for m in range(k + 1):
        for j in range(m + 1):
            B[m, j] = (-1) ** j * math.comb(m, j)
    return B @ A


def _rms(v: np.ndarray) -> float:
    return float(np.sqrt(np.mean(v * v)))


def _factor(err: float, p: int) -> float:
    return math.inf if err == 0.0 else err ** (-1.0 / p)


class BdfFailure(RuntimeError):
    pass


def bdf_integrate(f, jac, t_end: float, y0: np.ndarray, wabs: np.ndarray, rtol: float,
                  max_attempts: int = 100000):
    """Integrate y' = f(t, y) from t = 0 to t_end.

    f(t, y) -> f;  jac(t, y) -> (f, J) with J = df/dy.  wabs: absolute error
    weights (array); rtol: relative tolerance.  Returns (y(t_end), stats)."""
    n = y0.shape[0]
    y0 = np.asarray(y0, dtype=np.float64)
    eta = newton_tol(rtol)
    stats = dict(steps=0, rejected=0, newton_failures=0, f_evals=0, jac_evals=0, orders=[])
    # starting step (Hairer, Norsett & Wanner, Sec. II.4, order 1)
    f0 = f(0.0, y0)
    stats["f_evals"] += 1
    w = wabs + rtol * np.abs(y0)
    d0, d1 = _rms(y0 / w), _rms(f0 / w)
    h0 = 1e-6 if (d0 < 1e-5 or d1 < 1e-5) else 0.01 * d0 / d1
    h0 = min(h0, t_end)
    f1 = f(h0, y0 + h0 * f0)
    stats["f_evals"] += 1
    d2 = _rms((f1 - f0) / w) / h0
    dm = max(d1, d2)
    h1 = max(1e-6, 1e-3 * h0) if dm <= 1e-15 else math.sqrt(0.01 / dm)
    h = min(100.0 * h0, h1, t_end)

    D = np.zeros((MAX_ORDER + 3, n))
    D[0] = y0
    D[1] = h * f0
    k = 1
    n_equal = 0
    t = 0.0
    attempts = 0
    lu, c_lu, since_lu = None, 1.0, 0
    while t < t_end:
        attempts += 1
        if attempts > max_attempts or h <= 1e-14 * t_end:
            raise BdfFailure(f"step size collapsed at t = {t} (h = {h})")
        last = False
        if t + h >= t_end:
            rho = (t_end - t) / h
            D[:k + 1] = rescale_matrix(k, rho) @ D[:k + 1]
            h = t_end - t
            n_equal = 0
            last = True
        y_pred = D[:k + 1].sum(axis=0)
        psi = (GAMMA[1:k + 1] @ D[1:k + 1]) / GAMMA[k]
        c = h / GAMMA[k]
        w = wabs + rtol * np.abs(D[0])
        fresh = lu is None or since_lu >= LU_MAX_STEPS or abs(c / c_lu - 1.0) > LU_MAX_CHANGE
        if fresh:
            fy, J = jac(t + h, y_pred)
            stats["jac_evals"] += 1
            lu = sla.lu_factor(np.eye(n) - c * J)
            c_lu = c
            since_lu = 0
        else:
            fy = f(t + h, y_pred)
        stats["f_evals"] += 1
        # a matrix factored at another c: scale the correction (VODE's rule)
        scale = 2.0 / (1.0 + c / c_lu)
        d = np.zeros(n)
        y = y_pred.copy()
        converged = False
        dn_old = None
        for it in range(NEWTON_MAXITER):
            if it > 0:
                fy = f(t + h, y)
                stats["f_evals"] += 1
            delta = scale * sla.lu_solve(lu, c * fy - psi - d)
            y = y + delta
            d = d + delta
            dn = _rms(delta / w)
            if dn == 0.0:
                converged = True
                break
            if it > 0:
                rate = dn / dn_old
                if rate >= 1.0 or rate ** (NEWTON_MAXITER - it) / (1.0 - rate) * dn > eta:
                    break
                if rate / (1.0 - rate) * dn < eta:
                    converged = True
                    break
            dn_old = dn
        if not converged:
            stats["newton_failures"] += 1
            if not fresh:
                lu = None                 # retry the step with a new Jacobian
                continue
            D[:k + 1] = rescale_matrix(k, 0.5) @ D[:k + 1]
            h *= 0.5
            n_equal = 0
            continue
        err = _rms(d / (k + 1) / w)
        if err > 1.0:
            stats["rejected"] += 1
            factor = max(MIN_FACTOR, SAFETY * _factor(err, k + 1))
            D[:k + 1] = rescale_matrix(k, factor) @ D[:k + 1]
            h *= factor
            n_equal = 0
            continue
        # accepted: t_{n+1}, and the differences of y_{n+1}
        t = t_end if last else t + h
        since_lu += 1
        stats["steps"] += 1
        stats["orders"].append(k)
        D[k + 2] = d - D[k + 1]
        D[k + 1] = d
        for m in range(k, -1, -1):
            D[m] = D[m] + D[m + 1]
        n_equal += 1
        if t >= t_end:
            break
        if n_equal < k + 1:
            continue
        f_lo = _factor(_rms(D[k] / k / w), k) if k > 1 else 0.0
        f_0 = _factor(err, k + 1)
        f_hi = _factor(_rms(D[k + 2] / (k + 2) / w), k + 2) if k < MAX_ORDER else 0.0
        best, k_new = f_0, k
        if f_lo > best:
            best, k_new = f_lo, k - 1
        if f_hi > best:
            best, k_new = f_hi, k + 1
        factor = min(MAX_FACTOR, SAFETY * best)
        k = k_new
        D[:k + 1] = rescale_matrix(k, factor) @ D[:k + 1]
        h *= factor
        n_equal = 0
    return D[0].copy(), stats
