"""Ideal-gas mixture thermodynamics and primitive variables (Sec. 2.1).

Oracle, test infrastructure only.  Readings where the paper is silent:

* NASA 7-coefficient polynomials, one temperature range, for each species:
  cp/R = a1 + a2 T + a3 T^2 + a4 T^3 + a5 T^4,
  h/(R T) = a1 + a2 T/2 + a3 T^2/3 + a4 T^3/4 + a5 T^4/5 + a6/T,
  s/R = a1 ln T + a2 T + a3 T^2/2 + a4 T^3/3 + a5 T^4/4 + a7.
* E in eq. cns is internal plus kinetic energy with e = sum_k Y_k e_k(T),
  e_k = h_k - R_u T / W_k (formation enthalpies included), so the
  chemistry adds no energy source.
* T is recovered from e by Newton's method from a fixed first guess,
  stopping when |dT| <= tol * T (tol = 1e-13), at most 50 iterations.
"""
from __future__ import annotations

import numpy as np

R_U = 8.31446261815324e7        # erg / (mol K)
R_CAL = 1.98720425864083        # cal / (mol K)
P_ATM = 1.01325e6               # dyn / cm^2


def cp_R(nasa: np.ndarray, T: np.ndarray) -> np.ndarray:
    """[ns, ...] dimensionless molar heat capacity cp_k / R."""
    a = nasa.reshape(nasa.shape + (1,) * T.ndim)
    return a[:, 0] + a[:, 1] * T + a[:, 2] * T ** 2 + a[:, 3] * T ** 3 + a[:, 4] * T ** 4


def h_RT(nasa: np.ndarray, T: np.ndarray) -> np.ndarray:
    """[ns, ...] dimensionless molar enthalpy h_k / (R T)."""
    a = nasa.reshape(nasa.shape + (1,) * T.ndim)
    return (a[:, 0] + a[:, 1] * T / 2 + a[:, 2] * T ** 2 / 3 + a[:, 3] * T ** 3 / 4
            + a[:, 4] * T ** 4 / 5 + a[:, 5] / T)


def s_R(nasa: np.ndarray, T: np.ndarray) -> np.ndarray:
    """[ns, ...] dimensionless molar entropy s_k / R at the standard pressure."""
    a = nasa.reshape(nasa.shape + (1,) * T.ndim)
    return (a[:, 0] * np.log(T) + a[:, 1] * T + a[:, 2] * T ** 2 / 2 + a[:, 3] * T ** 3 / 3
            + a[:, 4] * T ** 4 / 4 + a[:, 6])


def _per_mass(W: np.ndarray, T: np.ndarray) -> np.ndarray:
    return (R_U / W).reshape((-1,) + (1,) * T.ndim)


def h_k(nasa, W, T):
    """[ns, ...] specific enthalpies (erg/g)."""
    return _per_mass(W, T) * T * h_RT(nasa, T)


def cp_k(nasa, W, T):
    return _per_mass(W, T) * cp_R(nasa, T)


def e_k(nasa, W, T):
    """[ns, ...] specific internal energies e_k = h_k - R_u T / W_k."""
    return h_k(nasa, W, T) - _per_mass(W, T) * T


def cv_k(nasa, W, T):
    return cp_k(nasa, W, T) - _per_mass(W, T)


def temperature(nasa, W, Y: np.ndarray, e: np.ndarray, T0: float = 1000.0,
                tol: float = 1e-13, maxit: int = 50):
    """Solve sum_k Y_k e_k(T) = e for T by Newton's method.

    Returns (T, converged mask).  Every cell iterates from T0; a cell stops
    changing once its own step satisfied |dT| <= tol * T.
    """
    T = np.full(e.shape, T0, dtype=e.dtype)
    done = np.zeros(e.shape, dtype=bool)
    for _ in range(maxit):
        f = np.sum(Y * e_k(nasa, W, T), axis=0) - e
        fp = np.sum(Y * cv_k(nasa, W, T), axis=0)
        dT = f / fp
        Tn = T - dT
        T = np.where(done, T, Tn)
        done = done | (np.abs(dT) <= tol * np.abs(Tn))
        if done.all():
            break
    return T, done


def primitives(U: np.ndarray, nasa, W, T0: float = 1000.0) -> dict:
    """Primitive variables from the conserved state U = (rho, rho u, rho v,
    rho w, rho E, rho Y_1 .. rho Y_ns) of eq. cns."""
    ns = W.shape[0]
    rho = U[0]
    vel = U[1:4] / rho
    E = U[4] / rho
    Y = U[5:5 + ns] / rho
    e = E - 0.5 * np.sum(vel ** 2, axis=0)
    T, ok = temperature(nasa, W, Y, e, T0=T0)
    Wmix_inv = np.sum(Y / W.reshape((-1,) + (1,) * rho.ndim), axis=0)
    p = rho * R_U * T * Wmix_inv
    X = (Y / W.reshape((-1,) + (1,) * rho.ndim)) / Wmix_inv
    return dict(rho=rho, vel=vel, E=E, e=e, Y=Y, T=T, p=p, X=X, converged=ok,
                h=h_k(nasa, W, T), cp=np.sum(Y * cp_k(nasa, W, T), axis=0))


def conserved(prim: np.ndarray, nasa, W) -> np.ndarray:
    """U from prim = (u, v, w, T, p, Y_1..Y_ns): rho from the ideal-gas law,
    rho E = rho (sum_k Y_k e_k(T) + |u|^2 / 2)."""
    ns = W.shape[0]
    vel = prim[0:3]
    T = prim[3]
    p = prim[4]
    Y = prim[5:5 + ns]
    Wmix_inv = np.sum(Y / W.reshape((-1,) + (1,) * T.ndim), axis=0)
    rho = p / (R_U * T * Wmix_inv)
    e = np.sum(Y * e_k(nasa, W, T), axis=0)
    U = np.empty((5 + ns,) + T.shape, dtype=T.dtype)
    U[0] = rho
    U[1:4] = rho * vel
    U[4] = rho * (e + 0.5 * np.sum(vel ** 2, axis=0))
    U[5:] = rho * Y
    return U
