"""The reaction ODE of one cell over a coarse MRSDC interval, its Jacobian,
and its integration by the BDF integrator (oracle; test infrastructure only,
plain NumPy FP64).

MRSDC mode 2 (Sec. 3.2, eq. mrupdate2) takes the reactions as the coarse
component and evaluates their contribution implicitly "with VODE".  Reading
(the paper gives no more detail): over a coarse interval of length dt_p the
cell ODE

    dU/dtau = R(U) + G,      U(0) = U_p,   0 <= tau <= dt_p,

is integrated with the BDF method, G a constant forcing per cell (all
components) and R the mass-action source, which is non-zero only in the
species components.  Its non-species components therefore move linearly,
U_c(tau) = U_p,c + tau G_c, and the ODE proper is for y = (rho Y_k):

    dy/dtau = rho omega(rho(tau), T(tau, y), y) + G_Y,

T from sum_k (y_k / rho) e_k(T) = e(tau) (Newton, started at the
temperature of U_p), e(tau) = rho E / rho - |rho u|^2 / (2 rho^2) of the
linearly moving components.  The BDF error weights are
w_k = atol rho_p + rtol |y_k| (atol in mass-fraction units).

Jacobian (analytic): with c_j = y_j / W_j, the two terms of every reaction
F_r = k_f prod c^nu', B_r = k_r prod c^nu'' and q_r = F_r - B_r,

    J_kj = d(rho omega_k)/dy_j at fixed T + d(rho omega_k)/dT * dT/dy_j,
    dT/dy_j = -e_j(T) / (rho c_v)                    (fixed rho and e),
    d ln k_f/dT = b/T + Ea/(R_c T^2),
    d ln K_c/dT = sum_k nu_k h_k/(R_u T^2) - (sum_k nu_k)/T.
"""
from __future__ import annotations

import numpy as np

from . import bdf, chem
from .thermo import R_CAL, R_U, P_ATM, cp_k, e_k, h_RT, s_R, temperature, _per_mass


def cell_state(Uc: np.ndarray, Gc: np.ndarray, ns: int):
    """Closures for the non-species components moving linearly in tau."""
    def at(tau):
        rho = Uc[0] + tau * Gc[0]
        m = Uc[1:4] + tau * Gc[1:4]
        E = Uc[4] + tau * Gc[4]
        e = E / rho - 0.5 * float(np.sum((m / rho) ** 2))
        return rho, e
    return at


def _temperature(mech, y, rho, e, T0, tol=1e-13, maxit=50):
    Y = y / rho
    T, ok = temperature(mech.nasa7, np.asarray(mech.W), Y, np.asarray(e), T0=T0, tol=tol,
                        maxit=maxit)
    if not bool(ok):
        raise bdf.BdfFailure("temperature Newton did not converge")
    return float(T)


def jacobian(mech, rho: float, T: float, y: np.ndarray) -> np.ndarray:
    """d(rho omega)/dy at fixed rho and internal energy (module docstring)."""
    W = np.asarray(mech.W)
    ns = W.shape[0]
    Ta = np.asarray(T)
    c = y / W
    g = h_RT(mech.nasa7, Ta) - s_R(mech.nasa7, Ta)
    hRT = h_RT(mech.nasa7, Ta)
    dwdy = np.zeros((ns, ns))
    dwdT = np.zeros(ns)
    for r in range(mech.A.shape[0]):
        nf = mech.nu_f[r].astype(int)
        nr = mech.nu_r[r].astype(int)
        nu = (nr - nf).astype(np.float64)
        kf = mech.A[r] * T ** mech.b[r] * np.exp(-mech.Ea[r] / (R_CAL * T))
        Kc = np.exp(-float(nu @ g)) * (P_ATM / (R_U * T)) ** nu.sum()
        kr = kf / Kc
        Fr = kf * np.prod(c ** nf)
        Br = kr * np.prod(c ** nr)
        dF = np.zeros(ns)
        dB = np.zeros(ns)
        for j in range(ns):
            if nf[j]:
                others = np.prod([c[l] ** nf[l] for l in range(ns) if l != j])
                dF[j] = kf * nf[j] * c[j] ** (nf[j] - 1) * others / W[j]
            if nr[j]:
                others = np.prod([c[l] ** nr[l] for l in range(ns) if l != j])
                dB[j] = kr * nr[j] * c[j] ** (nr[j] - 1) * others / W[j]
        dlnkf = mech.b[r] / T + mech.Ea[r] / (R_CAL * T * T)
        dlnKc = float(nu @ hRT) / T - nu.sum() / T
        dq_dT = Fr * dlnkf - Br * (dlnkf - dlnKc)
        for k in range(ns):
            if nu[k] != 0.0:
                dwdy[k] += W[k] * nu[k] * (dF - dB)
                dwdT[k] += W[k] * nu[k] * dq_dT
    Y = y / rho
    cv = float(np.sum(Y * (cp_k(mech.nasa7, W, Ta) - _per_mass(W, Ta))))
    dTdy = -e_k(mech.nasa7, W, Ta) / (rho * cv)
    return dwdy + np.outer(dwdT, dTdy)


def cell_ode(Uc: np.ndarray, Gc: np.ndarray, mech, T0: float = 1000.0):
    """(f, jac, y0, rho0) of the reaction ODE of one cell (module docstring)."""
    ns = np.asarray(mech.W).shape[0]
    at = cell_state(Uc, Gc, ns)
    rho0, e0 = at(0.0)
    y0 = np.array(Uc[5:5 + ns], dtype=np.float64)
    Tstart = _temperature(mech, y0, rho0, e0, T0)
    gY = np.array(Gc[5:5 + ns], dtype=np.float64)

    def f(tau, y):
        rho, e = at(tau)
        T = _temperature(mech, y, rho, e, Tstart)
        w = chem.production_rates(np.asarray(rho), np.asarray(T), y / rho, mech)
        return w + gY

    def jac(tau, y):
        rho, e = at(tau)
        T = _temperature(mech, y, rho, e, Tstart)
        w = chem.production_rates(np.asarray(rho), np.asarray(T), y / rho, mech)
        return w + gY, jacobian(mech, rho, T, y)

    return f, jac, y0, rho0


def integrate_cell(Uc, Gc, dt: float, mech, rtol: float = 1e-8, atol: float = 1e-12,
                   T0: float = 1000.0):
    """U(dt) of one cell and the BDF statistics."""
    ns = np.asarray(mech.W).shape[0]
    f, jac, y0, rho0 = cell_ode(Uc, Gc, mech, T0)
    y, st = bdf.bdf_integrate(f, jac, dt, y0, np.full(ns, atol * rho0), rtol)
    out = np.array(Uc, dtype=np.float64) + dt * np.asarray(Gc, dtype=np.float64)
    out[5:5 + ns] = y
    return out, st


def integrate(U: np.ndarray, G: np.ndarray | None, dt: float, mech, rtol: float = 1e-8,
              atol: float = 1e-12, T0: float = 1000.0, cells=None):
    """U(dt) for every cell of U ([NV, ...]; G the same shape or None), or
    for the flat cell indices `cells` only (returns [NV, len(cells)])."""
    nv = U.shape[0]
    Uf = U.reshape(nv, -1)
    Gf = np.zeros_like(Uf) if G is None else G.reshape(nv, -1)
    idx = range(Uf.shape[1]) if cells is None else cells
    out = np.empty((nv, len(idx)))
    for i, cidx in enumerate(idx):
        out[:, i], _ = integrate_cell(Uf[:, cidx], Gf[:, cidx], dt, mech, rtol, atol, T0)
    return out.reshape(U.shape) if cells is None else out
