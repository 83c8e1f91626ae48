"""Species production rates rho*omega_k of eq. NS:rY (oracle; test only).

The paper names its mechanisms but prints no rate law.  Reading (standard
mass-action kinetics, no third-body or fall-off terms):

  c_k   = rho Y_k / W_k                               (mol/cm^3)
  k_f   = A T^b exp(-Ea / (R_c T))                    (Ea in cal/mol)
  g_k   = h_k/(R T) - s_k/R                           (molar, dimensionless)
  K_c   = exp(-sum_k nu_k g_k) (p_atm / (R_u T))^(sum_k nu_k),
          nu_k = nu''_k - nu'_k
  k_r   = k_f / K_c
  q     = k_f prod_k c_k^nu'_k - k_r prod_k c_k^nu''_k
  omega_k = sum_r nu_rk q_r,     rho omega_k = W_k omega_k  (g/(cm^3 s))
"""
from __future__ import annotations

import numpy as np

from .thermo import P_ATM, R_CAL, R_U, h_RT, s_R


def production_rates(rho, T, Y, mech) -> np.ndarray:
    """[ns, ...] rho*omega_k in g/(cm^3 s)."""
    W = np.asarray(mech.W)
    ns = W.shape[0]
    shape = (-1,) + (1,) * T.ndim
    c = rho[None] * Y / W.reshape(shape)
    g = h_RT(mech.nasa7, T) - s_R(mech.nasa7, T)
    wdot = np.zeros((ns,) + T.shape, dtype=T.dtype)
    for r in range(mech.A.shape[0]):
        nf = mech.nu_f[r]
        nr = mech.nu_r[r]
        nu = (nr - nf).astype(np.float64)
        kf = mech.A[r] * T ** mech.b[r] * np.exp(-mech.Ea[r] / (R_CAL * T))
        Kc = np.exp(-np.tensordot(nu, g, axes=(0, 0))) * (P_ATM / (R_U * T)) ** nu.sum()
        kr = kf / Kc
        fwd = kf.copy()
        rev = kr.copy()
        for k in range(ns):
            if nf[k]:
                fwd = fwd * c[k] ** int(nf[k])
            if nr[k]:
                rev = rev * c[k] ** int(nr[k])
        q = fwd - rev
        for k in range(ns):
            if nu[k] != 0.0:
                wdot[k] = wdot[k] + nu[k] * q
    return W.reshape(shape) * wdot
