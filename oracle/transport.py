"""Mixture transport coefficients (oracle; test infrastructure only).

The paper evaluates eta, xi, lambda and D_k with EGLIB (Sec. 5), which is
not used here.  The stand-in model (a reading of the paper, which names no
model of its own):

  eta      = eta_ref (T / T_ref)^eta_exp
  xi       = xi_ratio * eta                 (bulk viscosity, default 0)
  lambda   = cp_mix eta / Pr
  rho D_k  = lambda / (cp_mix Le_k)

with cp_mix = sum_k Y_k cp_k the mixture specific heat.
"""
from __future__ import annotations

import numpy as np


def coefficients(T, cp_mix, Le, eta_ref, T_ref, eta_exp, Pr, xi_ratio=0.0) -> dict:
    eta = eta_ref * (T / T_ref) ** eta_exp
    xi = xi_ratio * eta
    lam = cp_mix * eta / Pr
    rhoD = lam[None] / (cp_mix[None] * Le.reshape((-1,) + (1,) * T.ndim))
    return dict(eta=eta, xi=xi, lam=lam, rhoD=rhoD)
