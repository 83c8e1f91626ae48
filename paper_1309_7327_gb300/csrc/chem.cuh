// Pointwise thermodynamics and production rates (device functions).
#pragma once

#include "smc_internal.h"

namespace smc {

// cp/R of species k at T.
__device__ __forceinline__ double cpR(const Mech &m, int k, double T) {
  const double *c = m.cp[k];
  return c[0] + T * (c[1] + T * (c[2] + T * (c[3] + T * c[4])));
}

// h/R (units of K) of species k at T: T * (h/RT).
__device__ __forceinline__ double hR(const Mech &m, int k, double T) {
  const double *c = m.hT[k];
  return c[0] + T * (c[1] + T * (c[2] + T * (c[3] + T * (c[4] + T * c[5]))));
}

// s/R of species k at T (lnT = ln T).
__device__ __forceinline__ double sR(const Mech &m, int k, double T, double lnT) {
  const double *c = m.sR[k];
  return c[0] * lnT + c[1] + T * (c[2] + T * (c[3] + T * (c[4] + T * c[5])));
}

// Temperature from the specific internal energy e and mass fractions Y:
// Newton's method on sum_k Y_k e_k(T) = e, e_k = (R/W_k)(h_k/R - T), from the
// first guess T0, stopping when |dT| <= tol |T|.  Returns false if maxit steps
// did not converge.
__device__ __forceinline__ bool newton_T(const Mech &m, const double *Y, double e, double T0,
                                         double tol, int maxit, double &Tout) {
  const int ns = m.ns;
  double yr_sum = 0.0;
  for (int k = 0; k < ns; ++k) yr_sum += Y[k] * m.Ru_W[k];
  double T = T0;
  for (int it = 0; it < maxit; ++it) {
    double f = 0.0, fp = 0.0;
    for (int k = 0; k < ns; ++k) {
      const double yr = Y[k] * m.Ru_W[k];
      f += yr * hR(m, k, T);
      fp += yr * cpR(m, k, T);
    }
    f -= yr_sum * T + e;
    fp -= yr_sum;
    const double dT = f / fp;
    T -= dT;
    if (fabs(dT) <= tol * fabs(T)) {
      Tout = T;
      return true;
    }
  }
  Tout = T;
  return false;
}

// rho*omega_k (g/(cm^3 s)) by mass action with reversible Arrhenius rates and
// equilibrium constants from the Gibbs energies.  wdot[k] is overwritten.
__device__ __forceinline__ void production_rates(const Mech &m, const Reaction *__restrict__ rx,
                                                 double rho, double T, const double *Y,
                                                 double *wdot) {
  const int ns = m.ns;
  double c[SMC_MAX_NS], g[SMC_MAX_NS];
  const double lnT = log(T);
  const double invT = 1.0 / T;
  for (int k = 0; k < ns; ++k) {
    c[k] = rho * Y[k] * m.invW[k];
    g[k] = hR(m, k, T) * invT - sR(m, k, T, lnT);   // g_k / (R T)
    wdot[k] = 0.0;
  }
  const double ln_patm_RT = log(kPatm / kRu) - lnT;
  for (int r = 0; r < m.nr; ++r) {
    const Reaction &R = rx[r];
    const double lnkf = R.lnA + R.b * lnT - R.Ea_R * invT;
    double sg = 0.0;
    for (int i = 0; i < R.nr_; ++i) sg += R.rc[i] * g[R.rk[i]];
    for (int i = 0; i < R.nf; ++i) sg -= R.fc[i] * g[R.fk[i]];
    // ln Kc = -sum nu g + dnu ln(p_atm / (R T));   ln kr = ln kf - ln Kc
    const double lnKc = -sg + R.dnu * ln_patm_RT;
    double fwd = exp(lnkf);
    double rev = exp(lnkf - lnKc);
    for (int i = 0; i < R.nf; ++i)
      for (int j = 0; j < R.fc[i]; ++j) fwd *= c[R.fk[i]];
    for (int i = 0; i < R.nr_; ++i)
      for (int j = 0; j < R.rc[i]; ++j) rev *= c[R.rk[i]];
    const double q = fwd - rev;
    for (int i = 0; i < R.nf; ++i) wdot[R.fk[i]] -= R.fc[i] * q;
    for (int i = 0; i < R.nr_; ++i) wdot[R.rk[i]] += R.rc[i] * q;
  }
  for (int k = 0; k < ns; ++k) wdot[k] *= m.W[k];
}

}  // namespace smc
