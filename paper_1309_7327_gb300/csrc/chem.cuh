// Pointwise thermodynamics and production rates (device functions).
#pragma once

#include "smc_internal.h"

namespace smc {

// exp(x) in FP64 by the table-driven method of P. T. P. Tang (ACM TOMS 15,
// 1989): x = (256 k + j) ln2/256 + r with |r| <= ln2/512, so that
//   exp(x) = 2^k * 2^(j/256) * exp(r),
// 2^(j/256) from a 256-entry table and exp(r) - 1 from its Taylor polynomial
// to r^4 (truncation r^5/120 < 4e-17 relative).  n = 256 k + j is rounded with
// the 1.5 * 2^52 shift, and 2^k is applied to the exponent field with integer
// arithmetic.  |x| >= 512 is clamped to [-708, 709] (the normal range of the
// result).  About 11 FP64 operations; error within ~1 ulp.
__device__ __forceinline__ double fast_exp(const Mech &m, double x) {
  // clamp only when |x| >= 512 (exponent field test in integer arithmetic;
  // NaN also takes this branch and stays NaN)
  if ((__double2hiint(x) & 0x7ff00000) >= ((1023 + 9) << 20)) x = fmin(fmax(x, -708.0), 709.0);
  const double shift = 6755399441055744.0;                 // 1.5 * 2^52
  const double t = x * 369.3299304675746;                  // 256 / ln 2
  const double nd = (t + shift) - shift;                   // nearest integer
  const int n = __double2loint(t + shift);
  // ln2/256 split: L1 has 19 trailing zero bits so nd * L1 is exact for |n| < 2^19
  const double L1 = 0.002707606173999011, L2 = 6.327543041662719e-14;
  const double r = fma(-nd, L2, fma(-nd, L1, x));
  double q = 1.0 / 24.0;
  q = fma(q, r, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  const double p = fma(r * r, q, r);                       // exp(r) - 1
  const int j = n & 255;
  const int k = n >> 8;                                    // floor division
  const double tj = m.exp2tab[j];
  const double y = fma(tj, p, tj);
  return __hiloint2double(__double2hiint(y) + (k << 20), __double2loint(y));
}

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

// g/RT = h/RT - s/R of species k, folded into one polynomial in T plus the
// 1/T and ln T terms (the same value as hR(T)/T - sR(T) in fewer operations).
__device__ __forceinline__ double gRT(const Mech &m, int k, double T, double invT, double lnT) {
  const double *c = m.gR[k];
  const double poly = T * (c[3] + T * (c[4] + T * (c[5] + T * c[6])));
  return fma(c[0], invT, fma(c[2], lnT, c[1] + poly));
}

// Temperature from the specific internal energy e and mass fractions Y:
// Newton's method on sum_k Y_k e_k(T) = e, e_k = (R/W_k)(h_k/R - T), from the
// first guess T0, stopping when |dT| <= tol |T|.  The species sums are folded
// once into the coefficients of one mixture polynomial
//   e(T) = sum_j H_j T^j - T sum_k Y_k R/W_k,   H_j = sum_k Y_k (R/W_k) hT[k][j],
// so every iteration costs one Horner evaluation of e and of de/dT = c_v.
// Returns false if maxit steps did not converge.
__device__ __forceinline__ bool newton_T(const Mech &m, const double *Y, double e, double T0,
                                         double tol, int maxit, double &Tout,
                                         double *cp_mix = nullptr, double *h_mix = nullptr) {
  const int ns = m.ns;
  double H0 = 0.0, H1 = 0.0, H2 = 0.0, H3 = 0.0, H4 = 0.0, H5 = 0.0, yr_sum = 0.0;
  for (int k = 0; k < ns; ++k) {
    const double yr = Y[k] * m.Ru_W[k];
    const double *c = m.hT[k];
    H0 += yr * c[0];
    H1 += yr * c[1];
    H2 += yr * c[2];
    H3 += yr * c[3];
    H4 += yr * c[4];
    H5 += yr * c[5];
    yr_sum += yr;
  }
  H0 -= e;
  H1 -= yr_sum;
  const double D2 = 2.0 * H2, D3 = 3.0 * H3, D4 = 4.0 * H4, D5 = 5.0 * H5;
  double T = T0;
  bool ok = false;
  for (int it = 0; it < maxit; ++it) {
    const double f = H0 + T * (H1 + T * (H2 + T * (H3 + T * (H4 + T * H5))));
    const double fp = H1 + T * (D2 + T * (D3 + T * (D4 + T * D5)));
    const double dT = f / fp;
    T -= dT;
    if (fabs(dT) <= tol * fabs(T)) {
      ok = true;
      break;
    }
  }
  Tout = T;
  // mixture c_p = d(sum Y_k h_k)/dT = c_v + sum Y_k R/W_k, and h = e(T) + (sum Y_k R/W_k) T
  if (cp_mix) *cp_mix = H1 + T * (D2 + T * (D3 + T * (D4 + T * D5))) + yr_sum;
  if (h_mix) *h_mix = H0 + T * (H1 + T * (H2 + T * (H3 + T * (H4 + T * H5)))) + e + yr_sum * T;
  return ok;
}

// rho*omega_k (g/(cm^3 s)) by mass action with reversible Arrhenius rates and
// equilibrium constants from the Gibbs energies.  wdot[k] is overwritten.
//
// With g_k = g_k/(RT), a per-cell shift s (the species mean of g), z_k =
// c_k exp(g_k - s) and P = (R_u T / p_atm) exp(s), the net rate
//   q = k_f prod c^nu' - (k_f / K_c) prod c^nu''
// equals
//   q = exp(ln k_f - sum_reac nu' (g - s)) (prod_reac z^nu' - P^dnu prod_prod z^nu'')
// exactly (the exponential factors cancel), which needs one exponential per
// reaction and one per species instead of two per reaction.  The shift keeps
// z and the prefactor inside the FP64 range when the species' g spread over
// less than 400 (checked by smc_create for 200..3500 K) with at most three
// molecules per reaction side.
__device__ __forceinline__ void production_rates(const Mech &m, const Reaction *__restrict__ rx,
                                                 double rho, double T, const double *Y,
                                                 double *wdot, const double *rhoY = nullptr) {
  const int ns = m.ns;
  double z[SMC_MAX_NS], g[SMC_MAX_NS];
  const double lnT = log(T);
  const double invT = 1.0 / T;
  double gs = 0.0;
  for (int k = 0; k < ns; ++k) {
    g[k] = gRT(m, k, T, invT, lnT);   // g_k / (R T)
    gs += g[k];
  }
  gs *= m.inv_ns;
  for (int k = 0; k < ns; ++k) {
    g[k] -= gs;
    const double c = (rhoY ? rhoY[k] : rho * Y[k]) * m.invW[k];
    z[k] = c * fast_exp(m, g[k]);
    wdot[k] = 0.0;
  }
  // P^j for j = -4..4
  const double P1 = T * (kRu / kPatm) * fast_exp(m, gs), Pm1 = 1.0 / P1;
  const double P2 = P1 * P1, Pm2 = Pm1 * Pm1;
  const double Ppow[9] = {Pm2 * Pm2, Pm2 * Pm1, Pm2, Pm1, 1.0, P1, P2, P2 * P1, P2 * P2};
  for (int r = 0; r < m.nr; ++r) {
    const Reaction &R = rx[r];
    double ex = R.lnA + R.b * lnT - R.Ea_R * invT;
    double fwd = 1.0, rev = 1.0;
    for (int i = 0; i < R.nf; ++i) {
      const int k = R.fk[i];
      ex -= R.fcd[i] * g[k];
      for (int j = 0; j < R.fc[i]; ++j) fwd *= z[k];
    }
    for (int i = 0; i < R.nr_; ++i)
      for (int j = 0; j < R.rc[i]; ++j) rev *= z[R.rk[i]];
    const double q = fast_exp(m, ex) * fma(-Ppow[R.dn + 4], rev, fwd);
    for (int i = 0; i < R.nf; ++i) wdot[R.fk[i]] = fma(-R.fcw[i], q, wdot[R.fk[i]]);
    for (int i = 0; i < R.nr_; ++i) wdot[R.rk[i]] = fma(R.rcw[i], q, wdot[R.rk[i]]);
  }
}

}  // namespace smc
