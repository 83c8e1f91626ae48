// Host-side packing of a reaction mechanism (NASA 7-coefficient
// thermodynamics, Arrhenius rate constants, stoichiometry; Sec. 2.1) into the
// device tables Mech and Reaction, with the validity checks smc_create and
// smc_rhs_noalloc both apply.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "smc_internal.h"

namespace smc {

const char *pack_mechanism(const smc_mechanism *mech, int max_reactions, Mech &M,
                           std::vector<Reaction> &rx) {
  const int ns = mech->nspecies, nr = mech->nreactions;
  if (ns < 1 || ns > SMC_MAX_NS) return "nspecies must be 1..64";
  if (nr < 0 || nr > max_reactions) return "too many reactions";
  if (!mech->W || !mech->nasa7 || !mech->Le ||
      (nr > 0 && (!mech->nu_f || !mech->nu_r || !mech->A || !mech->b || !mech->Ea)))
    return "null mechanism array";
  memset(&M, 0, sizeof(M));
  M.ns = ns;
  M.nr = nr;
  for (int k = 0; k < ns; ++k) {
    const double W = mech->W[k];
    if (!(W > 0) || !(mech->Le[k] > 0)) return "W and Le must be positive";
    const double *a = mech->nasa7 + 7 * k;
    M.W[k] = W;
    M.invW[k] = 1.0 / W;
    M.Ru_W[k] = kRu / W;
    M.invLe[k] = 1.0 / mech->Le[k];
    for (int i = 0; i < 5; ++i) M.cp[k][i] = a[i];
    const double hT[6] = {a[5], a[0], a[1] / 2, a[2] / 3, a[3] / 4, a[4] / 5};
    const double sR[6] = {a[0], a[6], a[1], a[2] / 2, a[3] / 3, a[4] / 4};
    for (int i = 0; i < 6; ++i) {
      M.hT[k][i] = hT[i];
      M.sR[k][i] = sR[i];
    }
    // g/RT - ln W_k: the constant term carries -ln W_k, so that
    // exp(gW) c_k = exp(g/RT) rho Y_k / W_k needs no division by W_k
    const double gW[7] = {a[5], a[0] - a[6] - std::log(W), -a[0], -a[1] / 2, -a[2] / 6, -a[3] / 12,
                          -a[4] / 20};
    for (int i = 0; i < 7; ++i) M.gW[k][i] = gW[i];
    for (int i = 0; i <= 100; ++i) {
      const double T = 200.0 + 33.0 * i;
      const double cp = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
      if (!(cp > 0)) return "cp must be positive on 200..3500 K";
    }
  }
  if (!(mech->eta_ref > 0) || !(mech->T_ref > 0) || !(mech->Pr > 0))
    return "transport parameters must be positive";
  M.inv_ns = 1.0 / ns;
  M.alu = 1;
  for (int j = 0; j < SMC_EXP_TABLE; ++j) {
    const long double t = exp2l((long double)j / (long double)SMC_EXP_TABLE);
    M.exp2tab[j] = (double)t;
    M.exp2tabf[j] = (float)t;
  }
  for (int i = 0; i <= 100; ++i) {
    // the production rates need g/RT - ln W over the species to spread over
    // less than 400 (the range argument of production_rates)
    const double T = 200.0 + 33.0 * i, lnT = std::log(T);
    double gmin = 1e300, gmax = -1e300;
    for (int k = 0; k < ns; ++k) {
      const double *a = mech->nasa7 + 7 * k;
      const double hRT = a[0] + T * (a[1] / 2 + T * (a[2] / 3 + T * (a[3] / 4 + T * a[4] / 5))) + a[5] / T;
      const double sR = a[0] * lnT + T * (a[1] + T * (a[2] / 2 + T * (a[3] / 3 + T * a[4] / 4))) + a[6];
      const double g = hRT - sR - std::log(mech->W[k]);
      gmin = std::min(gmin, g);
      gmax = std::max(gmax, g);
    }
    if (!(gmax - gmin < 400.0)) return "species Gibbs energies g/RT spread over more than 400";
  }
  M.eta_ref = mech->eta_ref;
  M.inv_T_ref = 1.0 / mech->T_ref;
  M.eta_exp = mech->eta_exp;
  M.inv_Pr = 1.0 / mech->Pr;
  for (int k = 0; k < ns; ++k) {
    for (int i = 0; i < 6; ++i) M.hTf[k][i] = (float)M.hT[k][i];
    M.Ru_Wf[k] = (float)M.Ru_W[k];
    M.invLef[k] = (float)M.invLe[k];
  }
  M.eta_ref_f = (float)M.eta_ref;
  M.inv_T_ref_f = (float)M.inv_T_ref;
  M.eta_exp_f = (float)M.eta_exp;
  M.inv_Pr_f = (float)M.inv_Pr;

  rx.assign(nr, Reaction{});
  for (int r = 0; r < nr; ++r) {
    Reaction &R = rx[r];
    memset(&R, 0, sizeof(R));
    if (!(mech->A[r] > 0)) return "A must be positive";
    R.b = mech->b[r];
    R.Ea_R = mech->Ea[r] / kRc;
    double dnu = 0, mass = 0, scale = 0, lnW_f = 0;
    for (int k = 0; k < ns; ++k) {
      const int f = mech->nu_f[r * ns + k], p = mech->nu_r[r * ns + k];
      if (f < 0 || p < 0) return "negative stoichiometric coefficient";
      if (f > 0) {
        if (R.nf == SMC_MAX_SIDE) return "more than 4 reactant species";
        if (R.nfm + f > 3) return "more than three molecules on a reaction side";
        R.fk[R.nf] = k;
        R.fcd[R.nf] = f;
        R.fcw[R.nf] = f * mech->W[k];
        R.fcwf[R.nf++] = (float)(f * mech->W[k]);
        for (int j = 0; j < f; ++j) R.fm[R.nfm++] = k;
        lnW_f += f * std::log(mech->W[k]);
      }
      if (p > 0) {
        if (R.nr_ == SMC_MAX_SIDE) return "more than 4 product species";
        if (R.nrm + p > 3) return "more than three molecules on a reaction side";
        R.rk[R.nr_] = k;
        R.rcw[R.nr_] = p * mech->W[k];
        R.rcwf[R.nr_++] = (float)(p * mech->W[k]);
        for (int j = 0; j < p; ++j) R.rm[R.nrm++] = k;
      }
      dnu += p - f;
      mass += (p - f) * mech->W[k];
      scale += (p + f) * mech->W[k];
    }
    if (R.nf == 0 || R.nr_ == 0) return "empty reaction side";
    if (std::fabs(mass) > 1e-9 * scale) return "reaction does not conserve mass";
    // ln A - sum nu' ln W: the reactant Gibbs sum is taken over g/RT - ln W
    R.lnA = std::log(mech->A[r]) - lnW_f;
    R.dn = (int)dnu;
  }
  return nullptr;
}

}  // namespace smc
