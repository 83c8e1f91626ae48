// Implicit integration of the reaction ODE of every cell over one coarse
// interval (MRSDC mode 2, Sec. 3.2, eq. mrupdate2): variable-order (1..5),
// variable-step BDF in backward-difference form with a Newton iteration on
// an analytic Jacobian.
//
// One thread integrates one cell:
//   dy/dtau = rho omega(rho(tau), T(tau, y), y) + G_Y,  y = (rho Y_k),
// with the non-species components moving linearly, U_c(tau) = U_c + tau G_c,
// and T from the internal energy of those components (Newton, started at the
// cell's temperature at tau = 0).  The method:
//   * order-k BDF  gamma_k d + sum_{m=1}^{k} gamma_m nabla^m y_n = h f(y_pred + d),
//     y_pred = sum_{m=0}^{k} nabla^m y_n, d = nabla^{k+1} y_{n+1};
//   * Newton on d with the matrix I - (h/gamma_k) J, J = d(rho omega)/dy at
//     fixed rho and e; the residual, the rates and every state update are
//     FP64, J and its LU factors FP32 (they only set the convergence rate of
//     the iteration).  The factored matrix is kept across steps and rebuilt
//     (J at the predicted point) when there is none, after 20 steps, when
//     c = h/gamma_k has moved by more than 30%, or when the iteration failed
//     with an old one (the step is then retried with the same h); an old
//     matrix's corrections are scaled by 2 / (1 + c / c_lu);
//   * local error d/(k+1) in the RMS norm with weights atol rho_0 + rtol |y_n|;
//   * step changes resample the interpolating polynomial (quasi-constant
//     step size); order k-1, k or k+1 chosen after k+1 equal steps by the
//     predicted step factors; the starting step of Hairer, Norsett & Wanner.
// Each loop iteration of a thread performs exactly one rate evaluation, so
// the threads of a warp stay together in the expensive part whatever phase
// (start, new attempt, Newton iteration) each of them is in.
#include <cuda_runtime.h>

#include <cmath>

#include "chem.cuh"

namespace smc {
namespace {

constexpr int KMAX = 5;            // highest BDF order
constexpr int NEWTON_MAXITER = 4;
constexpr int LU_MAX_STEPS = 20;   // steps before the Newton matrix is rebuilt regardless
constexpr double LU_MAX_CHANGE = 0.3;

struct CellConst {
  double rho0, m0[3], E0;          // non-species components at tau = 0
  double grho, gm[3], gE;          // and their forcing
  double Tstart;                   // Newton start of every temperature solve
};

__device__ __forceinline__ void state_at(const CellConst &c, double tau, double &rho, double &e) {
  rho = fma(tau, c.grho, c.rho0);
  const double ir = 1.0 / rho;
  const double ux = fma(tau, c.gm[0], c.m0[0]) * ir;
  const double uy = fma(tau, c.gm[1], c.m0[1]) * ir;
  const double uz = fma(tau, c.gm[2], c.m0[2]) * ir;
  e = fma(tau, c.gE, c.E0) * ir - 0.5 * (ux * ux + uy * uy + uz * uz);
}

// rho omega_k (FP64) by mass action, as production_rates (same shift form),
// and, when J is not null, the Jacobian J[k][j] = d(rho omega_k)/dy_j at
// fixed rho and internal energy (FP32, row stride NS):
//   d q/d y_j |_T  from the molecule products (z_j = y_j exp(G_j - s)),
//   d q/d T       = F (b/T + Ea_R/T^2) - B (b/T + Ea_R/T^2 - d ln K_c/dT),
//   d ln K_c/dT   = (sum_k nu_k h_k/(R T) - sum_k nu_k) / T,
//   dT/dy_j       = -e_j(T) / (rho c_v),
// F and B the forward and reverse terms of q.
template <int NS>
__device__ void rates_jac(const Mech &m, const Reaction *__restrict__ rx, double rho, double T,
                          const double *y, double *wdot, float *J) {
  const int ns = m.ns;
  double g[NS], E[NS], z[NS];
  float dwdT[NS], hrt[NS];
  const double lnT = log(T);
  const double invT = 1.0 / T;
  double gs = 0.0;
  for (int k = 0; k < ns; ++k) {
    g[k] = gRT_W(m, k, T, invT, lnT);
    gs += g[k];
  }
  gs *= m.inv_ns;
  for (int k = 0; k < ns; ++k) {
    E[k] = mech_exp(m, g[k] - gs);
    z[k] = y[k] * E[k];
    wdot[k] = 0.0;
  }
  if (J) {
    for (int k = 0; k < ns; ++k) {
      dwdT[k] = 0.0f;
      hrt[k] = trunc_float(hR(m, k, T) * invT);
      for (int j = 0; j < ns; ++j) J[k * NS + j] = 0.0f;
    }
  }
  const double P1 = T * (kRu / kPatm) * mech_exp(m, gs), Pm1 = 1.0 / P1;
  const double P2 = P1 * P1, Pm2 = Pm1 * Pm1;
  const double Ppow[7] = {Pm2 * Pm1, Pm2, Pm1, 1.0, P1, P2, P2 * P1};
  const float invTf = trunc_float(invT);
  for (int r = 0; r < m.nr; ++r) {
    const Reaction &R = rx[r];
    double ex = fma(R.b, lnT, fma(-R.Ea_R, invT, R.lnA));
    for (int i = 0; i < R.nf; ++i) ex = fma(-R.fcd[i], g[R.fk[i]] - gs, ex);
    double fwd = z[R.fm[0]], rev = z[R.rm[0]];
    for (int i = 1; i < R.nfm; ++i) fwd *= z[R.fm[i]];
    for (int i = 1; i < R.nrm; ++i) rev *= z[R.rm[i]];
    const double K = mech_exp(m, ex);
    const double KP = K * Ppow[R.dn + 3];
    const double F = K * fwd, B = KP * rev;
    const double q = F - B;
    for (int i = 0; i < R.nf; ++i) wdot[R.fk[i]] = fma(-R.fcw[i], q, wdot[R.fk[i]]);
    for (int i = 0; i < R.nr_; ++i) wdot[R.rk[i]] = fma(R.rcw[i], q, wdot[R.rk[i]]);
    if (!J) continue;
    // d q / d y_j of every molecule of the reaction
    float dv[6];
    int dj[6];
    int nd = 0;
    for (int i = 0; i < R.nfm; ++i) {
      double p = K * E[R.fm[i]];
      for (int l = 0; l < R.nfm; ++l)
        if (l != i) p *= z[R.fm[l]];
      dv[nd] = trunc_float(p);
      dj[nd++] = R.fm[i];
    }
    for (int i = 0; i < R.nrm; ++i) {
      double p = -KP * E[R.rm[i]];
      for (int l = 0; l < R.nrm; ++l)
        if (l != i) p *= z[R.rm[l]];
      dv[nd] = trunc_float(p);
      dj[nd++] = R.rm[i];
    }
    for (int a = 0; a < R.nf; ++a) {
      float *row = J + R.fk[a] * NS;
      const float cf = -R.fcwf[a];
      for (int b = 0; b < nd; ++b) row[dj[b]] = fmaf(cf, dv[b], row[dj[b]]);
    }
    for (int a = 0; a < R.nr_; ++a) {
      float *row = J + R.rk[a] * NS;
      const float cf = R.rcwf[a];
      for (int b = 0; b < nd; ++b) row[dj[b]] = fmaf(cf, dv[b], row[dj[b]]);
    }
    // d q / d T
    float sh = -(float)R.dn;
    for (int i = 0; i < R.nrm; ++i) sh += hrt[R.rm[i]];
    for (int i = 0; i < R.nfm; ++i) sh -= hrt[R.fm[i]];
    const double a = fma(R.Ea_R * invT, invT, R.b * invT);
    const double dlnKc = float_to_double(sh * invTf);
    const float dq = trunc_float(fma(F, a, -B * (a - dlnKc)));
    for (int i = 0; i < R.nf; ++i) dwdT[R.fk[i]] = fmaf(-R.fcwf[i], dq, dwdT[R.fk[i]]);
    for (int i = 0; i < R.nr_; ++i) dwdT[R.rk[i]] = fmaf(R.rcwf[i], dq, dwdT[R.rk[i]]);
  }
  if (!J) return;
  // dT/dy_j = -e_j / (rho c_v) (fixed rho and e)
  const float Tf = trunc_float(T);
  float cv = 0.0f;
  float ej[NS];
  const double ir = 1.0 / rho;
  for (int k = 0; k < ns; ++k) {
    const float RW = trunc_float(m.Ru_W[k]);
    cv = fmaf(trunc_float(y[k] * ir) * RW, trunc_float(cpR(m, k, T)) - 1.0f, cv);
    ej[k] = RW * (hrt[k] - 1.0f) * Tf;
  }
  const float sc = -1.0f / (trunc_float(rho) * cv);
  for (int k = 0; k < ns; ++k)
    for (int j = 0; j < ns; ++j) J[k * NS + j] = fmaf(dwdT[k], sc * ej[j], J[k * NS + j]);
}

// f(tau, y) of the cell ODE (and its Jacobian when J is not null).  False
// when the temperature solve failed or the state is not physical.
template <int NS>
__device__ bool ode_eval(const DevState &s, const CellConst &c, double tau, const double *y,
                         const double *gY, double *f, float *J) {
  const Mech &m = *s.mech;
  const int ns = s.ns;
  double rho, e;
  state_at(c, tau, rho, e);
  double Y[NS];
  const double ir = 1.0 / rho;
  for (int k = 0; k < ns; ++k) Y[k] = y[k] * ir;
  double T;
  const bool ok = newton_T(m, Y, e, c.Tstart, s.opt.tol, s.opt.maxit, T);
  if (!ok || !(T > 0.0) || !isfinite(T) || !(rho > 0.0)) return false;
  if (s.opt.reactions && m.nr > 0) {
    rates_jac<NS>(m, s.rx, rho, T, y, f, J);
  } else {
    for (int k = 0; k < ns; ++k) f[k] = 0.0;
    if (J)
      for (int k = 0; k < ns * NS; ++k) J[k] = 0.0f;
  }
  for (int k = 0; k < ns; ++k) f[k] += gY[k];
  return true;
}

// Backward differences (rows 0..k) for a step change h -> rho h: the
// interpolating polynomial P(t_n + s h) = sum_m [s (s+1)..(s+m-1)/m!] nabla^m
// is resampled at s = -j rho and differenced again.
template <int NS>
__device__ void rescale(double (*D)[NS], int ns, int k, double rho) {
  const double inv[KMAX + 1] = {1.0, 1.0, 0.5, 1.0 / 3.0, 0.25, 0.2};
  double A[KMAX + 1][KMAX + 1];
  for (int j = 0; j <= k; ++j) {
    const double sj = -j * rho;
    double v = 1.0;
    A[j][0] = 1.0;
    for (int mm = 1; mm <= k; ++mm) {
      v *= (sj + (mm - 1)) * inv[mm];
      A[j][mm] = v;
    }
  }
  // T = B A with B[mm][j] = (-1)^j C(mm, j)
  const double C[KMAX + 1][KMAX + 1] = {{1, 0, 0, 0, 0, 0},  {1, -1, 0, 0, 0, 0},
                                        {1, -2, 1, 0, 0, 0}, {1, -3, 3, -1, 0, 0},
                                        {1, -4, 6, -4, 1, 0}, {1, -5, 10, -10, 5, -1}};
  double Tm[KMAX + 1][KMAX + 1];
  for (int mm = 0; mm <= k; ++mm) {
    for (int c = 0; c <= k; ++c) {
      double acc = 0.0;
      for (int j = 0; j <= mm; ++j) acc = fma(C[mm][j], A[j][c], acc);
      Tm[mm][c] = acc;
    }
  }
  for (int sp = 0; sp < ns; ++sp) {
    double old[KMAX + 1];
    for (int c = 0; c <= k; ++c) old[c] = D[c][sp];
    for (int mm = 1; mm <= k; ++mm) {
      double acc = 0.0;
      for (int c = 0; c <= k; ++c) acc = fma(Tm[mm][c], old[c], acc);
      D[mm][sp] = acc;
    }
  }
}

// LU factors with partial pivoting of M = I - ch J, in place (FP32).
template <int NS>
__device__ bool lu_factor(float *J, int *piv, int ns, float ch) {
  for (int r = 0; r < ns; ++r)
    for (int c = 0; c < ns; ++c) J[r * NS + c] = (r == c ? 1.0f : 0.0f) - ch * J[r * NS + c];
  for (int p = 0; p < ns; ++p) {
    int pr = p;
    float best = fabsf(J[p * NS + p]);
    for (int r = p + 1; r < ns; ++r) {
      const float v = fabsf(J[r * NS + p]);
      if (v > best) {
        best = v;
        pr = r;
      }
    }
    piv[p] = pr;
    if (!(best > 0.0f) || !isfinite(best)) return false;
    if (pr != p)
      for (int c = 0; c < ns; ++c) {
        const float t = J[p * NS + c];
        J[p * NS + c] = J[pr * NS + c];
        J[pr * NS + c] = t;
      }
    const float ip = 1.0f / J[p * NS + p];
    for (int r = p + 1; r < ns; ++r) {
      const float l = J[r * NS + p] * ip;
      J[r * NS + p] = l;
      for (int c = p + 1; c < ns; ++c) J[r * NS + c] = fmaf(-l, J[p * NS + c], J[r * NS + c]);
    }
  }
  return true;
}

template <int NS>
__device__ void lu_solve(const float *LU, const int *piv, int ns, float *b) {
  for (int p = 0; p < ns; ++p) {
    const int q = piv[p];
    if (q != p) {
      const float t = b[p];
      b[p] = b[q];
      b[q] = t;
    }
  }
  for (int r = 1; r < ns; ++r) {
    float acc = b[r];
    for (int c = 0; c < r; ++c) acc = fmaf(-LU[r * NS + c], b[c], acc);
    b[r] = acc;
  }
  for (int r = ns - 1; r >= 0; --r) {
    float acc = b[r];
    for (int c = r + 1; c < ns; ++c) acc = fmaf(-LU[r * NS + c], b[c], acc);
    b[r] = acc / LU[r * NS + r];
  }
}

template <int NS>
__device__ __forceinline__ double wrms(const double *v, const double *w, int ns, double scale) {
  double acc = 0.0;
  for (int k = 0; k < ns; ++k) {
    const double x = v[k] * scale / w[k];
    acc = fma(x, x, acc);
  }
  return sqrt(acc / ns);
}

__device__ __forceinline__ double step_factor(double err, int p) {
  return err == 0.0 ? INFINITY : exp(-log(err) / p);
}

enum { PH_F0 = 0, PH_F1, PH_ATTEMPT, PH_NEWTON };

// One cell: integrate, write its outputs, add its counters to cnt[4] and
// its accepted steps to the running maximum mx.
template <int NS>
__device__ __forceinline__ void bdf_cell(const DevState &s, const BdfParams &P, long long i,
                                         unsigned *cnt, unsigned &mx) {
  const long long N = s.ncells;
  const int ns = s.ns;
  unsigned flag = 0;
  CellConst c;
  c.rho0 = P.U[i];
  c.m0[0] = P.U[N + i];
  c.m0[1] = P.U[2 * N + i];
  c.m0[2] = P.U[3 * N + i];
  c.E0 = P.U[4 * N + i];
  c.grho = P.G ? P.G[i] : 0.0;
  c.gm[0] = P.G ? P.G[N + i] : 0.0;
  c.gm[1] = P.G ? P.G[2 * N + i] : 0.0;
  c.gm[2] = P.G ? P.G[3 * N + i] : 0.0;
  c.gE = P.G ? P.G[4 * N + i] : 0.0;
  double D[KMAX + 3][NS];
  double gY[NS], y[NS], d[NS], psi[NS], w[NS], f[NS];
  float J[NS * NS];
  float b[NS];
  int piv[NS];
  for (int k = 0; k < ns; ++k) {
    D[0][k] = P.U[(5 + k) * N + i];
    gY[k] = P.G ? P.G[(5 + k) * N + i] : 0.0;
    for (int m = 1; m < KMAX + 3; ++m) D[m][k] = 0.0;
  }
  {
    double rho, e;
    state_at(c, 0.0, rho, e);
    for (int k = 0; k < ns; ++k) y[k] = D[0][k] / rho;
    double T;
    const bool ok = newton_T(*s.mech, y, e, s.opt.T0, s.opt.tol, s.opt.maxit, T);
    if (!ok) flag |= ST_NONCONV;
    if (!(rho > 0.0) || !(T > 0.0)) flag |= ST_NONPHYS;
    if (!isfinite(rho) || !isfinite(T)) flag |= ST_NONFINITE;
    c.Tstart = T;
  }
  const double T_end = P.dtp;
  const double wabs = P.atol * c.rho0;
  double t = 0.0, h = 0.0, h0 = 0.0, ch = 0.0, dn_old = 0.0, d1 = 0.0;
  double c_lu = 1.0, corr = 1.0;
  int k = 1, n_equal = 0, it = 0, attempts = 0, phase = PH_F0, since_lu = 0;
  bool last = false, have_lu = false, fresh = false;
  unsigned long long n_steps = 0, n_rej = 0, n_fail = 0, n_eval = 0;
  bool done = flag != 0 || !(T_end > 0.0);
  while (!done) {
    // ---- the point of this iteration's one evaluation
    const double *yv = y;
    double tau = t + h;
    bool wantJ = false;
    if (phase == PH_F0) {
      yv = D[0];
      tau = 0.0;
    } else if (phase == PH_F1) {
      tau = h0;
    } else if (phase == PH_ATTEMPT) {
      if (++attempts > P.max_attempts || h <= 1e-14 * T_end) {
        flag |= ST_NONCONV;
        break;
      }
      last = false;
      if (t + h >= T_end) {
        rescale<NS>(D, ns, k, (T_end - t) / h);
        h = T_end - t;
        n_equal = 0;
        last = true;
      }
      const double ig = 1.0 / P.gam[k];
      for (int j = 0; j < ns; ++j) {
        double yp = D[0][j], ps = 0.0;
        for (int mm = 1; mm <= k; ++mm) {
          yp += D[mm][j];
          ps = fma(P.gam[mm], D[mm][j], ps);
        }
        y[j] = yp;
        psi[j] = ps * ig;
        d[j] = 0.0;
        w[j] = fma(P.rtol, fabs(D[0][j]), wabs);
      }
      ch = h * ig;
      tau = t + h;
      fresh = !have_lu || since_lu >= LU_MAX_STEPS || fabs(ch / c_lu - 1.0) > LU_MAX_CHANGE;
      wantJ = fresh;
      it = 0;
    }
    bool ok = true;
    if (phase == PH_F0 && P.F0) {
      // f(0, y_0) = R(U_0) + G_Y from the caller's reaction rates at U_0
      for (int j = 0; j < ns; ++j) f[j] = P.F0[(long long)j * N + i] + gY[j];
    } else {
      ok = ode_eval<NS>(s, c, tau, yv, gY, f, wantJ ? J : nullptr);
      ++n_eval;
    }
    if (phase == PH_F0 || phase == PH_F1) {
      if (!ok) {
        flag |= ST_NONCONV;
        break;
      }
    }
    if (phase == PH_F0) {
      // starting step, first part: d0 = |y0|, d1 = |f0|
      for (int j = 0; j < ns; ++j) {
        psi[j] = f[j];
        w[j] = fma(P.rtol, fabs(D[0][j]), wabs);
      }
      const double d0 = wrms<NS>(D[0], w, ns, 1.0);
      d1 = wrms<NS>(f, w, ns, 1.0);
      h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
      h0 = fmin(h0, T_end);
      for (int j = 0; j < ns; ++j) y[j] = fma(h0, f[j], D[0][j]);
      phase = PH_F1;
      continue;
    }
    if (phase == PH_F1) {
      for (int j = 0; j < ns; ++j) d[j] = f[j] - psi[j];
      const double d2 = wrms<NS>(d, w, ns, 1.0) / h0;
      const double dm = fmax(d1, d2);
      const double h1 = dm <= 1e-15 ? fmax(1e-6, 1e-3 * h0) : sqrt(0.01 / dm);
      h = fmin(fmin(100.0 * h0, h1), T_end);
      for (int j = 0; j < ns; ++j) D[1][j] = h * psi[j];
      k = 1;
      n_equal = 0;
      t = 0.0;
      phase = PH_ATTEMPT;
      continue;
    }
    bool conv = false, fail = !ok;
    if (!fail && phase == PH_ATTEMPT && fresh) {
      have_lu = lu_factor<NS>(J, piv, ns, trunc_float(ch));
      fail = !have_lu;
      c_lu = ch;
      since_lu = 0;
    }
    if (phase == PH_ATTEMPT) corr = 2.0 / (1.0 + ch / c_lu);
    if (!fail) {
      // Newton correction: (I - c_lu J) delta = ch f - psi - d
      for (int j = 0; j < ns; ++j) b[j] = trunc_float(fma(ch, f[j], -psi[j]) - d[j]);
      lu_solve<NS>(J, piv, ns, b);
      double acc = 0.0;
      for (int j = 0; j < ns; ++j) {
        const double dd = corr * float_to_double(b[j]);
        y[j] += dd;
        d[j] += dd;
        const double x = dd / w[j];
        acc = fma(x, x, acc);
      }
      const double dn = sqrt(acc / ns);
      if (!isfinite(dn)) {
        fail = true;
      } else if (dn == 0.0) {
        conv = true;
      } else if (it > 0) {
        const double rate = dn / dn_old;
        double rp = 1.0;
        for (int e = it; e < NEWTON_MAXITER; ++e) rp *= rate;
        if (rate >= 1.0 || rp / (1.0 - rate) * dn > P.eta) fail = true;
        else if (rate / (1.0 - rate) * dn < P.eta) conv = true;
      }
      dn_old = dn;
      ++it;
      if (!conv && !fail && it >= NEWTON_MAXITER) fail = true;
    }
    if (fail && !fresh) {
      // an old matrix: retry the step with a new Jacobian
      ++n_fail;
      have_lu = false;
      phase = PH_ATTEMPT;
      continue;
    }
    if (fail) {
      ++n_fail;
      rescale<NS>(D, ns, k, 0.5);
      h *= 0.5;
      n_equal = 0;
      phase = PH_ATTEMPT;
      continue;
    }
    if (!conv) {
      phase = PH_NEWTON;
      continue;
    }
    const double err = wrms<NS>(d, w, ns, 1.0 / (k + 1));
    if (err > 1.0) {
      ++n_rej;
      const double factor = fmax(0.2, 0.9 * step_factor(err, k + 1));
      rescale<NS>(D, ns, k, factor);
      h *= factor;
      n_equal = 0;
      phase = PH_ATTEMPT;
      continue;
    }
    // accepted: the differences of y_{n+1}
    t = last ? T_end : t + h;
    ++since_lu;
    ++n_steps;
    for (int j = 0; j < ns; ++j) {
      D[k + 2][j] = d[j] - D[k + 1][j];
      D[k + 1][j] = d[j];
      for (int mm = k; mm >= 0; --mm) D[mm][j] += D[mm + 1][j];
    }
    ++n_equal;
    phase = PH_ATTEMPT;
    if (t >= T_end) break;
    if (n_equal < k + 1) continue;
    const double f_lo = k > 1 ? step_factor(wrms<NS>(D[k], w, ns, 1.0 / k), k) : 0.0;
    const double f_0 = step_factor(err, k + 1);
    const double f_hi = k < KMAX ? step_factor(wrms<NS>(D[k + 2], w, ns, 1.0 / (k + 2)), k + 2) : 0.0;
    double best = f_0;
    int k_new = k;
    if (f_lo > best) {
      best = f_lo;
      k_new = k - 1;
    }
    if (f_hi > best) {
      best = f_hi;
      k_new = k + 1;
    }
    const double factor = fmin(10.0, 0.9 * best);
    k = k_new;
    rescale<NS>(D, ns, k, factor);
    h *= factor;
    n_equal = 0;
  }
  // ---- outputs
  if (P.Rbar)
    for (int j = 0; j < ns; ++j)
      P.Rbar[(long long)j * N + i] = (D[0][j] - P.U[(5 + j) * N + i]) / T_end - gY[j];
  if (P.Uout) {
    P.Uout[i] = fma(T_end, c.grho, c.rho0);
    P.Uout[N + i] = fma(T_end, c.gm[0], c.m0[0]);
    P.Uout[2 * N + i] = fma(T_end, c.gm[1], c.m0[1]);
    P.Uout[3 * N + i] = fma(T_end, c.gm[2], c.m0[2]);
    P.Uout[4 * N + i] = fma(T_end, c.gE, c.E0);
    for (int j = 0; j < ns; ++j) P.Uout[(5 + j) * N + i] = D[0][j];
  }
  if (flag) atomicOr(s.status, flag);
  cnt[0] += (unsigned)n_steps;
  cnt[1] += (unsigned)n_rej;
  cnt[2] += (unsigned)n_fail;
  cnt[3] += (unsigned)n_eval;
  mx = max(mx, (unsigned)n_steps);
}

// One thread per cell.  MINB caps the registers so that MINB blocks fit on
// an SM: the kernel waits on its per-thread arrays in local memory, and more
// resident warps hide more of that latency.  Measured at 21 species (ms per
// launch over 4.7 M cells): 4 blocks/SM 614, 8 543, 12 490, 16 449, the
// extra spills notwithstanding; a persistent grid with fewer resident
// threads, which keeps those arrays in cache, was slower still.
template <int NS, int MINB>
__global__ void __launch_bounds__(128, MINB) k_react_bdf(const DevState s, const BdfParams P) {
  unsigned cnt[4] = {0u, 0u, 0u, 0u}, mx = 0u;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < s.ncells;
       i += (long long)gridDim.x * blockDim.x)
    bdf_cell<NS>(s, P, i, cnt, mx);
  if (P.counters) {
    // every lane of the warp is here (blocks are whole warps)
    for (int q = 0; q < 4; ++q) {
      const unsigned tot = __reduce_add_sync(0xffffffffu, cnt[q]);
      if ((threadIdx.x & 31) == 0 && tot) atomicAdd(P.counters + q, (unsigned long long)tot);
    }
    const unsigned m = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(P.counters + 4, (unsigned long long)m);
  }
}

}  // namespace

int bdf_species_limit() { return 32; }

void launch_react_bdf(const DevState &s, const BdfParams &P, cudaStream_t st) {
  const int block = 128;
  const long long nb = (s.ncells + block - 1) / block;
  if (nb == 0) return;
  if (s.ns <= 8) k_react_bdf<8, 16><<<(unsigned)nb, block, 0, st>>>(s, P);
  else if (s.ns <= 16) k_react_bdf<16, 16><<<(unsigned)nb, block, 0, st>>>(s, P);
  else if (s.ns <= 24) k_react_bdf<24, 16><<<(unsigned)nb, block, 0, st>>>(s, P);
  else k_react_bdf<32, 16><<<(unsigned)nb, block, 0, st>>>(s, P);
}

}  // namespace smc
