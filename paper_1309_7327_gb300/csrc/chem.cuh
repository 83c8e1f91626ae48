// Pointwise thermodynamics and production rates (device functions).
#pragma once

#include "smc_internal.h"

namespace smc {

// Truncating double -> float conversion in integer arithmetic (keeps the
// FP64 pipe free): the top 23 stored mantissa bits are kept; magnitudes below
// the float normal range flush to zero.  Exact when x has at most 24
// significant bits.
__device__ __forceinline__ float trunc_float(double x) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
  const unsigned sign = (unsigned)((unsigned long long)b >> 63) << 31;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((unsigned)e << 23) | (unsigned)((b >> 29) & 0x7fffff));
}


// exp(x) in FP64 by the table-driven method of P. T. P. Tang (ACM TOMS 15,
// 1989): x = (2048 k + j) ln2/2048 + r with |r| <= ln2/4096, so that
//   exp(x) = 2^k * 2^(j/2048) * exp(r),
// 2^(j/2048) from a 2048-entry table and exp(r) - 1 from its Taylor
// polynomial to r^3 (truncation r^4/24 < 4e-17 relative).  n = 2048 k + j is
// rounded with the 1.5 * 2^52 shift inside one FMA (the product x * 2048/ln2
// is exact inside it), and 2^k is applied to the exponent field with integer
// arithmetic.  |x| >= 512 is clamped to [-708, 709] (the normal range of the
// result).  Eight FP64 operations; error within about 1 ulp.
__device__ __forceinline__ double fast_exp(const Mech &m, double x) {
  // clamp only when |x| >= 512 (exponent field test in integer arithmetic;
  // NaN also takes this branch and is returned as it is)
  if ((__double2hiint(x) & 0x7ff00000) >= ((1023 + 9) << 20)) {
    if (x != x) return x;
    if (x > 709.0) x = 709.0;
    if (x < -708.0) x = -708.0;
  }
  const double shift = 6755399441055744.0;                 // 1.5 * 2^52
  const double u = fma(x, 2954.639443740597, shift);       // 2048 / ln 2
  const double nd = u - shift;                             // nearest integer to x 2048/ln2
  const int n = __double2loint(u);
  // ln2/2048 split: L1 has 29 significant bits, so nd * L1 is exact for |n| < 2^22
  const double L1 = 0.0003384507717782981, L2 = -2.0512280628325608e-14;
  const double r = fma(-nd, L2, fma(-nd, L1, x));
  const double q = fma(r, 1.0 / 6.0, 0.5);
  const double p = fma(r * r, q, r);                       // exp(r) - 1
  const int j = n & (SMC_EXP_TABLE - 1);
  const int k = n >> 11;                                   // floor division
  const double tj = m.exp2tab[j];
  const double y = fma(tj, p, tj);
  return __hiloint2double(__double2hiint(y) + (k << 20), __double2loint(y));
}

// A float's value truncated toward zero to a 64-bit integer, in integer
// arithmetic (a float-to-int64 conversion instruction would occupy the FP64
// pipe); for |v| < 2^62.
__device__ __forceinline__ long long float_to_ll(float v) {
  const unsigned b = __float_as_uint(v);
  const int e = (int)((b >> 23) & 0xff) - 150;          // v = m 2^e, m the 24-bit significand
  const long long m = (long long)((b & 0x7fffffu) | 0x800000u);
  long long r = 0;
  if ((b & 0x7f800000u) != 0) r = e >= 0 ? (m << e) : (e > -24 ? (m >> -e) : 0);
  return (b >> 31) ? -r : r;
}

// exp(x) to the accuracy of fast_exp without FP64 arithmetic on its main
// path.  On this GPU the FP64 pipe issues one operation for every 64 of the
// FP32 pipe, and exponentials are a third of the FP64 operations of the
// production rates; here every step runs on the integer and FP32 pipes.  The
// decomposition is fast_exp's, x = (2048 k + j) ln2/2048 + r:
//  * t = x 2048/ln2 in 64-bit fixed point: x's 53-bit significand times
//    2048/ln2 held to 128 bits (CI + CR 2^-64, both scaled by 2^52), so that
//    n = round(t) and u = t - n carry no rounding error that matters
//    (|t| < 2^22 for the clamped range);
//  * r = u ln2/2048 and exp(r) - 1 = r + r^2/2 + r^3/6 + r^4/24 as a float
//    pair (hi + lo); |r| <= ln2/4096, so the pair's ~46 bits are far below
//    the double rounding of the result and the omitted r^5/120 < 2e-21;
//  * exp(x) = 2^k T_j (1 + p): T_j = 2^(j/2048) from the FP64 table, the sum
//    T_j + T_j p formed in 64-bit fixed point (2^62 scale) and rounded once
//    to 53 bits, 2^k added to the exponent field.
// |x| < 2^-20 is left to fast_exp (the fixed point would keep too few bits
// of so small a t); |x| >= 512, infinities and NaN are clamped or passed as
// in fast_exp.  Error within about 1 ulp.
__device__ __forceinline__ double exp_alu(const Mech &m, double x) {
  long long b = __double_as_longlong(x);
  int ef = (int)((b >> 52) & 0x7ff);
  if (ef < 1023 - 20) return fast_exp(m, x);
  if (ef >= 1023 + 9) {
    if (x != x) return x;
    if (x > 709.0) x = 709.0;
    if (x < -708.0) x = -708.0;
    b = __double_as_longlong(x);
    ef = (int)((b >> 52) & 0x7ff);
  }
  // |x| = M 2^(ef - 1075), 2048/ln2 = (CI + CR 2^-64) 2^-52, so
  // t 2^64 = M (CI + CR 2^-64) 2^(ef - 1063); s = 1063 - ef is in 31..60
  const unsigned long long CI = 0xb8aa3b295c17f0bbULL, CR = 0xbe87fed0691d3e88ULL;
  const unsigned long long M = ((unsigned long long)b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
  const int s = 1063 - ef;
  const unsigned long long ph = __umul64hi(M, CI), pl = M * CI;
  const unsigned long long corr = __umul64hi(M, CR) >> s;
  unsigned long long ip = ph >> s;
  unsigned long long fr = (pl >> s) | (ph << (64 - s));
  const unsigned long long fr2 = fr + corr;
  ip += fr2 < fr ? 1ULL : 0ULL;
  // round to nearest: a fraction of 1/2 or more counts as a negative u
  const long long f = (long long)fr2;
  const int na = (int)ip + (f < 0 ? 1 : 0);
  // u = f 2^-64 in [-1/2, 1/2): its top 48 bits as two exact floats
  const float u1 = (float)(int)(f >> 40) * 0x1p-24f;
  const float u2 = (float)(int)((f >> 16) & 0xFFFFFF) * 0x1p-48f;
  // r = u ln2/2048 with ln2/2048 = LH + LL
  const float LH = 0x1.62e43p-12f, LL = -0x1.05c61p-40f;
  float rh = u1 * LH;
  float rl = fmaf(u1, LH, -rh) + fmaf(u1, LL, u2 * LH);
  int n = na;
  if (b < 0) {
    n = -na;
    rh = -rh;
    rl = -rl;
  }
  // p = exp(r) - 1 as a float pair
  const float sq = rh * rh;
  const float sqe = fmaf(rh, rh, -sq);
  const float h2 = 0.5f * sq;
  const float ph2 = rh + h2;                         // |rh| > |h2|: exact error below
  const float phe = h2 - (ph2 - rh);
  const float c34 = sq * rh * fmaf(rh, 1.0f / 24.0f, 1.0f / 6.0f);
  const float pl2 = phe + rl + fmaf(0.5f, sqe, rh * rl) + c34;
  // T_j (1 + p) in fixed point, T_j = MT 2^-52 in [1, 2)
  const int j = n & (SMC_EXP_TABLE - 1);
  const int k = n >> 11;
  const unsigned long long MT =
      ((unsigned long long)__double_as_longlong(m.exp2tab[j]) & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
  const float th = (float)(unsigned)(MT >> 29) * 0x1p-23f;
  const float tl = (float)(unsigned)(MT & 0x1FFFFFFFULL) * 0x1p-52f;
  const float q1 = th * ph2;
  const float q2 = fmaf(th, ph2, -q1) + fmaf(th, pl2, tl * ph2);
  const long long Y = (long long)(MT << 10) + float_to_ll(q1 * 0x1p62f) + float_to_ll(q2 * 0x1p62f);
  int sh = 10, eadj = 0;
  if (Y < (1LL << 62)) {
    sh = 9;
    eadj = -1;
  }
  unsigned long long mr = ((unsigned long long)Y + (1ULL << (sh - 1))) >> sh;
  if (mr >> 53) {
    mr >>= 1;
    eadj += 1;
  }
  return __longlong_as_double((long long)((unsigned long long)(1023 + k + eadj) << 52) |
                              (long long)(mr & 0xFFFFFFFFFFFFFULL));
}

// The exponential the mechanism's flag selects (SMC_OPT_ALU).
__device__ __forceinline__ double mech_exp(const Mech &m, double x) {
  return m.alu ? exp_alu(m, x) : fast_exp(m, x);
}

// a * b rounded to nearest (ties to even) exactly as the FP64 unit rounds it,
// in integer arithmetic: the 106-bit product of the two 53-bit significands
// (one shifted left by 11, so that the top word of the product holds the 52
// or 53 leading bits), normalised, rounded once on its round and sticky bits,
// and packed with the summed exponents.  Zero, subnormal, infinite and NaN
// operands, and products that could leave the normal range, go to the FP64
// unit (a * b).
__device__ __forceinline__ double dmul_alu(double a, double b) {
  const unsigned long long ua = (unsigned long long)__double_as_longlong(a);
  const unsigned long long ub = (unsigned long long)__double_as_longlong(b);
  const int ea = (int)((ua >> 52) & 0x7ff), eb = (int)((ub >> 52) & 0x7ff);
  int e = ea + eb - 1023;
  if ((unsigned)(ea - 1) > 2045u || (unsigned)(eb - 1) > 2045u || (unsigned)(e - 1) > 2043u)
    return a * b;
  const unsigned long long ma = (ua & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
  const unsigned long long mb = (ub & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
  const unsigned long long x = ma << 11;
  const unsigned long long hi = __umul64hi(x, mb);     // ma mb 2^11 = hi 2^64 + lo
  const unsigned long long lo = x * mb;
  unsigned long long m, rest;                          // 53 result bits, the bits below them
  if (hi >> 52) {                                      // ma mb in [2^105, 2^106)
    m = hi;
    rest = lo;
    e += 1;
  } else {                                             // ma mb in [2^104, 2^105)
    m = (hi << 1) | (lo >> 63);
    rest = lo << 1;
  }
  m += ((rest >> 63) && ((rest << 1) != 0 || (m & 1))) ? 1ULL : 0ULL;
  if (m >> 53) {
    m >>= 1;
    e += 1;
  }
  return __longlong_as_double((long long)(((ua ^ ub) & 0x8000000000000000ULL) |
                                          ((unsigned long long)e << 52) | (m & 0xFFFFFFFFFFFFFULL)));
}

// The product the mechanism's flag selects (SMC_OPT_ALU); both round alike.
__device__ __forceinline__ double mech_mul(bool alu_mul, double a, double b) {
  return alu_mul ? dmul_alu(a, b) : a * b;
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

// g/RT - ln W_k of species k: h/RT - s/R folded into one polynomial in T
// plus the 1/T and ln T terms, with -ln W_k in the constant term.
__device__ __forceinline__ double gRT_W(const Mech &m, int k, double T, double invT, double lnT) {
  const double *c = m.gW[k];
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
// With rho_scale != 0, Y holds rho Y_k and the mass fractions are formed as
// Y[k] * rho_scale on the fly (the same roundings as a Y array made first,
// without keeping that array).
__device__ __forceinline__ bool newton_T(const Mech &m, const double *Y, double e, double T0,
                                         double tol, int maxit, double &Tout,
                                         double *cp_mix = nullptr, double *h_mix = nullptr,
                                         double rho_scale = 0.0) {
  const int ns = m.ns;
  const bool amul = m.alu >= 2;
  double H0 = 0.0, H1 = 0.0, H2 = 0.0, H3 = 0.0, H4 = 0.0, H5 = 0.0, yr_sum = 0.0;
  for (int k = 0; k < ns; ++k) {
    const double yk = rho_scale != 0.0 ? mech_mul(amul, Y[k], rho_scale) : Y[k];
    const double yr = mech_mul(amul, yk, m.Ru_W[k]);
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
// With G_k = g_k/(RT) - ln W_k, a per-cell shift s (the species mean of G),
// z_k = rho Y_k exp(G_k - s) = c_k exp(g_k/RT - s) and P = (R_u T / p_atm) exp(s),
// the net rate
//   q = k_f prod c^nu' - (k_f / K_c) prod c^nu''
// equals
//   q = exp(ln k_f - sum_reac nu' (ln W + G - s)) (prod_reac z^nu' - P^dnu prod_prod z^nu'')
// exactly (the exponential factors cancel; the shift may be any number), which
// needs one exponential per reaction and one per species instead of two per
// reaction.  sum nu' ln W is folded into ln A when the mechanism is packed.
// The shift keeps z and the prefactor inside the FP64 range when G spreads
// over less than 400 (checked when the mechanism is packed, 200..3500 K) with
// at most three molecules per reaction side.
__device__ __forceinline__ void production_rates(const Mech &m, const Reaction *__restrict__ rx,
                                                 double rho, double T, const double *Y,
                                                 double *wdot, const double *rhoY = nullptr) {
  const int ns = m.ns;
  const bool alu = m.alu != 0, amul = m.alu >= 2;
  double z[SMC_MAX_NS], g[SMC_MAX_NS];
  const double lnT = log(T);
  const double invT = 1.0 / T;
  double gs = 0.0;
  for (int k = 0; k < ns; ++k) {
    g[k] = gRT_W(m, k, T, invT, lnT);
    gs += g[k];
  }
  gs *= m.inv_ns;
  for (int k = 0; k < ns; ++k) {
    g[k] -= gs;
    z[k] = mech_mul(amul, rhoY ? rhoY[k] : rho * Y[k], alu ? exp_alu(m, g[k]) : fast_exp(m, g[k]));
    wdot[k] = 0.0;
  }
  // P^j for j = -3..3
  const double P1 = T * (kRu / kPatm) * (alu ? exp_alu(m, gs) : fast_exp(m, gs)), Pm1 = 1.0 / P1;
  const double P2 = P1 * P1, Pm2 = Pm1 * Pm1;
  const double Ppow[7] = {Pm2 * Pm1, Pm2, Pm1, 1.0, P1, P2, P2 * P1};
  for (int r = 0; r < m.nr; ++r) {
    const Reaction &R = rx[r];
    double ex = fma(R.b, lnT, fma(-R.Ea_R, invT, R.lnA));
    for (int i = 0; i < R.nf; ++i) ex = fma(-R.fcd[i], g[R.fk[i]], ex);
    double fwd = z[R.fm[0]], rev = z[R.rm[0]];
    for (int i = 1; i < R.nfm; ++i) fwd = mech_mul(amul, fwd, z[R.fm[i]]);
    for (int i = 1; i < R.nrm; ++i) rev = mech_mul(amul, rev, z[R.rm[i]]);
    const double q = mech_mul(amul, alu ? exp_alu(m, ex) : fast_exp(m, ex), fma(-Ppow[R.dn + 3], rev, fwd));
    for (int i = 0; i < R.nf; ++i) wdot[R.fk[i]] = fma(-R.fcw[i], q, wdot[R.fk[i]]);
    for (int i = 0; i < R.nr_; ++i) wdot[R.rk[i]] = fma(R.rcw[i], q, wdot[R.rk[i]]);
  }
}

// ---------------------------------------------------------------- mixed
// Production rates with FP32 mantissas (the mixed-precision path).  The
// Gibbs energies, the reaction exponents and the argument reduction of every
// exponential stay in FP64 (their absolute errors become relative errors of
// the rates); what follows the reduction -- exp(r) on |r| <= ln2/4096, the
// products of concentrations, the two terms of q and the accumulation of
// rho omega_k -- runs in FP32.  Values outside the float range (z_k, the
// rate prefactors) are carried as a float mantissa m and an integer
// exponent e, m 2^e.

struct xf {
  float m;
  int e;
};

__device__ __forceinline__ xf xf_mul(xf a, xf b) { return xf{a.m * b.m, a.e + b.e}; }

// x (double) as m 2^e with |m| in [1, 2) (mantissa truncated to 24 bits);
// zero and subnormal x give 0
__device__ __forceinline__ xf xf_from_double(double x) {
  const long long b = __double_as_longlong(x);
  const int eb = (int)((b >> 52) & 0x7ff);
  const unsigned sign = (unsigned)((unsigned long long)b >> 63) << 31;
  if (eb == 0) return xf{0.0f, 0};
  return xf{__uint_as_float(sign | 0x3f800000u | (unsigned)((b >> 29) & 0x7fffff)), eb - 1023};
}

// m 2^e as a float; below the float range it is negligible and flushes to 0
__device__ __forceinline__ float xf_to_float(xf a) {
  if (a.e < -126) return 0.0f;
  const int e = a.e < 127 ? a.e : 127;
  return a.m * __int_as_float((e + 127) << 23);
}

// float to double in integer arithmetic (subnormals flush to zero)
__device__ __forceinline__ double float_to_double(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned ef = (b >> 23) & 0xff;
  const unsigned sign = b & 0x80000000u;
  if (ef == 0) return __hiloint2double((int)sign, 0);
  const unsigned ed = ef == 0xff ? 0x7ffu : ef - 127 + 1023;
  return __hiloint2double((int)(sign | (ed << 20) | ((b & 0x7fffff) >> 3)), (int)(b << 29));
}

// exp(x) as m 2^e: the reduction x = n ln2/2048 + r of fast_exp in FP64
// (three operations), then 2^(j/2048) (1 + r + r^2/2) in FP32 (the next
// term, r^3/6 < 1e-12, is far below FP32 rounding)
__device__ __forceinline__ xf exp_xf(const Mech &m, double x) {
  if ((__double2hiint(x) & 0x7ff00000) >= ((1023 + 9) << 20)) {
    if (x != x) return xf{__int_as_float(0x7fffffff), 0};
    if (x > 709.0) x = 709.0;
    if (x < -708.0) x = -708.0;
  }
  const double shift = 6755399441055744.0;                 // 1.5 * 2^52
  const double u = fma(x, 2954.639443740597, shift);       // 2048 / ln 2
  const double nd = u - shift;
  const int n = __double2loint(u);
  const float r = trunc_float(fma(-nd, 3.384507717577858e-4, x));   // ln2 / 2048
  const float p = fmaf(0.5f * r, r, r);
  const float t = m.exp2tabf[n & (SMC_EXP_TABLE - 1)];
  return xf{fmaf(t, p, t), n >> 11};
}

// rho*omega_k as production_rates (same shift and rewrite of q), FP32 after
// the reductions; wdot[k] is overwritten with the FP64 value of the FP32 sum.
__device__ __forceinline__ void production_rates_m(const Mech &m, const Reaction *__restrict__ rx,
                                                   double T, const double *rhoY, double *wdot) {
  const int ns = m.ns;
  double g[SMC_MAX_NS];
  xf z[SMC_MAX_NS];
  float wf[SMC_MAX_NS];
  const double lnT = log(T);
  const double invT = 1.0 / T;
  double gs = 0.0;
  for (int k = 0; k < ns; ++k) {
    g[k] = gRT_W(m, k, T, invT, lnT);
    gs += g[k];
  }
  gs *= m.inv_ns;
  for (int k = 0; k < ns; ++k) {
    g[k] -= gs;
    z[k] = xf_mul(xf_from_double(rhoY[k]), exp_xf(m, g[k]));
    wf[k] = 0.0f;
  }
  // P^j, j = -3..3
  const xf P1 = xf_mul(xf_from_double(T * (kRu / kPatm)), exp_xf(m, gs));
  const xf Pm1 = xf{1.0f / P1.m, -P1.e};
  const xf P2 = xf_mul(P1, P1), Pm2 = xf_mul(Pm1, Pm1);
  const xf Ppow[7] = {xf_mul(Pm2, Pm1), Pm2, Pm1, xf{1.0f, 0}, P1, P2, xf_mul(P2, P1)};
  for (int r = 0; r < m.nr; ++r) {
    const Reaction &R = rx[r];
    double ex = fma(R.b, lnT, fma(-R.Ea_R, invT, R.lnA));
    for (int i = 0; i < R.nf; ++i) ex = fma(-R.fcd[i], g[R.fk[i]], ex);
    const xf E = exp_xf(m, ex);
    xf fwd = z[R.fm[0]], rev = z[R.rm[0]];
    for (int i = 1; i < R.nfm; ++i) fwd = xf_mul(fwd, z[R.fm[i]]);
    for (int i = 1; i < R.nrm; ++i) rev = xf_mul(rev, z[R.rm[i]]);
    const float q = xf_to_float(xf_mul(E, fwd)) - xf_to_float(xf_mul(xf_mul(E, Ppow[R.dn + 3]), rev));
    for (int i = 0; i < R.nf; ++i) wf[R.fk[i]] = fmaf(-R.fcwf[i], q, wf[R.fk[i]]);
    for (int i = 0; i < R.nr_; ++i) wf[R.rk[i]] = fmaf(R.rcwf[i], q, wf[R.rk[i]]);
  }
  for (int k = 0; k < ns; ++k) wdot[k] = float_to_double(wf[k]);
}

}  // namespace smc
