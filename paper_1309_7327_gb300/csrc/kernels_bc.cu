// x-direction terms at the cells next to non-periodic x ends with the
// boundary-lowered stencils of Sec. 2.2 (boundary paragraph): every x
// derivative of the right-hand side -- narrow diffusion, convective D,
// mixed viscous D, correction velocity -- in the four cells next to each
// end, evaluated in FP64 and stored over the values the x line kernel left
// there.  No characteristic boundary correction (outflow only).
#include "bc.cuh"
#include "smc_internal.h"

namespace smc {

enum Field { F_U, F_T, F_P, F_K, F_HMIX, F_RHO, F_RHOH, F_C43, F_ETA, F_C23, F_LAM, F_AP, F_SB,
             F_Y, F_X, F_RY, F_RD, F_RDH, F_B };

// FP64 primitive planes
struct AccD {
  const double *__restrict__ Q;
  const double *__restrict__ G;
  size_t NG;
  int ns;
  __device__ double f(Field F, int c, long long g) const {
    int pl = 0;
    switch (F) {
      case F_U: pl = Q_U + c; break;
      case F_T: pl = Q_T; break;
      case F_P: pl = Q_P; break;
      case F_K: pl = Q_KX + c; break;
      case F_HMIX: pl = Q_HMIX; break;
      case F_RHO: pl = Q_RHO; break;
      case F_RHOH: pl = Q_RHOH; break;
      case F_C43: pl = Q_C43; break;
      case F_ETA: pl = Q_ETA; break;
      case F_C23: pl = Q_C23; break;
      case F_LAM: pl = Q_LAM; break;
      case F_AP: pl = Q_AP; break;
      case F_SB: pl = Q_SB; break;
      case F_Y: pl = qY(ns) + c; break;
      case F_X: pl = qX(ns) + c; break;
      case F_RY: pl = qRY(ns) + c; break;
      case F_RD: pl = qRD(ns) + c; break;
      case F_RDH: pl = qRDH(ns) + c; break;
      case F_B: pl = qB(ns) + c; break;
    }
    return __ldg(Q + (size_t)pl * NG + g);
  }
  __device__ double grad(int e, int c, long long g) const { return __ldg(G + (size_t)(3 * e + c) * NG + g); }
};

// mixed-precision planes: float pairs for the differenced fields, floats
// for the coefficients, float gradients; read back into FP64
struct AccM {
  const float *__restrict__ Q;
  const float *__restrict__ G;
  size_t NG;
  int ns;
  __device__ double pair(int pl, long long g) const {
    return (double)__ldg(Q + (size_t)pl * NG + g) + (double)__ldg(Q + (size_t)(pl + 1) * NG + g);
  }
  __device__ double single(int pl, long long g) const { return (double)__ldg(Q + (size_t)pl * NG + g); }
  __device__ double f(Field F, int c, long long g) const {
    switch (F) {
      case F_U: return pair(PM_U + 2 * c, g);
      case F_T: return pair(PM_T, g);
      case F_P: return pair(PM_P, g);
      case F_K: return pair(PM_KX + 2 * c, g);
      case F_HMIX: return pair(PM_HMIX, g);
      case F_RHO: return pair(PM_RHO, g);
      case F_RHOH: return pair(PM_RHOH, g);
      case F_C43: return single(PM_C43, g);
      case F_ETA: return single(PM_ETA, g);
      case F_C23: return single(PM_C23, g);
      case F_LAM: return single(PM_LAM, g);
      case F_AP: return single(PM_AP, g);
      case F_SB: return single(PM_SB, g);
      case F_Y: return pair(pmY(ns, c), g);
      case F_X: return pair(pmX(ns, c), g);
      case F_RY: return pair(pmRY(ns, c), g);
      case F_RD: return single(pmRD(ns, c), g);
      case F_RDH: return single(pmRDH(ns, c), g);
      case F_B: return single(pmB(ns, c), g);
    }
    return 0.0;
  }
  __device__ double grad(int e, int c, long long g) const {
    return (double)__ldg(G + (size_t)(3 * e + c) * NG + g);
  }
};

struct XbcParams {
  double ih, ih2;                 // 1/h_x and 1/h_x^2
  LoweredM L;
};

// The x-direction terms of one cell (DIR = x, E = y, F = z); out[NV] and the
// species divergence sum.
template <class A>
__device__ void xbc_cell(const DevState &s, const A &q, const XbcParams &P, const BcCell &c,
                         double *out, double &sumN) {
  const int ns = s.ns, mode = s.opt.mode, ref = s.opt.ref;
  const int k = c.k;
  const long long sg = c.side == 0 ? 1 : -1;
  const long long base = c.g - sg * k;               // the end cell
  double a[7], v[7];
  auto narrow = [&](Field fa, int ca, Field fu, int cu) {
    for (int j = 0; j < 7; ++j) {
      a[j] = q.f(fa, ca, base + sg * j);
      v[j] = q.f(fu, cu, base + sg * j);
    }
    return lowered_n(P.L, a, v, k) * P.ih2;
  };
  auto deriv = [&](Field fu, int cu) {
    for (int j = 0; j < 7; ++j) v[j] = q.f(fu, cu, base + sg * j);
    return (double)sg * lowered_d(v, k) * P.ih;
  };
  // narrow-stencil terms (eq. DaDu)
  out[0] = 0.0;
  out[1] = narrow(F_C43, 0, F_U, 0);
  out[2] = narrow(F_ETA, 0, F_U, 1);
  out[3] = narrow(F_ETA, 0, F_U, 2);
  out[4] = narrow(F_C43, 0, F_K, 0) + narrow(F_ETA, 0, F_K, 1) + narrow(F_ETA, 0, F_K, 2) +
           narrow(F_LAM, 0, F_T, 0) + narrow(F_AP, 0, F_P, 0);
  sumN = 0.0;
  for (int sp = 0; sp < ns; ++sp) {
    double N = 0.0;
    if (!(mode == 1 && sp == ref)) {
      N = narrow(F_RD, sp, F_X, sp) + narrow(F_B, sp, F_P, 0);
      out[4] += narrow(F_RDH, sp, F_X, sp);
    }
    out[5 + sp] = N;
    sumN += N;
  }
  if (mode == 1) out[5 + ref] = -sumN;
  // convective fluxes with the mixed viscous terms, -D_x of each
  double fl[5][7];
  for (int j = 0; j < 7; ++j) {
    const long long g = base + sg * j;
    const double rho = q.f(F_RHO, 0, g), ud = q.f(F_U, 0, g), ue = q.f(F_U, 1, g);
    const double uf = q.f(F_U, 2, g), p = q.f(F_P, 0, g), rH = q.f(F_RHOH, 0, g);
    const double c23 = q.f(F_C23, 0, g), eta = q.f(F_ETA, 0, g);
    const double Gee = q.grad(1, 1, g), Gff = q.grad(2, 2, g);
    const double Ged = q.grad(1, 0, g), Gfd = q.grad(2, 0, g);
    const double tdiv = c23 * (Gee + Gff);
    const double mass = rho * ud;
    fl[0][j] = mass;
    fl[1][j] = mass * ud + p - tdiv;
    fl[2][j] = mass * ue - eta * Ged;
    fl[3][j] = mass * uf - eta * Gfd;
    fl[4][j] = rH * ud - (tdiv * ud + eta * (Ged * ue + Gfd * uf));
  }
  for (int cc = 0; cc < 5; ++cc) out[cc] -= (double)sg * lowered_d(fl[cc], k) * P.ih;
  for (int sp = 0; sp < ns; ++sp) {
    for (int j = 0; j < 7; ++j) {
      const long long g = base + sg * j;
      v[j] = q.f(F_RY, sp, g) * q.f(F_U, 0, g);
    }
    out[5 + sp] -= (double)sg * lowered_d(v, k) * P.ih;
  }
  // correction velocity (Sec. 2.4) at the cell and the chain-rule terms
  if (mode == 0) {
    double Vc = -q.f(F_SB, 0, c.g) * deriv(F_P, 0);
    for (int l = 0; l < ns; ++l) Vc -= q.f(F_RD, l, c.g) * deriv(F_X, l);
    for (int sp = 0; sp < ns; ++sp) out[5 + sp] += deriv(F_Y, sp) * Vc;
    out[4] += deriv(F_HMIX, 0) * Vc;
  }
}

__global__ void __launch_bounds__(128) k_xbc(const DevState s, const XbcParams P,
                                             double *__restrict__ dU) {
  const AccD q{s.Q, s.G, (size_t)s.nghost, s.ns};
  const size_t NI = (size_t)s.ncells;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < s.n_bc;
       t += (long long)gridDim.x * blockDim.x) {
    const BcCell c = s.bc_cells[t];
    double out[5 + SMC_MAX_NS], sumN;
    xbc_cell(s, q, P, c, out, sumN);
    for (int cc = 0; cc < s.nv; ++cc) dU[cc * NI + c.i] = out[cc];
    if (s.opt.mode == 0) s.divacc[c.i] = sumN;
  }
}

__global__ void __launch_bounds__(128) k_xbc_m(const DevState s, const XbcParams P,
                                               float *__restrict__ dUf) {
  const AccM q{reinterpret_cast<const float *>(s.Q), reinterpret_cast<const float *>(s.G),
               (size_t)s.nghost, s.ns};
  const size_t NI = (size_t)s.ncells;
  float *__restrict__ divf = reinterpret_cast<float *>(s.divacc);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < s.n_bc;
       t += (long long)gridDim.x * blockDim.x) {
    const BcCell c = s.bc_cells[t];
    double out[5 + SMC_MAX_NS], sumN;
    xbc_cell(s, q, P, c, out, sumN);
    for (int cc = 0; cc < s.nv; ++cc) dUf[cc * NI + c.i] = (float)out[cc];
    if (s.opt.mode == 0) divf[c.i] = (float)sumN;
  }
}

static XbcParams xbc_params(const DevState &s) {
  XbcParams P;
  // D[0][0] = (4/5) / h_x
  P.ih = s.hcoef->D[0][0] * 1.25;
  P.ih2 = P.ih * P.ih;
  P.L = lowered_matrices();
  return P;
}

static int xbc_grid(long long n) {
  long long b = (n + 127) / 128;
  if (b > 152LL * 16) b = 152LL * 16;
  return (int)(b < 1 ? 1 : b);
}

void launch_xbc(const DevState &s, double *dU, cudaStream_t st) {
  if (!s.x_outflow || s.n_bc == 0) return;
  k_xbc<<<xbc_grid(s.n_bc), 128, 0, st>>>(s, xbc_params(s), dU);
}

void launch_xbc_m(const DevState &s, float *dUf, cudaStream_t st) {
  if (!s.x_outflow || s.n_bc == 0) return;
  k_xbc_m<<<xbc_grid(s.n_bc), 128, 0, st>>>(s, xbc_params(s), dUf);
}

}  // namespace smc
