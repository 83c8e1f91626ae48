// Right-hand-side kernels, FP64 path (Sec. 2.1 eq. cns, Sec. 2.2, Sec. 2.4).
//
//   k_prim   ghosted cell -> primitives, transport coefficients and the
//            per-cell coefficient products the stencils need (Q scratch)
//   k_grad   velocity gradients D_e u_c for the mixed viscous terms
//   k_march  one direction d: the narrow-stencil flux differences of every
//            (a u_x)_x term, -D_d of the convective plus mixed viscous fluxes
//            and the correction-velocity chain-rule terms, one grid-line
//            segment per thread
//   k_final  pointwise: Y_k div V_c, h div V_c and rho*omega_k
#include <cstdio>

#include "bc.cuh"
#include "chem.cuh"
#include "smc_internal.h"

namespace smc {

#define QF(f, g) __ldg(Q + (size_t)(f) * NG + (g))

// ---------------------------------------------------------------- k_prim
// INTERIOR: one thread per interior cell (the ghost cells are then filled by
// k_halo from their periodic images); otherwise one per ghosted cell, each
// reading U through the ghost-cell gather map.
template <bool INTERIOR>
__global__ void __launch_bounds__(128) k_prim(const DevState s, const double *__restrict__ U) {
  const Mech &m = *s.mech;
  const int ns = s.ns;
  const long long NG = s.nghost, NI = s.ncells;
  double *__restrict__ Q = s.Q;
  const int mode = s.opt.mode, ref = s.opt.ref;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (INTERIOR ? NI : NG);
       t += (long long)gridDim.x * blockDim.x) {
    const long long g = INTERIOR ? s.imap[t] : t;
    const long long src = INTERIOR ? t : (long long)s.gmap[t];
    const double rho = U[src];
    const double invrho = 1.0 / rho;
    const double u = U[NI + src] * invrho;
    const double v = U[2 * NI + src] * invrho;
    const double w = U[3 * NI + src] * invrho;
    const double rhoE = U[4 * NI + src];
    double Y[SMC_MAX_NS], h[SMC_MAX_NS];
    for (int k = 0; k < ns; ++k) Y[k] = U[(5 + k) * NI + src] * invrho;
    const double e = rhoE * invrho - 0.5 * (u * u + v * v + w * w);
    double T, cpm, hm;
    const bool ok = newton_T(m, Y, e, s.opt.T0, s.opt.tol, s.opt.maxit, T, &cpm, &hm);
    unsigned flag = 0;
    if (!ok) flag |= ST_NONCONV;
    if (!(rho > 0.0) || !(T > 0.0)) flag |= ST_NONPHYS;
    if (!isfinite(rho) || !isfinite(rhoE) || !isfinite(T)) flag |= ST_NONFINITE;
    if (flag) atomicOr(s.status, flag);

    double wmix = 0.0;
    for (int k = 0; k < ns; ++k) {
      wmix += Y[k] * m.invW[k];
      h[k] = m.Ru_W[k] * hR(m, k, T);
    }
    const double p = rho * kRu * T * wmix;
    const double invp = 1.0 / p;
    const double inv_wmix = 1.0 / wmix;
    // eta_ref (T / T_ref)^eta_exp as exp(eta_exp ln(T / T_ref)) with the
    // library's exponential (one log and one table exponential instead of a
    // general power)
    const double eta = m.eta_ref * mech_exp(m, m.eta_exp * log(T * m.inv_T_ref));
    const double xi = s.opt.xi_ratio * eta;
    const double lam = cpm * eta * m.inv_Pr;
    const double rd0 = lam / cpm;

    Q[(size_t)Q_U * NG + g] = u;
    Q[(size_t)Q_V * NG + g] = v;
    Q[(size_t)Q_W * NG + g] = w;
    Q[(size_t)Q_T * NG + g] = T;
    Q[(size_t)Q_P * NG + g] = p;
    Q[(size_t)Q_RHO * NG + g] = rho;
    Q[(size_t)Q_RHOH * NG + g] = rhoE + p;
    Q[(size_t)Q_C43 * NG + g] = 4.0 / 3.0 * eta + xi;
    Q[(size_t)Q_ETA * NG + g] = eta;
    Q[(size_t)Q_C23 * NG + g] = xi - 2.0 / 3.0 * eta;
    Q[(size_t)Q_LAM * NG + g] = lam;
    Q[(size_t)Q_HMIX * NG + g] = hm;
    Q[(size_t)Q_KX * NG + g] = 0.5 * u * u;
    Q[(size_t)Q_KY * NG + g] = 0.5 * v * v;
    Q[(size_t)Q_KZ * NG + g] = 0.5 * w * w;
    const double href = (mode == 1) ? h[ref] : 0.0;
    double ap = 0.0, sb = 0.0;
    for (int k = 0; k < ns; ++k) {
      const double X = Y[k] * m.invW[k] * inv_wmix;
      const double rd = rd0 * m.invLe[k];
      const double B = rd * (X - Y[k]) * invp;
      const double hp = h[k] - href;
      if (mode == 0) {
        ap += h[k] * B;
        sb += B;
      } else if (k != ref) {
        ap += hp * B;
      }
      Q[(size_t)(qY(ns) + k) * NG + g] = Y[k];
      Q[(size_t)(qX(ns) + k) * NG + g] = X;
      Q[(size_t)(qRY(ns) + k) * NG + g] = U[(5 + k) * NI + src];
      Q[(size_t)(qRD(ns) + k) * NG + g] = rd;
      Q[(size_t)(qRDH(ns) + k) * NG + g] = rd * hp;
      Q[(size_t)(qB(ns) + k) * NG + g] = B;
    }
    Q[(size_t)Q_AP * NG + g] = ap;
    Q[(size_t)Q_SB * NG + g] = sb;
  }
}

// ---------------------------------------------------------------- k_grad
struct GradParams {
  double D[3][4];
  double ihx;                     // 1/h_x (boundary-lowered x derivatives)
};

__device__ __forceinline__ int find_box_g(const Box *__restrict__ b, int nb, long long g) {
  int lo = 0, hi = nb - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (b[mid].off_g <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(128) k_grad(const DevState s, const GradParams P) {
  const long long NG = s.nghost;
  const double *__restrict__ Q = s.Q;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < NG;
       g += (long long)gridDim.x * blockDim.x) {
    const Box B = s.boxes[find_box_g(s.boxes, s.nboxes, g)];
    const long long l = g - B.off_g;
    const int ix = (int)(l % B.gx) - SMC_GHOST;
    const int iy = (int)((l / B.gx) % B.gy) - SMC_GHOST;
    const int iz = (int)(l / ((long long)B.gx * B.gy)) - SMC_GHOST;
    const int crd[3] = {ix, iy, iz};
    const int n[3] = {B.nx, B.ny, B.nz};
    const long long stride[3] = {1, B.gx, (long long)B.gx * B.gy};
    int nghost_dirs = 0;
    for (int e = 0; e < 3; ++e) nghost_dirs += (crd[e] < 0 || crd[e] >= n[e]);
    // cells next to non-periodic x ends take the lowered x derivative
    const int gxi = B.lo[0] + ix;
    const int kb = !s.x_outflow ? -1
                   : (gxi >= 0 && gxi < 4) ? gxi
                   : (gxi >= s.nx_domain - 4 && gxi < s.nx_domain) ? s.nx_domain - 1 - gxi : -1;
    for (int e = 0; e < 3; ++e) {
      if (crd[e] < 0 || crd[e] >= n[e]) continue;   // D_e needs e-interior cells
      if (nghost_dirs > 1) continue;                // edges are never read
      for (int c = 0; c < 3; ++c) {
        double acc = 0.0;
        if (e == 0 && kb >= 0) {
          const long long sg = gxi < 4 ? 1 : -1;
          double v[7];
          for (int j = 0; j < 7; ++j) v[j] = QF(Q_U + c, g + sg * (j - kb));
          acc = (double)sg * lowered_d(v, kb) * P.ihx;
        } else {
#pragma unroll
          for (int k = 1; k <= 4; ++k)
            acc += P.D[e][k - 1] * (QF(Q_U + c, g + k * stride[e]) - QF(Q_U + c, g - k * stride[e]));
        }
        s.G[(size_t)(3 * e + c) * NG + g] = acc;
      }
    }
  }
}

// ---------------------------------------------------------------- k_march
struct MarchParams {
  double M[8][8];   // narrow-stencil matrix / h_d^2, rows m = -3..4, cols n = -3..4
  double D[4];      // first-derivative weights / h_d
};

// Difference-first narrow stencil.  Every row of M sums to zero, so for the
// face between window cells 3 and 4 (the face's left cell is window cell 3)
//   H = sum_m a_m sum_n M_mn u_n = sum_m a_m sum_{n != 3} M_mn (u_n - u_3)
// exactly.  The differences carry the variation of u instead of its offset
// (p ~ 1e6 dyn/cm^2 varies by percent), which removes most of the rounding
// and costs no extra operation: column 3 drops out.

// w[m] = sum_{n != 3} M[m][n] (x[n] - x[3])   (M is banded: |m - n| <= 4)
__device__ __forceinline__ void mat_vec(const MarchParams &P, const double *x, double *w) {
  double d[8];
#pragma unroll
  for (int n = 0; n < 8; ++n) d[n] = (n == 3) ? 0.0 : x[n] - x[3];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    double acc = 0.0;
#pragma unroll
    for (int n = 0; n < 8; ++n)
      if (n != 3 && m - n <= 4 && n - m <= 4) acc += P.M[m][n] * d[n];
    w[m] = acc;
  }
}

// v[n] = sum_m a[m] M[m][n] for n != 3 (column 3 is never used)
__device__ __forceinline__ void vec_mat(const MarchParams &P, const double *a, double *v) {
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < 8; ++m)
      if (n != 3 && m - n <= 4 && n - m <= 4) acc += a[m] * P.M[m][n];
    v[n] = acc;
  }
}

__device__ __forceinline__ double dot8(const double *a, const double *b) {
  double acc = 0.0;
#pragma unroll
  for (int t = 0; t < 8; ++t) acc += a[t] * b[t];
  return acc;
}

// sum_{n != 3} v[n] (x[n] - x[3])
__device__ __forceinline__ double dot_diff(const double *v, const double *x) {
  double acc = 0.0;
#pragma unroll
  for (int n = 0; n < 8; ++n)
    if (n != 3) acc += v[n] * (x[n] - x[3]);
  return acc;
}

template <int DIR>
__device__ __forceinline__ void face_fluxes(const DevState &s, const MarchParams &P, long long gw,
                                            int sg, double *H) {
  // gw: ghosted index of the first window cell (4 cells left of the right cell)
  constexpr int E = (DIR + 1) % 3, F = (DIR + 2) % 3;
  const long long NG = s.nghost;
  const double *__restrict__ Q = s.Q;
  const int ns = s.ns, mode = s.opt.mode, ref = s.opt.ref;
  double win[8], wp[8], vA[8], vB[8], wk[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) win[t] = QF(Q_P, gw + t * sg);
  mat_vec(P, win, wp);
#pragma unroll
  for (int t = 0; t < 8; ++t) win[t] = QF(Q_C43, gw + t * sg);
  vec_mat(P, win, vA);
#pragma unroll
  for (int t = 0; t < 8; ++t) win[t] = QF(Q_ETA, gw + t * sg);
  vec_mat(P, win, vB);
  // momentum: (c43 u_d,d)_d, (eta u_e,d)_d, (eta u_f,d)_d
#pragma unroll
  for (int t = 0; t < 8; ++t) win[t] = QF(Q_U + DIR, gw + t * sg);
  H[0] = dot_diff(vA, win);
#pragma unroll
  for (int t = 0; t < 8; ++t) win[t] = QF(Q_U + E, gw + t * sg);
  H[1] = dot_diff(vB, win);
#pragma unroll
  for (int t = 0; t < 8; ++t) win[t] = QF(Q_U + F, gw + t * sg);
  H[2] = dot_diff(vB, win);
  // energy: viscous work in flux form, (c43 (u_d^2/2)_d)_d + (eta ((u_e^2+u_f^2)/2)_d)_d
  double HE;
#pragma unroll
  for (int t = 0; t < 8; ++t) win[t] = QF(Q_KX + DIR, gw + t * sg);
  HE = dot_diff(vA, win);
#pragma unroll
  for (int t = 0; t < 8; ++t) win[t] = QF(Q_KX + E, gw + t * sg);
  HE += dot_diff(vB, win);
#pragma unroll
  for (int t = 0; t < 8; ++t) win[t] = QF(Q_KX + F, gw + t * sg);
  HE += dot_diff(vB, win);
  // heat conduction (lambda T_d)_d
#pragma unroll
  for (int t = 0; t < 8; ++t) win[t] = QF(Q_T, gw + t * sg);
  mat_vec(P, win, wk);
#pragma unroll
  for (int t = 0; t < 8; ++t) win[t] = QF(Q_LAM, gw + t * sg);
  HE += dot8(win, wk);
  // enthalpy flux, pressure part: (A_p p_d)_d
#pragma unroll
  for (int t = 0; t < 8; ++t) win[t] = QF(Q_AP, gw + t * sg);
  HE += dot8(win, wp);
  // species: (rhoD_k X_k,d)_d + (B_k p_d)_d, energy (rhoD_k h'_k X_k,d)_d
  for (int k = 0; k < ns; ++k) {
    if (mode == 1 && k == ref) {
      H[4 + k] = 0.0;
      continue;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) win[t] = QF(qX(ns) + k, gw + t * sg);
    mat_vec(P, win, wk);
#pragma unroll
    for (int t = 0; t < 8; ++t) win[t] = QF(qRD(ns) + k, gw + t * sg);
    double hk = dot8(win, wk);
#pragma unroll
    for (int t = 0; t < 8; ++t) win[t] = QF(qB(ns) + k, gw + t * sg);
    hk += dot8(win, wp);
    H[4 + k] = hk;
#pragma unroll
    for (int t = 0; t < 8; ++t) win[t] = QF(qRDH(ns) + k, gw + t * sg);
    HE += dot8(win, wk);
  }
  H[3] = HE;
}

template <int DIR>
__global__ void __launch_bounds__(128, 3) k_march(const DevState s, const MarchParams P,
                                               double *__restrict__ dU, int first) {
  const long long item = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (item >= s.nlines[DIR]) return;
  const LineItem L = s.lines[DIR][item];
  constexpr int E = (DIR + 1) % 3, F = (DIR + 2) % 3;
  const int ns = s.ns, nv = s.nv, mode = s.opt.mode, ref = s.opt.ref;
  const long long NG = s.nghost, NI = s.ncells;
  const double *__restrict__ Q = s.Q;
  const double *__restrict__ G = s.G;
  const int sg = L.sg;

  double Hp[4 + SMC_MAX_NS], Hn[4 + SMC_MAX_NS], out[5 + SMC_MAX_NS];
  face_fluxes<DIR>(s, P, L.g0 - 4LL * sg, sg, Hp);
  for (int c = 0; c < L.len; ++c) {
    const long long gc = L.g0 + (long long)c * sg;
    const long long ic = L.i0 + (long long)c * L.si;
    face_fluxes<DIR>(s, P, gc - 3LL * sg, sg, Hn);   // right face of cell c

    // narrow-stencil flux differences (eq. DaDu; 1/h^2 folded into M)
    out[0] = 0.0;
    out[1 + DIR] = Hn[0] - Hp[0];
    out[1 + E] = Hn[1] - Hp[1];
    out[1 + F] = Hn[2] - Hp[2];
    out[4] = Hn[3] - Hp[3];
    double sumN = 0.0;
    for (int k = 0; k < ns; ++k) {
      const double N = Hn[4 + k] - Hp[4 + k];
      out[5 + k] = N;
      sumN += N;
    }
    if (mode == 1) out[5 + ref] = -sumN;

    // -D_d of the convective fluxes plus the mixed viscous terms
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0, a4 = 0.0;
    double udp[4], udm[4];
#pragma unroll
    for (int n = 1; n <= 4; ++n) {
      double fl[2][5];
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const long long j = side == 0 ? gc + n * sg : gc - n * sg;
        const double rho = QF(Q_RHO, j), ud = QF(Q_U + DIR, j), ue = QF(Q_U + E, j);
        const double uf = QF(Q_U + F, j), p = QF(Q_P, j), rH = QF(Q_RHOH, j);
        const double c23 = QF(Q_C23, j), eta = QF(Q_ETA, j);
        const double Gee = __ldg(G + (size_t)(3 * E + E) * NG + j);
        const double Gff = __ldg(G + (size_t)(3 * F + F) * NG + j);
        const double Ged = __ldg(G + (size_t)(3 * E + DIR) * NG + j);
        const double Gfd = __ldg(G + (size_t)(3 * F + DIR) * NG + j);
        const double tdiv = c23 * (Gee + Gff);
        const double mass = rho * ud;
        fl[side][0] = mass;
        fl[side][1] = mass * ud + p - tdiv;
        fl[side][2] = mass * ue - eta * Ged;
        fl[side][3] = mass * uf - eta * Gfd;
        fl[side][4] = rH * ud - (tdiv * ud + eta * (Ged * ue + Gfd * uf));
        if (side == 0) udp[n - 1] = ud; else udm[n - 1] = ud;
      }
      const double dn = P.D[n - 1];
      a0 += dn * (fl[0][0] - fl[1][0]);
      a1 += dn * (fl[0][1] - fl[1][1]);
      a2 += dn * (fl[0][2] - fl[1][2]);
      a3 += dn * (fl[0][3] - fl[1][3]);
      a4 += dn * (fl[0][4] - fl[1][4]);
    }
    out[0] -= a0;
    out[1 + DIR] -= a1;
    out[1 + E] -= a2;
    out[1 + F] -= a3;
    out[4] -= a4;
    for (int k = 0; k < ns; ++k) {
      double acc = 0.0;
#pragma unroll
      for (int n = 1; n <= 4; ++n)
        acc += P.D[n - 1] * (QF(qRY(ns) + k, gc + n * sg) * udp[n - 1] -
                             QF(qRY(ns) + k, gc - n * sg) * udm[n - 1]);
      out[5 + k] -= acc;
    }

    // correction velocity (Sec. 2.4): V_c,d = sum_l Fbar_l,d at the cell,
    // then grad Y_k . V_c and grad h . V_c (chain rule)
    if (mode == 0) {
      double Dp = 0.0;
#pragma unroll
      for (int n = 1; n <= 4; ++n) Dp += P.D[n - 1] * (QF(Q_P, gc + n * sg) - QF(Q_P, gc - n * sg));
      double Vc = -QF(Q_SB, gc) * Dp;
      for (int l = 0; l < ns; ++l) {
        double DX = 0.0;
#pragma unroll
        for (int n = 1; n <= 4; ++n)
          DX += P.D[n - 1] * (QF(qX(ns) + l, gc + n * sg) - QF(qX(ns) + l, gc - n * sg));
        Vc -= QF(qRD(ns) + l, gc) * DX;
      }
      for (int k = 0; k < ns; ++k) {
        double DY = 0.0;
#pragma unroll
        for (int n = 1; n <= 4; ++n)
          DY += P.D[n - 1] * (QF(qY(ns) + k, gc + n * sg) - QF(qY(ns) + k, gc - n * sg));
        out[5 + k] += DY * Vc;
      }
      double Dh = 0.0;
#pragma unroll
      for (int n = 1; n <= 4; ++n)
        Dh += P.D[n - 1] * (QF(Q_HMIX, gc + n * sg) - QF(Q_HMIX, gc - n * sg));
      out[4] += Dh * Vc;
      if (first) s.divacc[ic] = sumN; else s.divacc[ic] += sumN;
    }

    if (first) {
      for (int c2 = 0; c2 < nv; ++c2) dU[(size_t)c2 * NI + ic] = out[c2];
    } else {
      for (int c2 = 0; c2 < nv; ++c2) dU[(size_t)c2 * NI + ic] += out[c2];
    }
    for (int x = 0; x < 4 + ns; ++x) Hp[x] = Hn[x];
  }
}

// ---------------------------------------------------------------- k_final
__global__ void __launch_bounds__(128) k_final(const DevState s, double *__restrict__ dU,
                                               int transport, int chemistry) {
  const Mech &m = *s.mech;
  const int ns = s.ns;
  const long long NG = s.nghost, NI = s.ncells;
  const double *__restrict__ Q = s.Q;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < NI;
       i += (long long)gridDim.x * blockDim.x) {
    const long long g = s.imap[i];
    double add[SMC_MAX_NS];
    for (int k = 0; k < ns; ++k) add[k] = 0.0;
    if (transport && s.opt.mode == 0) {
      const double divVc = -s.divacc[i];
      dU[4 * NI + i] += QF(Q_HMIX, g) * divVc;
      for (int k = 0; k < ns; ++k) add[k] = QF(qY(ns) + k, g) * divVc;
    }
    if (chemistry) {
      double Y[SMC_MAX_NS], wd[SMC_MAX_NS];
      for (int k = 0; k < ns; ++k) Y[k] = QF(qY(ns) + k, g);
      production_rates(m, s.rx, QF(Q_RHO, g), QF(Q_T, g), Y, wd);
      for (int k = 0; k < ns; ++k) add[k] += wd[k];
    }
    if (transport) {
      for (int k = 0; k < ns; ++k) dU[(5 + k) * NI + i] += add[k];
    } else {
      for (int c = 0; c < 5; ++c) dU[c * NI + i] = 0.0;
      for (int k = 0; k < ns; ++k) dU[(5 + k) * NI + i] = add[k];
    }
  }
}

// ---------------------------------------------------------------- prim -> cons
__global__ void __launch_bounds__(128) k_prim_to_cons(const DevState s, const double *__restrict__ prim,
                                                      double *__restrict__ U) {
  const Mech &m = *s.mech;
  const int ns = s.ns;
  const long long NI = s.ncells;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < NI;
       i += (long long)gridDim.x * blockDim.x) {
    const double u = prim[i], v = prim[NI + i], w = prim[2 * NI + i];
    const double T = prim[3 * NI + i], p = prim[4 * NI + i];
    double wmix = 0.0, e = 0.0;
    for (int k = 0; k < ns; ++k) {
      const double Y = prim[(5 + k) * NI + i];
      wmix += Y * m.invW[k];
      e += Y * m.Ru_W[k] * (hR(m, k, T) - T);
    }
    const double rho = p / (kRu * T * wmix);
    U[i] = rho;
    U[NI + i] = rho * u;
    U[2 * NI + i] = rho * v;
    U[3 * NI + i] = rho * w;
    U[4 * NI + i] = rho * (e + 0.5 * (u * u + v * v + w * w));
    for (int k = 0; k < ns; ++k) U[(5 + k) * NI + i] = rho * prim[(5 + k) * NI + i];
  }
}

// ---------------------------------------------------------------- launchers
static int grid_for(long long n, int block) {
  long long b = (n + block - 1) / block;
  const long long cap = 152LL * 64;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

void launch_prim(const DevState &s, const double *U, cudaStream_t st) {
  k_prim<false><<<grid_for(s.nghost, 128), 128, 0, st>>>(s, U);
}

// Copy every plane of the primitive scratch from each ghost cell's periodic
// image (an interior cell of some box) to the ghost cell: the halo fill of
// the box array (Sec. 4), done once on the primitives instead of repeating
// the temperature solve and transport evaluation at every ghost cell.
template <typename T>
__global__ void __launch_bounds__(256) k_halo(const long long *__restrict__ dst,
                                              const long long *__restrict__ src, long long nh,
                                              T *__restrict__ Q, long long NG, int planes) {
  // blockIdx.y picks a group of 8 planes: eight independent loads in flight
  // per thread before the stores
  const int p0 = blockIdx.y * 8;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nh;
       j += (long long)gridDim.x * blockDim.x) {
    const long long gd = dst[j], gs = src[j];
    T v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (p0 + q < planes) v[q] = Q[(size_t)(p0 + q) * NG + gs];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (p0 + q < planes) Q[(size_t)(p0 + q) * NG + gd] = v[q];
  }
}

void launch_prim_interior(const DevState &s, const double *U, cudaStream_t st) {
  k_prim<true><<<grid_for(s.ncells, 128), 128, 0, st>>>(s, U);
}

void launch_halo(const DevState &s, int planes, int esize, cudaStream_t st) {
  if (s.nhalo == 0) return;
  long long bx = (s.nhalo + 255) / 256;
  if (bx > 152LL * 16) bx = 152LL * 16;
  const dim3 grid((unsigned)bx, (unsigned)((planes + 7) / 8));
  if (esize == 8)
    k_halo<double><<<grid, 256, 0, st>>>(s.halo_dst, s.halo_src, s.nhalo, s.Q, s.nghost, planes);
  else
    k_halo<float><<<grid, 256, 0, st>>>(s.halo_dst, s.halo_src, s.nhalo,
                                        reinterpret_cast<float *>(s.Q), s.nghost, planes);
}

void launch_grad(const DevState &s, cudaStream_t st) {
  GradParams P;
  const Coef *hc = s.hcoef;
  for (int d = 0; d < 3; ++d)
    for (int k = 0; k < 4; ++k) P.D[d][k] = hc->D[d][k];
  P.ihx = hc->D[0][0] * 1.25;
  k_grad<<<grid_for(s.nghost, 128), 128, 0, st>>>(s, P);
}

void launch_march(const DevState &s, int dir, double *dUdt, int first, cudaStream_t st) {
  const Coef *hc = s.hcoef;
  MarchParams P;
  for (int m = 0; m < 8; ++m)
    for (int n = 0; n < 8; ++n) P.M[m][n] = hc->M[dir][m][n];
  for (int k = 0; k < 4; ++k) P.D[k] = hc->D[dir][k];
  const long long n = s.nlines[dir];
  if (n == 0) return;
  const int blocks = (int)((n + 127) / 128);
  if (dir == 0) k_march<0><<<blocks, 128, 0, st>>>(s, P, dUdt, first);
  else if (dir == 1) k_march<1><<<blocks, 128, 0, st>>>(s, P, dUdt, first);
  else k_march<2><<<blocks, 128, 0, st>>>(s, P, dUdt, first);
}

void launch_final(const DevState &s, double *dUdt, int transport, int chemistry, cudaStream_t st) {
  k_final<<<grid_for(s.ncells, 128), 128, 0, st>>>(s, dUdt, transport, chemistry);
}

void launch_prim_to_cons(const DevState &s, const double *prim, double *U, cudaStream_t st) {
  k_prim_to_cons<<<grid_for(s.ncells, 128), 128, 0, st>>>(s, prim, U);
}

}  // namespace smc
