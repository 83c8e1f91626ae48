// FP64 stencil-line kernel with sliding register windows (Sec. 2.2 narrow
// stencil, eqs. DaDu/H; 8th-order D of the convective and mixed viscous
// fluxes; the correction-velocity terms of Sec. 2.4).
//
// The same terms and the same arithmetic per term as k_march (difference-
// first narrow products, D applied to pointwise fluxes), organised for data
// reuse.  Each thread walks its line segment in chunks of up to CH cells.
// Every field is held in a 9-cell register window (cells c-4 .. c+4 of the
// current cell c) that slides by one cell per step, so a primitive value is
// loaded once per cell and field instead of once per face and stencil point:
// the kernel streams the primitive planes once per direction, where the
// per-face kernel's eight-fold re-reads from every line in flight overflow
// the L2 cache.  The terms are taken in sub-passes over small groups of
// fields (momentum, kinetic energy, heat, convective fluxes, then two passes
// per species) to bound the live registers; the per-cell energy, correction
// velocity and species divergence sum are carried between sub-passes in
// shared memory.  Convective fluxes are formed once per window
// cell rather than once per stencil point.
#include "smc_internal.h"

namespace smc {
namespace {

constexpr int NT = 128;

struct ParamsW {
  double M[8][8];   // narrow-stencil matrix / h_d^2, rows m = -3..4, cols n = -3..4
  double D[4];      // first-derivative weights / h_d
};

struct Win {
  const double *__restrict__ Q;
  const double *__restrict__ G;
  size_t NG;
  long long gb;     // ghosted index of the chunk's first cell
  int sg;
  __device__ __forceinline__ double q(int plane, int r) const {
    return __ldg(Q + (size_t)plane * NG + gb + (long long)r * sg);
  }
  __device__ __forceinline__ double g(int plane, int r) const {
    return __ldg(G + (size_t)plane * NG + gb + (long long)r * sg);
  }
};

// v[n] = sum_m a[o+m] M[m][n] for n != 3 (M is banded: |m - n| <= 4)
__device__ __forceinline__ void vm(const ParamsW &P, const double *a, int o, double *v) {
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < 8; ++m)
      if (n != 3 && m - n <= 4 && n - m <= 4) acc = fma(a[o + m], P.M[m][n], acc);
    v[n] = acc;
  }
}
// w[m] = sum_{n != 3} M[m][n] (x[o+n] - x[o+3])  (rows of M sum to zero)
__device__ __forceinline__ void mv(const ParamsW &P, const double *x, int o, double *w) {
  double d[8];
#pragma unroll
  for (int n = 0; n < 8; ++n) d[n] = (n == 3) ? 0.0 : x[o + n] - x[o + 3];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    double acc = 0.0;
#pragma unroll
    for (int n = 0; n < 8; ++n)
      if (n != 3 && m - n <= 4 && n - m <= 4) acc = fma(P.M[m][n], d[n], acc);
    w[m] = acc;
  }
}
// sum_{n != 3} v[n] (x[o+n] - x[o+3])
__device__ __forceinline__ double dpd(const double *v, const double *x, int o) {
  double acc = 0.0;
#pragma unroll
  for (int n = 0; n < 8; ++n)
    if (n != 3) acc = fma(v[n], x[o + n] - x[o + 3], acc);
  return acc;
}
// sum_t a[o+t] w[t]
__device__ __forceinline__ double ds(const double *a, int o, const double *w) {
  double acc = 0.0;
#pragma unroll
  for (int t = 0; t < 8; ++t) acc = fma(a[o + t], w[t], acc);
  return acc;
}
// centred D at the middle (index 4) of a 9-cell window
__device__ __forceinline__ double Dc(const ParamsW &P, const double *w) {
  double acc = 0.0;
#pragma unroll
  for (int n = 1; n <= 4; ++n) acc = fma(P.D[n - 1], w[4 + n] - w[4 - n], acc);
  return acc;
}
__device__ __forceinline__ void slide(double *w) {
#pragma unroll
  for (int i = 0; i < 8; ++i) w[i] = w[i + 1];
}
// Store, or add without waiting for the old value (the add goes out as a
// reduction).  Each cell is updated by one thread per launch, in program
// order, so the sums are deterministic.
__device__ __forceinline__ void put(double *__restrict__ dU, size_t NI, int comp, long long i,
                                    double v, bool store) {
  double *q = dU + (size_t)comp * NI + i;
  if (store) *q = v; else atomicAdd(q, v);
}

// transverse momentum fluxes rho u_d u_t - eta u_d,t (t = e, f) at window offset r
template <int DIR>
__device__ __forceinline__ void flux_ef(const Win &x, int r, double &fe, double &ff) {
  constexpr int E_ = (DIR + 1) % 3, F_ = (DIR + 2) % 3;
  const double m = x.q(Q_RHO, r) * x.q(Q_U + DIR, r);
  const double eta = x.q(Q_ETA, r);
  fe = m * x.q(Q_U + E_, r) - eta * x.g(3 * E_ + DIR, r);
  ff = m * x.q(Q_U + F_, r) - eta * x.g(3 * F_ + DIR, r);
}

// energy flux rho H u_d - [c23 (u_e,e + u_f,f) u_d + eta (u_d,e u_e + u_d,f u_f)]
template <int DIR>
__device__ __forceinline__ double flux_E(const Win &x, int r) {
  constexpr int E_ = (DIR + 1) % 3, F_ = (DIR + 2) % 3;
  const double ud = x.q(Q_U + DIR, r);
  const double tdiv = x.q(Q_C23, r) * (x.g(3 * E_ + E_, r) + x.g(3 * F_ + F_, r));
  return x.q(Q_RHOH, r) * ud -
         (tdiv * ud + x.q(Q_ETA, r) * (x.g(3 * E_ + DIR, r) * x.q(Q_U + E_, r) +
                                      x.g(3 * F_ + DIR, r) * x.q(Q_U + F_, r)));
}

// the d-momentum flux rho u_d u_d + p - c23 (u_e,e + u_f,f)
template <int DIR>
__device__ __forceinline__ double flux_d(const Win &x, int r) {
  constexpr int E_ = (DIR + 1) % 3, F_ = (DIR + 2) % 3;
  const double ud = x.q(Q_U + DIR, r);
  const double tdiv = x.q(Q_C23, r) * (x.g(3 * E_ + E_, r) + x.g(3 * F_ + F_, r));
  return x.q(Q_RHO, r) * ud * ud + x.q(Q_P, r) - tdiv;
}

// CH: cells per chunk.  The three per-cell arrays live in dynamic shared
// memory, 3 CH NT doubles.  WP: the pressure products w = M (p - p_3) of
// the chunk's CH + 1 faces are also kept in shared memory (8 (CH + 1) NT
// more doubles), formed once in the heat pass and read by every species'
// pressure term, instead of formed again for every species; MINB is the
// resident blocks per SM the registers are sized for.
template <int DIR, int CH, bool WP, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_march_w(const DevState s, const ParamsW P,
                                                      double *__restrict__ dU, int first) {
  extern __shared__ double w_smem[];
  double(*sE)[NT] = reinterpret_cast<double(*)[NT]>(w_smem);
  double(*sV)[NT] = sE + CH;
  double(*sN)[NT] = sV + CH;
  double(*sW)[NT] = sN + CH;       // [(face * 8 + m)][thread], WP only
  const int tid = threadIdx.x;
  constexpr int E_ = (DIR + 1) % 3, F_ = (DIR + 2) % 3;
  const int ns = s.ns, mode = s.opt.mode, ref = s.opt.ref;
  const size_t NI = (size_t)s.ncells;
  const bool st = first != 0;
  // one line segment per thread and iteration (a grid smaller than the
  // segment count loops); no block-wide barrier below
  for (long long item = blockIdx.x * (long long)blockDim.x + tid; item < s.nlines[DIR];
       item += (long long)gridDim.x * blockDim.x) {
  const LineItem L = s.lines[DIR][item];
  Win x;
  x.Q = s.Q;
  x.G = s.G;
  x.NG = (size_t)s.nghost;
  x.sg = L.sg;

  for (int c0 = 0; c0 < L.len; c0 += CH) {
    const int n = min(CH, L.len - c0);
    x.gb = L.g0 + (long long)c0 * L.sg;
    const long long ib = L.i0 + (long long)c0 * L.si;
    for (int c = 0; c < n; ++c) {
      sE[c][tid] = 0.0;
      sN[c][tid] = 0.0;
      sV[c][tid] = 0.0;
    }

    // (c43 u_d,d)_d and (c43 (u_d^2/2)_d)_d
    {
      double a[9], u[9], k[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        a[i] = x.q(Q_C43, i - 4);
        u[i] = x.q(Q_U + DIR, i - 4);
        k[i] = x.q(Q_KX + DIR, i - 4);
      }
      double v[8];
      vm(P, a, 0, v);
      double Hm = dpd(v, u, 0), He = dpd(v, k, 0);
#pragma unroll 1
      for (int c = 0; c < n; ++c) {
        vm(P, a, 1, v);
        const double Hm2 = dpd(v, u, 1), He2 = dpd(v, k, 1);
        put(dU, NI, 1 + DIR, ib + (long long)c * L.si, Hm2 - Hm, st);
        sE[c][tid] += He2 - He;
        Hm = Hm2;
        He = He2;
        if (c + 1 < n) {
          slide(a); slide(u); slide(k);
          a[8] = x.q(Q_C43, c + 5);
          u[8] = x.q(Q_U + DIR, c + 5);
          k[8] = x.q(Q_KX + DIR, c + 5);
        }
      }
    }
    // (eta u_t,d)_d and (eta (u_t^2/2)_d)_d for the two transverse components t
#pragma unroll 1
    for (int tt = 0; tt < 2; ++tt) {
      const int t = tt == 0 ? E_ : F_;
      double a[9], u[9], k[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        a[i] = x.q(Q_ETA, i - 4);
        u[i] = x.q(Q_U + t, i - 4);
        k[i] = x.q(Q_KX + t, i - 4);
      }
      double v[8];
      vm(P, a, 0, v);
      double Hm = dpd(v, u, 0), He = dpd(v, k, 0);
#pragma unroll 1
      for (int c = 0; c < n; ++c) {
        vm(P, a, 1, v);
        const double Hm2 = dpd(v, u, 1), He2 = dpd(v, k, 1);
        put(dU, NI, 1 + t, ib + (long long)c * L.si, Hm2 - Hm, st);
        sE[c][tid] += He2 - He;
        Hm = Hm2;
        He = He2;
        if (c + 1 < n) {
          slide(a); slide(u); slide(k);
          a[8] = x.q(Q_ETA, c + 5);
          u[8] = x.q(Q_U + t, c + 5);
          k[8] = x.q(Q_KX + t, c + 5);
        }
      }
    }
    // (lambda T_d)_d, then (A_p p_d)_d with the pressure part of the
    // correction velocity, V_c,d = -(sum_l rhoD_l X_l,d + (sum_l B_l) p_d)
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      const int pc = pass == 0 ? Q_LAM : Q_AP, pf = pass == 0 ? Q_T : Q_P;
      double a[9], f[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        a[i] = x.q(pc, i - 4);
        f[i] = x.q(pf, i - 4);
      }
      double w[8];
      mv(P, f, 0, w);
      if (WP && pass == 1)
        for (int m = 0; m < 8; ++m) sW[m][tid] = w[m];
      double H = ds(a, 0, w);
#pragma unroll 1
      for (int c = 0; c < n; ++c) {
        if (pass == 1 && mode == 0) sV[c][tid] = -x.q(Q_SB, c) * Dc(P, f);
        mv(P, f, 1, w);
        if (WP && pass == 1)
          for (int m = 0; m < 8; ++m) sW[(c + 1) * 8 + m][tid] = w[m];
        const double H2 = ds(a, 1, w);
        sE[c][tid] += H2 - H;
        H = H2;
        if (c + 1 < n) {
          slide(a); slide(f);
          a[8] = x.q(pc, c + 5);
          f[8] = x.q(pf, c + 5);
        }
      }
    }
    // -D_d(rho u_d) and -D_d(rho u_d u_d + p - c23 (u_e,e + u_f,f))
    {
      double ms[9], fd[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        ms[i] = x.q(Q_RHO, i - 4) * x.q(Q_U + DIR, i - 4);
        fd[i] = flux_d<DIR>(x, i - 4);
      }
#pragma unroll 1
      for (int c = 0; c < n; ++c) {
        const long long i = ib + (long long)c * L.si;
        put(dU, NI, 0, i, -Dc(P, ms), st);
        put(dU, NI, 1 + DIR, i, -Dc(P, fd), false);
        if (c + 1 < n) {
          slide(ms); slide(fd);
          ms[8] = x.q(Q_RHO, c + 5) * x.q(Q_U + DIR, c + 5);
          fd[8] = flux_d<DIR>(x, c + 5);
        }
      }
    }
    // -D_d of the transverse momentum fluxes
    {
      double fe[9], ff[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) flux_ef<DIR>(x, i - 4, fe[i], ff[i]);
#pragma unroll 1
      for (int c = 0; c < n; ++c) {
        const long long i = ib + (long long)c * L.si;
        put(dU, NI, 1 + E_, i, -Dc(P, fe), false);
        put(dU, NI, 1 + F_, i, -Dc(P, ff), false);
        if (c + 1 < n) {
          slide(fe); slide(ff);
          flux_ef<DIR>(x, c + 5, fe[8], ff[8]);
        }
      }
    }
    // -D_d of the energy flux
    {
      double fE[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) fE[i] = flux_E<DIR>(x, i - 4);
#pragma unroll 1
      for (int c = 0; c < n; ++c) {
        sE[c][tid] -= Dc(P, fE);
        if (c + 1 < n) {
          slide(fE);
          fE[8] = flux_E<DIR>(x, c + 5);
        }
      }
    }
    // species, first pass: (rhoD_k X_k,d)_d, its energy part (rhoD_k h'_k
    // X_k,d)_d and the species part of the correction velocity, -rhoD_k X_k,d
#pragma unroll 1
    for (int k = 0; k < ns; ++k) {
      if (mode == 1 && k == ref) {
        if (st)
          for (int c = 0; c < n; ++c) put(dU, NI, 5 + k, ib + (long long)c * L.si, 0.0, true);
        continue;
      }
      double X[9], rd[9], rdh[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        X[i] = x.q(qX(ns) + k, i - 4);
        rd[i] = x.q(qRD(ns) + k, i - 4);
        rdh[i] = x.q(qRDH(ns) + k, i - 4);
      }
      double w[8];
      mv(P, X, 0, w);
      double H = ds(rd, 0, w), He = ds(rdh, 0, w);
#pragma unroll 1
      for (int c = 0; c < n; ++c) {
        if (mode == 0) sV[c][tid] -= rd[4] * Dc(P, X);
        mv(P, X, 1, w);
        const double H2 = ds(rd, 1, w), He2 = ds(rdh, 1, w);
        put(dU, NI, 5 + k, ib + (long long)c * L.si, H2 - H, st);
        sN[c][tid] += H2 - H;
        sE[c][tid] += He2 - He;
        H = H2;
        He = He2;
        if (c + 1 < n) {
          slide(X); slide(rd); slide(rdh);
          X[8] = x.q(qX(ns) + k, c + 5);
          rd[8] = x.q(qRD(ns) + k, c + 5);
          rdh[8] = x.q(qRDH(ns) + k, c + 5);
        }
      }
    }
    // species, second pass (V_c complete): (B_k p_d)_d, -D_d(rho Y_k u_d) and
    // Y_k,d V_c,d
#pragma unroll 1
    for (int k = 0; k < ns; ++k) {
      const bool narrow = !(mode == 1 && k == ref);
      double p[9], B[9], Fk[9], Yk[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        p[i] = x.q(Q_P, i - 4);
        B[i] = x.q(qB(ns) + k, i - 4);
        Fk[i] = x.q(qRY(ns) + k, i - 4) * x.q(Q_U + DIR, i - 4);
        Yk[i] = mode == 0 ? x.q(qY(ns) + k, i - 4) : 0.0;
      }
      double w[8];
      if (WP) {
        for (int m = 0; m < 8; ++m) w[m] = sW[m][tid];
      } else {
        mv(P, p, 0, w);
      }
      double H = ds(B, 0, w);
#pragma unroll 1
      for (int c = 0; c < n; ++c) {
        double o = -Dc(P, Fk);
        if (mode == 0) o = fma(Dc(P, Yk), sV[c][tid], o);
        if (narrow) {
          if (WP) {
            for (int m = 0; m < 8; ++m) w[m] = sW[(c + 1) * 8 + m][tid];
          } else {
            mv(P, p, 1, w);
          }
          const double H2 = ds(B, 1, w);
          o += H2 - H;
          sN[c][tid] += H2 - H;
          H = H2;
        }
        put(dU, NI, 5 + k, ib + (long long)c * L.si, o, false);
        if (c + 1 < n) {
          slide(p); slide(B); slide(Fk);
          p[8] = x.q(Q_P, c + 5);
          B[8] = x.q(qB(ns) + k, c + 5);
          Fk[8] = x.q(qRY(ns) + k, c + 5) * x.q(Q_U + DIR, c + 5);
          if (mode == 0) {
            slide(Yk);
            Yk[8] = x.q(qY(ns) + k, c + 5);
          }
        }
      }
    }
    if (mode == 1) {
      for (int c = 0; c < n; ++c)
        put(dU, NI, 5 + ref, ib + (long long)c * L.si, -sN[c][tid], false);
    } else {
      // h,d V_c,d
      double hm[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) hm[i] = x.q(Q_HMIX, i - 4);
#pragma unroll 1
      for (int c = 0; c < n; ++c) {
        sE[c][tid] = fma(Dc(P, hm), sV[c][tid], sE[c][tid]);
        if (c + 1 < n) {
          slide(hm);
          hm[8] = x.q(Q_HMIX, c + 5);
        }
      }
      for (int c = 0; c < n; ++c) {
        const long long i = ib + (long long)c * L.si;
        if (st) s.divacc[i] = sN[c][tid]; else s.divacc[i] += sN[c][tid];
      }
    }
    for (int c = 0; c < n; ++c) put(dU, NI, 4, ib + (long long)c * L.si, sE[c][tid], st);
  }
  }
}

template <int CH, bool WP, int MINB>
void launch_variant(const DevState &s, int dir, const ParamsW &P, double *dU, int first,
                    int blocks, cudaStream_t st) {
  const size_t smem = (3 * CH + (WP ? 8 * (CH + 1) : 0)) * NT * sizeof(double);
  // the attribute is per device: set it once per device, on the first
  // (eager) launch, before any stream capture
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    cudaFuncSetAttribute(k_march_w<0, CH, WP, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    cudaFuncSetAttribute(k_march_w<1, CH, WP, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    cudaFuncSetAttribute(k_march_w<2, CH, WP, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr_set[dev] = true;
  }
  if (s.opt.persistent) {
    static int cache[64] = {};
    const int r = resident_blocks(k_march_w<1, CH, WP, MINB>, NT, smem, cache);
    if (blocks > r) blocks = r;
  }
  if (dir == 0) k_march_w<0, CH, WP, MINB><<<blocks, NT, smem, st>>>(s, P, dU, first);
  else if (dir == 1) k_march_w<1, CH, WP, MINB><<<blocks, NT, smem, st>>>(s, P, dU, first);
  else k_march_w<2, CH, WP, MINB><<<blocks, NT, smem, st>>>(s, P, dU, first);
}

}  // namespace

void launch_march_w(const DevState &s, int dir, double *dUdt, int first, int variant,
                    cudaStream_t st) {
  const Coef *hc = s.hcoef;
  ParamsW P;
  for (int m = 0; m < 8; ++m)
    for (int n = 0; n < 8; ++n) P.M[m][n] = hc->M[dir][m][n];
  for (int k = 0; k < 4; ++k) P.D[k] = hc->D[dir][k];
  const long long n = s.nlines[dir];
  if (n == 0) return;
  const int blocks = (int)((n + NT - 1) / NT);
  if (variant == 3) launch_variant<8, true, 2>(s, dir, P, dUdt, first, blocks, st);
  else if (variant == 2) launch_variant<32, false, 3>(s, dir, P, dUdt, first, blocks, st);
  else launch_variant<16, false, 3>(s, dir, P, dUdt, first, blocks, st);
}

}  // namespace smc
