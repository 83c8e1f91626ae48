// Mixed-precision right-hand side: stencil, transport and correction-velocity
// arithmetic in FP32; temperature inversion, Gibbs energies, exponentials,
// production rates and the result accumulation in FP64.
//
// Fields that enter differences (velocities, T, p, kinetic energies, h, rho,
// rho H, Y_k, X_k, rho Y_k) are stored as float pairs hi + lo with
// hi = fl32(x), lo = fl32(x - hi) (about 48 significant bits); a difference
// x_a - x_b is formed as (hi_a - hi_b) + (lo_a - lo_b), accurate to FP32
// rounding of the difference itself rather than of x.  Coefficients (eta,
// lambda, rho D_k, B_k, ...) are plain floats.  Products that form
// convective fluxes (rho u_d, rho u_c u_d, rho H u_d, rho Y_k u_d) are
// carried as float pairs through an FMA-based exact product.
#include "bc.cuh"
#include "chem.cuh"
#include "smc_internal.h"

namespace smc {

int nQm(int ns) { return PM_NBASE + 9 * ns; }

struct f2 {
  float h, l;
};

// x = hi + lo with hi the truncation of x to 24 bits (exactly representable)
// and lo the remainder truncated to 24 bits: about 48 significant bits.  In
// integer arithmetic only (the FP64 pipe is the scarce one): hi keeps the
// top 23 stored mantissa bits; lo is the low 29 bits, x - hi exactly,
// normalised and truncated to a float.  Zero, subnormal and tiny remainders
// flush to zero, as trunc_float does.
__device__ __forceinline__ void put_pair(float *Qf, size_t NG, int plane, long long g, double x) {
  const long long b = __double_as_longlong(x);
  Qf[(size_t)plane * NG + g] = trunc_float(__longlong_as_double(b & (long long)0xFFFFFFFFE0000000ULL));
  const unsigned m = (unsigned)(b & 0x1FFFFFFFLL);                 // x - hi = m 2^(e - 52)
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  float lo = 0.0f;
  if (m != 0u && e > -1022 && e < 1024) {
    const int p = 31 - __clz(m);                                    // leading bit of m, 0..28
    const int fe = e - 52 + p + 127;                                // float exponent field
    if (fe > 0) {
      const unsigned frac = (p >= 23 ? (m >> (p - 23)) : (m << (23 - p))) & 0x7fffffu;
      lo = __uint_as_float((unsigned)((unsigned long long)b >> 63) << 31 | (unsigned)fe << 23 | frac);
    }
  }
  Qf[(size_t)(plane + 1) * NG + g] = lo;
}

// x rounded to the nearest float (ties away from zero) in integer
// arithmetic: half a float ulp added to the magnitude, then truncated.
// For finite x in the float range.
__device__ __forceinline__ float round_float(double x) {
  return trunc_float(__longlong_as_double(__double_as_longlong(x) + (1LL << 28)));
}

__device__ __forceinline__ f2 get_pair(const float *__restrict__ Qf, size_t NG, int plane,
                                       long long g) {
  f2 r;
  r.h = __ldg(Qf + (size_t)plane * NG + g);
  r.l = __ldg(Qf + (size_t)(plane + 1) * NG + g);
  return r;
}

__device__ __forceinline__ float diff(f2 a, f2 b) { return (a.h - b.h) + (a.l - b.l); }

// a * b as a float pair (exact product of the high parts plus the cross terms)
__device__ __forceinline__ f2 mul(f2 a, f2 b) {
  f2 r;
  r.h = a.h * b.h;
  r.l = fmaf(a.h, b.h, -r.h) + fmaf(a.h, b.l, a.l * b.h);
  return r;
}

__device__ __forceinline__ f2 mulf(f2 a, float b) {
  f2 r;
  r.h = a.h * b;
  r.l = fmaf(a.h, b, -r.h) + a.l * b;
  return r;
}

// ------------------------------------------------------------ k_prim_m
// INTERIOR: one thread per interior cell (ghost cells filled by k_halo);
// otherwise one per ghosted cell through the gather map.
template <bool INTERIOR>
__global__ void __launch_bounds__(128) k_prim_m(const DevState s, const double *__restrict__ U) {
  const Mech &m = *s.mech;
  const int ns = s.ns;
  const long long NG = s.nghost, NI = s.ncells;
  float *__restrict__ Qf = reinterpret_cast<float *>(s.Q);
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
    double Y[SMC_MAX_NS];
    for (int k = 0; k < ns; ++k) Y[k] = U[(5 + k) * NI + src] * invrho;
    const double e = rhoE * invrho - 0.5 * (u * u + v * v + w * w);
    // first guess: this cell's temperature from the handle's previous mixed
    // evaluation when there is one (a nearby state: two Newton steps instead
    // of four or five from the fixed guess), else the fixed guess
    double T0 = s.opt.T0;
    if (INTERIOR && s.warm_T) {
      const f2 tp = get_pair(Qf, NG, PM_T, g);
      const double tg = (double)tp.h + (double)tp.l;
      if (tg > 0.0 && isfinite(tg)) T0 = tg;
    }
    double T, cpd, hm;
    const bool ok = newton_T(m, Y, e, T0, s.opt.tol, s.opt.maxit, T, &cpd, &hm);
    unsigned flag = 0;
    if (!ok) flag |= ST_NONCONV;
    if (!(rho > 0.0) || !(T > 0.0)) flag |= ST_NONPHYS;
    if (!isfinite(rho) || !isfinite(rhoE) || !isfinite(T)) flag |= ST_NONFINITE;
    if (flag) atomicOr(s.status, flag);

    double wmix = 0.0;
    const float Tf = trunc_float(T);
    float h32[SMC_MAX_NS];
    for (int k = 0; k < ns; ++k) {
      wmix += Y[k] * m.invW[k];
      // species enthalpies only enter coefficients: FP32
      const float *c = m.hTf[k];
      const float hRf = c[0] + Tf * (c[1] + Tf * (c[2] + Tf * (c[3] + Tf * (c[4] + Tf * c[5]))));
      h32[k] = m.Ru_Wf[k] * hRf;
    }
    const double p = rho * kRu * T * wmix;
    const double inv_wmix = 1.0 / wmix;
    // Transport coefficients: computed in FP64 from the FP64 temperature and
    // rounded once to float.  They multiply stencil products whose face sums
    // cancel (a species' gradient and pressure fluxes can be several times its
    // net flux, and a face flux tens of times its divergence), so rounding
    // noise from a chain of FP32 operations would be amplified by as much.
    const double eta_d = m.eta_ref * mech_exp(m, m.eta_exp * log(T * m.inv_T_ref));
    const double xi_d = s.opt.xi_ratio * eta_d;
    const double rd0_d = eta_d * m.inv_Pr;           // lambda / cp = rho D_k Le_k
    const double bq = rd0_d / p;                     // B_k = bq (X_k - Y_k) / Le_k
    const float eta = round_float(eta_d);
    const float lam = round_float(cpd * rd0_d);
    put_pair(Qf, NG, PM_U, g, u);
    put_pair(Qf, NG, PM_V, g, v);
    put_pair(Qf, NG, PM_W, g, w);
    put_pair(Qf, NG, PM_T, g, T);
    put_pair(Qf, NG, PM_P, g, p);
    put_pair(Qf, NG, PM_KX, g, 0.5 * u * u);
    put_pair(Qf, NG, PM_KY, g, 0.5 * v * v);
    put_pair(Qf, NG, PM_KZ, g, 0.5 * w * w);
    put_pair(Qf, NG, PM_HMIX, g, hm);
    put_pair(Qf, NG, PM_RHO, g, rho);
    put_pair(Qf, NG, PM_RHOH, g, rhoE + p);
    Qf[(size_t)PM_C43 * NG + g] = round_float(4.0 / 3.0 * eta_d + xi_d);
    Qf[(size_t)PM_ETA * NG + g] = eta;
    Qf[(size_t)PM_C23 * NG + g] = round_float(xi_d - 2.0 / 3.0 * eta_d);
    Qf[(size_t)PM_LAM * NG + g] = lam;
    const float href = (mode == 1) ? h32[ref] : 0.0f;
    float ap = 0.0f;
    double sb = 0.0;                                 // sum_k B_k: its terms cancel (sum X = sum Y)
    for (int k = 0; k < ns; ++k) {
      const double X = Y[k] * m.invW[k] * inv_wmix;
      const float rd = round_float(rd0_d * m.invLe[k]);
      const double Bd = bq * m.invLe[k] * (X - Y[k]);
      const float B = round_float(Bd);
      const float hp = h32[k] - href;
      if (mode == 0) {
        ap += h32[k] * B;
        sb += Bd;
      } else if (k != ref) {
        ap += hp * B;
      }
      put_pair(Qf, NG, pmY(ns, k), g, Y[k]);
      put_pair(Qf, NG, pmX(ns, k), g, X);
      put_pair(Qf, NG, pmRY(ns, k), g, U[(5 + k) * NI + src]);
      Qf[(size_t)pmRD(ns, k) * NG + g] = rd;
      Qf[(size_t)pmRDH(ns, k) * NG + g] = rd * hp;
      Qf[(size_t)pmB(ns, k) * NG + g] = B;
    }
    Qf[(size_t)PM_AP * NG + g] = ap;
    Qf[(size_t)PM_SB * NG + g] = round_float(sb);
  }
}

// ------------------------------------------------------------ k_grad_m
struct GradParamsM {
  float D[3][4];
  double ihx;                     // 1/h_x (boundary-lowered x derivatives, FP64)
};

__device__ __forceinline__ int find_box_m(const Box *__restrict__ b, int nb, long long g) {
  int lo = 0, hi = nb - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (b[mid].off_g <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(128) k_grad_m(const DevState s, const GradParamsM P) {
  const long long NG = s.nghost;
  const float *__restrict__ Qf = reinterpret_cast<const float *>(s.Q);
  float *__restrict__ Gf = reinterpret_cast<float *>(s.G);
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < NG;
       g += (long long)gridDim.x * blockDim.x) {
    const Box B = s.boxes[find_box_m(s.boxes, s.nboxes, g)];
    const long long l = g - B.off_g;
    const int crd[3] = {(int)(l % B.gx) - SMC_GHOST, (int)((l / B.gx) % B.gy) - SMC_GHOST,
                        (int)(l / ((long long)B.gx * B.gy)) - SMC_GHOST};
    const int n[3] = {B.nx, B.ny, B.nz};
    const long long stride[3] = {1, B.gx, (long long)B.gx * B.gy};
    int ng = 0;
    for (int e = 0; e < 3; ++e) ng += (crd[e] < 0 || crd[e] >= n[e]);
    // cells next to non-periodic x ends take the lowered x derivative (FP64)
    const int gxi = B.lo[0] + crd[0];
    const int kb = !s.x_outflow ? -1
                   : (gxi >= 0 && gxi < 4) ? gxi
                   : (gxi >= s.nx_domain - 4 && gxi < s.nx_domain) ? s.nx_domain - 1 - gxi : -1;
    for (int e = 0; e < 3; ++e) {
      if (crd[e] < 0 || crd[e] >= n[e] || ng > 1) continue;
      for (int c = 0; c < 3; ++c) {
        float acc = 0.0f;
        if (e == 0 && kb >= 0) {
          const long long sg = gxi < 4 ? 1 : -1;
          double v[7];
          for (int j = 0; j < 7; ++j) {
            const f2 pr = get_pair(Qf, NG, PM_U + 2 * c, g + sg * (j - kb));
            v[j] = (double)pr.h + (double)pr.l;
          }
          acc = (float)((double)sg * lowered_d(v, kb) * P.ihx);
        } else {
#pragma unroll
          for (int k = 1; k <= 4; ++k)
            acc += P.D[e][k - 1] * diff(get_pair(Qf, NG, PM_U + 2 * c, g + k * stride[e]),
                                        get_pair(Qf, NG, PM_U + 2 * c, g - k * stride[e]));
        }
        Gf[(size_t)(3 * e + c) * NG + g] = acc;
      }
    }
  }
}

// ------------------------------------------------------------ line-kernel constants
struct MarchParamsM {
  float M[8][8];
  float D[4];
  float2 MT2[8][4];               // (M[2j][t], M[2j+1][t]): two rows of a column, for FFMA2
};

// ------------------------------------------------------------ k_final_m
// dUdt (FP64) = float stencil sum + correction terms (FP32) + rho omega_k (FP64)
__global__ void __launch_bounds__(128) k_final_m(const DevState s, const double *__restrict__ U,
                                                 const float *__restrict__ dUf,
                                                 double *__restrict__ dU, int transport,
                                                 int chemistry) {
  const Mech &m = *s.mech;
  const int ns = s.ns;
  const size_t NG = (size_t)s.nghost, NI = (size_t)s.ncells;
  const float *__restrict__ Qf = reinterpret_cast<const float *>(s.Q);
  const float *__restrict__ divf = reinterpret_cast<const float *>(s.divacc);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)NI;
       i += (long long)gridDim.x * blockDim.x) {
    const long long g = s.imap[i];
    double add[SMC_MAX_NS];
    for (int k = 0; k < ns; ++k) add[k] = 0.0;
    if (chemistry) {
      // the temperature of the primitive pass, then the rates (FP64, or with
      // FP32 mantissas when SMC_OPT_RATES is 1)
      double rhoY[SMC_MAX_NS], wd[SMC_MAX_NS];
      for (int k = 0; k < ns; ++k) rhoY[k] = U[(size_t)(5 + k) * NI + i];
      const f2 Tp = get_pair(Qf, NG, PM_T, g);
      const double T = (double)Tp.h + (double)Tp.l;
      if (s.opt.rates32) production_rates_m(m, s.rx, T, rhoY, wd);
      else production_rates(m, s.rx, 0.0, T, nullptr, wd, rhoY);
      for (int k = 0; k < ns; ++k) add[k] = wd[k];
    }
    if (transport) {
      float corr[SMC_MAX_NS];
      float corrE = 0.0f;
      for (int k = 0; k < ns; ++k) corr[k] = 0.0f;
      if (s.opt.mode == 0) {
        const float divVc = -divf[i];
        const f2 hm = get_pair(Qf, NG, PM_HMIX, g);
        corrE = (hm.h + hm.l) * divVc;
        for (int k = 0; k < ns; ++k) {
          const f2 y = get_pair(Qf, NG, pmY(ns, k), g);
          corr[k] = (y.h + y.l) * divVc;
        }
      }
      for (int c = 0; c < 4; ++c) dU[(size_t)c * NI + i] = (double)dUf[(size_t)c * NI + i];
      dU[4 * NI + i] = (double)(dUf[4 * NI + i] + corrE);
      for (int k = 0; k < ns; ++k)
        dU[(5 + k) * NI + i] = (double)(dUf[(5 + k) * NI + i] + corr[k]) + add[k];
    } else {
      for (int c = 0; c < 5; ++c) dU[(size_t)c * NI + i] = 0.0;
      for (int k = 0; k < ns; ++k) dU[(5 + k) * NI + i] = add[k];
    }
  }
}

// ------------------------------------------------------------ launchers
static int grid_for(long long n, int block) {
  long long b = (n + block - 1) / block;
  const long long cap = 152LL * 64;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

void launch_prim_m(const DevState &s, const double *U, cudaStream_t st) {
  if (s.nhalo > 0) {
    k_prim_m<true><<<grid_for(s.ncells, 128), 128, 0, st>>>(s, U);
    launch_halo(s, nQm(s.ns), 4, st);
  } else {
    k_prim_m<false><<<grid_for(s.nghost, 128), 128, 0, st>>>(s, U);
  }
}

void launch_grad_m(const DevState &s, cudaStream_t st) {
  GradParamsM P;
  for (int d = 0; d < 3; ++d)
    for (int k = 0; k < 4; ++k) P.D[d][k] = (float)s.hcoef->D[d][k];
  P.ihx = s.hcoef->D[0][0] * 1.25;
  k_grad_m<<<grid_for(s.nghost, 128), 128, 0, st>>>(s, P);
}

void launch_final_m(const DevState &s, const double *U, const float *dUf, double *dU, int transport,
                    int chemistry, cudaStream_t st) {
  k_final_m<<<grid_for(s.ncells, 128), 128, 0, st>>>(s, U, dUf, dU, transport, chemistry);
}



// ------------------------------------------------------------ k_march_m2
// The same terms as k_march_m, organised for data reuse.  Each thread walks
// its line segment in chunks of up to CH cells.  Every field is held in a
// 9-cell register window (cells c-4 .. c+4 of the current cell c) that slides
// by one cell per step, so a field value is loaded once per cell rather than
// once per face or per stencil point.  The terms are taken in sub-passes over
// small groups of fields (momentum, heat, convective fluxes, correction
// velocity, then one species at a time) to bound the live registers; the
// per-cell energy, correction velocity, species divergence sum and species
// narrow term are carried between sub-passes in shared memory.
constexpr int M2_NT = 128;

namespace m2 {

struct Win {
  const float *__restrict__ Qf;
  const float *__restrict__ Gf;
  size_t NG;
  long long gb;   // ghosted index of the chunk's first cell
  int sg;
  __device__ __forceinline__ float s(int plane, int r) const {
    return __ldg(Qf + (size_t)plane * NG + gb + (long long)r * sg);
  }
  __device__ __forceinline__ float g(int plane, int r) const {
    return __ldg(Gf + (size_t)plane * NG + gb + (long long)r * sg);
  }
  __device__ __forceinline__ f2 p(int plane, int r) const {
    f2 v;
    v.h = __ldg(Qf + (size_t)plane * NG + gb + (long long)r * sg);
    v.l = __ldg(Qf + (size_t)(plane + 1) * NG + gb + (long long)r * sg);
    return v;
  }
};

// v[n] = sum_m a[o+m] M[m][n] for n != 3, two columns per paired FMA
__device__ __forceinline__ void vm(const MarchParamsM &P, const float *a, int o, float *v) {
#pragma unroll
  for (int np = 0; np < 4; ++np) {
    float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int mm = 0; mm < 8; ++mm) {
      const int n0 = 2 * np, n1 = 2 * np + 1;
      const bool nz = (mm - n0 <= 4 && n0 - mm <= 4) || (mm - n1 <= 4 && n1 - mm <= 4);
      if (nz)
        acc = __ffma2_rn(make_float2(a[o + mm], a[o + mm]),
                         make_float2(P.M[mm][n0], P.M[mm][n1]), acc);
    }
    v[2 * np] = acc.x;
    v[2 * np + 1] = acc.y;
  }
}
// the differences x[o+t] - x[o+3] of a pair window, one paired add each
__device__ __forceinline__ void diffs(const f2 *x, int o, float *d) {
  const float2 m3 = make_float2(-x[o + 3].h, -x[o + 3].l);
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    if (t == 3) {
      d[t] = 0.0f;
    } else {
      const float2 e = __fadd2_rn(make_float2(x[o + t].h, x[o + t].l), m3);
      d[t] = e.x + e.y;
    }
  }
}
// w[m] = sum_{n != 3} M[m][n] (x[o+n] - x[o+3]), two rows per paired FMA
__device__ __forceinline__ void mv(const MarchParamsM &P, const f2 *x, int o, float *w) {
  float d[8];
  diffs(x, o, d);
  float2 acc[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) acc[j] = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    if (t == 3) continue;
    const float2 dd = make_float2(d[t], d[t]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m0 = 2 * j, m1 = 2 * j + 1;
      const bool nz = (m0 - t <= 4 && t - m0 <= 4) || (m1 - t <= 4 && t - m1 <= 4);
      if (nz) acc[j] = __ffma2_rn(P.MT2[t][j], dd, acc[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    w[2 * j] = acc[j].x;
    w[2 * j + 1] = acc[j].y;
  }
}
// w[m] = sum_{n != 3} M[m][n] d[n] for given differences d (d[3] unused)
__device__ __forceinline__ void mvd(const MarchParamsM &P, const float *d, float *w) {
  float2 acc[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) acc[j] = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    if (t == 3) continue;
    const float2 dd = make_float2(d[t], d[t]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m0 = 2 * j, m1 = 2 * j + 1;
      const bool nz = (m0 - t <= 4 && t - m0 <= 4) || (m1 - t <= 4 && t - m1 <= 4);
      if (nz) acc[j] = __ffma2_rn(P.MT2[t][j], dd, acc[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    w[2 * j] = acc[j].x;
    w[2 * j + 1] = acc[j].y;
  }
}
// For the 9-cell pair window x (cells c-4 .. c+4) the change, from the face
// left of cell c (window cells 0..7) to the face right of it (1..8), of the
// differences the narrow stencil multiplies: with d_f[n] = x[f+n] - x[f+3],
//   dd[n] = d_1[n] - d_0[n] = (x[n+1] - x[n]) - (x[4] - x[3]),
// formed from the pairs' neighbour differences (the high parts of neighbouring
// values subtract exactly), so dd carries the second differences of x at
// FP32 precision relative to themselves.
__device__ __forceinline__ void ddiffs(const f2 *x, float *dd) {
  const float d3h = x[4].h - x[3].h, d3l = x[4].l - x[3].l;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    if (t == 3) {
      dd[t] = 0.0f;
    } else {
      const float2 e = __fadd2_rn(make_float2(x[t + 1].h - x[t].h, x[t + 1].l - x[t].l),
                                  make_float2(-d3h, -d3l));
      dd[t] = e.x + e.y;
    }
  }
}
// The flux difference H_1 - H_0 of a narrow term between the faces right and
// left of cell c, with H_f = sum_m a[f+m] w_f[m], formed directly:
//   H_1 - H_0 = sum_m a[1+m] (w_1 - w_0)[m] + (a[1+m] - a[m]) w_0[m],
// w_1 - w_0 = M dd (ddiffs).  Every product is of the size of the result,
// instead of the face fluxes' (which can be tens of times larger and cancel),
// so FP32 rounding is not amplified by that ratio.  w0: the left face's w.
__device__ __forceinline__ float flux_diff(const MarchParamsM &P, const float *a, const f2 *x,
                                           const float *w0) {
  float dd[8], dw[8];
  ddiffs(x, dd);
  mvd(P, dd, dw);
  float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int t = 0; t < 8; t += 2) {
    acc = __ffma2_rn(make_float2(a[1 + t], a[2 + t]), make_float2(dw[t], dw[t + 1]), acc);
    acc = __ffma2_rn(make_float2(a[1 + t] - a[t], a[2 + t] - a[1 + t]), make_float2(w0[t], w0[t + 1]), acc);
  }
  return acc.x + acc.y;
}
// flux_diff with the face products given: dw = M dd and w0 (the left face's w)
__device__ __forceinline__ float flux_diff_w(const float *a, const float *dw, const float *w0) {
  float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int t = 0; t < 8; t += 2) {
    acc = __ffma2_rn(make_float2(a[1 + t], a[2 + t]), make_float2(dw[t], dw[t + 1]), acc);
    acc = __ffma2_rn(make_float2(a[1 + t] - a[t], a[2 + t] - a[1 + t]), make_float2(w0[t], w0[t + 1]), acc);
  }
  return acc.x + acc.y;
}
// sum_{n != 3} v[n] (x[o+n] - x[o+3])
__device__ __forceinline__ float dp(const float *v, const f2 *x, int o) {
  float d[8];
  diffs(x, o, d);
  float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int t = 0; t < 8; t += 2) acc = __ffma2_rn(make_float2(v[t], v[t + 1]), make_float2(d[t], d[t + 1]), acc);
  return acc.x + acc.y;
}
// sum_t a[o+t] w[t]
__device__ __forceinline__ float ds(const float *a, int o, const float *w) {
  float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int t = 0; t < 8; t += 2) acc = __ffma2_rn(make_float2(a[o + t], a[o + t + 1]), make_float2(w[t], w[t + 1]), acc);
  return acc.x + acc.y;
}
template <typename T>
__device__ __forceinline__ void slide(T *w) {
#pragma unroll
  for (int i = 0; i < 8; ++i) w[i] = w[i + 1];
}
// centred D at the middle (index 4) of a 9-cell window
__device__ __forceinline__ float Dp(const MarchParamsM &P, const f2 *w) {
  float acc = 0.0f;
#pragma unroll
  for (int nn = 1; nn <= 4; ++nn) acc = fmaf(P.D[nn - 1], diff(w[4 + nn], w[4 - nn]), acc);
  return acc;
}
__device__ __forceinline__ float Ds(const MarchParamsM &P, const float *w) {
  float acc = 0.0f;
#pragma unroll
  for (int nn = 1; nn <= 4; ++nn) acc = fmaf(P.D[nn - 1], w[4 + nn] - w[4 - nn], acc);
  return acc;
}

// Store, or add without waiting for the old value: the add goes out as a
// reduction (no result returned), so the thread does not stall on a global
// load in every step of the march.  Each cell is updated by one thread per
// launch, in program order, so the sums are deterministic.
__device__ __forceinline__ void put(float *__restrict__ dUf, size_t NI, int comp, long long i, float v,
                                    bool store) {
  float *q = dUf + (size_t)comp * NI + i;
  if (store) *q = v; else atomicAdd(q, v);
}

// transverse momentum fluxes rho u_d u_t - eta u_d,t (t = e, f) at window offset r
template <int DIR>
__device__ __forceinline__ void flux_ef(const Win &x, int r, f2 &fe, f2 &ff) {
  constexpr int E_ = (DIR + 1) % 3, F_ = (DIR + 2) % 3;
  const f2 m = mul(x.p(PM_RHO, r), x.p(PM_U + 2 * DIR, r));
  fe = mul(m, x.p(PM_U + 2 * E_, r));
  ff = mul(m, x.p(PM_U + 2 * F_, r));
  const float eta = x.s(PM_ETA, r);
  fe.l -= eta * x.g(3 * E_ + DIR, r);
  ff.l -= eta * x.g(3 * F_ + DIR, r);
}

// energy flux rho H u_d - [c23 (u_e,e + u_f,f) u_d + eta (u_d,e u_e + u_d,f u_f)]
template <int DIR>
__device__ __forceinline__ f2 flux_E(const Win &x, int r) {
  constexpr int E_ = (DIR + 1) % 3, F_ = (DIR + 2) % 3;
  const f2 ud = x.p(PM_U + 2 * DIR, r), ue = x.p(PM_U + 2 * E_, r), uf = x.p(PM_U + 2 * F_, r);
  const float eta = x.s(PM_ETA, r);
  const float tdiv = x.s(PM_C23, r) * (x.g(3 * E_ + E_, r) + x.g(3 * F_ + F_, r));
  f2 fE = mul(x.p(PM_RHOH, r), ud);
  fE.l -= tdiv * (ud.h + ud.l) +
          eta * (x.g(3 * E_ + DIR, r) * (ue.h + ue.l) + x.g(3 * F_ + DIR, r) * (uf.h + uf.l));
  return fE;
}

}  // namespace m2

// CH: cells per chunk; MINB: resident blocks per SM the register budget is
// sized for (3: 168 registers, 2: 255).  The four per-cell arrays live in
// dynamic shared memory, 4 CH M2_NT floats.  WP: the pressure products of
// every cell's two faces (w of the left face, and w_right - w_left) are
// formed once in the heat pass and kept in shared memory (16 CH M2_NT more
// floats) for every species' pressure term, instead of formed again per
// species.
template <int DIR, int CH, int MINB, bool WP>
__global__ void __launch_bounds__(M2_NT, MINB) k_march_m2(const DevState s, const MarchParamsM P,
                                                          float *__restrict__ dUf, int first) {
  using namespace m2;
  extern __shared__ float m2_smem[];
  float(*sE)[M2_NT] = reinterpret_cast<float(*)[M2_NT]>(m2_smem);
  float(*sV)[M2_NT] = sE + CH;
  float(*sN)[M2_NT] = sV + CH;
  float(*sO)[M2_NT] = sN + CH;
  float(*sW)[M2_NT] = sO + CH;     // [(cell * 16 + m)][thread], WP only
  const int tid = threadIdx.x;
  constexpr int E_ = (DIR + 1) % 3, F_ = (DIR + 2) % 3;
  const int ns = s.ns, mode = s.opt.mode, ref = s.opt.ref;
  const size_t NI = (size_t)s.ncells;
  float *__restrict__ divf = reinterpret_cast<float *>(s.divacc);
  const bool st = first != 0;
  // one line segment per thread and iteration (a grid smaller than the
  // segment count loops); no block-wide barrier below
  for (long long item = blockIdx.x * (long long)blockDim.x + tid; item < s.nlines[DIR];
       item += (long long)gridDim.x * blockDim.x) {
  const LineItem L = s.lines[DIR][item];
  Win x;
  x.Qf = reinterpret_cast<const float *>(s.Q);
  x.Gf = reinterpret_cast<const float *>(s.G);
  x.NG = (size_t)s.nghost;
  x.sg = L.sg;

  for (int c0 = 0; c0 < L.len; c0 += CH) {
    const int n = min(CH, L.len - c0);
    x.gb = L.g0 + (long long)c0 * L.sg;
    const long long ib = L.i0 + (long long)c0 * L.si;
    for (int c = 0; c < n; ++c) {
      sE[c][tid] = 0.0f;
      sN[c][tid] = 0.0f;
    }

    // (c43 u_d,d)_d and (c43 (u_d^2/2)_d)_d
    {
      float a[9];
      f2 u[9], k[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        a[i] = x.s(PM_C43, i - 4);
        u[i] = x.p(PM_U + 2 * DIR, i - 4);
        k[i] = x.p(PM_KX + 2 * DIR, i - 4);
      }
      float v[8];
      vm(P, a, 0, v);
      float Hm = dp(v, u, 0), He = dp(v, k, 0);
#pragma unroll 1
      for (int c = 0; c < n; ++c) {
        vm(P, a, 1, v);
        const float Hm2 = dp(v, u, 1), He2 = dp(v, k, 1);
        put(dUf, NI, 1 + DIR, ib + (long long)c * L.si, Hm2 - Hm, st);
        sE[c][tid] += He2 - He;
        Hm = Hm2;
        He = He2;
        if (c + 1 < n) {
          slide(a); slide(u); slide(k);
          a[8] = x.s(PM_C43, c + 5);
          u[8] = x.p(PM_U + 2 * DIR, c + 5);
          k[8] = x.p(PM_KX + 2 * DIR, c + 5);
        }
      }
    }
    // (eta u_t,d)_d and (eta (u_t^2/2)_d)_d for the two transverse components t
#pragma unroll 1
    for (int tt = 0; tt < 2; ++tt) {
      const int t = tt == 0 ? E_ : F_;
      float a[9];
      f2 u[9], k[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        a[i] = x.s(PM_ETA, i - 4);
        u[i] = x.p(PM_U + 2 * t, i - 4);
        k[i] = x.p(PM_KX + 2 * t, i - 4);
      }
      float v[8];
      vm(P, a, 0, v);
      float Hm = dp(v, u, 0), He = dp(v, k, 0);
#pragma unroll 1
      for (int c = 0; c < n; ++c) {
        vm(P, a, 1, v);
        const float Hm2 = dp(v, u, 1), He2 = dp(v, k, 1);
        put(dUf, NI, 1 + t, ib + (long long)c * L.si, Hm2 - Hm, st);
        sE[c][tid] += He2 - He;
        Hm = Hm2;
        He = He2;
        if (c + 1 < n) {
          slide(a); slide(u); slide(k);
          a[8] = x.s(PM_ETA, c + 5);
          u[8] = x.p(PM_U + 2 * t, c + 5);
          k[8] = x.p(PM_KX + 2 * t, c + 5);
        }
      }
    }
    // (lambda T_d)_d, then (A_p p_d)_d
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      const int pc = pass == 0 ? PM_LAM : PM_AP, pf = pass == 0 ? PM_T : PM_P;
      float a[9];
      f2 f[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        a[i] = x.s(pc, i - 4);
        f[i] = x.p(pf, i - 4);
      }
      float w[8];
      mv(P, f, 0, w);
      float H = ds(a, 0, w);
#pragma unroll 1
      for (int c = 0; c < n; ++c) {
        // the pressure part of the correction velocity,
        // V_c,d = -(sum_l rhoD_l X_l,d + (sum_l B_l) p_d): p is in this pass's window
        if (pass == 1 && mode == 0) sV[c][tid] = -x.s(PM_SB, c) * Dp(P, f);
        if (WP && pass == 1) {
          float dd[8], dw[8];
          ddiffs(f, dd);
          mvd(P, dd, dw);
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            sW[c * 16 + m][tid] = w[m];
            sW[c * 16 + 8 + m][tid] = dw[m];
          }
        }
        mv(P, f, 1, w);
        const float H2 = ds(a, 1, w);
        sE[c][tid] += H2 - H;
        H = H2;
        if (c + 1 < n) {
          slide(a); slide(f);
          a[8] = x.s(pc, c + 5);
          f[8] = x.p(pf, c + 5);
        }
      }
    }
    // -D_d(rho u_d) and -D_d(rho u_d u_d)
    {
      f2 ms[9], fd[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const f2 ud = x.p(PM_U + 2 * DIR, i - 4);
        ms[i] = mul(x.p(PM_RHO, i - 4), ud);
        fd[i] = mul(ms[i], ud);
      }
#pragma unroll 1
      for (int c = 0; c < n; ++c) {
        const long long i = ib + (long long)c * L.si;
        put(dUf, NI, 0, i, -Dp(P, ms), st);
        sO[c][tid] = Dp(P, fd);
        if (c + 1 < n) {
          slide(ms); slide(fd);
          const f2 ud = x.p(PM_U + 2 * DIR, c + 5);
          ms[8] = mul(x.p(PM_RHO, c + 5), ud);
          fd[8] = mul(ms[8], ud);
        }
      }
    }
    // -D_d(p - c23 (u_e,e + u_f,f)) and the convective part above
    {
      f2 p[9];
      float td[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        p[i] = x.p(PM_P, i - 4);
        td[i] = x.s(PM_C23, i - 4) * (x.g(3 * E_ + E_, i - 4) + x.g(3 * F_ + F_, i - 4));
      }
#pragma unroll 1
      for (int c = 0; c < n; ++c) {
        put(dUf, NI, 1 + DIR, ib + (long long)c * L.si, Ds(P, td) - sO[c][tid] - Dp(P, p), false);
        if (c + 1 < n) {
          slide(p); slide(td);
          p[8] = x.p(PM_P, c + 5);
          td[8] = x.s(PM_C23, c + 5) * (x.g(3 * E_ + E_, c + 5) + x.g(3 * F_ + F_, c + 5));
        }
      }
    }
    // -D_d of the transverse momentum fluxes
    {
      f2 fe[9], ff[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) flux_ef<DIR>(x, i - 4, fe[i], ff[i]);
#pragma unroll 1
      for (int c = 0; c < n; ++c) {
        const long long i = ib + (long long)c * L.si;
        put(dUf, NI, 1 + E_, i, -Dp(P, fe), false);
        put(dUf, NI, 1 + F_, i, -Dp(P, ff), false);
        if (c + 1 < n) {
          slide(fe); slide(ff);
          flux_ef<DIR>(x, c + 5, fe[8], ff[8]);
        }
      }
    }
    // -D_d of the energy flux
    {
      f2 fE[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) fE[i] = flux_E<DIR>(x, i - 4);
#pragma unroll 1
      for (int c = 0; c < n; ++c) {
        sE[c][tid] -= Dp(P, fE);
        if (c + 1 < n) {
          slide(fE);
          fE[8] = flux_E<DIR>(x, c + 5);
        }
      }
    }
    // species, first pass: (rhoD_k X_k,d)_d, its energy part (rhoD_k h'_k X_k,d)_d
    // and the species part of the correction velocity, -rhoD_k X_k,d; the
    // narrow term goes straight to the accumulator
#pragma unroll 1
    for (int k = 0; k < ns; ++k) {
      if (mode == 1 && k == ref) {
        if (st)
          for (int c = 0; c < n; ++c) put(dUf, NI, 5 + k, ib + (long long)c * L.si, 0.0f, true);
        continue;
      }
      f2 X[9];
      float rd[9], rdh[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        X[i] = x.p(pmX(ns, k), i - 4);
        rd[i] = x.s(pmRD(ns, k), i - 4);
        rdh[i] = x.s(pmRDH(ns, k), i - 4);
      }
      float w[8];
      mv(P, X, 0, w);
      float He = ds(rdh, 0, w);
#pragma unroll 1
      for (int c = 0; c < n; ++c) {
        if (mode == 0) sV[c][tid] -= rd[4] * Dp(P, X);
        const float N = flux_diff(P, rd, X, w);
        mv(P, X, 1, w);
        const float He2 = ds(rdh, 1, w);
        put(dUf, NI, 5 + k, ib + (long long)c * L.si, N, st);
        sN[c][tid] += N;
        sE[c][tid] += He2 - He;
        He = He2;
        if (c + 1 < n) {
          slide(X); slide(rd); slide(rdh);
          X[8] = x.p(pmX(ns, k), c + 5);
          rd[8] = x.s(pmRD(ns, k), c + 5);
          rdh[8] = x.s(pmRDH(ns, k), c + 5);
        }
      }
    }
    // species, second pass (V_c complete): (B_k p_d)_d, -D_d(rho Y_k u_d) and
    // Y_k,d V_c,d
#pragma unroll 1
    for (int k = 0; k < ns; ++k) {
      const bool narrow = !(mode == 1 && k == ref);
      f2 p[9], Fk[9], Yk[9];
      float B[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        if (!WP) p[i] = x.p(PM_P, i - 4);
        B[i] = x.s(pmB(ns, k), i - 4);
        Fk[i] = mul(x.p(pmRY(ns, k), i - 4), x.p(PM_U + 2 * DIR, i - 4));
        if (mode == 0) Yk[i] = x.p(pmY(ns, k), i - 4);
      }
      float w[8];
      if (!WP) mv(P, p, 0, w);
#pragma unroll 1
      for (int c = 0; c < n; ++c) {
        float o = -Dp(P, Fk);
        if (mode == 0) o = fmaf(Dp(P, Yk), sV[c][tid], o);
        if (narrow) {
          float N;
          if (WP) {
            float w0[8], dw[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) {
              w0[m] = sW[c * 16 + m][tid];
              dw[m] = sW[c * 16 + 8 + m][tid];
            }
            N = flux_diff_w(B, dw, w0);
          } else {
            N = flux_diff(P, B, p, w);
            mv(P, p, 1, w);
          }
          o += N;
          sN[c][tid] += N;
        }
        put(dUf, NI, 5 + k, ib + (long long)c * L.si, o, false);
        if (c + 1 < n) {
          slide(B); slide(Fk);
          if (!WP) {
            slide(p);
            p[8] = x.p(PM_P, c + 5);
          }
          B[8] = x.s(pmB(ns, k), c + 5);
          Fk[8] = mul(x.p(pmRY(ns, k), c + 5), x.p(PM_U + 2 * DIR, c + 5));
          if (mode == 0) {
            slide(Yk);
            Yk[8] = x.p(pmY(ns, k), c + 5);
          }
        }
      }
    }
    if (mode == 1) {
      for (int c = 0; c < n; ++c)
        put(dUf, NI, 5 + ref, ib + (long long)c * L.si, -sN[c][tid], false);
    } else {
      // h,d V_c,d
      f2 hm[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) hm[i] = x.p(PM_HMIX, i - 4);
#pragma unroll 1
      for (int c = 0; c < n; ++c) {
        sE[c][tid] = fmaf(Dp(P, hm), sV[c][tid], sE[c][tid]);
        if (c + 1 < n) {
          slide(hm);
          hm[8] = x.p(PM_HMIX, c + 5);
        }
      }
      for (int c = 0; c < n; ++c) {
        const long long i = ib + (long long)c * L.si;
        if (st) divf[i] = sN[c][tid]; else divf[i] += sN[c][tid];
      }
    }
    for (int c = 0; c < n; ++c) put(dUf, NI, 4, ib + (long long)c * L.si, sE[c][tid], st);
  }
  }
}

template <int CH, int MINB, bool WP>
static void launch_m2_variant(const DevState &s, int dir, const MarchParamsM &P, float *dUf,
                              int first, int blocks, cudaStream_t st) {
  const size_t smem = (4 * CH + (WP ? 16 * CH : 0)) * M2_NT * sizeof(float);
  // the attribute is per device: set it once per device and instantiation,
  // on the first (eager) launch, before any stream capture
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    cudaFuncSetAttribute(k_march_m2<0, CH, MINB, WP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    cudaFuncSetAttribute(k_march_m2<1, CH, MINB, WP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    cudaFuncSetAttribute(k_march_m2<2, CH, MINB, WP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr_set[dev] = true;
  }
  if (s.opt.persistent) {
    static int cache[64] = {};
    const int r = resident_blocks(k_march_m2<1, CH, MINB, WP>, M2_NT, smem, cache);
    if (blocks > r) blocks = r;
  }
  if (dir == 0) k_march_m2<0, CH, MINB, WP><<<blocks, M2_NT, smem, st>>>(s, P, dUf, first);
  else if (dir == 1) k_march_m2<1, CH, MINB, WP><<<blocks, M2_NT, smem, st>>>(s, P, dUf, first);
  else k_march_m2<2, CH, MINB, WP><<<blocks, M2_NT, smem, st>>>(s, P, dUf, first);
}

void launch_march_m2(const DevState &s, int dir, float *dUf, int first, int variant,
                     cudaStream_t st) {
  MarchParamsM P;
  for (int a = 0; a < 8; ++a)
    for (int b = 0; b < 8; ++b) P.M[a][b] = (float)s.hcoef->M[dir][a][b];
  for (int k = 0; k < 4; ++k) P.D[k] = (float)s.hcoef->D[dir][k];
  for (int t = 0; t < 8; ++t)
    for (int j = 0; j < 4; ++j) P.MT2[t][j] = make_float2(P.M[2 * j][t], P.M[2 * j + 1][t]);
  const long long n = s.nlines[dir];
  if (n == 0) return;
  const int blocks = (int)((n + M2_NT - 1) / M2_NT);
  if (variant == 2) launch_m2_variant<32, 3, false>(s, dir, P, dUf, first, blocks, st);
  else if (variant == 3) launch_m2_variant<8, 2, true>(s, dir, P, dUf, first, blocks, st);
  else launch_m2_variant<16, 3, false>(s, dir, P, dUf, first, blocks, st);
}

}  // namespace smc
