// Time-integration kernels: the SDC node update (Sec. 3.1, eq. expsdc) as a
// linear combination of state and right-hand-side arrays, and the mode-1
// multirate fine-node chain (Sec. 3.2, eq. mrupdate) in which every cell
// advances through the reaction substeps of one coarse interval on its own.
#include <algorithm>

#include "chem.cuh"
#include "smc_internal.h"

namespace smc {

static int grid_for(long long n, int block) {
  long long b = (n + block - 1) / block;
  const long long cap = 152LL * 64;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// out = in + sum_j c_j src_j  (elementwise; in may alias out)
__global__ void __launch_bounds__(256) k_combo(const double *in, double *out, const Combo cb,
                                               long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double acc = in ? in[i] : 0.0;
    for (int j = 0; j < cb.nsrc; ++j) acc += cb.c[j] * cb.src[j][i];
    out[i] = acc;
  }
}

void launch_combo(const double *in, double *out, const Combo &cb, long long n, cudaStream_t st) {
  k_combo<<<grid_for(n, 256), 256, 0, st>>>(in, out, cb, n);
}

// Reaction right-hand side f2 at one cell from its conserved state.  Tg is
// the Newton first guess on entry and the temperature on return.  MIX: the
// mixed-precision rates (FP32 after the FP64 reductions).
template <bool MIX>
__device__ __forceinline__ bool cell_reactions(const DevState &s, const double *Uc, double *f2,
                                               unsigned &flag, double &Tg) {
  const Mech &m = *s.mech;
  const int ns = s.ns;
  const double rho = Uc[0];
  const double invrho = 1.0 / rho;
  const double u = Uc[1] * invrho, v = Uc[2] * invrho, w = Uc[3] * invrho;
  const double e = Uc[4] * invrho - 0.5 * (u * u + v * v + w * w);
  double T;
  // mass fractions Uc[5 + k] / rho formed inside the solve (no Y array)
  const bool ok = newton_T(m, Uc + 5, e, Tg, s.opt.tol, s.opt.maxit, T, nullptr, nullptr, invrho);
  if (ok) Tg = T;
  if (!ok) flag |= ST_NONCONV;
  if (!(rho > 0.0) || !(T > 0.0)) flag |= ST_NONPHYS;
  if (!isfinite(rho) || !isfinite(T)) flag |= ST_NONFINITE;
  if (s.opt.reactions && m.nr > 0) {
    if (MIX) production_rates_m(m, s.rx, T, Uc + 5, f2);
    else production_rates(m, s.rx, rho, T, nullptr, f2, Uc + 5);
  } else {
    for (int k = 0; k < ns; ++k) f2[k] = 0.0;
  }
  return ok;
}

template <bool MIX>
__global__ void __launch_bounds__(128) k_chem_only(const DevState s, const double *__restrict__ U,
                                                   double *__restrict__ F2) {
  const int ns = s.ns, nv = s.nv;
  const long long NI = s.ncells;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < NI;
       i += (long long)gridDim.x * blockDim.x) {
    double Uc[5 + SMC_MAX_NS], f2[SMC_MAX_NS];
    for (int c = 0; c < nv; ++c) Uc[c] = U[(size_t)c * NI + i];
    unsigned flag = 0;
    double Tg = s.opt.T0;
    cell_reactions<MIX>(s, Uc, f2, flag, Tg);
    if (flag) atomicOr(s.status, flag);
    for (int k = 0; k < ns; ++k) F2[(size_t)k * NI + i] = f2[k];
  }
}

void launch_chem_only(const DevState &s, const double *U, double *F2, cudaStream_t st) {
  if (s.opt.rates32) k_chem_only<true><<<grid_for(s.ncells, 128), 128, 0, st>>>(s, U, F2);
  else k_chem_only<false><<<grid_for(s.ncells, 128), 128, 0, st>>>(s, U, F2);
}

// Fine substeps q = q0 .. q0+nsub-1 of eq. mrupdate for every cell:
//   U_{q+1} = U_q + dt_q [f1(U^{k+1}_p) - f1(U^k_p)] + dt_q [f2(U^{k+1}_q) - f2(U^k_q)]
//             + dt (S22 F2^k)_q + dt (S21 F1^k)_q
// f1 is frozen at the coarse node p on the left; f2 (reactions, species
// components only) is evaluated at every fine node.  f1(U^k_p) and f2(U^k_q)
// are nodes of the two quadratures, so their -dt_q terms are folded into the
// weights s21[.][p] and s22[.][q - q0] on the host.
template <bool MIX>
__global__ void __launch_bounds__(128) k_fine_chain(const DevState s, const double *__restrict__ Uin,
                                                    double *__restrict__ Uout, const FineChain fc) {
  const int ns = s.ns, nv = s.nv, M1 = fc.M1;
  const long long NI = s.ncells;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < NI;
       i += (long long)gridDim.x * blockDim.x) {
    double Uc[5 + SMC_MAX_NS], f2[SMC_MAX_NS];
    for (int c = 0; c < nv; ++c) Uc[c] = Uin[(size_t)c * NI + i];
    unsigned flag = 0;
    // each substep's Newton solve starts from the previous substep's
    // temperature (a deterministic sequence within the chain)
    double Tg = s.opt.T0;
    for (int sidx = 0; sidx < fc.nsub; ++sidx) {
      if (sidx > 0 || fc.eval_first) {
        cell_reactions<MIX>(s, Uc, f2, flag, Tg);
        for (int k = 0; k < ns; ++k) fc.F2new[sidx][(size_t)k * NI + i] = f2[k];
      } else {
        for (int k = 0; k < ns; ++k) f2[k] = fc.F2old[0][(size_t)k * NI + i];
      }
      const double dq = fc.dtq[sidx];
      for (int c = 0; c < nv; ++c) {
        const size_t o = (size_t)c * NI + i;
        double acc = dq * fc.F1new_p[o];
        for (int j = 0; j <= M1; ++j) acc = fma(fc.s21[sidx][j], fc.F1old[j][o], acc);
        if (c >= 5) {
          const int k = c - 5;
          const size_t ok = (size_t)k * NI + i;
          acc = fma(dq, f2[k], acc);
          for (int t = 0; t <= fc.nsub; ++t) acc = fma(fc.s22[sidx][t], fc.F2old[t][ok], acc);
        }
        Uc[c] += acc;
      }
    }
    if (fc.eval_last) {
      cell_reactions<MIX>(s, Uc, f2, flag, Tg);
      for (int k = 0; k < ns; ++k) fc.F2new[fc.nsub][(size_t)k * NI + i] = f2[k];
    }
    if (flag) atomicOr(s.status, flag);
    for (int c = 0; c < nv; ++c) Uout[(size_t)c * NI + i] = Uc[c];
  }
}

// [z][y][x] -> [x][z][y] within each ghosted box, 32 x 32 (x, y) tiles through
// shared memory so that both the reads and the writes are coalesced.  The
// (plane, box, z, tile) work items are enumerated in one flat grid-stride loop.
template <typename T>
__global__ void __launch_bounds__(256) k_transpose_x(const Box *__restrict__ boxes, int nboxes,
                                                     const long long *__restrict__ tiles,
                                                     long long NG, const T *__restrict__ src,
                                                     T *__restrict__ dst, int planes) {
  __shared__ T tile[32][33];
  const long long per_plane = tiles[nboxes];
  const long long total = per_plane * planes;
  for (long long w = blockIdx.x; w < total; w += gridDim.x) {
    const int plane = (int)(w / per_plane);
    const long long r = w - (long long)plane * per_plane;
    int lo = 0, hi = nboxes - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tiles[mid] <= r) lo = mid; else hi = mid - 1;
    }
    const Box B = boxes[lo];
    const long long t = r - tiles[lo];
    const int tilesx = (B.gx + 31) / 32, tilesy = (B.gy + 31) / 32;
    const int z = (int)(t / ((long long)tilesx * tilesy));
    const int rr = (int)(t % ((long long)tilesx * tilesy));
    const int x0 = (rr % tilesx) * 32, y0 = (rr / tilesx) * 32;
    const size_t pbase = (size_t)plane * NG + B.off_g;
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
      const int x = x0 + threadIdx.x, y = y0 + j;
      if (x < B.gx && y < B.gy)
        tile[j][threadIdx.x] = src[pbase + ((size_t)z * B.gy + y) * B.gx + x];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
      const int y = y0 + threadIdx.x, x = x0 + j;
      if (x < B.gx && y < B.gy)
        dst[pbase + ((size_t)x * B.gz + z) * B.gy + y] = tile[threadIdx.x][j];
    }
  }
}

void launch_transpose_x(const DevState &s, const void *src, void *dst, int planes, int esize,
                        cudaStream_t st) {
  dim3 block(32, 8);
  const int grid = 152 * 8;
  if (esize == 8)
    k_transpose_x<double><<<grid, block, 0, st>>>(s.boxes, s.nboxes, s.xt_tiles, s.nghost,
                                                  (const double *)src, (double *)dst, planes);
  else
    k_transpose_x<float><<<grid, block, 0, st>>>(s.boxes, s.nboxes, s.xt_tiles, s.nghost,
                                                 (const float *)src, (float *)dst, planes);
}

// Collocation residual of eq. residual, R = U_0 - U_M + sum_j c1_j F1_j (all
// components) + sum_t c2_t F2_t (species components, F2 arrays hold ns
// components), reduced per component to max|R| (out[c]) and max|U_0|
// (out[nv + c]).  Non-negative doubles order like their bit patterns, so the
// maxima reduce with integer atomicMax; out must be zeroed before the launch.
__global__ void __launch_bounds__(256) k_residual(const double *__restrict__ U0,
                                                  const double *__restrict__ UM,
                                                  const ResidualTable *__restrict__ tab, int nv,
                                                  long long NI,
                                                  unsigned long long *__restrict__ out) {
  const long long n = (long long)nv * NI;
  const int n1 = tab->n1, n2 = tab->n2;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n;
       base += (long long)gridDim.x * blockDim.x) {
    const long long i = base + threadIdx.x;
    double r = 0.0, u = 0.0;
    int c = -1;
    if (i < n) {
      c = (int)(i / NI);
      r = U0[i] - UM[i];
      for (int j = 0; j < n1; ++j) r = fma(tab->c1[j], tab->src1[j][i], r);
      if (c >= 5)
        for (int t = 0; t < n2; ++t) r = fma(tab->c2[t], tab->src2[t][i - 5 * NI], r);
      r = fabs(r);
      u = fabs(U0[i]);
    }
    // one atomic per component present in the warp (a warp spans at most
    // two components when NI >= 32)
    const unsigned mask = 0xffffffffu;
    const int c0 = __shfl_sync(mask, c, 0);
    for (int cc = c0; cc >= 0; ) {
      double rr = (c == cc) ? r : 0.0, uu = (c == cc) ? u : 0.0;
      for (int off = 16; off; off >>= 1) {
        rr = fmax(rr, __shfl_xor_sync(mask, rr, off));
        uu = fmax(uu, __shfl_xor_sync(mask, uu, off));
      }
      if ((threadIdx.x & 31) == 0) {
        atomicMax(out + cc, (unsigned long long)__double_as_longlong(rr));
        atomicMax(out + nv + cc, (unsigned long long)__double_as_longlong(uu));
      }
      // the next component present in this warp, if any
      const int nxt = (c > cc) ? c : 0x7fffffff;
      int m = nxt;
      for (int off = 16; off; off >>= 1) m = min(m, __shfl_xor_sync(mask, m, off));
      cc = (m == 0x7fffffff) ? -1 : m;
    }
  }
}

void launch_residual(const double *U0, const double *UM, const ResidualTable *tab, int nv,
                     long long NI, unsigned long long *out, cudaStream_t st) {
  const long long n = (long long)nv * NI;
  long long blocks = (n + 255) / 256;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  k_residual<<<(int)blocks, 256, 0, st>>>(U0, UM, tab, nv, NI, out);
}

template <bool ALU>
__global__ void __launch_bounds__(256) k_exp(const Mech *__restrict__ m, const double *__restrict__ x,
                                             double *__restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = ALU ? exp_alu(*m, x[i]) : fast_exp(*m, x[i]);
}

void launch_exp(const Mech *m, const double *x, double *y, long long n, int variant,
                cudaStream_t st) {
  if (variant == 1) k_exp<true><<<grid_for(n, 256), 256, 0, st>>>(m, x, y, n);
  else k_exp<false><<<grid_for(n, 256), 256, 0, st>>>(m, x, y, n);
}

__global__ void __launch_bounds__(256) k_dmul(const double *__restrict__ a, const double *__restrict__ b,
                                              double *__restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = dmul_alu(a[i], b[i]);
}

void launch_dmul(const double *a, const double *b, double *y, long long n, cudaStream_t st) {
  k_dmul<<<grid_for(n, 256), 256, 0, st>>>(a, b, y, n);
}

// The chain's per-thread arrays (state, rates, Gibbs terms) live in local
// memory; capping the resident blocks per SM (by reserving shared memory the
// kernel does not use) trades FP64 latency hiding for L1 hits on them.
void launch_fine_chain(const DevState &s, const double *Uin, double *Uout, const FineChain &fc,
                       cudaStream_t st) {
  size_t smem = 0;
  if (s.opt.chain_blocks > 0) {
    smem = (size_t)(227 * 1024) / (size_t)s.opt.chain_blocks;
    smem = smem > 1024 ? smem - 1024 : 0;
    static bool attr_set[64] = {};  // per device, on the first (eager) launch
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
      cudaFuncSetAttribute(k_fine_chain<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      cudaFuncSetAttribute(k_fine_chain<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      attr_set[dev] = true;
    }
  }
  int blocks = grid_for(s.ncells, 128);
  if (s.opt.persistent) {
    // the chain is a grid-stride loop: a grid of the resident capacity
    // leaves no partly filled last wave
    static int cache[2][64] = {};
    const int r = s.opt.rates32 ? resident_blocks(k_fine_chain<true>, 128, smem, cache[1])
                                : resident_blocks(k_fine_chain<false>, 128, smem, cache[0]);
    const long long need = (s.ncells + 127) / 128;
    blocks = (int)(need < r ? need : r);
  }
  if (s.opt.rates32) k_fine_chain<true><<<blocks, 128, smem, st>>>(s, Uin, Uout, fc);
  else k_fine_chain<false><<<blocks, 128, smem, st>>>(s, Uin, Uout, fc);
}

}  // namespace smc
