// smc_rhs_noalloc: the FP64 right-hand side of one periodic box without any
// device allocation (see include/smc.h).
//
// Some callers cannot call cudaMalloc: applications whose framework owns
// every byte of device memory in a fixed arena (a cudaMalloc outside it
// fails or breaks the arena's accounting), and loops that must not pay the
// implicit device synchronisation of cudaMalloc/cudaFree.  This entry point
// runs the same kernels as smc_rhs, but every scratch array, table and
// constant lives in one file-scope static device array of fixed size
// (kScratchBytes), reserved on every device that loads the library until the
// process exits.
//
// The call copies its tables from host memory and waits for its stream
// before it returns (it reads the evaluation's device status back), so it
// must not be issued while that stream is being captured into a CUDA graph.
//
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (with that device current).  Calls share the array and
// it keeps the last call's contents: calls that overlap on the GPU
// (different streams, or different host threads) race and must be
// serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "smc_internal.h"

namespace {

using namespace smc;

constexpr size_t kScratchBytes = 20u << 20;   // 20 MiB
constexpr int kMaxDevices = 64;
constexpr int kMaxReactions = 256;
// no box side above this can fit the scratch (its ghost-cell map alone is
// 4 (n + 8) 9 9 bytes); checked before any size product is formed
constexpr int kMaxSide = 1 << 16;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

void *g_dev_ptr[kMaxDevices] = {};

// host staging: filled per call, copied with cudaMemcpyAsync (pageable
// source, so the copy has completed when the call returns)
static unsigned char g_host_stage[kScratchBytes];
static Coef g_coef;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

smc_status scratch_ptr(unsigned char **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SMC_ERR_CUDA;
  if (!g_dev_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SMC_ERR_CUDA;
    g_dev_ptr[dev] = p;
  }
  *out = static_cast<unsigned char *>(g_dev_ptr[dev]);
  return SMC_OK;
}

}  // namespace

extern "C" smc_status smc_rhs_noalloc(const int n[3], const double dx[3],
                                      const smc_mechanism *mech, const double *U, double *dUdt,
                                      void *stream) {
  if (!n || !dx || !mech || !U || !dUdt) return SMC_ERR_ARG;
  for (int d = 0; d < 3; ++d)
    if (n[d] < 1 || n[d] > kMaxSide || !(dx[d] > 0)) return SMC_ERR_ARG;
  // U and dUdt must be device memory of the current device (no staging: a
  // host array would need a device buffer)
  {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return SMC_ERR_CUDA;
    const void *ptrs[2] = {U, dUdt};
    for (const void *p : ptrs) {
      cudaPointerAttributes a;
      if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return SMC_ERR_ARG;
      }
      if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return SMC_ERR_ARG;
      if (a.type == cudaMemoryTypeDevice && a.device != cur) return SMC_ERR_ARG;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int ns = mech->nspecies;
  if (ns < 1 || ns > SMC_MAX_NS) return SMC_ERR_ARG;
  const long long NI = (long long)n[0] * n[1] * n[2];
  const int gx = n[0] + 2 * SMC_GHOST, gy = n[1] + 2 * SMC_GHOST, gz = n[2] + 2 * SMC_GHOST;
  const long long NG = (long long)gx * gy * gz;

  // layout of the static array (host staging mirrors it byte for byte)
  size_t off = 0;
  const size_t o_mech = off; off = align256(off + sizeof(Mech));
  const size_t o_rx = off; off = align256(off + sizeof(Reaction) * kMaxReactions);
  const size_t o_box = off; off = align256(off + sizeof(Box));
  const size_t o_status = off; off = align256(off + sizeof(unsigned));
  size_t ol[3];
  const long long nlines[3] = {(long long)n[1] * n[2], (long long)n[0] * n[2], (long long)n[0] * n[1]};
  for (int d = 0; d < 3; ++d) { ol[d] = off; off = align256(off + sizeof(LineItem) * nlines[d]); }
  const size_t o_gmap = off; off = align256(off + sizeof(int) * NG);
  const size_t o_imap = off; off = align256(off + sizeof(long long) * NI);
  const size_t table_end = off;
  const size_t o_Q = off; off = align256(off + sizeof(double) * (size_t)nQ(ns) * NG);
  const size_t o_G = off; off = align256(off + sizeof(double) * 9 * (size_t)NG);
  const size_t o_div = off; off = align256(off + sizeof(double) * (size_t)NI);
  if (off > kScratchBytes) return SMC_ERR_ARG;   // box too large for the fixed scratch

  unsigned char *base = nullptr;
  smc_status s0 = scratch_ptr(&base);
  if (s0 != SMC_OK) return s0;

  // host side of the tables
  unsigned char *hs = g_host_stage;
  Mech &M = *reinterpret_cast<Mech *>(hs + o_mech);
  Reaction *rx = reinterpret_cast<Reaction *>(hs + o_rx);
  {
    std::vector<Reaction> hrx;   // host memory only
    if (pack_mechanism(mech, kMaxReactions, M, hrx)) return SMC_ERR_ARG;
    if (!hrx.empty()) memcpy(rx, hrx.data(), hrx.size() * sizeof(Reaction));
  }
  Box &B = *reinterpret_cast<Box *>(hs + o_box);
  B.nx = n[0]; B.ny = n[1]; B.nz = n[2];
  B.gx = gx; B.gy = gy; B.gz = gz;
  B.off_g = 0; B.off_i = 0;
  B.lo[0] = B.lo[1] = B.lo[2] = 0;
  B.pad = 0;
  *reinterpret_cast<unsigned *>(hs + o_status) = 0u;   // the status word starts at zero
  int *gmap = reinterpret_cast<int *>(hs + o_gmap);
  long long *imap = reinterpret_cast<long long *>(hs + o_imap);
  for (int k = -SMC_GHOST; k < n[2] + SMC_GHOST; ++k)
    for (int j = -SMC_GHOST; j < n[1] + SMC_GHOST; ++j)
      for (int i = -SMC_GHOST; i < n[0] + SMC_GHOST; ++i) {
        const int x = ((i % n[0]) + n[0]) % n[0];
        const int y = ((j % n[1]) + n[1]) % n[1];
        const int z = ((k % n[2]) + n[2]) % n[2];
        const long long g = ((long long)(k + SMC_GHOST) * gy + (j + SMC_GHOST)) * gx + (i + SMC_GHOST);
        gmap[g] = (int)(((long long)z * n[1] + y) * n[0] + x);
        if (i >= 0 && i < n[0] && j >= 0 && j < n[1] && k >= 0 && k < n[2])
          imap[((long long)k * n[1] + j) * n[0] + i] = g;
      }
  const long long gs[3] = {1, gx, (long long)gx * gy};
  const long long is[3] = {1, n[0], (long long)n[0] * n[1]};
  for (int d = 0; d < 3; ++d) {
    LineItem *L = reinterpret_cast<LineItem *>(hs + ol[d]);
    const int e0 = (d == 0) ? 1 : 0, e1 = (d == 2) ? 1 : 2;
    long long t = 0;
    for (int t1 = 0; t1 < n[e1]; ++t1)
      for (int t0 = 0; t0 < n[e0]; ++t0) {
        int crd[3];
        crd[d] = 0;
        crd[e0] = t0;
        crd[e1] = t1;
        long long go = 0, io = 0;
        for (int c = 0; c < 3; ++c) {
          go += (long long)(crd[c] + SMC_GHOST) * gs[c];
          io += (long long)crd[c] * is[c];
        }
        L[t].g0 = go;
        L[t].i0 = io;
        L[t].sg = (int)gs[d];
        L[t].si = (int)is[d];
        L[t].len = n[d];
        L[t].pad = 0;
        ++t;
      }
  }
  if (cudaMemcpyAsync(base, hs, table_end, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return SMC_ERR_CUDA;

  // stencil coefficients (default free parameters, Sec. 2.2)
  {
    double M[8][8];
    narrow8_matrix(3557.0 / 44100.0, -2083.0 / 117600.0, M);
    const double D8[4] = {4.0 / 5, -1.0 / 5, 4.0 / 105, -1.0 / 280};
    for (int d = 0; d < 3; ++d) {
      const double ih2 = 1.0 / (dx[d] * dx[d]);
      for (int r = 0; r < 8; ++r)
        for (int c = 0; c < 8; ++c) g_coef.M[d][r][c] = M[r][c] * ih2;
      for (int k = 0; k < 4; ++k) g_coef.D[d][k] = D8[k] / dx[d];
    }
  }

  DevState s;
  memset(&s, 0, sizeof(s));
  s.ns = ns;
  s.nv = 5 + ns;
  s.nq = nQ(ns);
  s.nboxes = 1;
  s.ncells = NI;
  s.nghost = NG;
  s.mech = reinterpret_cast<const Mech *>(base + o_mech);
  s.rx = reinterpret_cast<const Reaction *>(base + o_rx);
  s.hcoef = &g_coef;
  s.boxes = reinterpret_cast<const Box *>(base + o_box);
  s.gmap = reinterpret_cast<const int *>(base + o_gmap);
  s.imap = reinterpret_cast<const long long *>(base + o_imap);
  for (int d = 0; d < 3; ++d) {
    s.lines[d] = reinterpret_cast<const LineItem *>(base + ol[d]);
    s.nlines[d] = nlines[d];
  }
  s.Q = reinterpret_cast<double *>(base + o_Q);
  s.G = reinterpret_cast<double *>(base + o_G);
  s.divacc = reinterpret_cast<double *>(base + o_div);
  s.status = reinterpret_cast<unsigned *>(base + o_status);
  s.opt.mode = 0;
  s.opt.ref = ns - 1;
  s.opt.reactions = 1;
  s.opt.maxit = 50;
  s.opt.tol = 1e-13;
  s.opt.T0 = 1000.0;
  s.opt.xi_ratio = 0.0;

  launch_prim(s, U, st);
  launch_grad(s, st);
  for (int d = 0; d < 3; ++d) launch_march(s, d, dUdt, d == 0, st);
  launch_final(s, dUdt, 1, mech->nreactions > 0, st);
  if (cudaGetLastError() != cudaSuccess) return SMC_ERR_CUDA;
  unsigned flags = 0;
  if (cudaMemcpyAsync(&flags, base + o_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SMC_ERR_CUDA;
  if (flags & ST_NONCONV) return SMC_ERR_NONCONVERGED;
  if (flags & (ST_NONPHYS | ST_NONFINITE)) return SMC_ERR_NONPHYSICAL;
  return SMC_OK;
}
