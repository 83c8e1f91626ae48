// The appendix heat-equation problems (App. A, T1 and T2) on the GPU:
//   u_t = (a u_x)_x + (b u_y)_y + exp(-t) G
// on a periodic N x N grid, both second-derivative terms by the 8th-order
// narrow stencil of Sec. 2.2 (eqs. DaDu/H) and time by SDC (Sec. 3.1,
// eq. expsdc).  The second benchmark of the narrow stencil and the SDC
// update, independent of the reacting-flow right-hand side.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "smc_internal.h"

namespace smc {

struct HeatParams {
  double M[8][8];                 // narrow-stencil matrix scaled by 1/h^2
};

// H at the face between window cells 3 and 4 of an 8-cell window (cells
// c-4 .. c+3 for the face left of cell c), difference-first:
//   H = sum_m a_m sum_{n != 3} M_mn (u_n - u_3),
// exact since every row of M sums to zero; M is banded (|m - n| <= 4).
__device__ __forceinline__ double face_h(const HeatParams &P, const double *a, int as,
                                         const double *u, int us) {
  double du[8];
#pragma unroll
  for (int n = 0; n < 8; ++n) du[n] = u[n * us] - u[3 * us];
  double acc = 0.0;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    double w = 0.0;
#pragma unroll
    for (int n = 0; n < 8; ++n)
      if (n != 3 && m - n <= 4 && n - m <= 4) w = fma(P.M[m][n], du[n], w);
    acc = fma(a[m * as], w, acc);
  }
  return acc;
}

// F = (a u_x)_x + (b u_y)_y + gs G on a periodic N x N grid.  A block owns
// a 32 x 16 tile: u, a and b with their 4-cell halos are staged in shared
// memory, every face of the tile is computed once (33 x 16 x-faces,
// 32 x 17 y-faces) and each cell takes the difference of its two faces per
// direction, so the FP64 work per cell is about two faces instead of four.
constexpr int HTX = 32, HTY = 16;

__global__ void __launch_bounds__(256) k_heat_rhs(int N, const HeatParams P,
                                                  const double *__restrict__ a,
                                                  const double *__restrict__ b,
                                                  const double *__restrict__ G, double gs,
                                                  const double *__restrict__ u,
                                                  double *__restrict__ F) {
  __shared__ double su[HTY + 8][HTX + 8];
  __shared__ double sa[HTY][HTX + 8];
  __shared__ double sb[HTY + 8][HTX];
  __shared__ double hx[HTY][HTX + 1];
  __shared__ double hy[HTY + 1][HTX];
  const int x0 = blockIdx.x * HTX, y0 = blockIdx.y * HTY;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nt = blockDim.x * blockDim.y;
  auto wrap = [N](int i) {
    i %= N;
    return i < 0 ? i + N : i;
  };
  for (int idx = tid; idx < (HTY + 8) * (HTX + 8); idx += nt) {
    const int r = idx / (HTX + 8), c = idx % (HTX + 8);
    su[r][c] = __ldg(u + (size_t)wrap(y0 + r - 4) * N + wrap(x0 + c - 4));
  }
  for (int idx = tid; idx < HTY * (HTX + 8); idx += nt) {
    const int r = idx / (HTX + 8), c = idx % (HTX + 8);
    sa[r][c] = __ldg(a + (size_t)wrap(y0 + r) * N + wrap(x0 + c - 4));
  }
  for (int idx = tid; idx < (HTY + 8) * HTX; idx += nt) {
    const int r = idx / HTX, c = idx % HTX;
    sb[r][c] = __ldg(b + (size_t)wrap(y0 + r - 4) * N + wrap(x0 + c));
  }
  __syncthreads();
  for (int idx = tid; idx < HTY * (HTX + 1); idx += nt) {
    const int r = idx / (HTX + 1), f = idx % (HTX + 1);
    hx[r][f] = face_h(P, &sa[r][f], 1, &su[r + 4][f], 1);
  }
  for (int idx = tid; idx < (HTY + 1) * HTX; idx += nt) {
    const int f = idx / HTX, c = idx % HTX;
    hy[f][c] = face_h(P, &sb[f][c], HTX, &su[f][c + 4], HTX + 8);
  }
  __syncthreads();
  for (int idx = tid; idx < HTY * HTX; idx += nt) {
    const int r = idx / HTX, c = idx % HTX;
    const int gx = x0 + c, gy = y0 + r;
    if (gx >= N || gy >= N) continue;
    const size_t o = (size_t)gy * N + gx;
    double f = hx[r][c + 1] - hx[r][c];
    f += hy[r + 1][c] - hy[r][c];
    if (G) f = fma(gs, __ldg(G + o), f);
    F[o] = f;
  }
}

}  // namespace smc

using namespace smc;

namespace {

bool on_device(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" smc_status smc_heat2d(int N, double h, const double *a, const double *b,
                                 const double *G, double m47, double m48, double t0, double dt,
                                 int nsteps, int nodes, int sweeps, double *u,
                                 long long *n_evals, void *stream) {
  if (N < 8 || N > 16384 || !(h > 0) || !(dt > 0) || !std::isfinite(dt) || nsteps < 0 ||
      nodes < 2 || nodes > 9 || sweeps < 1 || sweeps > 64 || !a || !b || !u)
    return SMC_ERR_ARG;
  if (!on_device(a) || !on_device(b) || !on_device(u) || (G && !on_device(G))) return SMC_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  HeatParams P;
  narrow8_matrix(m47, m48, P.M);
  for (int r = 0; r < 8; ++r)
    for (int c = 0; c < 8; ++c) P.M[r][c] /= h * h;
  std::vector<double> tau, S;
  lobatto_nodes(nodes, tau);
  node_to_node_matrix(tau, S);
  const int M = nodes - 1;
  const size_t n = (size_t)N * N;
  // U_0 plus two sets of M node values of F and the shared F(U_0)
  const int nbuf = 2 + 2 * M;
  double *buf = nullptr;
  if (cudaMalloc(&buf, nbuf * n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return SMC_ERR_OOM;
  }
  double *U0 = buf;
  auto Fp = [&](int k) { return buf + (size_t)(1 + k) * n; };   // k = 0 .. 2M
  const dim3 blk(32, 8), grd((N + HTX - 1) / HTX, (N + HTY - 1) / HTY);
  long long evals = 0;
  smc_status status = SMC_OK;
  auto rhs = [&](const double *x, double *F, double t) {
    k_heat_rhs<<<grd, blk, 0, st>>>(N, P, a, b, G, std::exp(-t), x, F);
    ++evals;
  };
  double t = t0;
  // F(U_0) at slot 0; node values of sweep k in slots 1..M or M+1..2M
  rhs(u, Fp(0), t);
  std::vector<int> fold(M + 1, 0), fnew(M + 1, 0);
  for (int step = 0; step < nsteps && status == SMC_OK; ++step) {
    if (cudaMemcpyAsync(U0, u, n * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
      status = SMC_ERR_CUDA;
      break;
    }
    for (int m = 0; m <= M; ++m) fold[m] = 0;   // spread start: F(U_0) at every node
    int set = 0;
    for (int k = 0; k < sweeps; ++k) {
      fnew[0] = 0;
      for (int m = 1; m <= M; ++m) fnew[m] = set * M + m;
      for (int m = 0; m < M; ++m) {
        if (m > 0) rhs(u, Fp(fnew[m]), t + dt * tau[m]);
        // eq. expsdc: U_{m+1} = U_m + dt_m (F^{k+1}_m - F^k_m) + dt (S F^k)_m
        const double dtm = dt * (tau[m + 1] - tau[m]);
        Combo cb;
        cb.nsrc = 0;
        cb.c[cb.nsrc] = dtm;
        cb.src[cb.nsrc++] = Fp(fnew[m]);
        cb.c[cb.nsrc] = -dtm;
        cb.src[cb.nsrc++] = Fp(fold[m]);
        for (int j = 0; j <= M; ++j) {
          cb.c[cb.nsrc] = dt * S[m * (M + 1) + j];
          cb.src[cb.nsrc++] = Fp(fold[j]);
        }
        launch_combo(m == 0 ? U0 : u, u, cb, (long long)n, st);
      }
      rhs(u, Fp(fnew[M]), t + dt);
      fold = fnew;
      set ^= 1;
    }
    // F(U_M) becomes the next step's F(U_0)
    if (cudaMemcpyAsync(Fp(0), Fp(fold[M]), n * sizeof(double), cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess)
      status = SMC_ERR_CUDA;
    t += dt;
  }
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
    status = SMC_ERR_CUDA;
  cudaFree(buf);
  if (n_evals) *n_evals = evals;
  return status;
}
