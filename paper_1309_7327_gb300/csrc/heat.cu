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

// H at the faces left (window offset 0) and right (offset 1) of the middle
// cell of a 9-cell window, difference-first: H = sum_m a_m sum_{n != 3}
// M_mn (u_n - u_3), exact since every row of M sums to zero.
__device__ __forceinline__ double face_diff(const HeatParams &P, const double *a, const double *u) {
  double H[2];
#pragma unroll
  for (int o = 0; o < 2; ++o) {
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      double w = 0.0;
#pragma unroll
      for (int n = 0; n < 8; ++n)
        if (n != 3 && m - n <= 4 && n - m <= 4) w = fma(P.M[m][n], u[o + n] - u[o + 3], w);
      acc = fma(a[o + m], w, acc);
    }
    H[o] = acc;
  }
  return H[1] - H[0];
}

// F = (a u_x)_x + (b u_y)_y + gs G, one thread per cell, periodic windows
__global__ void __launch_bounds__(256) k_heat_rhs(int N, const HeatParams P,
                                                  const double *__restrict__ a,
                                                  const double *__restrict__ b,
                                                  const double *__restrict__ G, double gs,
                                                  const double *__restrict__ u,
                                                  double *__restrict__ F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= N || j >= N) return;
  double wa[9], wu[9];
  const size_t row = (size_t)j * N;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    int ii = i + k - 4;
    ii += ii < 0 ? N : 0;
    ii -= ii >= N ? N : 0;
    wa[k] = __ldg(a + row + ii);
    wu[k] = __ldg(u + row + ii);
  }
  double f = face_diff(P, wa, wu);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    int jj = j + k - 4;
    jj += jj < 0 ? N : 0;
    jj -= jj >= N ? N : 0;
    wa[k] = __ldg(b + (size_t)jj * N + i);
    wu[k] = __ldg(u + (size_t)jj * N + i);
  }
  f += face_diff(P, wa, wu);
  if (G) f = fma(gs, __ldg(G + row + i), f);
  F[row + i] = f;
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
  const dim3 blk(32, 8), grd((N + 31) / 32, (N + 7) / 8);
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
