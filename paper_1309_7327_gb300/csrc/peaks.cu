// Throughput of the SM's fused multiply-add pipes, measured on the device the
// library runs on.  These are the denominators of the arithmetic rooflines:
// the FP64 path (the temperature solve, the production rates, the FP64
// stencil kernels) is bound by the FP64 pipe, the mixed path's stencil
// arithmetic by the FP32 pipe.  Sec. 2.3 of the paper counts flops per
// stencil application; this measures the rate those flops can run at.
//
// Every thread carries eight independent chains x <- x * a + b for `iters`
// iterations (a, b kernel arguments, so nothing folds at compile time) and
// stores the sum of its chains, so no chain is dead code.  The grid is
// sm_count x 4 blocks of 256 threads: 8 warps per SM sub-partition, each with
// 8 independent instructions in flight, enough to cover the FMA latency of
// every pipe.
#include <cuda_runtime.h>

#include "smc.h"

namespace smc {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

__global__ void __launch_bounds__(kThreads) k_dfma(double *out, long long iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = (threadIdx.x + j) * 1e-3;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  out[blockIdx.x * (long long)blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_ffma(float *out, long long iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = (threadIdx.x + j) * 1e-3f;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  out[blockIdx.x * (long long)blockDim.x + threadIdx.x] = s;
}

// FP64 FMAs with one active lane per warp (the other lanes skip the loop):
// what scalar FP64 work costs inside warp-cooperative code
__global__ void __launch_bounds__(kThreads) k_dfma_lane0(double *out, long long iters, double a,
                                                         double b) {
  double s = 0.0;
  if ((threadIdx.x & 31) == 0) {
    double x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = (threadIdx.x + j) * 1e-3;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], a, b);
    }
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
  }
  out[blockIdx.x * (long long)blockDim.x + threadIdx.x] = s;
}

// two FP32 FMAs per lane and instruction (the paired form the mixed line
// kernels use for their stencil products)
__global__ void __launch_bounds__(kThreads) k_ffma2(float *out, long long iters, float a, float b) {
  float2 x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = make_float2((threadIdx.x + j) * 1e-3f, (threadIdx.x - j) * 1e-3f);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = __ffma2_rn(x[j], a2, b2);
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j].x + x[j].y;
  out[blockIdx.x * (long long)blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace smc

extern "C" smc_status smc_fma_throughput(int kind, long long iters, double *flops_per_s,
                                         double *ms, int *sm_count) {
  using namespace smc;
  if (kind < 0 || kind > 3 || iters < 1 || iters > (1LL << 40) || !flops_per_s) return SMC_ERR_ARG;
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    return SMC_ERR_CUDA;
  const int sms = prop.multiProcessorCount;
  const int blocks = sms * kBlocksPerSm;
  const long long threads = (long long)blocks * kThreads;
  void *out = nullptr;
  if (cudaMalloc(&out, (size_t)threads * sizeof(double)) != cudaSuccess) return SMC_ERR_OOM;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  smc_status rc = SMC_OK;
  float t = 0.0f;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = SMC_ERR_CUDA;
  } else {
    // one untimed launch (clocks up, code loaded), then the timed one
    for (int rep = 0; rep < 2 && rc == SMC_OK; ++rep) {
      const long long it = rep == 0 ? (iters + 7) / 8 : iters;
      if (rep == 1) cudaEventRecord(e0, st);
      if (kind == 0) k_dfma<<<blocks, kThreads, 0, st>>>((double *)out, it, 0.999999, 1e-7);
      else if (kind == 1) k_ffma<<<blocks, kThreads, 0, st>>>((float *)out, it, 0.999999f, 1e-7f);
      else if (kind == 2) k_ffma2<<<blocks, kThreads, 0, st>>>((float *)out, it, 0.999999f, 1e-7f);
      else k_dfma_lane0<<<blocks, kThreads, 0, st>>>((double *)out, it, 0.999999, 1e-7);
      if (rep == 1) cudaEventRecord(e1, st);
      if (cudaGetLastError() != cudaSuccess) rc = SMC_ERR_CUDA;
    }
    if (rc == SMC_OK && (cudaStreamSynchronize(st) != cudaSuccess ||
                         cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
      rc = SMC_ERR_CUDA;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(out);
  if (rc != SMC_OK) return rc;
  const double fma_per_thread = (double)iters * kChains * (kind == 2 ? 2.0 : 1.0);
  const double active = kind == 3 ? (double)threads / 32.0 : (double)threads;
  *flops_per_s = 2.0 * fma_per_thread * active / (t * 1e-3);
  if (ms) *ms = t;
  if (sm_count) *sm_count = sms;
  return SMC_OK;
}
