// FMA throughput of this GPU, measured: the denominator of the rooflines of
// the FP64 and FP32 element kernels, which are bound by their arithmetic
// pipes rather than by HBM. Not part of the method; it only measures the
// machine the method runs on.
//
// Every thread runs kChains independent multiply-add chains x <- x a + b
// (a just below 1, b small, so that the values stay finite and normal) for
// a fixed number of rounds, and adds its chains into one output word so
// that nothing is dead code. The grid fills every SM with 1024 threads in
// blocks of 256. One untimed launch, then the best of kReps timed ones
// (CUDA events on the caller's stream). Work is fixed; nothing waits.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/tmop.h"

namespace tmop {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kReps = 3;

template <class R>
__global__ void __launch_bounds__(kThreads) k_fma_rate(R* out, int rounds, R a, R b) {
  R x[kChains];
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = R(1) + R(1e-3) * R((tid + c) & 1023);
#pragma unroll 1
  for (int r = 0; r < rounds; ++r) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  R s = R(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[tid] = s;
}

// FP32 pairs: each __ffma2_rn is two independent FP32 multiply-adds
__global__ void __launch_bounds__(kThreads) k_fma_rate_f32x2(float* out, int rounds, float a, float b) {
  float2 x[kChains];
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = make_float2(1.f + 1e-3f * ((tid + c) & 1023), 1.f - 1e-3f * ((tid + c) & 511));
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll 1
  for (int r = 0; r < rounds; ++r) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
  out[tid] = s;
}

}  // namespace
}  // namespace tmop

using namespace tmop;

extern "C" int tmop_fma_peak(int kind, void* scratch, size_t scratch_bytes, double* gflops, double* ms,
                             void* stream) {
  if (!gflops || !scratch || (kind != TMOP_PEAK_FP64 && kind != TMOP_PEAK_FP32 && kind != TMOP_PEAK_FP32X2))
    return TMOP_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return TMOP_ERR_CUDA;
  const int blocks = sms * (1024 / kThreads);
  const size_t elt = kind == TMOP_PEAK_FP64 ? sizeof(double) : sizeof(float);
  if (scratch_bytes < elt * (size_t)blocks * kThreads) return TMOP_ERR_CAPACITY;
  // rounds sized for a few milliseconds per launch at the expected rates
  // (FP64 ~1 TFLOP/s, FP32 ~80 TFLOP/s on this part)
  const int rounds = kind == TMOP_PEAK_FP64 ? 64 : 4096;
  const double fma_per_launch = (double)blocks * kThreads * rounds * 16 * kChains * (kind == TMOP_PEAK_FP32X2 ? 2 : 1);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return TMOP_ERR_CUDA;
  }
  auto launch = [&]() {
    if (kind == TMOP_PEAK_FP64)
      k_fma_rate<double><<<blocks, kThreads, 0, s>>>(static_cast<double*>(scratch), rounds, 0.999999999, 1e-9);
    else if (kind == TMOP_PEAK_FP32)
      k_fma_rate<float><<<blocks, kThreads, 0, s>>>(static_cast<float*>(scratch), rounds, 0.9999999f, 1e-7f);
    else
      k_fma_rate_f32x2<<<blocks, kThreads, 0, s>>>(static_cast<float*>(scratch), rounds, 0.9999999f, 1e-7f);
  };
  int rc = TMOP_OK;
  float best = 0.f;
  launch();
  for (int r = 0; r < kReps && rc == TMOP_OK; ++r) {
    float t = 0.f;
    if (cudaEventRecord(e0, s) != cudaSuccess) rc = TMOP_ERR_CUDA;
    launch();
    if (rc == TMOP_OK && (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
                          cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
      rc = TMOP_ERR_CUDA;
    if (rc == TMOP_OK && (best == 0.f || t < best)) best = t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != TMOP_OK) return rc;
  if (!(best > 0.f)) return TMOP_ERR_CUDA;
  *gflops = 2.0 * fma_per_launch / (best * 1e-3) / 1e9;
  if (ms) *ms = best;
  return TMOP_OK;
}
