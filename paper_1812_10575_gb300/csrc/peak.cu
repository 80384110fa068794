// Measured FP32 FMA throughput of this GPU: the ALU roofline of the direct
// O(N^2) sum, which is bound by its FP32 arithmetic (Sec. 1: N - 1 pair
// evaluations per particle and step).  Every thread runs eight independent
// chains of fused multiply-adds, as scalar instructions or as packed two-lane
// instructions, on a grid of eight 256-thread blocks per SM.
#include <cuda_runtime.h>

#include <cstdio>

#include "rbm.h"
#include "rbm_internal.h"

namespace rbm {
namespace {

constexpr int kChains = 8;     // independent FMA chains per thread
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

template <bool kPacked>
__global__ void __launch_bounds__(kThreads) k_fma_peak(float* sink, int iters, float a, float b) {
  float v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = 1e-3f * static_cast<float>(threadIdx.x + c);
  if (kPacked) {
    unsigned long long w[kChains / 2], a2, b2;
    asm("mov.b64 %0, {%1, %1};" : "=l"(a2) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(b2) : "f"(b));
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) asm("mov.b64 %0, {%1, %2};" : "=l"(w[c]) : "f"(v[2 * c]), "f"(v[2 * c + 1]));
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kChains / 2; ++c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(w[c]) : "l"(a2), "l"(b2));
    }
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) asm("mov.b64 {%0, %1}, %2;" : "=f"(v[2 * c]), "=f"(v[2 * c + 1]) : "l"(w[c]));
  } else {
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(v[c]) : "f"(a), "f"(b));
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  if (s == -1.0f) sink[0] = s;  // never true for these inputs; keeps the chains live
}

}  // namespace
}  // namespace rbm

extern "C" rbm_status rbm_fp32_fma_peak(int32_t packed, double* tflops, void* cuda_stream) {
  using namespace rbm;
  if (!tflops || (packed != 0 && packed != 1)) {
    set_last_error_text("rbm_fp32_fma_peak: tflops must not be null and packed must be 0 or 1");
    return RBM_ERR_INVALID;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  float* sink = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(float));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  constexpr int kIters = 8192, kReps = 5;
  const unsigned grid = static_cast<unsigned>(sms) * kBlocksPerSm;
  float best = 0.0f;
  for (int r = 0; r <= kReps && e == cudaSuccess; ++r) {  // the first launch warms up
    e = cudaEventRecord(e0, st);
    if (packed) k_fma_peak<true><<<grid, kThreads, 0, st>>>(sink, kIters, 0.999999f, 1e-7f);
    else k_fma_peak<false><<<grid, kThreads, 0, st>>>(sink, kIters, 0.999999f, 1e-7f);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) {
    char msg[160];
    snprintf(msg, sizeof(msg), "rbm_fp32_fma_peak: %s", cudaGetErrorString(e));
    set_last_error_text(msg);
    return RBM_ERR_CUDA;
  }
  const double flop = 2.0 * kChains * static_cast<double>(kIters) * kThreads * grid;
  *tflops = flop / (best * 1e-3) / 1e12;
  return RBM_OK;
}
