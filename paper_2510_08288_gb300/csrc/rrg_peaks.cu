// rrg_peaks.cu -- throughput of the arithmetic units the rollouts use,
// measured on the current device: binary32 FMA, binary64 FMA and the MUFU
// exp2 the compressor term issues.  Each thread runs 8 independent chains of
// the operation (enough to cover the pipeline latency), with 64 warps per SM;
// CUDA events time the launch.
#include <cuda_runtime.h>

#include "../../include/rrg.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_kernel(T* out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = static_cast<T>(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == static_cast<T>(12345.678)) out[blockIdx.x] = s;  // keeps the chains alive
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__global__ void __launch_bounds__(kThreads) mufu_kernel(float* out, int iters) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = -1.0f - 1e-3f * static_cast<float>(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = -ex2_approx(x[c]);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678f) out[blockIdx.x] = s;
}

template <typename K>
int time_kernel(K launch, int blocks, float* ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return RRG_ECUDA;
  launch(blocks);  // warm-up
  cudaEventRecord(a);
  launch(blocks);
  cudaEventRecord(b);
  const cudaError_t e = cudaEventSynchronize(b);
  cudaEventElapsedTime(ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return (e == cudaSuccess && cudaGetLastError() == cudaSuccess) ? RRG_OK : RRG_ECUDA;
}

}  // namespace

extern "C" int rrg_alu_peaks(double* fp32_tflops, double* fp64_tflops, double* mufu_tops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return RRG_ECUDA;
  const int blocks = sms * 8;  // 64 warps per SM
  void* out = nullptr;
  if (cudaMalloc(&out, blocks * sizeof(double)) != cudaSuccess) return RRG_ENOMEM;
  const double threads = static_cast<double>(blocks) * kThreads;
  int rc = RRG_OK;
  float ms = 0.0f;
  const int it32 = 2048, it64 = 64, itm = 512;
  if (fp32_tflops && rc == RRG_OK) {
    rc = time_kernel([&](int nb) { fma_kernel<float><<<nb, kThreads>>>(static_cast<float*>(out), it32,
                                                                       0.999999f, 1e-7f); },
                     blocks, &ms);
    *fp32_tflops = 2.0 * kChains * 16.0 * it32 * threads / (ms * 1e-3) / 1e12;
  }
  if (fp64_tflops && rc == RRG_OK) {
    rc = time_kernel([&](int nb) { fma_kernel<double><<<nb, kThreads>>>(static_cast<double*>(out), it64,
                                                                        0.999999, 1e-7); },
                     blocks, &ms);
    *fp64_tflops = 2.0 * kChains * 16.0 * it64 * threads / (ms * 1e-3) / 1e12;
  }
  if (mufu_tops && rc == RRG_OK) {
    rc = time_kernel([&](int nb) { mufu_kernel<<<nb, kThreads>>>(static_cast<float*>(out), itm); },
                     blocks, &ms);
    *mufu_tops = kChains * 16.0 * itm * threads / (ms * 1e-3) / 1e12;
  }
  cudaFree(out);
  return rc;
}
