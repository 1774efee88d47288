// Throughput probe of the SIMT fused multiply-add pipes (FP32 scalar, FP32
// packed pairs and FP64) on the current device.  The benchmark states the
// FP64 form's roofline against the measured DFMA rate; the paper has no
// counterpart of this.  Each thread runs independent multiply-add chains
// a <- a b + c long enough that launch costs vanish; nothing but the SIMT pipes
// is exercised.  Clocks and power settings are left as they are.
#include <cuda_runtime.h>

#include "../../include/mbo.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T* out, int iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (T)(threadIdx.x + 1) * (T)1e-3 + (T)i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  T s = (T)0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == (T)-1) out[0] = s;  // never true: keeps the chains live
}

__global__ void __launch_bounds__(kThreads) k_ffma2_chains(float* out, int iters, float b, float c) {
  float2 a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = make_float2((threadIdx.x + 1) * 1e-3f + i, i * 0.5f);
  const float2 bb = make_float2(b, b), cc = make_float2(c, c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = __ffma2_rn(a[i], bb, cc);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i].x + a[i].y;
  if (s == -1.f) out[0] = s;
}

// Best of five timed launches (after one warm-up); returns ms.
template <class F> float best_ms(F launch) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 1e30f;
  for (int k = 0; k < 6; ++k) {
    cudaEventRecord(a);
    launch();
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (k > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

}  // namespace

extern "C" mbo_status mbo_measure_fma_peaks(double* fp32_tflops, double* fp32x2_tflops,
                                             double* fp64_tflops) {
  if (!fp32_tflops || !fp32x2_tflops || !fp64_tflops) return MBO_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MBO_ERR_CUDA;
  void* out = nullptr;
  if (cudaMalloc(&out, 64) != cudaSuccess) return MBO_ERR_OOM;
  const int blocks = sms * 8;  // 64 warps per SM
  const double threads = (double)blocks * kThreads;
  const int it32 = 16384, it64 = 256;
  const float m32 = best_ms([&] {
    k_fma_chains<float><<<blocks, kThreads>>>(static_cast<float*>(out), it32, 0.999f, 1e-3f);
  });
  const float m2 = best_ms([&] {
    k_ffma2_chains<<<blocks, kThreads>>>(static_cast<float*>(out), it32, 0.999f, 1e-3f);
  });
  const float m64 = best_ms([&] {
    k_fma_chains<double><<<blocks, kThreads>>>(static_cast<double*>(out), it64, 0.999, 1e-3);
  });
  const cudaError_t e = cudaGetLastError();
  cudaFree(out);
  if (e != cudaSuccess) return MBO_ERR_CUDA;
  *fp32_tflops = 2.0 * threads * kChains * it32 / (m32 * 1e-3) / 1e12;
  *fp32x2_tflops = 4.0 * threads * kChains * it32 / (m2 * 1e-3) / 1e12;
  *fp64_tflops = 2.0 * threads * kChains * it64 / (m64 * 1e-3) / 1e12;
  return MBO_OK;
}
