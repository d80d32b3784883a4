// Peak probes for the roofline denominators: sustained rates of the arithmetic pipes the
// step kernels use (float64 FMA for the float64 step; integer multiply-add and 64-bit
// high products for the fixed-point relaxation; float32 FMA for the FP32 step).  Each
// thread runs 8 independent dependency chains so that the pipe, not the latency of one
// chain, sets the rate.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lbm_d2q37.h"

namespace {

constexpr int kIters = 4096;
constexpr int kChains = 8;
constexpr int kThreads = 256;

template <class T, class Op>
__device__ __forceinline__ void run_chains(T* out, T seed, Op op) {
  T v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = seed + (T)(threadIdx.x * kChains + c);
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = op(v[c]);
  }
  T s = v[0];
#pragma unroll
  for (int c = 1; c < kChains; ++c) s = s + v[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(kThreads) k_probe_dfma(double* out, double a, double b) {
  run_chains<double>(out, 1e-3, [&](double v) { return fma(v, a, b); });
}
__global__ void __launch_bounds__(kThreads) k_probe_ffma(float* out, float a, float b) {
  run_chains<float>(out, 1e-3f, [&](float v) { return fmaf(v, a, b); });
}
__global__ void __launch_bounds__(kThreads) k_probe_imad(unsigned* out, unsigned a, unsigned b) {
  run_chains<unsigned>(out, 7u, [&](unsigned v) { return v * a + b; });
}
__global__ void __launch_bounds__(kThreads) k_probe_mulhi(long long* out, long long a, long long b) {
  run_chains<long long>(out, 977, [&](long long v) { return __mul64hi(v, a) ^ b; });
}
__global__ void __launch_bounds__(kThreads) k_probe_umulhi(unsigned long long* out, unsigned long long a,
                                                          unsigned long long b) {
  run_chains<unsigned long long>(out, 977ull, [&](unsigned long long v) { return __umul64hi(v, a) ^ b; });
}

}  // namespace

extern "C" int32_t lbm_probe_peak(int32_t kind, double* ops_per_second) {
  if (!ops_per_second || kind < LBM_PROBE_DFMA || kind > LBM_PROBE_UMULHI64) return LBM_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LBM_ECUDA;
  const int blocks = sms * 8;
  void* buf = nullptr;
  if (cudaMalloc(&buf, (size_t)blocks * kThreads * 8) != cudaSuccess) return LBM_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&]() {
    switch (kind) {
      case LBM_PROBE_DFMA: k_probe_dfma<<<blocks, kThreads>>>((double*)buf, 1.0000001, 1e-9); break;
      case LBM_PROBE_FFMA: k_probe_ffma<<<blocks, kThreads>>>((float*)buf, 1.0000001f, 1e-9f); break;
      case LBM_PROBE_IMAD: k_probe_imad<<<blocks, kThreads>>>((unsigned*)buf, 1664525u, 1013904223u); break;
      case LBM_PROBE_MULHI64:
        k_probe_mulhi<<<blocks, kThreads>>>((long long*)buf, 0x5851F42D4C957F2DLL, 1442695040888963407LL);
        break;
      default:
        k_probe_umulhi<<<blocks, kThreads>>>((unsigned long long*)buf, 0x5851F42D4C957F2DULL,
                                             1442695040888963407ULL);
    }
  };
  launch();  // warm-up
  cudaEventRecord(e0);
  launch();
  cudaEventRecord(e1);
  const cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  const cudaError_t last = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (err != cudaSuccess || last != cudaSuccess || ms <= 0.0f) return LBM_ECUDA;
  *ops_per_second = (double)blocks * kThreads * kChains * kIters / (ms * 1e-3);
  return LBM_OK;
}
