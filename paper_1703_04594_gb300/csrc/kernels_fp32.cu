// FP32 shifted-deviation storage kernels (step, init, moments, kinetic energy).
// The precision split of the step is described in step_fp32.cuh.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"
#include "step_fp32.cuh"

namespace d2q37 {

#ifndef LBM_FP32_MIN_BLOCKS
#define LBM_FP32_MIN_BLOCKS 6  // 80 registers; measured best among 4..8 blocks per SM
#endif
// The conserved-moment form holds all 37 outputs and eight sum lanes until its
// correction: 5 blocks per SM (96 registers) instead of spilling at 80.
#ifndef LBM_FP32C_MIN_BLOCKS
#define LBM_FP32C_MIN_BLOCKS 5
#endif
template <bool PERIODIC, bool SCALED, bool CONSERVE>
__global__ void __launch_bounds__(128, CONSERVE ? LBM_FP32C_MIN_BLOCKS : LBM_FP32_MIN_BLOCKS) k_step_fp32(
    const float* __restrict__ fin,
                                                                       float* __restrict__ fout, StepArgs a) {
  const int x = blockIdx.y * 4 + threadIdx.y;
  if (x >= a.lx) return;  // uniform per warp
  step_strip_fp32<PERIODIC, SCALED, CONSERVE>(fin, fout, a, a, x, blockIdx.x * 32, LdReadOnly());
}

// g_i = f_i^eq(rho, u, T) - w_i rho0, equilibrium evaluated in float64 then rounded.
__global__ void __launch_bounds__(128) k_init_fp32(const double* __restrict__ rho, const double* __restrict__ ux,
                                                   const double* __restrict__ uy, const double* __restrict__ T,
                                                   float* __restrict__ fout, StepArgs a) {
  const int x = blockIdx.y * 4 + threadIdx.y;
  const int y = blockIdx.x * 32 + threadIdx.x;
  if (x >= a.lx || y >= a.ly) return;
  const long long fi = (long long)x * a.ly + y;
  double f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] = 0.0;
  float* dst = fout + (long long)x * a.pitch + y;
  const double rho0 = a.rho0;
  relax_site(f, 0.0, rho[fi], C * ux[fi], C * uy[fi], T[fi] - 1.0,
             [&](int i, double v) { dst[i * a.pop] = (float)(v - weight(i) * rho0); });
}

__device__ __forceinline__ void site_fields_fp32(const float (&g)[Q], const StepScalars& a, double& rho, double& ux,
                                                 double& uy, double& T) {
  const double rho0 = a.rho0;
  const DevMoments<double> m = moments_fix<double, true>(g, a);
  rho = m.drho + rho0;
  const double inv = 1.0 / rho;
  ux = C * m.jx * inv;
  uy = C * m.jy * inv;
  const double etot = m.de + rho0 * (D / C2);
  T = (C2 * etot * inv - fma(ux, ux, uy * uy)) / D;
}

__global__ void __launch_bounds__(128) k_moments_fp32(const float* __restrict__ fin, double* __restrict__ rho,
                                                      double* __restrict__ ux, double* __restrict__ uy,
                                                      double* __restrict__ T, StepArgs a) {
  const int x = blockIdx.y * 4 + threadIdx.y;
  const int y = blockIdx.x * 32 + threadIdx.x;
  if (x >= a.lx || y >= a.ly) return;
  const long long o = (long long)x * a.pitch + y;
  float g[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) g[i] = __ldg(fin + o + i * a.pop);
  const long long fi = (long long)x * a.ly + y;
  site_fields_fp32(g, a, rho[fi], ux[fi], uy[fi], T[fi]);
}

__global__ void __launch_bounds__(128) k_ke_partial_fp32(const float* __restrict__ fin, double* __restrict__ part,
                                                         StepArgs a) {
  const int x = blockIdx.y * 4 + threadIdx.y;
  const int y = blockIdx.x * 32 + threadIdx.x;
  double ke = 0.0;
  if (x < a.lx && y < a.ly) {
    const long long o = (long long)x * a.pitch + y;
    float g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = __ldg(fin + o + i * a.pop);
    double rho, ux, uy, T;
    site_fields_fp32(g, a, rho, ux, uy, T);
    ke = 0.5 * rho * fma(ux, ux, uy * uy);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) ke += __shfl_down_sync(0xffffffffu, ke, off);
  __shared__ double warp_sum[4];
  if (threadIdx.x == 0) warp_sum[threadIdx.y] = ke;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0)
    part[blockIdx.y * gridDim.x + blockIdx.x] = (warp_sum[0] + warp_sum[1]) + (warp_sum[2] + warp_sum[3]);
}

static inline dim3 site_grid(const StepArgs& a) { return dim3((a.ly + 31) / 32, (a.lx + 3) / 4); }
static const dim3 kSiteBlock(32, 4);

template <bool PERIODIC, bool SCALED>
static void launch_fp32(const float* fin, float* fout, const StepArgs& a, cudaStream_t s) {
  if (a.conserve) k_step_fp32<PERIODIC, SCALED, true><<<site_grid(a), kSiteBlock, 0, s>>>(fin, fout, a);
  else k_step_fp32<PERIODIC, SCALED, false><<<site_grid(a), kSiteBlock, 0, s>>>(fin, fout, a);
}

cudaError_t launch_step_fp32(const float* fin, float* fout, const StepArgs& a, cudaStream_t s) {
  const bool scaled = a.fix_back != 1.0 / 4503599627370496.0;
  if (a.periodic) {
    if (scaled) launch_fp32<true, true>(fin, fout, a, s);
    else launch_fp32<true, false>(fin, fout, a, s);
  } else {
    if (scaled) launch_fp32<false, true>(fin, fout, a, s);
    else launch_fp32<false, false>(fin, fout, a, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_init_fp32(const double* rho, const double* ux, const double* uy, const double* T, float* f,
                             const StepArgs& a, cudaStream_t s) {
  k_init_fp32<<<site_grid(a), kSiteBlock, 0, s>>>(rho, ux, uy, T, f, a);
  return cudaGetLastError();
}

cudaError_t launch_moments_fp32(const float* f, double* rho, double* ux, double* uy, double* T,
                                const StepArgs& a, cudaStream_t s) {
  k_moments_fp32<<<site_grid(a), kSiteBlock, 0, s>>>(f, rho, ux, uy, T, a);
  return cudaGetLastError();
}

cudaError_t launch_kinetic_energy_fp32(const float* f, double* out, double* part, const StepArgs& a,
                                       cudaStream_t s) {
  k_ke_partial_fp32<<<site_grid(a), kSiteBlock, 0, s>>>(f, part, a);
  return launch_reduce_sum(part, ke_partial_count(a), out, s);
}

}  // namespace d2q37
