// FP64 kernels: fused pull step, the separate propagate / bc / collide kernels,
// equilibrium initialisation, moments and the kinetic-energy reduction.
//
// Thread mapping (all site kernels): block = 32 x 4 threads; threadIdx.x runs along y
// (the contiguous axis, Sec. 4 "column-major, Y innermost"), so each warp owns 32
// consecutive sites of one column x and every population load/store of a warp is one
// contiguous 256-byte run (shifted by the hop's vy for loads).
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"
#include "step_fix64.cuh"

namespace d2q37 {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int wrap(int v, int n) { return wrap_index(v, n); }

// Source column offsets x_s * pitch for hops vx = -3..3 (index vx + 3), x periodic.
__device__ __forceinline__ void source_columns(int x, const StepArgs& a, long long (&col)[7]) {
#pragma unroll
  for (int d = 0; d < 7; ++d) col[d] = (long long)wrap(x - (d - 3), a.lx) * a.pitch;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Fused step: gather (propagate + bc) -> collide -> streaming store (step_fp64.cuh).
template <bool PERIODIC>
__global__ void __launch_bounds__(128, 4) k_step_fp64(const double* __restrict__ fin, double* __restrict__ fout,
                                                   StepArgs a) {
  const int x = blockIdx.y * 4 + threadIdx.y;
  if (x >= a.lx) return;  // uniform per warp
  step_strip_fp64<PERIODIC>(fin, fout, a, a, x, blockIdx.x * 32, LdReadOnly());
}

// The same fused step with the fixed-point relaxation of collide_fix64.cuh.
#ifndef LBM_FIX64_MIN_BLOCKS
#define LBM_FIX64_MIN_BLOCKS 5
#endif
template <bool PERIODIC>
__global__ void __launch_bounds__(128, LBM_FIX64_MIN_BLOCKS) k_step_fix64(const double* __restrict__ fin,
                                                                         double* __restrict__ fout, StepArgs a) {
  __shared__ double staged[kFixWarps][Q * 32];  // 37 populations x 32 sites per warp
  const int x = blockIdx.y * 4 + threadIdx.y;
  if (x >= a.lx) return;  // uniform per warp
  step_strip_fix64<PERIODIC>(fin, fout, a, a, x, blockIdx.x * 32, LdReadOnly(), staged[threadIdx.y]);
}

// ---------------------------------------------------------------------------------------
// Separate kernels (the paper's propagate -> bc -> collide sequence, Sec. 5).
template <bool PERIODIC>
__global__ void __launch_bounds__(128) k_propagate_fp64(const double* __restrict__ fin,
                                                        double* __restrict__ ftmp, StepArgs a) {
  const int x = blockIdx.y * 4 + threadIdx.y;
  const int y = blockIdx.x * 32 + threadIdx.x;
  if (x >= a.lx || y >= a.ly) return;
  long long col[7];
  source_columns(x, a, col);
  double* dst = ftmp + (long long)x * a.pitch + y;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    int ys = y - vy(i);
    if (PERIODIC) ys = wrap(ys, a.ly);
    else if (ys < 0 || ys >= a.ly) continue;  // left for bc
    __stcs(dst + i * a.pop, __ldg(fin + i * a.pop + col[vx(i) + 3] + ys));
  }
}

// Push form of propagate: site (x, y) sends each of its populations to (x + vx, y + vy).
// A warp reads 32 consecutive y of one population (one aligned 256-byte run) and writes
// them shifted by the hop, so the writes are the unaligned side.  Moves that leave the fluid
// in y are dropped; the entries they would have fed from outside are left for bc.
template <bool PERIODIC>
__global__ void __launch_bounds__(128) k_propagate_push_fp64(const double* __restrict__ fin,
                                                             double* __restrict__ ftmp, StepArgs a) {
  const int x = blockIdx.y * 4 + threadIdx.y;
  const int y = blockIdx.x * 32 + threadIdx.x;
  if (x >= a.lx || y >= a.ly) return;
  long long col[7];  // destination column offsets for vx = -3..3
#pragma unroll
  for (int d = 0; d < 7; ++d) col[d] = (long long)wrap(x + (d - 3), a.lx) * a.pitch;
  const double* src = fin + (long long)x * a.pitch + y;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    int yd = y + vy(i);
    if (PERIODIC) yd = wrap(yd, a.ly);
    else if (yd < 0 || yd >= a.ly) continue;  // leaves the fluid
    __stcs(ftmp + i * a.pop + col[vx(i) + 3] + yd, __ldg(src + i * a.pop));
  }
}

// One thread per (column x, wall row r in 0..5): rows 0,1,2 and ly-3, ly-2, ly-1.
__global__ void __launch_bounds__(128) k_bc_fp64(const double* __restrict__ fin, double* __restrict__ ftmp,
                                                 StepArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.lx * 6) return;
  const int x = t / 6, r = t % 6;
  const bool bottom = r < 3;
  const int y = bottom ? r : a.ly - 6 + r;
  const int wall_row = bottom ? 0 : a.ly - 1;
  double* dst = ftmp + (long long)x * a.pitch + y;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int ys = y - vy(i);
    const bool outside = bottom ? (ys < 0) : (ys >= a.ly);
    if (!outside) continue;
    const double* src = fin + (long long)wrap(x - vx(i), a.lx) * a.pitch + wall_row;
    double rw = 0.0;
#pragma unroll
    for (int j = 0; j < Q; ++j) rw += __ldg(src + j * a.pop);
    dst[i * a.pop] = rw * (bottom ? a.wall_b[i] : a.wall_t[i]);
  }
}

__global__ void __launch_bounds__(128) k_collide_fp64(const double* __restrict__ ftmp, double* __restrict__ fout,
                                                      StepArgs a) {
  const int x = blockIdx.y * 4 + threadIdx.y;
  const int y = blockIdx.x * 32 + threadIdx.x;
  if (x >= a.lx || y >= a.ly) return;
  const long long o = (long long)x * a.pitch + y;
  double f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] = __ldg(ftmp + o + i * a.pop);
  double* dst = fout + o;
  collide_site(f, a.cc, [&](int i, double v) { __stcs(dst + i * a.pop, v); });
}

// ---------------------------------------------------------------------------------------
// f_i = f_i^eq(rho, u, T) from [lx][ly] fields.
__global__ void __launch_bounds__(128) k_init_fp64(const double* __restrict__ rho, const double* __restrict__ ux,
                                                   const double* __restrict__ uy, const double* __restrict__ T,
                                                   double* __restrict__ fout, StepArgs a) {
  const int x = blockIdx.y * 4 + threadIdx.y;
  const int y = blockIdx.x * 32 + threadIdx.x;
  if (x >= a.lx || y >= a.ly) return;
  const long long fi = (long long)x * a.ly + y;
  double f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] = 0.0;
  double* dst = fout + (long long)x * a.pitch + y;
  relax_site(f, 0.0, rho[fi], C * ux[fi], C * uy[fi], T[fi] - 1.0, [&](int i, double v) { dst[i * a.pop] = v; });
}

__device__ __forceinline__ void site_fields(const double (&f)[Q], double& rho, double& ux, double& uy, double& T) {
  double jx, jy, e;
  moments_int(f, rho, jx, jy, e);
  const double inv_rho = 1.0 / rho;
  ux = C * jx * inv_rho;
  uy = C * jy * inv_rho;
  T = (C2 * e * inv_rho - fma(ux, ux, uy * uy)) / D;
}

__global__ void __launch_bounds__(128) k_moments_fp64(const double* __restrict__ fin, double* __restrict__ rho,
                                                      double* __restrict__ ux, double* __restrict__ uy,
                                                      double* __restrict__ T, StepArgs a) {
  const int x = blockIdx.y * 4 + threadIdx.y;
  const int y = blockIdx.x * 32 + threadIdx.x;
  if (x >= a.lx || y >= a.ly) return;
  const long long o = (long long)x * a.pitch + y;
  double f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] = __ldg(fin + o + i * a.pop);
  const long long fi = (long long)x * a.ly + y;
  site_fields(f, rho[fi], ux[fi], uy[fi], T[fi]);
}

// Kinetic energy: per-block partial sums (fixed order), then one block sums the partials.
__global__ void __launch_bounds__(128) k_ke_partial_fp64(const double* __restrict__ fin, double* __restrict__ part,
                                                         StepArgs a) {
  const int x = blockIdx.y * 4 + threadIdx.y;
  const int y = blockIdx.x * 32 + threadIdx.x;
  double ke = 0.0;
  if (x < a.lx && y < a.ly) {
    const long long o = (long long)x * a.pitch + y;
    double f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = __ldg(fin + o + i * a.pop);
    double rho, ux, uy, T;
    site_fields(f, rho, ux, uy, T);
    ke = 0.5 * rho * fma(ux, ux, uy * uy);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) ke += __shfl_down_sync(FULL, ke, off);
  __shared__ double warp_sum[4];
  if (threadIdx.x == 0) warp_sum[threadIdx.y] = ke;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0)
    part[blockIdx.y * gridDim.x + blockIdx.x] = (warp_sum[0] + warp_sum[1]) + (warp_sum[2] + warp_sum[3]);
}

__global__ void __launch_bounds__(256) k_reduce_sum(const double* __restrict__ part, long long n,
                                                    double* __restrict__ out) {
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(FULL, s, off);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += ws[w];
    *out = t;
  }
}

// ---------------------------------------------------------------------------------------
// Host-side launchers.
static inline dim3 site_grid(const StepArgs& a) { return dim3((a.ly + 31) / 32, (a.lx + 3) / 4); }
static const dim3 kSiteBlock(32, 4);

cudaError_t launch_step_fp64(const double* fin, double* fout, const StepArgs& a, cudaStream_t s) {
  if (a.periodic) k_step_fp64<true><<<site_grid(a), kSiteBlock, 0, s>>>(fin, fout, a);
  else k_step_fp64<false><<<site_grid(a), kSiteBlock, 0, s>>>(fin, fout, a);
  return cudaGetLastError();
}

cudaError_t launch_step_fix64(const double* fin, double* fout, const StepArgs& a, cudaStream_t s) {
  if (a.periodic) k_step_fix64<true><<<site_grid(a), kSiteBlock, 0, s>>>(fin, fout, a);
  else k_step_fix64<false><<<site_grid(a), kSiteBlock, 0, s>>>(fin, fout, a);
  return cudaGetLastError();
}

cudaError_t launch_propagate_fp64(const double* fin, double* ftmp, const StepArgs& a, cudaStream_t s) {
  if (a.periodic) k_propagate_fp64<true><<<site_grid(a), kSiteBlock, 0, s>>>(fin, ftmp, a);
  else k_propagate_fp64<false><<<site_grid(a), kSiteBlock, 0, s>>>(fin, ftmp, a);
  return cudaGetLastError();
}

cudaError_t launch_propagate_push_fp64(const double* fin, double* ftmp, const StepArgs& a, cudaStream_t s) {
  if (a.periodic) k_propagate_push_fp64<true><<<site_grid(a), kSiteBlock, 0, s>>>(fin, ftmp, a);
  else k_propagate_push_fp64<false><<<site_grid(a), kSiteBlock, 0, s>>>(fin, ftmp, a);
  return cudaGetLastError();
}

cudaError_t launch_bc_fp64(const double* fin, double* ftmp, const StepArgs& a, cudaStream_t s) {
  if (a.periodic) return cudaSuccess;
  const int n = a.lx * 6;
  k_bc_fp64<<<(n + 127) / 128, 128, 0, s>>>(fin, ftmp, a);
  return cudaGetLastError();
}

cudaError_t launch_collide_fp64(const double* ftmp, double* fout, const StepArgs& a, cudaStream_t s) {
  k_collide_fp64<<<site_grid(a), kSiteBlock, 0, s>>>(ftmp, fout, a);
  return cudaGetLastError();
}

cudaError_t launch_init_fp64(const double* rho, const double* ux, const double* uy, const double* T, double* f,
                             const StepArgs& a, cudaStream_t s) {
  k_init_fp64<<<site_grid(a), kSiteBlock, 0, s>>>(rho, ux, uy, T, f, a);
  return cudaGetLastError();
}

cudaError_t launch_moments_fp64(const double* f, double* rho, double* ux, double* uy, double* T,
                                const StepArgs& a, cudaStream_t s) {
  k_moments_fp64<<<site_grid(a), kSiteBlock, 0, s>>>(f, rho, ux, uy, T, a);
  return cudaGetLastError();
}

long long ke_partial_count(const StepArgs& a) {
  const dim3 g = site_grid(a);
  return (long long)g.x * g.y;
}

cudaError_t launch_reduce_sum(const double* part, long long n, double* out, cudaStream_t s) {
  k_reduce_sum<<<1, 256, 0, s>>>(part, n, out);
  return cudaGetLastError();
}

cudaError_t launch_kinetic_energy_fp64(const double* f, double* out, double* part, const StepArgs& a,
                                       cudaStream_t s) {
  k_ke_partial_fp64<<<site_grid(a), kSiteBlock, 0, s>>>(f, part, a);
  return launch_reduce_sum(part, ke_partial_count(a), out, s);
}

}  // namespace d2q37
