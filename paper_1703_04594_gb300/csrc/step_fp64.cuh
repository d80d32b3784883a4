// One warp-strip of the fused FP64 pull step: 32 consecutive sites (x, y0 .. y0+31) of
// one column, gathered (propagate + bc, Sec. 3 eq. "master2", Sec. 5), collided
// (collide_fp64.cuh) and stored.  Shared by the single-lattice kernel and the batched
// kernels; `Ld` chooses the load path (read-only cache, or L2-only inside a persistent
// kernel whose source buffers were written earlier in the same launch).
#pragma once
#include "collide_fp64.cuh"
#include "kernels.h"

namespace d2q37 {

// kL1: the loads may be served from L1 (sources written by earlier launches only), which
// also allows staging through L1-cached asynchronous copies.
struct LdReadOnly {
  static constexpr bool kL1 = true;
  template <class T>
  __device__ __forceinline__ T operator()(const T* p) const { return __ldg(p); }
};
struct LdL2 {
  static constexpr bool kL1 = false;
  template <class T>
  __device__ __forceinline__ T operator()(const T* p) const { return __ldcg(p); }
};

__device__ __forceinline__ int wrap_index(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Wall densities rho(x_s, 0) and rho(x_s, ly-1) of the seven source columns, computed by
// lanes 0..6 (bottom) and 8..14 (top) of the warp and broadcast to all lanes.
// Every lane of the warp must call this (it shuffles with the full mask).
template <class Ld>
__device__ __forceinline__ void wall_densities_fp64(const double* __restrict__ fin, int x, const StepScalars& a,
                                                    double (&rb)[7], double (&rt)[7], Ld ld) {
  const int lane = threadIdx.x & 31;
  const int d = lane & 7;
  const int row = lane < 8 ? 0 : a.ly - 1;
  double r = 0.0;
  if (d < 7 && lane < 16) {
    const double* src = fin + (long long)wrap_index(x - (d - 3), a.lx) * a.pitch + row;
#pragma unroll
    for (int i = 0; i < Q; ++i) r += ld(src + i * a.pop);
  }
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    rb[j] = __shfl_sync(0xffffffffu, r, j);
    rt[j] = __shfl_sync(0xffffffffu, r, 8 + j);
  }
}

// Pull-gather of the 37 populations of site (x, yc) with the wall values for sources
// outside the fluid.  Must be called by all 32 lanes of a warp strip (x, y0..y0+31); yc is
// the lane's row clamped into the lattice.
template <bool PERIODIC, class Ld>
__device__ __forceinline__ void gather_strip_fp64(const double* __restrict__ fin, const StepScalars& a,
                                                  const StepWalls& w, int x, int y0, int yc, double (&f)[Q], Ld ld) {
  long long col[7];
#pragma unroll
  for (int d = 0; d < 7; ++d) col[d] = (long long)wrap_index(x - (d - 3), a.lx) * a.pitch;
  const bool wall_warp = !PERIODIC && (y0 < 3 || y0 + 32 > a.ly - 3);
  if (wall_warp) {
    double rb[7], rt[7];
    wall_densities_fp64(fin, x, a, rb, rt, ld);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int ys = yc - vy(i);
      const double* src = fin + i * a.pop + col[vx(i) + 3];
      if (vy(i) > 0 && ys < 0) f[i] = rb[vx(i) + 3] * w.wall_b[i];
      else if (vy(i) < 0 && ys >= a.ly) f[i] = rt[vx(i) + 3] * w.wall_t[i];
      else f[i] = ld(src + ys);
    }
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      int ys = yc - vy(i);
      if (PERIODIC) ys = wrap_index(ys, a.ly);
      f[i] = ld(fin + i * a.pop + col[vx(i) + 3] + ys);
    }
  }
}

// One warp-strip of the fused step.  Must be called by all 32 lanes of a warp
// (lane = y - y0).  Lanes with y >= ly gather clamped data and store nothing.
template <bool PERIODIC, class Ld>
__device__ __forceinline__ void step_strip_fp64(const double* __restrict__ fin, double* __restrict__ fout,
                                                const StepScalars& a, const StepWalls& w, int x, int y0, Ld ld) {
  const int y = y0 + (threadIdx.x & 31);
  const bool active = y < a.ly;
  const int yc = active ? y : a.ly - 1;
  double f[Q];
  gather_strip_fp64<PERIODIC>(fin, a, w, x, y0, yc, f, ld);
  if (!active) return;
  double* dst = fout + (long long)x * a.pitch + y;
  collide_site(f, a.cc, [&](int i, double v) { __stcs(dst + i * a.pop, v); });
}

}  // namespace d2q37
