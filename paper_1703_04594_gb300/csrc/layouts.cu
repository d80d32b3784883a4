// Alternative population layouts for the fused FP64 step (the layout comparison of Sec. 4,
// Tables "propagate-kernel"/"collide-kernel": AoS, SoA, CSoA, CAoSoA).  Same arithmetic as
// the SoA step (collide_site) on the same gathered values; only the addresses of the 37
// gathers and stores change.  Walls only (no periodic-y mode).
//
//   SoA:    the production layout.  With pitch a multiple of 32 it is the paper's CSoA with
//           cluster width 32: a warp's 32 consecutive y are one aligned 256-byte cluster.
//   AoS:    element (i, x, y) at (x * pitch + y) * 37 + i: the 37 populations of a site are
//           contiguous (Sec. 4 "AoS").  A warp still owns 32 consecutive y of one column, so
//           each of its loads touches 32 records 296 bytes apart.
//   PSoA:   element (i, x, y) at ((i * lx + x) * P + j) * 32 + k with y = k * P + j and
//           P = pitch / 32: every population column is split into 32 partitions of P rows
//           and the k-th elements of the partitions form a 32-wide cluster (the partitioning
//           of the paper's CAoSoA, one array per population).
//   CAoSoA: the same clusters, with the 37 clusters of one (x, j) adjacent (Sec. 4
//           "CAoSoA"): element (i, x, y) at ((x * P + j) * 37 + i) * 32 + k.
// In both partitioned layouts a warp owns cluster (x, j): lane k is site y = k * P + j, so a
// hop by vy reads cluster j - vy of the same lanes, one aligned 256-byte run, except across
// a partition edge, where lane k reads lane k -/+ 1 of cluster j - vy +/- P.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lbm_d2q37.h"
#include "kernels.h"
#include "step_fp64.cuh"

namespace d2q37 {

namespace {

__device__ __forceinline__ long long aos_index(const StepArgs& a, int i, int x, int y) {
  return ((long long)x * a.pitch + y) * Q + i;
}

// Element k of cluster j of population i in column x, partitioned layouts.
template <int L>
__device__ __forceinline__ long long cluster_index(const StepArgs& a, int i, int x, long long j, long long k) {
  const long long P = a.pitch >> 5;
  if (L == LBM_LAYOUT_CAOSOA) return (((long long)x * P + j) * Q + i) * 32 + k;
  return (((long long)i * a.lx + x) * P + j) * 32 + k;
}

constexpr bool partitioned(int L) { return L == LBM_LAYOUT_PSOA || L == LBM_LAYOUT_CAOSOA; }

template <int L>
__device__ __forceinline__ long long lindex(const StepArgs& a, int i, int x, int y) {
  if (L == LBM_LAYOUT_AOS) return aos_index(a, i, x, y);
  if (partitioned(L)) {
    const long long P = a.pitch >> 5;
    const long long k = y / P;
    return cluster_index<L>(a, i, x, y - k * P, k);
  }
  return (long long)i * a.pop + (long long)x * a.pitch + y;
}

// rho at (x_s, row) summed over the 37 populations, any layout.
template <int L>
__device__ __forceinline__ double column_density(const double* __restrict__ f, const StepArgs& a, int xs, int row) {
  double r = 0.0;
#pragma unroll
  for (int i = 0; i < Q; ++i) r += __ldg(f + lindex<L>(a, i, xs, row));
  return r;
}

// Fused step of site (x, y) in layout L (walls).  All lanes of a warp share x; in the
// partitioned layouts the warp is cluster j (uniform) and lane k is row y = k * P + j.
template <int L>
__device__ __forceinline__ void step_site_layout(const double* __restrict__ fin, double* __restrict__ fout,
                                                 const StepArgs& a, int x, int y, int j, bool active) {
  const int lane = threadIdx.x & 31;
  const bool near_wall = __any_sync(0xffffffffu, active && (y < 3 || y >= a.ly - 3));
  double rb[7], rt[7];
  if (near_wall) {
    const int d = lane & 7;
    double r = 0.0;
    if (d < 7 && lane < 16) r = column_density<L>(fin, a, wrap_index(x - (d - 3), a.lx), lane < 8 ? 0 : a.ly - 1);
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      rb[k] = __shfl_sync(0xffffffffu, r, k);
      rt[k] = __shfl_sync(0xffffffffu, r, 8 + k);
    }
  }
  const long long P = a.pitch >> 5;
  double f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int xs = wrap_index(x - vx(i), a.lx);
    long long idx;
    int ys;
    if (partitioned(L)) {
      int js = j - vy(i), ks = lane;  // partition arithmetic: uniform branches on js
      if (P >= 3) {                   // a hop crosses at most one partition edge
        if (js < 0) {
          js += (int)P;
          ks -= 1;
        } else if (js >= (int)P) {
          js -= (int)P;
          ks += 1;
        }
      } else {                        // partitions shorter than a hop (pitch < 96)
        while (js < 0) {
          js += (int)P;
          ks -= 1;
        }
        while (js >= (int)P) {
          js -= (int)P;
          ks += 1;
        }
      }
      ys = ks * (int)P + js;
      idx = cluster_index<L>(a, i, xs, js, ks);
    } else {
      ys = y - vy(i);
      idx = aos_index(a, i, xs, ys);
    }
    if (active && ys < 0) f[i] = near_wall ? rb[vx(i) + 3] * a.wall_b[i] : 0.0;
    else if (active && ys >= a.ly) f[i] = near_wall ? rt[vx(i) + 3] * a.wall_t[i] : 0.0;
    else f[i] = (active && ys >= 0 && ys < a.ly) ? __ldg(fin + idx) : 0.0;
  }
  if (!active) return;
  collide_site(f, a.cc, [&](int i, double v) { __stcs(fout + lindex<L>(a, i, x, y), v); });
}

}  // namespace

template <int L>
__global__ void __launch_bounds__(128) k_step_layout(const double* __restrict__ fin, double* __restrict__ fout,
                                                     StepArgs a) {
  const int x = blockIdx.y * 4 + threadIdx.y;
  if (x >= a.lx) return;  // uniform per warp
  int y, j = 0;
  if (partitioned(L)) {
    j = blockIdx.x;  // cluster j, lane k = threadIdx.x
    y = (int)threadIdx.x * (int)(a.pitch >> 5) + j;
  } else {
    y = blockIdx.x * 32 + threadIdx.x;
  }
  step_site_layout<L>(fin, fout, a, x, y, j, y < a.ly);
}

// Layout conversion: dst(layout Lt) <- src(layout Ls), one thread per site.
template <int Ls, int Lt>
__global__ void __launch_bounds__(128) k_convert(const double* __restrict__ src, double* __restrict__ dst, StepArgs a) {
  const int x = blockIdx.y * 4 + threadIdx.y;
  const int y = blockIdx.x * 32 + threadIdx.x;
  if (x >= a.lx || y >= a.ly) return;
#pragma unroll
  for (int i = 0; i < Q; ++i) dst[lindex<Lt>(a, i, x, y)] = src[lindex<Ls>(a, i, x, y)];
}

template <int L>
cudaError_t launch_step_layout(const double* fin, double* fout, const StepArgs& a, cudaStream_t s) {
  const dim3 grid(partitioned(L) ? (unsigned)(a.pitch >> 5) : (unsigned)((a.ly + 31) / 32),
                  (unsigned)((a.lx + 3) / 4));
  k_step_layout<L><<<grid, dim3(32, 4), 0, s>>>(fin, fout, a);
  return cudaGetLastError();
}

cudaError_t launch_convert(int from, int to, const double* src, double* dst, const StepArgs& a, cudaStream_t s) {
  const dim3 grid((a.ly + 31) / 32, (a.lx + 3) / 4), blk(32, 4);
#define LBM_CONV(F, T) \
  if (from == F && to == T) k_convert<F, T><<<grid, blk, 0, s>>>(src, dst, a);
  LBM_CONV(LBM_LAYOUT_SOA, LBM_LAYOUT_AOS)
  LBM_CONV(LBM_LAYOUT_SOA, LBM_LAYOUT_PSOA)
  LBM_CONV(LBM_LAYOUT_SOA, LBM_LAYOUT_CAOSOA)
  LBM_CONV(LBM_LAYOUT_AOS, LBM_LAYOUT_SOA)
  LBM_CONV(LBM_LAYOUT_PSOA, LBM_LAYOUT_SOA)
  LBM_CONV(LBM_LAYOUT_CAOSOA, LBM_LAYOUT_SOA)
#undef LBM_CONV
  return cudaGetLastError();
}

}  // namespace d2q37

using namespace d2q37;

extern "C" {

int32_t lbm_convert_layout(const lbm_params* p, int32_t from, const void* src, int32_t to, void* dst, void* stream) {
  const auto other = [](int32_t l) {
    return l == LBM_LAYOUT_AOS || l == LBM_LAYOUT_PSOA || l == LBM_LAYOUT_CAOSOA;
  };
  const bool ok_pair = (from == LBM_LAYOUT_SOA && other(to)) || (to == LBM_LAYOUT_SOA && other(from));
  if (!params_valid(p) || p->precision != LBM_FP64 || !ok_pair || !src || !dst || src == dst ||
      ((uintptr_t)src % 16) || ((uintptr_t)dst % 16))
    return LBM_EINVAL;
  const StepArgs a = make_step_args(p);
  return launch_convert(from, to, (const double*)src, (double*)dst, a, (cudaStream_t)stream) == cudaSuccess
             ? LBM_OK
             : LBM_ECUDA;
}

int32_t lbm_step_layout(const lbm_params* p, int32_t layout, const void* fin, void* fout, void* stream) {
  if (!params_valid(p) || p->precision != LBM_FP64 || p->bc != LBM_BC_WALLS || !fin || !fout ||
      lbm_buffer_bytes(p) <= 0 || ((uintptr_t)fin < (uintptr_t)fout + lbm_buffer_bytes(p) &&
                                   (uintptr_t)fout < (uintptr_t)fin + lbm_buffer_bytes(p)) ||
      ((uintptr_t)fin % 16) || ((uintptr_t)fout % 16))
    return LBM_EINVAL;
  const StepArgs a = make_step_args(p);
  cudaError_t e;
  switch (layout) {
    case LBM_LAYOUT_AOS: e = launch_step_layout<LBM_LAYOUT_AOS>((const double*)fin, (double*)fout, a, (cudaStream_t)stream); break;
    case LBM_LAYOUT_PSOA: e = launch_step_layout<LBM_LAYOUT_PSOA>((const double*)fin, (double*)fout, a, (cudaStream_t)stream); break;
    case LBM_LAYOUT_CAOSOA: e = launch_step_layout<LBM_LAYOUT_CAOSOA>((const double*)fin, (double*)fout, a, (cudaStream_t)stream); break;
    default: return LBM_EINVAL;
  }
  return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

}  // extern "C"
