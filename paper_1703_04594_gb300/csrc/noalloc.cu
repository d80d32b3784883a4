// Kinetic energy without caller scratch: lbm_kinetic_energy_noalloc.
//
// Some callers cannot allocate device memory once they are running: a host application
// whose device memory is entirely reserved up front by its own pool, or a time-critical
// stepping loop that must not pay for cudaMalloc (which can synchronise the device).  They
// can still hand in the state and the output scalar, but not the per-tile scratch that
// lbm_kinetic_energy needs.  This entry point takes that scratch from a fixed array that
// is part of the library image instead.
//
// The array holds LBM_NOALLOC_MAX_TILES doubles (2 MiB) and exists once on every GPU that
// loads the library, until the process exits.  Lattices needing more partial sums than
// that are rejected with LBM_ESIZE.  Every call shares the array and leaves its partial
// sums in it; the reduction only reads the entries the same call has just written, so
// nothing has to start at zero.  Two calls whose kernels overlap on the GPU (different
// streams, no ordering between them) race on the array.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lbm_d2q37.h"

namespace {

__device__ __align__(256) double g_ke_partials[LBM_NOALLOC_MAX_TILES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_partials_dev[kMaxDevices] = {};  // device address of g_ke_partials, per device

// Device address of the array on the current device.  In host code the name
// g_ke_partials is only a host-side stand-in, so the address has to be looked up once
// per device with that device current.  The cached address is not refreshed after a
// cudaDeviceReset (the header says so).
int32_t partials_on_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return LBM_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return LBM_EINVAL;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_partials_dev[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_ke_partials);
    if (e != cudaSuccess || p == nullptr) return LBM_ECUDA;
    g_partials_dev[dev] = static_cast<double*>(p);
  }
  *out = g_partials_dev[dev];
  return LBM_OK;
}

}  // namespace

extern "C" int32_t lbm_kinetic_energy_noalloc(const lbm_params* p, const void* f_dev, double* out_dev,
                                              void* stream) {
  const int64_t need = lbm_reduce_scratch_bytes(p);  // validates p; -1 if invalid
  if (need < 0) return LBM_EINVAL;
  if (need > (int64_t)sizeof(double) * LBM_NOALLOC_MAX_TILES) return LBM_ESIZE;
  double* scratch = nullptr;
  const int32_t st = partials_on_current_device(&scratch);
  if (st != LBM_OK) return st;
  return lbm_kinetic_energy(p, f_dev, out_dev, scratch, sizeof(double) * (size_t)LBM_NOALLOC_MAX_TILES, stream);
}
