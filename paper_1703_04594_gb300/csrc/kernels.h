// Internal launch interface between the C-ABI layer (lbm_api.cu) and the kernels.
#pragma once
#include <cuda_runtime.h>

#include "collide_fp64.cuh"

namespace d2q37 {

// Everything a site kernel needs, passed by value as the kernel parameter.
struct StepArgs {
  int lx, ly;
  long long pitch;      // elements per y-column
  long long pop;        // elements per population plane = lx * pitch
  int periodic;         // 1: y wraps (test mode), 0: thermal walls
  CollideConst cc;
  double wall_b[Q];     // w_i P_i(T_bottom): ghost value = rho_w * wall_b[i]
  double wall_t[Q];     // w_i P_i(T_top)
};

cudaError_t launch_step_fp64(const double* fin, double* fout, const StepArgs& a, cudaStream_t s);
cudaError_t launch_propagate_fp64(const double* fin, double* ftmp, const StepArgs& a, cudaStream_t s);
cudaError_t launch_bc_fp64(const double* fin, double* ftmp, const StepArgs& a, cudaStream_t s);
cudaError_t launch_collide_fp64(const double* ftmp, double* fout, const StepArgs& a, cudaStream_t s);
cudaError_t launch_init_fp64(const double* rho, const double* ux, const double* uy, const double* T, double* f,
                             const StepArgs& a, cudaStream_t s);
cudaError_t launch_moments_fp64(const double* f, double* rho, double* ux, double* uy, double* T,
                                const StepArgs& a, cudaStream_t s);
long long ke_partial_count(const StepArgs& a);
cudaError_t launch_kinetic_energy_fp64(const double* f, double* out, double* part, const StepArgs& a,
                                       cudaStream_t s);

}  // namespace d2q37
