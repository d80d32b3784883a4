// Internal launch interface between the C-ABI layer (lbm_api.cu) and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lbm_d2q37.h"
#include "collide_fp64.cuh"

namespace d2q37 {

// Per-lattice scalars every site needs (small: kept in registers by the batched kernels).
struct StepScalars {
  int lx, ly;
  long long pitch;      // elements per y-column
  long long pop;        // elements per population plane = lx * pitch
  int periodic;         // 1: y wraps (test mode), 0: thermal walls
  CollideConst cc;
  double rho0;          // FP32 shifted storage: g_i = f_i - w_i rho0
  // Float copies of cc for the FP32 collision.  Their rounding must not bias the
  // collision: a relative bias e of the equilibrium's momentum multiplies the momentum by
  // (1 + omega e) every step, which compounds over a run.  So f_om1 = 1 - f_omega exactly
  // (for 1/2 <= omega <= 2), and the velocity is scaled by c2_iso = 1 / sum_s w_s M_s with
  // the float32 shell weights w_s the collision uses (M_s = sum of vx^2 over shell s;
  // exactly c^2 with exact weights), instead of c^2.  (The gravity shift's rounding only
  // adds a bias of the forcing, about 6e-8 of it, which does not compound.)
  float f_omega, f_om1, f_cgx, f_cgy;
  double c2_iso;
  // FP32_CONSERVED: gravity over c (gx / c, gy / c) and |g|^2 / c^2 (with the momentum,
  // the energy the collision adds, in integer-velocity units), and the mass and energy
  // correction's basis over all 37 populations with the float32 weights: 1 / sum w,
  // m = sum w |v|^2 / sum w and 1 / sum w (|v|^2 - m)^2
  double corr_gx, corr_gy, corr_g2, corr_iw, corr_m, corr_ivar;
  // float copies for the correction's float32 arithmetic (gravity over c as hi + lo pairs)
  float f_corr_gx_hi, f_corr_gx_lo, f_corr_gy_hi, f_corr_gy_lo, f_corr_g2, f_corr_iw, f_corr_m, f_corr_ivar,
      f_c2_iso;
  int conserve;  // 1 for LBM_FP32_CONSERVED
  // FP32 moment sums: of g_i 2^(52-k), 2^k <= rho0 < 2^(k+1) (k >= 0), valid for
  // |g_i| < f_fix_range = 8 * 2^k; split constants 48 * 2^k, 1.5 * 2^(k-18), 2^(52-k)
  // (step_fp32.cuh); fix_back = 2^(k-52) turns the sums into moments
  float f_split_c1, f_split_c2, f_split_s, f_fix_range, f_fix_back;
  int i_split_b1, i_split_b2;  // bit patterns of f_split_c1, f_split_c2
  double fix_back;
};

// Wall tables, read only by the warps next to a wall.
struct StepWalls {
  double wall_b[Q];     // w_i P_i(T_bottom): ghost value = rho_w * wall_b[i]
  double wall_t[Q];     // w_i P_i(T_top)
  float gb_scale[Q];    // ghost deviation = drho_w * gb_scale[i] + gb_bias[i]  (bottom wall)
  float gb_bias[Q];     //   with gb_scale = w_i P_i(T_b), gb_bias = w_i rho0 (P_i(T_b) - 1)
  float gt_scale[Q];    // same for the top wall
  float gt_bias[Q];
};

// Everything a site kernel needs, passed by value as the kernel parameter.
struct StepArgs : StepScalars, StepWalls {};

cudaError_t launch_step_fp64(const double* fin, double* fout, const StepArgs& a, cudaStream_t s);
cudaError_t launch_step_fix64(const double* fin, double* fout, const StepArgs& a, cudaStream_t s);
cudaError_t launch_propagate_fp64(const double* fin, double* ftmp, const StepArgs& a, cudaStream_t s);
cudaError_t launch_propagate_push_fp64(const double* fin, double* ftmp, const StepArgs& a, cudaStream_t s);
cudaError_t launch_bc_fp64(const double* fin, double* ftmp, const StepArgs& a, cudaStream_t s);
cudaError_t launch_collide_fp64(const double* ftmp, double* fout, const StepArgs& a, cudaStream_t s);
cudaError_t launch_init_fp64(const double* rho, const double* ux, const double* uy, const double* T, double* f,
                             const StepArgs& a, cudaStream_t s);
cudaError_t launch_moments_fp64(const double* f, double* rho, double* ux, double* uy, double* T,
                                const StepArgs& a, cudaStream_t s);
long long ke_partial_count(const StepArgs& a);
// Sums n doubles of part (one block, fixed order) into *out.
cudaError_t launch_reduce_sum(const double* part, long long n, double* out, cudaStream_t s);
cudaError_t launch_kinetic_energy_fp64(const double* f, double* out, double* part, const StepArgs& a,
                                       cudaStream_t s);

// Parameter validation and launch arguments shared by the C-ABI files (lbm_api.cu).
bool params_valid(const lbm_params* p);
StepArgs make_step_args(const lbm_params* p);
cudaError_t launch_step(const void* fin, void* fout, const StepArgs& a, int32_t precision, cudaStream_t s);

// FP32 shifted-deviation storage
cudaError_t launch_step_fp32(const float* fin, float* fout, const StepArgs& a, cudaStream_t s);
cudaError_t launch_init_fp32(const double* rho, const double* ux, const double* uy, const double* T, float* f,
                             const StepArgs& a, cudaStream_t s);
cudaError_t launch_moments_fp32(const float* f, double* rho, double* ux, double* uy, double* T,
                                const StepArgs& a, cudaStream_t s);
cudaError_t launch_kinetic_energy_fp32(const float* f, double* out, double* part, const StepArgs& a,
                                       cudaStream_t s);

}  // namespace d2q37
