// C-ABI layer: argument validation, per-call launch parameters, dispatch.
// Declarations and the contract of every entry point: include/lbm_d2q37.h.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <cmath>

#include "../../include/lbm_d2q37.h"
#include "kernels.h"

using namespace d2q37;

namespace {

thread_local int32_t g_last_cuda_error = 0;

int32_t cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return LBM_OK;
  g_last_cuda_error = (int32_t)e;
  return LBM_ECUDA;
}

}  // namespace

bool d2q37::params_valid(const lbm_params* p) {
  if (!p) return false;
  if (p->lx < 4 || p->ly < 6) return false;
  if (!(p->tau > 0.5) || !(p->tau < 1e6)) return false;
  if (p->precision != LBM_FP64 && p->precision != LBM_FP32_SHIFTED && p->precision != LBM_FP64_FIXED &&
      p->precision != LBM_FP32_CONSERVED)
    return false;
  if (p->bc != LBM_BC_WALLS && p->bc != LBM_BC_PERIODIC_Y) return false;
  // grid.y = ceil(lx / 4) must fit in 65535; 37 * lx * pitch must fit the index math
  if (p->lx > 4 * 65535) return false;
  const double sites = (double)p->lx * (double)p->ly;
  if (sites * Q > (double)(1LL << 40)) return false;
  // one population plane (lx * pitch elements) must be addressable with 32-bit offsets
  if ((double)p->lx * (double)(((int64_t)p->ly + 31) / 32 * 32) >= 4294967296.0) return false;
  const double vals[] = {p->gx, p->gy, p->t_bottom, p->t_top, p->rho0, p->tau};
  for (double v : vals)
    if (!(v == v) || v > 1e300 || v < -1e300) return false;  // NaN / inf
  if (!(p->t_bottom > 0) || !(p->t_top > 0)) return false;
  return true;
}

namespace {

bool params_ok(const lbm_params* p) { return params_valid(p); }

int64_t pitch_of(const lbm_params* p) { return ((int64_t)p->ly + 31) / 32 * 32; }
bool fp32_storage(const lbm_params* p) {
  return p->precision == LBM_FP32_SHIFTED || p->precision == LBM_FP32_CONSERVED;
}
int64_t elem_size(const lbm_params* p) { return fp32_storage(p) ? 4 : 8; }
int64_t state_bytes(const lbm_params* p) { return (int64_t)Q * p->lx * pitch_of(p) * elem_size(p); }

bool aligned16(const void* ptr) { return ptr && ((uintptr_t)ptr % 16) == 0; }
bool aligned8(const void* ptr) { return ptr && ((uintptr_t)ptr % 8) == 0; }

bool overlap(const void* a, const void* b, int64_t bytes) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + (uintptr_t)bytes && y < x + (uintptr_t)bytes;
}

// Rest-state equilibrium per unit density at wall temperature T (fourth-order Hermite
// form at u = 0): w_i [1 + th (q - D)/2 + th^2 (q^2 - 2(D+2) q + D(D+2))/8], th = T - 1.
double wall_multiplier(int i, double T) {
  const double th = T - 1.0, q = C2 * (double)v2(i);
  return weight(i) * (1.0 + 0.5 * th * (q - D) + th * th * (q * q - 2.0 * (D + 2.0) * q + D * (D + 2.0)) / 8.0);
}

}  // namespace

StepArgs d2q37::make_step_args(const lbm_params* p) {
  StepArgs a;
  memset(&a, 0, sizeof(a));
  a.lx = p->lx;
  a.ly = p->ly;
  a.pitch = pitch_of(p);
  a.pop = (long long)p->lx * a.pitch;
  a.periodic = p->bc == LBM_BC_PERIODIC_Y;
  const double tau = p->tau;
  a.cc.omega = 1.0 / tau;
  a.cc.om1 = 1.0 - 1.0 / tau;
  a.cc.cgx = C * tau * p->gx;
  a.cc.cgy = C * tau * p->gy;
  a.cc.tshift = tau * (1.0 - tau) * (p->gx * p->gx + p->gy * p->gy) / D - 1.0;
  a.rho0 = p->rho0;
  a.f_omega = (float)a.cc.omega;
  a.f_om1 = 1.0f - a.f_omega;  // exact for 1/2 <= omega <= 2
  a.f_cgx = (float)a.cc.cgx;
  a.f_cgy = (float)a.cc.cgy;
  {
    double s = 0.0;  // sum_s w_s M_s with the float32 weights of the FP32 collision
    for (int i = 0; i < Q; ++i) s += (double)(float)weight(i) * (double)(vx(i) * vx(i));
    a.c2_iso = 1.0 / s;
    // the mass and energy correction's basis: all 37 populations, float32 weights
    double sw = 0.0, swq = 0.0;
    for (int i = 0; i < Q; ++i) {
      const double w = (double)(float)weight(i);
      sw += w;
      swq += w * v2(i);
    }
    const double m = swq / sw;
    double var = 0.0;
    for (int i = 0; i < Q; ++i) var += (double)(float)weight(i) * (v2(i) - m) * (v2(i) - m);
    a.corr_iw = 1.0 / sw;
    a.corr_m = m;
    a.corr_ivar = 1.0 / var;
  }
  a.corr_gx = p->gx / C;
  a.corr_gy = p->gy / C;
  a.corr_g2 = (p->gx * p->gx + p->gy * p->gy) / C2;
  a.conserve = p->precision == LBM_FP32_CONSERVED;
  a.f_corr_gx_hi = (float)a.corr_gx;
  a.f_corr_gx_lo = (float)(a.corr_gx - (double)a.f_corr_gx_hi);
  a.f_corr_gy_hi = (float)a.corr_gy;
  a.f_corr_gy_lo = (float)(a.corr_gy - (double)a.f_corr_gy_hi);
  a.f_corr_g2 = (float)a.corr_g2;
  a.f_corr_iw = (float)a.corr_iw;
  a.f_corr_m = (float)a.corr_m;
  a.f_corr_ivar = (float)a.corr_ivar;
  a.f_c2_iso = (float)a.c2_iso;
  int k = 0;  // 2^k <= rho0 < 2^(k+1), k >= 0
  while (k < 100 && p->rho0 >= std::ldexp(1.0, k + 1)) ++k;
  a.f_split_c1 = (float)std::ldexp(48.0, k);
  a.f_split_c2 = (float)std::ldexp(1.5, k - 18);
  a.f_split_s = (float)std::ldexp(1.0, 52 - k);
  a.f_fix_range = (float)std::ldexp(8.0, k);
  memcpy(&a.i_split_b1, &a.f_split_c1, sizeof(int));
  memcpy(&a.i_split_b2, &a.f_split_c2, sizeof(int));
  a.fix_back = std::ldexp(1.0, k - 52);
  a.f_fix_back = (float)a.fix_back;
  for (int i = 0; i < Q; ++i) {
    a.wall_b[i] = wall_multiplier(i, p->t_bottom);
    a.wall_t[i] = wall_multiplier(i, p->t_top);
    a.gb_scale[i] = (float)a.wall_b[i];
    a.gb_bias[i] = (float)(p->rho0 * (a.wall_b[i] - weight(i)));
    a.gt_scale[i] = (float)a.wall_t[i];
    a.gt_bias[i] = (float)(p->rho0 * (a.wall_t[i] - weight(i)));
  }
  return a;
}

cudaError_t d2q37::launch_step(const void* fin, void* fout, const StepArgs& a, int32_t precision, cudaStream_t s) {
  if (precision == LBM_FP32_SHIFTED || precision == LBM_FP32_CONSERVED)
    return launch_step_fp32((const float*)fin, (float*)fout, a, s);
  if (precision == LBM_FP64_FIXED) return launch_step_fix64((const double*)fin, (double*)fout, a, s);
  return launch_step_fp64((const double*)fin, (double*)fout, a, s);
}

namespace {

StepArgs make_args(const lbm_params* p) { return make_step_args(p); }

cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

}  // namespace

extern "C" {

int32_t lbm_version(void) { return 1; }

int32_t lbm_model(double* c, double* w37, int32_t* vx37, int32_t* vy37) {
  if (c) *c = C;
  for (int i = 0; i < Q; ++i) {
    if (w37) w37[i] = weight(i);
    if (vx37) vx37[i] = vx(i);
    if (vy37) vy37[i] = vy(i);
  }
  return LBM_OK;
}

int64_t lbm_pitch(const lbm_params* p) { return params_ok(p) ? pitch_of(p) : -1; }

int64_t lbm_buffer_bytes(const lbm_params* p) { return params_ok(p) ? state_bytes(p) : -1; }

int32_t lbm_init(const lbm_params* p, const double* rho, const double* ux, const double* uy, const double* T,
                 void* f, void* stream) {
  if (!params_ok(p) || !aligned8(rho) || !aligned8(ux) || !aligned8(uy) || !aligned8(T) || !aligned16(f))
    return LBM_EINVAL;
  const StepArgs a = make_args(p);
  if (fp32_storage(p))
    return cuda_status(launch_init_fp32(rho, ux, uy, T, (float*)f, a, as_stream(stream)));
  return cuda_status(launch_init_fp64(rho, ux, uy, T, (double*)f, a, as_stream(stream)));
}

int32_t lbm_step(const lbm_params* p, const void* fin, void* fout, void* stream) {
  if (!params_ok(p) || !aligned16(fin) || !aligned16(fout)) return LBM_EINVAL;
  if (overlap(fin, fout, state_bytes(p))) return LBM_EINVAL;
  const StepArgs a = make_args(p);
  return cuda_status(launch_step(fin, fout, a, p->precision, as_stream(stream)));
}

int32_t lbm_run(const lbm_params* p, void* fa, void* fb, int32_t n_steps, void* stream) {
  if (!params_ok(p) || !aligned16(fa) || !aligned16(fb) || n_steps < 0) return LBM_EINVAL;
  if (overlap(fa, fb, state_bytes(p))) return LBM_EINVAL;
  const StepArgs a = make_args(p);
  for (int32_t n = 0; n < n_steps; ++n) {
    const void* src = (n & 1) ? fb : fa;
    void* dst = (n & 1) ? fa : fb;
    const int32_t st = cuda_status(launch_step(src, dst, a, p->precision, as_stream(stream)));
    if (st != LBM_OK) return st;
  }
  return LBM_OK;
}

int32_t lbm_propagate(const lbm_params* p, const void* fin, void* ftmp, void* stream) {
  if (!params_ok(p) || !aligned16(fin) || !aligned16(ftmp) || p->precision != LBM_FP64) return LBM_EINVAL;
  if (overlap(fin, ftmp, state_bytes(p))) return LBM_EINVAL;
  const StepArgs a = make_args(p);
  return cuda_status(launch_propagate_fp64((const double*)fin, (double*)ftmp, a, as_stream(stream)));
}

int32_t lbm_propagate_push(const lbm_params* p, const void* fin, void* ftmp, void* stream) {
  if (!params_ok(p) || !aligned16(fin) || !aligned16(ftmp) || p->precision != LBM_FP64) return LBM_EINVAL;
  if (overlap(fin, ftmp, state_bytes(p))) return LBM_EINVAL;
  const StepArgs a = make_args(p);
  return cuda_status(launch_propagate_push_fp64((const double*)fin, (double*)ftmp, a, as_stream(stream)));
}

int32_t lbm_bc(const lbm_params* p, const void* fin, void* ftmp, void* stream) {
  if (!params_ok(p) || !aligned16(fin) || !aligned16(ftmp) || p->precision != LBM_FP64) return LBM_EINVAL;
  if (overlap(fin, ftmp, state_bytes(p))) return LBM_EINVAL;
  const StepArgs a = make_args(p);
  return cuda_status(launch_bc_fp64((const double*)fin, (double*)ftmp, a, as_stream(stream)));
}

int32_t lbm_collide(const lbm_params* p, const void* ftmp, void* fout, void* stream) {
  if (!params_ok(p) || !aligned16(ftmp) || !aligned16(fout) || p->precision != LBM_FP64) return LBM_EINVAL;
  if (overlap(ftmp, fout, state_bytes(p))) return LBM_EINVAL;
  const StepArgs a = make_args(p);
  return cuda_status(launch_collide_fp64((const double*)ftmp, (double*)fout, a, as_stream(stream)));
}

int32_t lbm_moments(const lbm_params* p, const void* f, double* rho, double* ux, double* uy, double* T,
                    void* stream) {
  if (!params_ok(p) || !aligned16(f) || !aligned8(rho) || !aligned8(ux) || !aligned8(uy) || !aligned8(T))
    return LBM_EINVAL;
  const StepArgs a = make_args(p);
  if (fp32_storage(p))
    return cuda_status(launch_moments_fp32((const float*)f, rho, ux, uy, T, a, as_stream(stream)));
  return cuda_status(launch_moments_fp64((const double*)f, rho, ux, uy, T, a, as_stream(stream)));
}

int64_t lbm_reduce_scratch_bytes(const lbm_params* p) {
  if (!params_ok(p)) return -1;
  return ke_partial_count(make_args(p)) * (int64_t)sizeof(double);
}

int32_t lbm_kinetic_energy(const lbm_params* p, const void* f, double* out, void* scratch, size_t scratch_bytes,
                           void* stream) {
  if (!params_ok(p) || !aligned16(f) || !aligned8(out) || !aligned8(scratch)) return LBM_EINVAL;
  const StepArgs a = make_args(p);
  if ((int64_t)scratch_bytes < ke_partial_count(a) * (int64_t)sizeof(double)) return LBM_EINVAL;
  if (fp32_storage(p))
    return cuda_status(launch_kinetic_energy_fp32((const float*)f, out, (double*)scratch, a, as_stream(stream)));
  return cuda_status(launch_kinetic_energy_fp64((const double*)f, out, (double*)scratch, a, as_stream(stream)));
}

int32_t lbm_simulate_host(const lbm_params* p, const double* rho_h, const double* ux_h, const double* uy_h,
                          const double* T_h, int32_t n_steps, double* rho_o, double* ux_o, double* uy_o,
                          double* T_o, void* fa, void* fb, double* fields, void* stream) {
  if (!params_ok(p) || !rho_h || !ux_h || !uy_h || !T_h || !rho_o || !ux_o || !uy_o || !T_o || !aligned8(fields) ||
      n_steps < 0)
    return LBM_EINVAL;
  cudaStream_t s = as_stream(stream);
  const size_t n = (size_t)p->lx * p->ly;
  const size_t bytes = n * sizeof(double);
  double* dev[4] = {fields, fields + n, fields + 2 * n, fields + 3 * n};
  const double* hin[4] = {rho_h, ux_h, uy_h, T_h};
  double* hout[4] = {rho_o, ux_o, uy_o, T_o};
  for (int k = 0; k < 4; ++k) {
    const int32_t st = cuda_status(cudaMemcpyAsync(dev[k], hin[k], bytes, cudaMemcpyHostToDevice, s));
    if (st != LBM_OK) return st;
  }
  int32_t st = lbm_init(p, dev[0], dev[1], dev[2], dev[3], fa, stream);
  if (st != LBM_OK) return st;
  st = lbm_run(p, fa, fb, n_steps, stream);
  if (st != LBM_OK) return st;
  st = lbm_moments(p, (n_steps & 1) ? fb : fa, dev[0], dev[1], dev[2], dev[3], stream);
  if (st != LBM_OK) return st;
  for (int k = 0; k < 4; ++k) {
    st = cuda_status(cudaMemcpyAsync(hout[k], dev[k], bytes, cudaMemcpyDeviceToHost, s));
    if (st != LBM_OK) return st;
  }
  return cuda_status(cudaStreamSynchronize(s));
}

const char* lbm_strerror(int32_t status) {
  switch (status) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument (parameters, pointer alignment, aliasing or sizes)";
    case LBM_ECUDA: return "CUDA launch or copy failed (see lbm_last_cuda_error)";
    case LBM_ETIMEOUT: return "device-side wait exceeded its iteration limit";
    case LBM_ENOMEM: return "out of memory";
    case LBM_ESIZE: return "lattice needs more than LBM_NOALLOC_MAX_TILES tiles of fixed scratch";
    default: return "unknown status";
  }
}

int32_t lbm_last_cuda_error(void) { return g_last_cuda_error; }

}  // extern "C"
