// FP32 shifted-deviation storage: the state holds g_i = f_i - w_i rho0 as float.
//
// Precision split (same step as the FP64 path: propagate -> bc -> collide, Sec. 5):
//  * moments (eq. "macro") are accumulated in fixed point with 2^-52 resolution: every
//    stored float of magnitude >= 2^-29 splits exactly into three int32 parts (split3),
//    the integer sums are exact and order-independent (error <= 37 * 2^-53 from the tiny
//    values, the same order as a float64 accumulation), and the sums are then converted
//    to float64.  The values summed are g_i 2^-k with 2^k <= rho0 < 2^(k+1) (k >= 0), so
//    range and resolution follow the reference density.  The fixed-point sums hold
//    magnitudes below 2^11, and sum |v_i|^2 |g_i 2^-k| < 216 * 8 when every
//    |g_i| < 8 * 2^k: that is the storage range of the form, |f_i - w_i rho0| < 8 * 2^k,
//    between 4 rho0 and 8 rho0 for rho0 >= 1.  A site outside it, or holding an infinity
//    or NaN, gets NaN moments and so NaN in every population;
//  * density, energy and the temperature t = T_s - 1 (the equilibrium's temperature
//    terms) are formed in float64 from those sums; 1/rho is a float32 seed refined by one
//    float64 Newton step;
//  * velocity, the Hermite coefficients and the BGK relaxation run in float32, written in
//    deviation form  g_i' = (1 - 1/tau) g_i + (1/tau) (f_i^eq - w_i rho0),
//    f_i^eq - w_i rho0 = w_i [ (rho - rho0) + rho (P_i(s) - 1) ],
//    so float32 rounds deviations, not whole populations.
#pragma once
#include "step_fp64.cuh"

namespace d2q37 {



// Exact split of a float |v| < 16 * 2^k into three integers with
// v * 2^(52-k) = H * 2^34 + R * 2^11 + L (|H|, |R| <= 2^22, |L| <= 2^10), done with float
// additions of power-of-two constants so that it runs on the FMA pipe instead of the
// integer pipe (k is the lattice's scale exponent, StepScalars::f_fix_range; k = 0 for
// rho0 <= 1, and the constants are then 48, 1.5 * 2^-18 and 2^52):
//   h1 = fl(v + 48 * 2^k) lies in [32, 64) 2^k, where floats are spaced 2^(k-18) apart, so
//   it rounds v to a multiple of 2^(k-18), and within that binade the bit pattern grows by
//   one per 2^(k-18): H = bits(h1) - bits(48 * 2^k).  r1 = v - (h1 - 48 * 2^k) is exact
//   (|r1| <= 2^(k-19)).  The same with 1.5 * 2^(k-18) (binade [2^(k-18), 2^(k-17)), spacing
//   2^(k-41)) gives R and an exact rest r2, |r2| <= 2^(k-42), and one FMA with 1.5 * 2^23
//   rounds r2 * 2^(52-k) to the integer L.
// Floats of magnitude >= 2^(k-29) convert exactly; smaller ones are rounded at 2^(k-52).
struct Fix3 {
  int H, R, L;
};

// The split constants of one lattice: 48 * 2^k, 1.5 * 2^(k-18) and 2^(52-k), and the bit
// patterns of the first two.
struct SplitConst {
  float c1, c2, s;
  int b1, b2;
};

__device__ __forceinline__ Fix3 split3(float v, const SplitConst& k) {
  constexpr float C3 = 12582912.0f;  // 1.5 * 2^23
  const float h1 = __fadd_rn(v, k.c1);
  const float r1 = __fsub_rn(v, __fsub_rn(h1, k.c1));
  const float h2 = __fadd_rn(r1, k.c2);
  const float r2 = __fsub_rn(r1, __fsub_rn(h2, k.c2));
  const float h3 = __fmaf_rn(r2, k.s, C3);
  return {__float_as_int(h1) - k.b1, __float_as_int(h2) - k.b2, __float_as_int(h3) - __float_as_int(C3)};
}

// The first two parts of split3: v * 2^(41-k) ~ H * 2^23 + R, dropping the rest r2
// (|r2| <= 2^(k-42)).  Enough for sums that only need an absolute error far below float32
// rounding (37 values: below 2^(k-36)).
struct Fix2 {
  int H, R;
};

__device__ __forceinline__ Fix2 split2(float v, const SplitConst& k) {
  const float h1 = __fadd_rn(v, k.c1);
  const float r1 = __fsub_rn(v, __fsub_rn(h1, k.c1));
  const float h2 = __fadd_rn(r1, k.c2);
  return {__float_as_int(h1) - k.b1, __float_as_int(h2) - k.b2};
}

// Running sums of the collision's outputs (mass, sum |v|^2 f, sum vx f, sum vy f) in the
// two lanes of split2.
struct OutSums {
  int rH = 0, rR = 0, eH = 0, eR = 0, xH = 0, xR = 0, yH = 0, yR = 0;
  // one opposite pair (v, -v): the sum and difference of the two values' lanes
  __device__ __forceinline__ void add_pair(float a, float b, int vx, int vy, const SplitConst& k) {
    const Fix2 za = split2(a, k), zb = split2(b, k);
    const int PH = za.H + zb.H, PR = za.R + zb.R, MH = za.H - zb.H, MR = za.R - zb.R;
    const int q = vx * vx + vy * vy;
    rH += PH;
    rR += PR;
    eH += q * PH;
    eR += q * PR;
    xH += vx * MH;
    xR += vx * MR;
    yH += vy * MH;
    yR += vy * MR;
  }
  __device__ __forceinline__ void add_rest(float a, const SplitConst& k) {
    const Fix2 z = split2(a, k);
    rH += z.H;
    rR += z.R;
  }
};

__device__ __forceinline__ long long join2(int H, int R) { return ((long long)H << 23) + (long long)R; }

// Moments of the stored deviations: sum g, sum vx g, sum vy g, sum |v|^2 g.  The step
// uses the momentum in float32 (JT = float), the moments kernels in float64.
template <class JT>
struct DevMoments {
  double drho, de;
  JT jx, jy;
};

__device__ __forceinline__ long long join3(int H, int R, int L) {
  return ((long long)H << 34) + ((long long)R << 11) + (long long)L;
}

// Streaming: each opposite pair is split and added to the four sums at once, in three
// int32 lanes per sum.  The sums are of g_i 2^(52-k) with 2^k <= rho0 < 2^(k+1) (k = 0
// for rho0 < 2), so their range and resolution follow the reference density: with every
// |g_i| < 8 * 2^k no lane overflows (|sum| < 216 * 2^22 per lane)
// and the joined 64-bit sums stay below 2^63 (see the file header).  That is the storage
// range of the form, |g_i| < 8 * 2^k: a site holding a larger deviation, an infinity or a
// NaN gets NaN moments, so every population it produces is NaN.  (A float64 fallback for
// such sites does not fit the step's 80-register budget.)
// SCALED = false is the common case k = 0 (rho0 < 2), with every constant an immediate;
// SCALED = true reads the lattice's constants (a separate instantiation, so the common
// one keeps its registers).
// The four exact sums of v_i 2^(52-k) over the 37 values (the lattice's split constants):
// sum, sum |v|^2, sum vx, sum vy.
struct FixSums {
  long long R, E, X, Y;
};

template <bool SCALED>
__device__ __forceinline__ SplitConst split_const(const StepScalars& a) {
  constexpr SplitConst s0 = {48.0f, 5.7220458984375e-06f, 4503599627370496.0f, 0x42400000, 0x36c00000};
  return SCALED ? SplitConst{a.f_split_c1, a.f_split_c2, a.f_split_s, a.i_split_b1, a.i_split_b2} : s0;
}

__device__ __forceinline__ FixSums fix_sums(const float (&g)[Q], const SplitConst& s) {
  const Fix3 z = split3(g[0], s);
  int rH = z.H, rR = z.R, rL = z.L;
  int eH = 0, eR = 0, eL = 0, xH = 0, xR = 0, xL = 0, yH = 0, yR = 0, yL = 0;
#pragma unroll
  for (int k = 1; k <= NPAIR; ++k) {
    const Fix3 a = split3(g[k], s), b = split3(g[k + NPAIR], s);
    const int PH = a.H + b.H, PR = a.R + b.R, PL = a.L + b.L;
    const int MH = a.H - b.H, MR = a.R - b.R, ML = a.L - b.L;
    rH += PH;
    rR += PR;
    rL += PL;
    eH += v2(k) * PH;
    eR += v2(k) * PR;
    eL += v2(k) * PL;
    if (rep_vx(k) != 0) {
      xH += rep_vx(k) * MH;
      xR += rep_vx(k) * MR;
      xL += rep_vx(k) * ML;
    }
    if (rep_vy(k) != 0) {
      yH += rep_vy(k) * MH;
      yR += rep_vy(k) * MR;
      yL += rep_vy(k) * ML;
    }
  }
  return {join3(rH, rR, rL), join3(eH, eR, eL), join3(xH, xR, xL), join3(yH, yR, yL)};
}

// Every |g_i| < 8 * 2^k (false for an infinity or NaN): the storage range of the form.
template <bool SCALED>
__device__ __forceinline__ bool fix_in_range(const float (&g)[Q], const StepScalars& a) {
  const float range = SCALED ? a.f_fix_range : 8.0f;
  bool in_range = true;
#pragma unroll
  for (int i = 0; i < Q; ++i) in_range &= fabsf(g[i]) < range;
  return in_range;
}

// 2^(k-52): from the fixed-point sums back to moments.
template <bool SCALED>
__device__ __forceinline__ double fix_back(const StepScalars& a) {
  return SCALED ? a.fix_back : 1.0 / 4503599627370496.0;
}

template <class JT, bool SCALED>
__device__ __forceinline__ DevMoments<JT> moments_of(const FixSums& f, bool in_range, const StepScalars& a) {
  const double back = fix_back<SCALED>(a);
  const JT back_j = SCALED ? (JT)(sizeof(JT) == 4 ? a.f_fix_back : a.fix_back) : (JT)(1.0 / 4503599627370496.0);
  DevMoments<JT> r;
  r.drho = (double)f.R * back;
  r.de = (double)f.E * back;
  r.jx = (JT)f.X * back_j;
  r.jy = (JT)f.Y * back_j;
  if (!in_range) r.drho = __longlong_as_double(0x7FF8000000000000LL);  // rho, and so every output, NaN
  return r;
}

template <class JT, bool SCALED>
__device__ __forceinline__ DevMoments<JT> moments_fix(const float (&g)[Q], const StepScalars& a) {
  return moments_of<JT, SCALED>(fix_sums(g, split_const<SCALED>(a)), fix_in_range<SCALED>(g, a), a);
}

// Collision of one site in the precision split described at the top of the file.
//
// CONSERVE: restore the exact post-collision mass, momentum and energy after the float32
// arithmetic.  Float32 rounding in the equilibrium changes a site's mass, momentum and
// energy by a few units of 2^-24 of the deviations; conserved quantities are never relaxed
// away, so that noise accumulates and dominates the velocity error of long runs (mass and
// energy as pressure noise early on, momentum more and more as the flow develops).  The
// collision's exact post-collision values are known in closed form (eq. "lbequation" with
// the shifted equilibrium, omega tau = 1): mass unchanged, momentum J + rho g, energy
// E + rho (2 u.g + |g|^2).  The outputs are summed as they are formed (split2: absolute
// error below 2^-36, against rounding noise of ~1e-8), and the difference is put back along
// the first Hermite polynomials over all 37 populations,
// delta_i = w_i [alpha + beta . v_i + gamma (|v_i|^2 - m)], m = sum w |v|^2 / sum w: the
// shape of the equilibrium's own density, velocity and temperature response, which disturbs
// the other moments least.
template <bool SCALED, bool CONSERVE, class Store>
__device__ __forceinline__ void collide_site_fp32(float (&g)[Q], const StepScalars& a, Store&& store) {
  const SplitConst sc = split_const<SCALED>(a);
  const bool in_range = fix_in_range<SCALED>(g, a);
  const FixSums in = fix_sums(g, sc);
  const DevMoments<float> m = moments_of<float, SCALED>(in, in_range, a);
  // float64: density, energy, temperature
  const double drho = m.drho;
  const double rho = a.rho0 + drho;
  const double etot = m.de + a.rho0 * (D / C2);  // sum |v|^2 f
  const float rho_f = (float)rho;
  const float r_f = __frcp_rn(rho_f);
  const double r0 = (double)r_f;
  const double inv = fma(r0, fma(-rho, r0, 1.0), r0);
  // float32: velocity c u = c^2 j / rho
  // c u = c^2 j / rho with the velocity scale c2_iso in place of c^2 (see StepScalars):
  // with it the float32 equilibrium's first-order momentum is exactly rho u
  const float c2ir_f = (float)(a.c2_iso * inv);
  const float Ux0 = (float)m.jx * c2ir_f, Uy0 = (float)m.jy * c2ir_f;
  const float uu = fmaf(Ux0, Ux0, Uy0 * Uy0) * (float)(1.0 / C2);
  // t = T_s - 1 = (c^2 e / rho - |u|^2) / D + tau (1 - tau) |g|^2 / D - 1: the large part in
  // float64, the small |u|^2 / D correction in float32
  const float t = (float)fma(etot, C2 * inv * (1.0 / D), a.cc.tshift) - uu * (float)(1.0 / D);
  const float drho_f = (float)drho;
  // float32: Hermite coefficients in deviation form and relaxation
  const float Ux = Ux0 + a.f_cgx, Uy = Uy0 + a.f_cgy;
  const float U = fmaf(Ux, Ux, Uy * Uy) * (float)(1.0 / C2);
  const float om = a.f_omega, om1 = a.f_om1;
  const float tU = t * U, t2 = t * t;
  const float a00m1 = fmaf(0.125f, U * U, fmaf(-0.5f, U, -t)) + (tU + t2);   // a00 - 1
  const float a01 = fmaf(-0.25f, tU, 0.5f * t) - t2;
  const float a02 = 0.125f * t2;
  const float a10 = fmaf(-0.5f, U, 1.0f) - 2.0f * t;
  const float a11 = 0.5f * t;
  const float a20 = fmaf(-0.25f, U, 0.5f) - 1.5f * t;
  const float a21 = 0.25f * t;
  const float R = om * rho_f, Rd = om * drho_f;
  float K0[8], K1[8], K2[8], K3[8], K4[8];
  K0[0] = (float)w_shell(0) * fmaf(R, a00m1, Rd);
#pragma unroll
  for (int s = 1; s < 8; ++s) {
    const float q = (float)q_shell(s);
    const float ws = (float)w_shell(s);
    const float W = R * ws;
    K0[s] = fmaf(W, fmaf(fmaf(a02, q, a01), q, a00m1), Rd * ws);
    K1[s] = W * fmaf(a11, q, a10);
    K2[s] = W * fmaf(a21, q, a20);
    K3[s] = W * (1.0f / 6.0f);
    K4[s] = W * (1.0f / 24.0f);
  }
  float X[4] = {0.0f, Ux, Ux + Ux, 0.0f}, Y[4] = {0.0f, Uy, Uy + Uy, 0.0f};
  X[3] = X[2] + Ux;
  Y[3] = Y[2] + Uy;
  OutSums os;
  // CONSERVE holds the outputs in g (each g_i is dead once its output is formed)
  const auto out = [&](int i, float v) {
    if (CONSERVE) g[i] = v;
    else store(i, v);
  };
  out(0, fmaf(om1, g[0], K0[0]));
  if (CONSERVE) os.add_rest(g[0], sc);
#pragma unroll
  for (int j = 1; j <= NPAIR; ++j) {
    const int sh = shell(j), vxk = rep_vx(j), vyk = rep_vy(j);
    float s;
    if (vyk == 0) s = X[vxk];
    else if (vxk == 0) s = Y[vyk];
    else s = vyk > 0 ? X[vxk] + Y[vyk] : X[vxk] - Y[-vyk];
    const float s2 = s * s;
    const float E = fmaf(fmaf(K4[sh], s2, K2[sh]), s2, K0[sh]);
    const float O = s * fmaf(K3[sh], s2, K1[sh]);
    out(j, fmaf(om1, g[j], E + O));
    out(j + NPAIR, fmaf(om1, g[j + NPAIR], E - O));
    if (CONSERVE) os.add_pair(g[j], g[j + NPAIR], vxk, vyk, sc);
  }
  if constexpr (CONSERVE) {
    // What the outputs lack, in integers: the exact input sums (units of 2^(k-52)) minus the
    // output sums (split2, units of 2^(k-41)); then, in float32 (the differences are ~1e-8),
    // plus the forcing.  No float64 arithmetic: this form is otherwise bound by that pipe.
    const float backf = SCALED ? a.f_fix_back : 2.220446049250313e-16f;  // 2^(k-52)
    const float dM = (float)(in.R - (join2(os.rH, os.rR) << 11)) * backf;
    const float dX = (float)(in.X - (join2(os.xH, os.xR) << 11)) * backf;
    const float dY = (float)(in.Y - (join2(os.yH, os.yR) << 11)) * backf;
    const float dEs = (float)(in.E - (join2(os.eH, os.eR) << 11)) * backf;
    // momentum: + rho g / c (the constant as a float pair, so the forcing keeps its value);
    // energy: + 2 j.g / c + rho |g|^2 / c^2
    const float dJx = fmaf(rho_f, a.f_corr_gx_hi, fmaf(rho_f, a.f_corr_gx_lo, dX));
    const float dJy = fmaf(rho_f, a.f_corr_gy_hi, fmaf(rho_f, a.f_corr_gy_lo, dY));
    const float dE = fmaf(rho_f, a.f_corr_g2, fmaf(2.0f * m.jx, a.f_corr_gx_hi, fmaf(2.0f * m.jy, a.f_corr_gy_hi, dEs)));
    const float alpha = dM * a.f_corr_iw;
    const float mf = a.f_corr_m;
    const float gamma = fmaf(-dM, mf, dE) * a.f_corr_ivar;
    // sum_i w_i vx_i^2 = 1 / c2_iso for the float32 weights (see StepScalars)
    const float bx = a.f_c2_iso * dJx, by = a.f_c2_iso * dJy;
    store(0, g[0] + (float)w_shell(0) * fmaf(gamma, -mf, alpha));
#pragma unroll
    for (int j = 1; j <= NPAIR; ++j) {
      const float ws = (float)w_shell(shell(j));
      const float A = ws * fmaf(gamma, (float)v2(j) - mf, alpha);
      const float B = fmaf(ws * (float)rep_vx(j), bx, (ws * (float)rep_vy(j)) * by);
      store(j, g[j] + (A + B));
      store(j + NPAIR, g[j + NPAIR] + (A - B));
    }
  }
}

// Wall deviations sum_j g_j at (x_s, 0) and (x_s, ly-1) of the seven source columns
// (lanes 0..6 bottom, 8..14 top), summed in float64, broadcast to the warp.
template <class Ld>
__device__ __forceinline__ void wall_drho(const float* __restrict__ fin, int x, const StepScalars& a, float (&rb)[7],
                                          float (&rt)[7], Ld ld) {
  const int lane = threadIdx.x & 31;
  const int d = lane & 7;
  const int row = lane < 8 ? 0 : a.ly - 1;
  double r = 0.0;
  if (d < 7 && lane < 16) {
    const float* src = fin + (long long)wrap_index(x - (d - 3), a.lx) * a.pitch + row;
#pragma unroll
    for (int i = 0; i < Q; ++i) r += (double)ld(src + i * a.pop);
  }
  const float rf = (float)r;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    rb[j] = __shfl_sync(0xffffffffu, rf, j);
    rt[j] = __shfl_sync(0xffffffffu, rf, 8 + j);
  }
}


// One warp-strip of the FP32 shifted step (see step_fp64.cuh for the strip contract).
// SCALED: the lattice's reference density is 2 or more (see moments_fix); CONSERVE: the
// collision restores the exact conserved moments (collide_site_fp32).
template <bool PERIODIC, bool SCALED, bool CONSERVE, class Ld>
__device__ __forceinline__ void step_strip_fp32(const float* __restrict__ fin, float* __restrict__ fout,
                                                const StepScalars& a, const StepWalls& w, int x, int y0, Ld ld) {
  const int y = y0 + (threadIdx.x & 31);
  const bool active = y < a.ly;
  const int yc = active ? y : a.ly - 1;
  long long col[7];
#pragma unroll
  for (int d = 0; d < 7; ++d) col[d] = (long long)wrap_index(x - (d - 3), a.lx) * a.pitch;
  float g[Q];
  const bool wall_warp = !PERIODIC && (y0 < 3 || y0 + 32 > a.ly - 3);
  if (wall_warp) {
    float rb[7], rt[7];
    wall_drho(fin, x, a, rb, rt, ld);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int ys = yc - vy(i);
      const float* src = fin + i * a.pop + col[vx(i) + 3];
      if (vy(i) > 0 && ys < 0) g[i] = fmaf(rb[vx(i) + 3], w.gb_scale[i], w.gb_bias[i]);
      else if (vy(i) < 0 && ys >= a.ly) g[i] = fmaf(rt[vx(i) + 3], w.gt_scale[i], w.gt_bias[i]);
      else g[i] = ld(src + ys);
    }
  } else if (PERIODIC) {
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = ld(fin + i * a.pop + col[vx(i) + 3] + wrap_index(yc - vy(i), a.ly));
  } else {
    // Interior warps: a population plane's base (fin + i * pop) is the same for every thread;
    // the per-thread part is one of seven 32-bit offsets (column x_s, row yc), shifted by -vy_i.
    unsigned off[7];
#pragma unroll
    for (int d = 0; d < 7; ++d) off[d] = (unsigned)(col[d] + yc);
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = ld(fin + i * a.pop + (off[vx(i) + 3] - vy(i)));
  }
  if (!active) return;
  const unsigned self = (unsigned)((long long)x * a.pitch + y);
  collide_site_fp32<SCALED, CONSERVE>(g, a, [&](int i, float v) { __stcs(fout + i * a.pop + self, v); });
}

}  // namespace d2q37
