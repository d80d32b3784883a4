// FP64 collision with the equilibrium polynomial and the relaxation in 64-bit fixed point.
//
// The same update as collide_site (Sec. 3, eq. "lbequation"; equilibrium and moments as in
// collide_fp64.cuh), with a different split of the work between the GPU's pipes.  The site
// scalars (moments, 1/rho, u, T and the gravity shift) stay in float64.  Everything after
// them runs in signed 64-bit fixed point on the integer pipes: the Hermite coefficients
// a_jk and their products with omega rho, the shell coefficients K0..K3 of
// omega rho w_s (C0 + C1 s + C2 s^2 + s^3/6 + s^4/24), and for each opposite pair
// s = xi . u_s, s^2, h = K3 s^2, the odd part O = s (K1 + h), the even part
// E = K0 + s^2 (K2 + h/4) and f_+/-' = (1 - omega) f_+/- + E +/- O.
//
// Formats.  Shell s is scaled by 2^e_s with w_s 2^e_s in [0.5, 1), so every scaled
// population and coefficient is of order rho whatever the weight.  A product keeps the
// high 64 bits of the 128-bit result (a truncation).  Each quantity has the number of
// fraction bits that makes its products land on their consumers' binary points with no
// shift:
//   outputs, E, O, K0, (1 - omega) f   58  (|v| < 32)      K2, K2 + h/4      60
//   K1, h = K3 s^2, K1 + h             59                  K3 61
//   s 63, s^2 62, |1 - omega| 63, f 59 + e_s
// Each output carries a few units of 2^-58 relative to its scaled size, below the 2^-53
// rounding unit of a float64 result.  The truncations (each -1/2 unit on average) are
// re-centred by small constant offsets to within half a unit of 2^-58, far below the
// systematic error that the float64 weights themselves put on mass conservation.
//
// Range.  The path is taken for sites with 2^-7 <= f_i 2^e_s < 8 for all i,
// 0 < omega rho < 3, |c u_s,x| and |c u_s,y| below 0.15 (so |s| < 0.6) and
// |T_s - 1| < 0.25; then every intermediate stays inside its format.  All other sites (and
// NaNs) take the float64 collision of collide_site, so results never depend on the range.
#pragma once
#include "collide_fp64.cuh"
#include "fixed64.cuh"

namespace d2q37 {

__host__ __device__ constexpr int shell_exp(int s) {
  constexpr int t[8] = {2, 3, 4, 6, 7, 9, 11, 11};
  return t[s];
}

// Compile-time fixed-point constants from the model's float64 constants, computed exactly
// in integers: a positive double is m 2^x with an integer m < 2^53.
struct DoubleParts {
  unsigned long long m;
  int x;
};
__host__ __device__ constexpr DoubleParts double_parts(double v) {  // v > 0, finite
  int x = 0;
  while (v >= 9007199254740992.0) { v *= 0.5; ++x; }
  while (v < 4503599627370496.0) { v *= 2.0; --x; }
  return DoubleParts{(unsigned long long)v, x};
}
// round(a b 2^k / d) for positive doubles a, b and a positive integer d (half up); the
// exact product of the two 53-bit significands fits 106 bits.
__host__ __device__ constexpr unsigned long long fx_const(double a, double b, int k, unsigned d = 1) {
  const DoubleParts pa = double_parts(a), pb = double_parts(b);
  const unsigned __int128 p = (unsigned __int128)pa.m * pb.m;
  const int sh = pa.x + pb.x + k;
  const unsigned __int128 n = sh >= 0 ? (p << sh) : ((p + ((unsigned __int128)1 << (-sh - 1))) >> (-sh));
  return (unsigned long long)((n + d / 2) / d);
}
// Shell constants with w' = w_s 2^e_s (signed formats need values below 2^63):
//   cw = w' (Q0.63), cq = w' q_s (Q4.59), cq2 = w' q_s^2 (Q8.55, with q_s^2 rounded to
//   64 bits first), cw6 = w' / 6 (unsigned Q0.64).
__host__ __device__ constexpr long long shell_cw(int s) {
  return (long long)fx_const(w_shell(s), 1.0, shell_exp(s) + 63);
}
__host__ __device__ constexpr long long shell_cq(int s) {
  return (long long)fx_const(w_shell(s), q_shell(s), shell_exp(s) + 59);
}
__host__ __device__ constexpr long long shell_cq2(int s) {
  // round(w' q q 2^55): the 106-bit product w' q is rounded to 64 significant bits, then
  // multiplied by q exactly (117 bits)
  const DoubleParts pw = double_parts(w_shell(s)), pq = double_parts(q_shell(s));
  unsigned __int128 p = (unsigned __int128)pw.m * pq.m;
  int x = pw.x + pq.x;
  while (p >= ((unsigned __int128)1 << 64)) {
    p = (p + 1) >> 1;
    ++x;
  }
  const unsigned __int128 p3 = p * pq.m;
  const int sh = x + pq.x + shell_exp(s) + 55;  // negative for every shell
  return (long long)((p3 + ((unsigned __int128)1 << (-sh - 1))) >> (-sh));
}
__host__ __device__ constexpr unsigned long long shell_cw_div(int s, unsigned d) {
  return fx_const(w_shell(s), 1.0, shell_exp(s) + 64, d);
}

// The tables, evaluated by the compiler (constexpr locals must be constant expressions), so
// kernels only ever read literals.
__host__ __device__ constexpr long long kCw(int s) {
  constexpr long long t[8] = {shell_cw(0), shell_cw(1), shell_cw(2), shell_cw(3),
                              shell_cw(4), shell_cw(5), shell_cw(6), shell_cw(7)};
  return t[s];
}
__host__ __device__ constexpr long long kCq(int s) {
  constexpr long long t[8] = {0, shell_cq(1), shell_cq(2), shell_cq(3), shell_cq(4), shell_cq(5), shell_cq(6),
                              shell_cq(7)};
  return t[s];
}
__host__ __device__ constexpr long long kCq2(int s) {
  constexpr long long t[8] = {0,            shell_cq2(1), shell_cq2(2), shell_cq2(3),
                              shell_cq2(4), shell_cq2(5), shell_cq2(6), shell_cq2(7)};
  return t[s];
}
__host__ __device__ constexpr unsigned long long kCw6(int s) {
  constexpr unsigned long long t[8] = {shell_cw_div(0, 6), shell_cw_div(1, 6), shell_cw_div(2, 6),
                                       shell_cw_div(3, 6), shell_cw_div(4, 6), shell_cw_div(5, 6),
                                       shell_cw_div(6, 6), shell_cw_div(7, 6)};
  return t[s];
}

// round(2^64 / c^2), exact from the float64 c^2 = m 2^x
__host__ __device__ constexpr unsigned long long inv_c2_64() {
  const DoubleParts p = double_parts(C2);
  const unsigned __int128 num = (unsigned __int128)1 << (64 - p.x);
  return (unsigned long long)((num + p.m / 2) / p.m);
}
constexpr unsigned long long kInvC2 = inv_c2_64();

// Per-pair data of representatives 1..18 as a constant-memory table (one uniform load per
// pair; cheaper in issue slots than unpacking the values from immediates).
struct PairFix {
  int vx, vy, v2, sh;
};
#define LBM_PAIR_FIX(j) \
  { rep_vx(j), rep_vy(j), rep_vx(j) * rep_vx(j) + rep_vy(j) * rep_vy(j), shell(j) }
static __constant__ PairFix c_pair_fix[NPAIR + 1] = {
    LBM_PAIR_FIX(0),  LBM_PAIR_FIX(1),  LBM_PAIR_FIX(2),  LBM_PAIR_FIX(3),  LBM_PAIR_FIX(4),
    LBM_PAIR_FIX(5),  LBM_PAIR_FIX(6),  LBM_PAIR_FIX(7),  LBM_PAIR_FIX(8),  LBM_PAIR_FIX(9),
    LBM_PAIR_FIX(10), LBM_PAIR_FIX(11), LBM_PAIR_FIX(12), LBM_PAIR_FIX(13), LBM_PAIR_FIX(14),
    LBM_PAIR_FIX(15), LBM_PAIR_FIX(16), LBM_PAIR_FIX(17), LBM_PAIR_FIX(18)};
#undef LBM_PAIR_FIX

// The Hermite coefficients of C0 = a00 + a01 q + a02 q^2, C1 = a10 + a11 q, C2 = a20 + a21 q
// (collide_fp64.cuh) in fixed point, from X1 = c u_s,x and Y1 = c u_s,y (63 fraction bits)
// and t = T_s - 1, each with the fraction bits (in brackets) that its size allows in the
// range of the fixed-point path (|X1|, |Y1| < 0.15, |t| < 0.25):
//   a00 = 1 - U/2 - t + U^2/8 + tU + t^2 [61]   a01 = t/2 - tU/4 - t^2 [65]   a02 = t^2/8 [69]
//   a10 = 1 - U/2 - 2t [62]   a11 = t/2 [65]   a20 = 1/2 - U/4 - 3t/2 [63]   a21 = t/4 [66]
// with U = |u_s|^2 = (Ux^2 + Uy^2) / c^2 [62]; a21 is the same integer as a11.
struct HermiteFix {
  long long U62, t63, a00, a01, a02, a10, a11, a20;
};

__device__ __forceinline__ HermiteFix hermite_fix(long long X1, long long Y1, double t) {
  bool unused = false;
  HermiteFix h;
  h.t63 = fx_from_double(t, 63, 64, unused);
  const unsigned long long ax = (unsigned long long)(X1 < 0 ? -X1 : X1), ay = (unsigned long long)(Y1 < 0 ? -Y1 : Y1);
  h.U62 = (long long)fx_umulhi(fx_umulhi(ax, ax) + fx_umulhi(ay, ay), kInvC2);
  const unsigned long long at = (unsigned long long)(h.t63 < 0 ? -h.t63 : h.t63);
  const long long tU = fx_mulhi_su(h.t63, (unsigned long long)h.U62);                             // 61
  const long long t2 = (long long)fx_umulhi(at, at);                                                // 62
  const long long U2 = (long long)fx_umulhi((unsigned long long)h.U62, (unsigned long long)h.U62);  // 60
  h.a00 = (1LL << 61) - (h.U62 >> 2) - (h.t63 >> 2) + (U2 >> 2) + tU + (t2 >> 1);
  h.a01 = h.t63 * 2 - tU * 4 - t2 * 8;
  h.a02 = t2 * 16;
  h.a10 = (1LL << 62) - (h.U62 >> 1) - h.t63;
  h.a11 = h.t63 * 2;
  h.a20 = (1LL << 62) - (h.U62 >> 1) - h.t63 - (h.t63 >> 1);
  return h;
}

// Positive float64 values order like their bit patterns.
constexpr long long kBitsR = 0x4008000000000000LL;  // 3.0
constexpr long long kBitsU = 0x3FC3333333333333LL;  // 0.15
constexpr long long kBitsT = 0x3FD0000000000000LL;  // 0.25
constexpr long long kAbs = 0x7FFFFFFFFFFFFFFFLL;

__device__ __forceinline__ bool fixed_range_ok(const SiteScalars& v) {
  const long long r = __double_as_longlong(v.R);
  return r > 0 && r < kBitsR && (__double_as_longlong(v.Ux) & kAbs) < kBitsU &&
         (__double_as_longlong(v.Uy) & kAbs) < kBitsU && (__double_as_longlong(v.t) & kAbs) < kBitsT;
}

}  // namespace d2q37
