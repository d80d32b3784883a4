// FP64 collision of one site, factored for the FP64 pipe.
//
// Computes the BGK update (Sec. 3, eq. "lbequation", dt = 1)
//     f_i' = f_i + (f_i^eq - f_i) / tau
// with the moments of eq. "macro" (xi_i = c v_i):
//     rho = sum f,  rho u = sum xi f,  D rho T = sum |xi - u|^2 f = c^2 sum |v|^2 f - rho |u|^2,
// and the fourth-order Hermite equilibrium evaluated at the gravity-shifted
// u_s = u + tau g, T_s = T + tau (1 - tau) |g|^2 / D.  Written as a polynomial in
// s = xi_i . u_s with t = T_s - 1, U = |u_s|^2, q = |xi_i|^2 (D = 2):
//     f_i^eq / (w_i rho) = C0(q) + C1(q) s + C2(q) s^2 + s^3/6 + s^4/24,
//     C2 = 1/2 - U/4 + t (q - D - 4)/4,   C1 = 1 - U/2 + t (q - D - 2)/2,
//     C0 = 1 - U/2 + t (q - D)/2 + U^2/8 + t U (D + 2 - q)/4 + t^2 (q^2 - 2(D+2) q + D(D+2))/8.
// Work saved against the textbook form (Sec. 3 quotes ~7000 flops per site):
//   * moments are sums over opposite pairs P = f_v + f_-v, M = f_v - f_-v with integer
//     velocity weights grouped by value, accumulated in 64-bit fixed point on the
//     integer pipe;
//   * C0..C2 are per shell (8 values of q), pre-multiplied by omega w_s rho;
//   * each opposite pair shares the even part E(s^2) and odd part O(s):
//     f_v^eq = E + O, f_-v^eq = E - O.
#pragma once
#include "d2q37_model.cuh"

namespace d2q37 {

// X * 2^-k for a signed 64-bit X and -960 <= k <= 1022 (the result is then normal for
// every X != 0), rounded to nearest even: the value (double)X * 2^-k, formed on the integer
// pipe (count of leading zeros, shift, round, exponent) instead of the float64 pipe's
// conversion and product.
__host__ __device__ __forceinline__ double fix_to_double_rn(long long X, int k) {
  const unsigned long long s = (unsigned long long)(X >> 63);  // 0 or all ones
  const unsigned long long A = ((unsigned long long)X ^ s) - s;
#ifdef __CUDA_ARCH__
  const int lz = __clzll((long long)A);
#else
  const int lz = A ? __builtin_clzll(A) : 64;
#endif
  const unsigned long long M = A << (lz & 63);                  // leading one at bit 63
  const unsigned long long mant = M >> 11;                      // 53 bits with the leading one
  const unsigned long long rem = M & 0x7FFull;
  const unsigned long long up = (rem > 0x400ull) | ((rem == 0x400ull) & mant);
  // (e - 1) << 52 plus the 53-bit significand: its leading one, and a carry out of the
  // rounding, land in the exponent field
  const unsigned long long bits = ((unsigned long long)(1085 - lz - k) << 52) + mant + (up & 1ull);
  const unsigned long long r = A == 0 ? 0ull : bits | (s & 0x8000000000000000ull);
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)r);
#else
  double d;
  __builtin_memcpy(&d, &r, 8);
  return d;
#endif
}

// x * 2^k as an integer addition to x's exponent field: GB300 runs float64 at 1/64 of its
// float32 rate, and these kernels are bound by that pipe, so the exact scalings by powers
// of two move to the integer pipe.  The result equals the float64 product bit for bit when
// x and the result are normal.  Zeros, subnormals, infinities and NaNs are returned
// unchanged, and a result below the normal range becomes a zero of x's sign; neither case
// arises from a valid state (|k| <= 52 and the values scaled here are far inside the
// normal range, never near its top).
__host__ __device__ __forceinline__ double pow2_scale(double x, int k) {
#ifdef __CUDA_ARCH__
  const long long b = __double_as_longlong(x);
#else
  long long b;
  __builtin_memcpy(&b, &x, 8);
#endif
  const int e = (int)((b >> 52) & 0x7ff);
  const long long sign = b & (long long)0x8000000000000000ull;
  const long long scaled = e + k > 0 ? b + (long long)((unsigned long long)(long long)k << 52) : sign;
  const long long r = e == 0 || e == 0x7ff ? b : scaled;
#ifdef __CUDA_ARCH__
  return __longlong_as_double(r);
#else
  double d;
  __builtin_memcpy(&d, &r, 8);
  return d;
#endif
}

struct CollideConst {
  double omega;   // 1 / tau
  double om1;     // 1 - 1 / tau
  double cgx;     // c * tau * gx   (shift of c * u_x)
  double cgy;     // c * tau * gy
  double tshift;  // tau (1 - tau) |g|^2 / D - 1
};

// Moments in integer-velocity units: rho = sum f, (jx, jy) = sum v f, e = sum |v|^2 f.
//
// The sums run on the integer pipe, which is idle in this FP64-bound kernel: every f_i is
// rounded to 64-bit fixed point with 2^-52 resolution (round to nearest),
// the fixed-point sums are exact, and the four sums are converted back to float64.  The
// error is at most 37 * 2^-53 absolute per moment, the same order as a float64
// summation, and it is order-independent.  This takes 88 additions off the FP64 pipe.
// The signed 64-bit sums hold magnitudes below 2^11.  With every |f_i| < 8 the largest
// of them, sum |v_i|^2 |f_i|, stays below 216 * 8 = 1728 (216 = sum_i |v_i|^2), so the
// fixed-point sums are used only then; a site with a population of magnitude 8 or more
// (a dense state, rho above ~30, or an infinity or NaN) sums in plain float64 instead.
constexpr int DFIX = 52;
constexpr int kFixSumMaxExp = 1025;  // largest biased exponent with |f| < 8

// Also returns the biased exponent field E of v.
__device__ __forceinline__ long long to_fix52_e(double v, int& E) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  E = (int)((b >> 52) & 0x7ffu);
  const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);  // 53-bit mantissa
  const int sh = E - 1023;  // v * 2^52 = m * 2^sh
  const int l = sh < 0 ? 0 : (sh < 10 ? sh : 10);   // left shift (|v| >= 1)
  const int r = sh < 0 ? (-sh < 55 ? -sh : 55) : 0;  // right shift (|v| < 1), rounded
  const long long half = r > 0 ? (1LL << (r - 1)) : 0;
  long long x = ((m + half) >> r) << l;
  x = E == 0 ? 0 : x;
  const long long s = (long long)((long long)b >> 63);  // 0 or -1
  return (x ^ s) - s;
}

// The same four moments as plain float64 sums over opposite pairs (P = f_v + f_-v and
// M = f_v - f_-v, times the integer velocity weights).  Reads every f_i again through fget.
template <class Fget>
__device__ __forceinline__ void moments_float64(Fget&& fget, double& rho, double& jx, double& jy, double& e) {
  double R = fget(0), Ei = 0.0, Jx = 0.0, Jy = 0.0;
#pragma unroll
  for (int k = 1; k <= NPAIR; ++k) {
    const double a = fget(k), b = fget(k + NPAIR);
    const double P = a + b, M = a - b;
    R += P;
    Ei = fma((double)v2(k), P, Ei);
    if (rep_vx(k) != 0) Jx = fma((double)rep_vx(k), M, Jx);
    if (rep_vy(k) != 0) Jy = fma((double)rep_vy(k), M, Jy);
  }
  rho = R;
  e = Ei;
  jx = Jx;
  jy = Jy;
}

// Streaming accumulation: each opposite pair is converted and added to the four sums
// at once, so only the sums stay live (the products by the small integer velocity
// weights are exact integer shifts and adds).  on_exp(i, E) sees the exponent field of
// every f_i (for range checks of callers; a no-op otherwise).
// `fget(i)` returns f_i (an array read, or a load); it is called once per population.
// `wide(rho, jx, jy, e)` computes the moments of a site outside the fixed-point sums'
// range (moments_float64 on the same values, possibly out of line).
template <class Fget, class OnExp, class Wide>
__device__ __forceinline__ void moments_get_or(Fget&& fget, double& rho, double& jx, double& jy, double& e,
                                               OnExp&& on_exp, Wide&& wide) {
  int E0, Ea, Eb;
  long long R = to_fix52_e(fget(0), E0), Ei = 0, Jx = 0, Jy = 0;
  on_exp(0, E0);
  int emax = E0;
#pragma unroll
  for (int k = 1; k <= NPAIR; ++k) {
    const long long a = to_fix52_e(fget(k), Ea), b = to_fix52_e(fget(k + NPAIR), Eb);
    on_exp(k, Ea);
    on_exp(k + NPAIR, Eb);
    emax = max(emax, max(Ea, Eb));
    const long long P = a + b, M = a - b;
    R += P;
    Ei += (long long)v2(k) * P;
    if (rep_vx(k) != 0) Jx += (long long)rep_vx(k) * M;
    if (rep_vy(k) != 0) Jy += (long long)rep_vy(k) * M;
  }
  rho = fix_to_double_rn(R, DFIX);  // the fixed-point sums are their values times 2^52
  e = fix_to_double_rn(Ei, DFIX);
  jx = fix_to_double_rn(Jx, DFIX);
  jy = fix_to_double_rn(Jy, DFIX);
  // outside the fixed-point sums' range (see kFixSumMaxExp): plain float64 sums, which
  // also carry infinities and NaNs into the moments as any float64 sum would
  if (emax > kFixSumMaxExp) wide(rho, jx, jy, e);
}

template <class Fget, class OnExp>
__device__ __forceinline__ void moments_get(Fget&& fget, double& rho, double& jx, double& jy, double& e,
                                            OnExp&& on_exp) {
  moments_get_or(fget, rho, jx, jy, e, on_exp,
                 [&](double& r, double& x, double& y, double& en) { moments_float64(fget, r, x, y, en); });
}

__device__ __forceinline__ void moments_int(const double (&f)[Q], double& rho, double& jx, double& jy, double& e) {
  moments_get([&](int i) { return f[i]; }, rho, jx, jy, e, [](int, int) {});
}

// Equilibrium coefficients of one site.  R = omega * rho for a collision (the result is
// omega f^eq), or rho for a plain equilibrium.  Outputs per shell s = 0..7 the Horner
// coefficients K0..K4 of R w_s (C0 + C1 s + C2 s^2 + s^3/6 + s^4/24).
struct ShellCoef {
  double K0[8], K1[8], K2[8], K3[8], K4[8];
};

// C0..C2 as polynomials in q: C0 = a00 + a01 q + a02 q^2, C1 = a10 + a11 q, C2 = a20 + a21 q.
struct HermiteA {
  double a00, a01, a02, a10, a11, a20, a21;
};

__device__ __forceinline__ HermiteA hermite_a(double t, double U) {
  const double tU = t * U, t2 = t * t;
  HermiteA h;
  h.a00 = fma(0.125, U * U, fma(-0.5, U, 1.0) - t) + (tU + t2);
  const double t_half = pow2_scale(t, -1);  // t / 2, exactly
  h.a01 = fma(-0.25, tU, t_half) - t2;
  h.a02 = pow2_scale(t2, -3);
  h.a10 = fma(-0.5, U, 1.0) - pow2_scale(t, 1);
  h.a11 = t_half;
  h.a20 = fma(-0.25, U, 0.5) - 1.5 * t;
  h.a21 = pow2_scale(t, -2);
  return h;
}

// K0..K4 of shell s >= 1 (K0 only for s = 0).
__device__ __forceinline__ void shell_coefficient(const HermiteA& h, double R, int s, double& K0, double& K1,
                                                  double& K2, double& K3, double& K4) {
  const double q = q_shell(s);
  const double W = R * w_shell(s);
  K0 = s == 0 ? W * h.a00 : W * fma(fma(h.a02, q, h.a01), q, h.a00);
  K1 = W * fma(h.a11, q, h.a10);
  K2 = W * fma(h.a21, q, h.a20);
  K3 = W * (1.0 / 6.0);
  K4 = pow2_scale(K3, -2);  // W / 24: the double nearest 1/24 is that nearest 1/6 over 4
}

__device__ __forceinline__ void shell_coefficients(double R, double t, double U, ShellCoef& k) {
  const HermiteA h = hermite_a(t, U);
  k.K0[0] = (R * w_shell(0)) * h.a00;
#pragma unroll
  for (int s = 1; s < 8; ++s) shell_coefficient(h, R, s, k.K0[s], k.K1[s], k.K2[s], k.K3[s], k.K4[s]);
}

// s = v . (Ux, Uy) for integer v with |vx|, |vy| <= 3, from precomputed multiples.
struct Multiples {
  double X[4], Y[4];
};
__device__ __forceinline__ Multiples make_multiples(double Ux, double Uy) {
  Multiples m;
  m.X[0] = 0.0; m.X[1] = Ux; m.X[2] = pow2_scale(Ux, 1); m.X[3] = m.X[2] + Ux;
  m.Y[0] = 0.0; m.Y[1] = Uy; m.Y[2] = pow2_scale(Uy, 1); m.Y[3] = m.Y[2] + Uy;
  return m;
}
__device__ __forceinline__ double dot_v(const Multiples& m, int vxk, int vyk) {
  // vxk >= 0 for representatives
  if (vyk == 0) return m.X[vxk];
  if (vxk == 0) return vyk > 0 ? m.Y[vyk] : -m.Y[-vyk];
  return vyk > 0 ? m.X[vxk] + m.Y[vyk] : m.X[vxk] - m.Y[-vyk];
}

// Relaxation: out_i = om1 * f_i + R w_i P_i(s_i), for a whole site.  With om1 = 0 and
// R = rho this is the plain equilibrium.  `store(i, value)` receives each population.
// Per opposite pair: E = K0 + s^2 (K2 + s^2 K4), O = s R1 with R1 = K1 + s^2 K3, and
// E +- O = fma(+-s, R1, E), so the odd part costs no product of its own (8 FP64
// operations per pair).
template <class Fget, class Store>
__device__ __forceinline__ void relax_site_get(Fget&& fget, double om1, double R, double Ux, double Uy, double t,
                                               Store&& store) {
  const double U = fma(Ux, Ux, Uy * Uy) * (1.0 / C2);
  ShellCoef k;
  shell_coefficients(R, t, U, k);
  const Multiples m = make_multiples(Ux, Uy);
  store(0, fma(om1, fget(0), k.K0[0]));
#pragma unroll
  for (int j = 1; j <= NPAIR; ++j) {
    const int sh = shell(j);
    const double s = dot_v(m, rep_vx(j), rep_vy(j));
    const double s2 = s * s;
    const double E = fma(fma(k.K4[sh], s2, k.K2[sh]), s2, k.K0[sh]);
    const double R1 = fma(k.K3[sh], s2, k.K1[sh]);  // O = s R1, folded into E +- O
    store(j, fma(om1, fget(j), fma(s, R1, E)));
    store(j + NPAIR, fma(om1, fget(j + NPAIR), fma(-s, R1, E)));
  }
}

template <class Store>
__device__ __forceinline__ void relax_site(const double (&f)[Q], double om1, double R, double Ux, double Uy,
                                           double t, Store&& store) {
  relax_site_get([&](int i) { return f[i]; }, om1, R, Ux, Uy, t, store);
}

// Site scalars of the collision: R = omega rho, the gravity-shifted c u_s and t = T_s - 1.
struct SiteScalars {
  double R, Ux, Uy, t;
};

__device__ __forceinline__ SiteScalars scalars_from_moments(double rho, double jx, double jy, double e,
                                                          const CollideConst& cc) {
  const double inv_rho = 1.0 / rho;
  const double c2ir = C2 * inv_rho;
  const double Ux0 = jx * c2ir, Uy0 = jy * c2ir;              // c * u
  const double uu = fma(Ux0, Ux0, Uy0 * Uy0) * (1.0 / C2);     // |u|^2
  const double TD = fma(e, c2ir, -uu);                         // D T
  SiteScalars r;
  r.t = fma(TD, 1.0 / D, cc.tshift);                           // T_s - 1
  r.R = cc.omega * rho;
  r.Ux = Ux0 + cc.cgx;
  r.Uy = Uy0 + cc.cgy;
  return r;
}

template <class Fget, class OnExp>
__device__ __forceinline__ SiteScalars site_scalars(Fget&& fget, const CollideConst& cc, OnExp&& on_exp) {
  double rho, jx, jy, e;
  moments_get(fget, rho, jx, jy, e, on_exp);
  return scalars_from_moments(rho, jx, jy, e, cc);
}

// Full collision of one site (moments -> gravity shift -> equilibrium -> BGK).
template <class Store>
__device__ __forceinline__ void collide_site(const double (&f)[Q], const CollideConst& cc, Store&& store) {
  const SiteScalars v = site_scalars([&](int i) { return f[i]; }, cc, [](int, int) {});
  relax_site(f, cc.om1, v.R, v.Ux, v.Uy, v.t, store);
}

}  // namespace d2q37
