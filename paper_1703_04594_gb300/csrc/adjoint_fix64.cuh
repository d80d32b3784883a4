// Vector-Jacobian product of the equilibrium in 64-bit fixed point (the adjoint's
// counterpart of collide_fix64.cuh).
//
// The VJP of f^eq_i = w_i rho P_i(s_i, U, t) against the adjoint vector mu (adjoint.cu,
// eq_vjp_pairs) costs ~32 float64 operations per opposite pair, which bounds the adjoint
// step by GB300's float64 pipe.  Here the per-shell polynomial coefficients, the per-pair
// polynomial values (P, dP/ds, dP/dU, dP/dt for the even and odd parts) and their
// contraction with mu run in fixed point on the integer pipes; only the site scalars and
// the final combination stay in float64.
//
// Formats.  mu is block floating point: every mu_i of the site is scaled by the same power
// of two, chosen from the largest exponent among the 37 values so that |mu'| < 2^57.
// Polynomial values have 59 fraction bits (all below 16 in the range of the path), s has
// 63 and s^2 62 (as in the forward path).  A product of mu' with a polynomial value keeps
// the high 64 bits, mu' P / 32; sums over a shell are multiplied by the shell weight w_s
// (64 fraction bits) and the four results are converted back to float64 with the block
// exponent.  The sums' unit is 2^-52 to 2^-51 of max_i |mu_i|; each high product rounds
// down by less than one unit, half a unit on average, which the sums add back (+1 per
// two products, +4 for the eight shell products), so a result carries an unbiased error
// of a few units, comparable to the float64 rounding of the same sums.  (Uncompensated,
// that bias is the same sign at every site and adds up in dL/dtau.)
//
// Range: |c u_s,x|, |c u_s,y| < 0.15 and |t| < 0.25 (as the forward path) and mu finite
// with max_i |mu_i| in [2^-922, 2^876] (or all zero); other sites use the float64 VJP.
#pragma once
#include "collide_fix64.cuh"

namespace d2q37 {

// Per-shell constants: q = c^2 |v|^2 (59 fraction bits), q^2 (55), (q - D - 4)/4 (61),
// (q - D - 2)/2 (60), w_s (64, unsigned).
struct AdjShellFix {
  long long q, q2, kq1, kq2;
  unsigned long long w;
};
__host__ __device__ constexpr long long fx_signed_const(double v, int k) {
  return v >= 0.0 ? (long long)fx_const(v, 1.0, k) : -(long long)fx_const(-v, 1.0, k);
}
#define LBM_ADJ_SHELL(s)                                                                          \
  {                                                                                               \
    s ? (long long)fx_const(q_shell(s), 1.0, 59) : 0LL,                                           \
        s ? (long long)fx_const(q_shell(s), q_shell(s), 55) : 0LL,                                \
        fx_signed_const((q_shell(s) - D - 4.0) / 4.0, 61), fx_signed_const((q_shell(s) - D - 2.0) / 2.0, 60), \
        fx_const(w_shell(s), 1.0, 64)                                                             \
  }
static __constant__ AdjShellFix c_adj_shell[8] = {LBM_ADJ_SHELL(0), LBM_ADJ_SHELL(1), LBM_ADJ_SHELL(2),
                                                  LBM_ADJ_SHELL(3), LBM_ADJ_SHELL(4), LBM_ADJ_SHELL(5),
                                                  LBM_ADJ_SHELL(6), LBM_ADJ_SHELL(7)};
#undef LBM_ADJ_SHELL

constexpr unsigned long long kInv6 = 3074457345618258603ull;   // round(2^64 / 6)
constexpr unsigned long long kInv24 = 768614336404564651ull;   // round(2^64 / 24)

// Sums of the VJP before the site factors: G = {Grho, sum w v_x X, sum w v_y X, sum w W,
// sum w T} (see eq_vjp_pairs in adjoint.cu for X, W, T), as float64.
struct VjpSums {
  double Gr, Ax, Ay, Wu, Gt;
};

__device__ __forceinline__ bool zero_sums(VjpSums& out) {
  out = VjpSums{0.0, 0.0, 0.0, 0.0, 0.0};
  return true;
}

// Returns false (and leaves `out` untouched) when the site is outside the fixed-point range.
// `mu(i)` returns mu_i; it is called twice per population (a scan for the block exponent,
// then the conversion).
template <class Mu>
__device__ __forceinline__ bool eq_vjp_sums_fix(double usx, double usy, double t, Mu&& mu, VjpSums& out) {
  const double Uxd = C * usx, Uyd = C * usy;
  const long long kU = 0x3FC3333333333333LL, kT = 0x3FD0000000000000LL, kA = 0x7FFFFFFFFFFFFFFFLL;
  if ((__double_as_longlong(Uxd) & kA) >= kU || (__double_as_longlong(Uyd) & kA) >= kU ||
      (__double_as_longlong(t) & kA) >= kT)
    return false;
  // block exponent of mu
  unsigned emax = 0;
#pragma unroll 1
  for (int i = 0; i < Q; ++i) {
    const unsigned e = (unsigned)((unsigned long long)__double_as_longlong(mu(i)) >> 52) & 0x7ffu;
    emax = e > emax ? e : emax;
  }
  // inf or NaN; or magnitudes whose sums could leave the normal float64 range
  if (emax >= 1900u || emax < 100u) return emax == 0u ? zero_sums(out) : false;
  const int kmu = 1079 - (int)emax;  // |mu| < 2^(emax - 1022)  =>  |mu 2^kmu| < 2^57
  bool unused = false;
  const long long X1 = fx_from_double(Uxd, 63, 64, unused), Y1 = fx_from_double(Uyd, 63, 64, unused);
  // the forward coefficients of c0, c1, c2 (collide_fix64.cuh), and those in q of dP/dU and
  // dP/dt at s = 0:  pue0 = b0 + b1 q,  pt0 = p0 + p1 q + p2 q^2
  const HermiteFix h = hermite_fix(X1, Y1, t);
  const long long U62 = h.U62, t63 = h.t63;
  const long long a00 = h.a00, a01 = h.a01, a02 = h.a02, a10 = h.a10, a11 = h.a11, a20 = h.a20;
  const long long a21 = h.a11;                                                                   // 66
  const long long b0 = -(1LL << 60) + (U62 >> 3) + (t63 >> 2);                                   // 61
  const long long b1 = -t63;                                                                     // 65
  const long long p0 = -(1LL << 61) + (U62 >> 1) + (t63 >> 1);                                   // 61
  const long long p1 = (1LL << 60) - (U62 >> 3) - (t63 >> 1);                                    // 61
  const long long p2 = t63 * 2;                                                                  // 66
  long long Gr = 0, Ax = 0, Ay = 0, Wu = 0, Gt = 0;
  int cur = -1;
  long long c0 = 0, c1 = 0, c2 = 0, pue0 = 0, pt0 = 0, kq1 = 0, kq2 = 0;
  unsigned long long w = 0;
  long long Rs = 0, Axs = 0, Ays = 0, Ws = 0, Ts = 0;
  const auto flush = [&]() {
    Gr += fx_mulhi_su(Rs, w);
    Ax += fx_mulhi_su(Axs, w);
    Ay += fx_mulhi_su(Ays, w);
    Wu += fx_mulhi_su(Ws, w);
    Gt += fx_mulhi_su(Ts, w);
    Rs = Axs = Ays = Ws = Ts = 0;
  };
  {  // rest population: s = 0, only E = c0, dP/dU = pue0 and dP/dt = pt0 at q = 0
    const long long m = fx_from_double(mu(0), kmu, 64, unused);
    const AdjShellFix& c = c_adj_shell[0];
    Rs = fx_mulhi(m, a00 >> 2);       // 59 fraction bits each
    Ws = fx_mulhi(m, b0 >> 2);
    Ts = fx_mulhi(m, p0 >> 2);
    w = c.w;
    flush();
  }
#pragma unroll 1
  for (int k = 1; k <= NPAIR; ++k) {
    const PairFix pk = c_pair_fix[k];
    if (pk.sh != cur) {  // uniform across the warp
      if (cur > 0) flush();
      cur = pk.sh;
      const AdjShellFix& c = c_adj_shell[cur];
      const unsigned long long q = (unsigned long long)c.q, q2 = (unsigned long long)c.q2;
      // values at 59 fraction bits: q (59) x a (65) -> 60, q^2 (55) x a (69) -> 60, ...
      c0 = (a00 >> 2) + (fx_mulhi_su(a01, q) >> 1) + (fx_mulhi_su(a02, q2) >> 1);
      c1 = (a10 >> 3) + (fx_mulhi_su(a11, q) >> 1);
      c2 = (a20 >> 4) + (fx_mulhi_su(a21, q) >> 2);
      pue0 = (b0 >> 2) + (fx_mulhi_su(b1, q) >> 1);
      pt0 = (p0 >> 2) + fx_mulhi_su(p1, q) * 8 + fx_mulhi_su(p2, q2) * 4;
      kq1 = c.kq1;
      kq2 = c.kq2;
      w = c.w;
    }
    const long long s = pk.vx * X1 + pk.vy * Y1;                                   // 63
    const unsigned long long as = (unsigned long long)(s < 0 ? -s : s);
    const unsigned long long s2 = fx_umulhi(as, as);                                // 62
    const long long h24 = (long long)(fx_umulhi(s2, kInv24) >> 3);                  // s^2/24, 59
    const long long h6 = (long long)(fx_umulhi(s2, kInv6) >> 3);                    // s^2/6, 59
    const long long E = c0 + fx_mulhi_su(c2 + h24, s2) * 4;                          // 57 -> 59
    const long long O = fx_mulhi(c1 + h6, s) * 2;                                    // 58 -> 59
    const long long Pse = c1 + (long long)(s2 >> 4);                                 // + s^2/2
    const long long Pso = fx_mulhi(2 * c2 + h6, s) * 2;                              // s (2 c2 + s^2/6)
    const long long PUe = pue0 - (long long)(s2 >> 5);                               // - s^2/4
    const long long PUo = -(s >> 5);                                                 // - s/2
    const long long Pte = pt0 + fx_mulhi_su(kq1, s2);                                // + (q-D-4)/4 s^2
    const long long Pto = fx_mulhi(s, kq2);                                          // (q-D-2)/2 s
    const long long mp = fx_from_double(mu(k), kmu, 64, unused);
    const long long mm = fx_from_double(mu(k + NPAIR), kmu, 64, unused);
    const long long S = mp + mm, Dm = mp - mm;
    // each high product rounds down, half a unit low on average: + 1 per two products
    // (without it the bias, ~2^-51 max|mu| per site, adds up over the sites of dL/dtau)
    Rs += fx_mulhi(S, E) + fx_mulhi(Dm, O) + 1;
    const long long X = fx_mulhi(Dm, Pse) + fx_mulhi(S, Pso) + 1;
    Axs += pk.vx * X;
    Ays += pk.vy * X;
    Ws += fx_mulhi(S, PUe) + fx_mulhi(Dm, PUo) + 1;
    Ts += fx_mulhi(S, Pte) + fx_mulhi(Dm, Pto) + 1;
  }
  flush();
  // the eight shell products of each sum (one per flush) likewise
  Gr += 4;
  Ax += 4;
  Ay += 4;
  Wu += 4;
  Gt += 4;
  // mu' P / 32 with mu' = mu 2^kmu: the sums are their values times 2^(kmu - 5)
  const int k = kmu - 5;
  // -826 < k <= 974: on the integer pipe, rounded to nearest even
  out.Gr = fix_to_double_rn(Gr, k);
  out.Ax = fix_to_double_rn(Ax, k);
  out.Ay = fix_to_double_rn(Ay, k);
  out.Wu = fix_to_double_rn(Wu, k);
  out.Gt = fix_to_double_rn(Gt, k);
  return true;
}

}  // namespace d2q37
