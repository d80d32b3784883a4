// One warp-strip of the fused FP64 step with the fixed-point relaxation of collide_fix64.cuh.
//
// Layout of the work, chosen for the integer pipes:
//   1. the 37 pull-gathered populations of the strip are copied global -> shared memory
//      with cp.async (no registers held while the loads are in flight);
//   2. moments: a rolled loop over opposite pairs reads shared memory and sums in 64-bit
//      fixed point (collide_fp64.cuh), checking the range of the fixed-point path;
//   3. site scalars in float64 (1/rho, u, T, gravity shift, Hermite coefficients);
//   4. relaxation: a rolled loop over opposite pairs re-reads shared memory and evaluates
//      the equilibrium polynomial and (1 - omega) f + omega f^eq in fixed point.
// Rolled loops keep the kernel's code small: the fully unrolled form of this arithmetic is
// ~8000 instructions per site, which thrashes the instruction cache.  Per-pair velocities
// and shells come from packed immediates, per-shell constants from a constant-memory table.
// Sites outside the fixed-point range take the float64 relaxation on the same staged values.
// Warps next to a wall (two strips per column) run the float64 strip of step_fp64.cuh.
#pragma once
#include "collide_fix64.cuh"
#include "step_fp64.cuh"

namespace d2q37 {

// Representatives 1..18 packed into 64-bit immediates: vx in 2 bits, vy + 3 and the shell in
// 3 bits each, pair j at bit (j - 1) times the width.
__host__ __device__ constexpr unsigned long long pack_pairs(int field) {
  unsigned long long r = 0;
  for (int j = 1; j <= NPAIR; ++j) {
    if (field == 0) r |= (unsigned long long)rep_vx(j) << (2 * (j - 1));
    if (field == 1) r |= (unsigned long long)(rep_vy(j) + 3) << (3 * (j - 1));
    if (field == 2) r |= (unsigned long long)shell(j) << (3 * (j - 1));
  }
  return r;
}
constexpr unsigned long long kPairVx = pack_pairs(0);
constexpr unsigned long long kPairVy = pack_pairs(1);
constexpr unsigned long long kPairShell = pack_pairs(2);

struct ShellFix {
  long long cw, cq, cq2;
  unsigned long long cw6, cw24;
  int e;  // shell scale exponent e_s
  int lim;  // largest exponent field with |f| 2^e_s < 8
};
#define LBM_SHELL_FIX(s) \
  { kCw(s), kCq(s), kCq2(s), kCw6(s), kCw24(s), shell_exp(s), 1025 - shell_exp(s) }
static __constant__ ShellFix c_shell_fix[8] = {LBM_SHELL_FIX(0), LBM_SHELL_FIX(1), LBM_SHELL_FIX(2),
                                               LBM_SHELL_FIX(3), LBM_SHELL_FIX(4), LBM_SHELL_FIX(5),
                                               LBM_SHELL_FIX(6), LBM_SHELL_FIX(7)};
#undef LBM_SHELL_FIX

// round(v 2^k) for a float64 v >= 0 with v 2^k < 2^62 (callers guarantee both); integer
// instructions only, round half up.  v 2^k = m 2^sh with the 53-bit significand m: the
// value is formed with one extra fraction bit, m 2^(sh + 1) = (m 2^11) >> (10 - sh), then
// rounded.  Values below half a unit (shifts past 63) give 0, as do zeros and subnormals.
__device__ __forceinline__ long long fx_from_nonneg(double v, int k) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int E = (int)(b >> 52);  // sign bit clear
  unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  m = E == 0 ? 0ull : m;
  const int r = 1085 - E - k;  // 10 - sh >= 1 when v 2^k < 2^62
  const unsigned long long t = r < 64 ? (m << 11) >> r : 0ull;
  return (long long)((t + 1) >> 1);
}

// 8-byte asynchronous global -> shared copy (sm_80+ LDGSTS), cached in L1.
__device__ __forceinline__ void cp_async8(double* smem_dst, const double* gmem_src) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Shared staging: one warp holds sf[i * 32 + lane] for its 32 sites.
constexpr int kFixWarps = 4;  // warps per block (block = 32 x 4 threads)

template <bool PERIODIC, class Ld>
__device__ __forceinline__ void step_strip_fix64(const double* __restrict__ fin, double* __restrict__ fout,
                                                 const StepScalars& a, const StepWalls& w, int x, int y0, Ld ld,
                                                 double* __restrict__ sf) {
  const bool wall_warp = !PERIODIC && (y0 < 3 || y0 + 32 > a.ly - 3);
  if (wall_warp) {
    step_strip_fp64<PERIODIC>(fin, fout, a, w, x, y0, ld);
    return;
  }
  const int lane = threadIdx.x & 31;
  const int y = y0 + lane;
  const bool active = y < a.ly;
  const int yc = active ? y : a.ly - 1;
  // 1. stage the pull-gather in shared memory
  {
    unsigned off[7];  // column x_s, row yc within a population plane (planes < 2^32 elements)
#pragma unroll
    for (int d = 0; d < 7; ++d) off[d] = (unsigned)((long long)wrap_index(x - (d - 3), a.lx) * a.pitch + yc);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double* src = PERIODIC ? fin + i * a.pop + (off[vx(i) + 3] - yc) + wrap_index(yc - vy(i), a.ly)
                                   : fin + i * a.pop + (off[vx(i) + 3] - vy(i));
      cp_async8(sf + i * 32 + lane, src);
    }
    cp_async_wait_all();
    __syncwarp();
  }
  sf += lane;
  // 2. moments in 64-bit fixed point, with the range check of the fixed-point path
  constexpr double S = 1.0 / 4503599627370496.0;  // 2^-52
  int E;
  long long R = to_fix52_e(sf[0], E), Ei = 0, Jx = 0, Jy = 0;
  bool out = E > 1025 - shell_exp(0);
  unsigned sign = (unsigned)(__double_as_longlong(sf[0]) >> 32);
#pragma unroll 1
  for (int k = 1; k <= NPAIR; ++k) {
    const int vxk = (int)((kPairVx >> (2 * (k - 1))) & 3);
    const int vyk = (int)((kPairVy >> (3 * (k - 1))) & 7) - 3;
    const int lim = c_shell_fix[(kPairShell >> (3 * (k - 1))) & 7].lim;
    const double fa = sf[k * 32], fb = sf[(k + NPAIR) * 32];
    int Ea, Eb;
    const long long va = to_fix52_e(fa, Ea), vb = to_fix52_e(fb, Eb);
    out |= (Ea > lim) | (Eb > lim);
    sign |= (unsigned)(__double_as_longlong(fa) >> 32) | (unsigned)(__double_as_longlong(fb) >> 32);
    const long long P = va + vb, M = va - vb;
    R += P;
    Ei += (long long)(vxk * vxk + vyk * vyk) * P;
    Jx += (long long)vxk * M;
    Jy += (long long)vyk * M;
  }
  out |= (sign >> 31) != 0;  // a negative population
  if (!active) return;
  // 3. site scalars in float64
  const SiteScalars v = scalars_from_moments((double)R * S, (double)Jx * S, (double)Jy * S, (double)Ei * S, a.cc);
  const unsigned self = (unsigned)((long long)x * a.pitch + y);
  const auto store = [&](int i, double val) { __stcs(fout + i * a.pop + self, val); };
  if (out || !fixed_range_ok(v)) {
    relax_site_get([&](int i) { return sf[i * 32]; }, a.cc.om1, v.R, v.Ux, v.Uy, v.t, store);
    return;
  }
  // 4. fixed-point relaxation
  const double U = fma(v.Ux, v.Ux, v.Uy * v.Uy) * (1.0 / C2);
  const HermiteA h = hermite_a(v.t, U);
  bool unused = false;  // the range check rules overflow out
  // omega rho times the Hermite coefficients a_jk (C0 = a00 + a01 q + a02 q^2, ...), each in
  // the format that keeps its products with the shell constants at 2^-57
  const long long A00 = fx_from_double(v.R * h.a00, FV, 64, unused);  // |A00| < 4
  const long long A01 = fx_from_double(v.R * h.a01, 62, 64, unused);  // |A01| < 0.6
  const long long A02 = fx_from_double(v.R * h.a02, 66, 64, unused);  // |A02| < 0.03
  const long long A10 = fx_from_double(v.R * h.a10, FV, 64, unused);  // |A10| < 5
  const long long A11 = fx_from_double(v.R * h.a11, 62, 64, unused);  // |A11| < 0.4
  const long long A20 = fx_from_double(v.R * h.a20, FV, 64, unused);  // |A20| < 3
  const long long A21 = fx_from_double(v.R * h.a21, 62, 64, unused);  // |A21| < 0.2
  const unsigned long long Rf = (unsigned long long)fx_from_double(v.R, 61, 64, unused);  // < 3
  const long long om1f = fx_from_double(a.cc.om1, FU, 64, unused);
  const long long X1 = fx_from_double(v.Ux, FU, 64, unused), Y1 = fx_from_double(v.Uy, FU, 64, unused);
  {
    constexpr int e = shell_exp(0);
    const long long K0 = fx_mulhi(kCw(0), A00) * 2 + 1;
    store(0, fx_to_double(fx_mulhi(om1f, fx_from_nonneg(sf[0], FV + e)) * 4 + 2 + K0, FV + e));
  }
  //   K0 = w' (A00 + q A01 + q^2 A02), K1 = w' (A10 + q A11), K2 = w' (A20 + q A21)  (Q5.58)
  //   K3 = omega rho w' / 6, K4 = omega rho w' / 24                                   (Q3.61)
  // formed at the first pair of each shell (pairs come grouped by shell).
  int cur = -1, e = 0;
  long long K0 = 0, K1 = 0, K2 = 0;
  unsigned long long K3 = 0, K4 = 0;
#pragma unroll 1
  for (int j = 1; j <= NPAIR; ++j) {
    const int sh = (int)((kPairShell >> (3 * (j - 1))) & 7);
    if (sh != cur) {  // uniform across the warp
      cur = sh;
      const ShellFix& c = c_shell_fix[sh];
      K0 = (fx_mulhi(c.cw, A00) + fx_mulhi(c.cq, A01) + fx_mulhi(c.cq2, A02)) * 2 + 3;
      K1 = (fx_mulhi(c.cw, A10) + fx_mulhi(c.cq, A11)) * 2 + 2;
      K2 = (fx_mulhi(c.cw, A20) + fx_mulhi(c.cq, A21)) * 2 + 2;
      K3 = fx_umulhi(Rf, c.cw6);
      K4 = fx_umulhi(Rf, c.cw24);
      e = c.e;
    }
    const int vxk = (int)((kPairVx >> (2 * (j - 1))) & 3);
    const int vyk = (int)((kPairVy >> (3 * (j - 1))) & 7) - 3;
    const long long s = vxk * X1 + vyk * Y1;                                          // Q1.62
    const unsigned long long as = (unsigned long long)(s < 0 ? -s : s);
    const unsigned long long s2 = fx_umulhi(as, as);                                  // Q4.60
    const long long e1 = K2 + (long long)fx_umulhi(K4, s2) * 2 + 1;                   // Q5.58
    const long long Ev = K0 + fx_mulhi(e1, (long long)s2) * 16 + 8;                   // 2^-54 -> Q5.58
    const long long o1 = K1 + (long long)fx_umulhi(K3, s2) * 2 + 1;                   // Q5.58
    const long long Ov = fx_mulhi(o1, s) * 4 + 2;                                     // 2^-56 -> Q5.58
    const long long rp = fx_mulhi(om1f, fx_from_nonneg(sf[j * 32], FV + e)) * 4 + 2;
    const long long rm = fx_mulhi(om1f, fx_from_nonneg(sf[(j + NPAIR) * 32], FV + e)) * 4 + 2;
    store(j, fx_to_double(rp + Ev + Ov, FV + e));
    store(j + NPAIR, fx_to_double(rm + Ev - Ov, FV + e));
  }
}

}  // namespace d2q37
