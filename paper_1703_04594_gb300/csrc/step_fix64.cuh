// One warp-strip of the fused FP64 step with the fixed-point relaxation of collide_fix64.cuh.
//
// Layout of the work, chosen for the integer pipes:
//   1. the 37 pull-gathered populations of the strip are copied global -> shared memory
//      with cp.async (no registers held while the loads are in flight; inside a persistent
//      kernel, whose sources were written earlier in the same launch, with L2 loads);
//   2. an unrolled loop over opposite pairs converts every population once to fixed point
//      (written back over its float64 in shared memory), checks the range of the
//      fixed-point path and sums the moments in 64-bit fixed point;
//   3. the site scalars in float64 (1/rho, u, T, gravity shift);
//   4. the Hermite coefficients and, per shell, K0..K3 in fixed point; then a loop over
//      opposite pairs (two per iteration) reads the fixed-point populations and evaluates
//      the equilibrium polynomial and (1 - omega) f + omega f^eq.
// The relaxation loop stays rolled to keep the kernel's code small (unrolled, it thrashes
// the instruction cache); its per-pair velocities and shells, and per-shell constants,
// come from constant-memory tables.  Sites outside the fixed-point range take the float64
// collision on their values loaded again from global memory; warps next to a wall (two
// strips per column) run the float64 strip of step_fp64.cuh.
#pragma once
#include "collide_fix64.cuh"
#include "step_fp64.cuh"

namespace d2q37 {

struct ShellFix {
  long long cw, cq, cq2;
  unsigned long long cw6;
  int e;  // shell scale exponent e_s
  int lim;  // largest exponent field with |f| 2^e_s < 8 (the range is checked by fx_exact_shift)
};
#define LBM_SHELL_FIX(s) \
  { kCw(s), kCq(s), kCq2(s), kCw6(s), shell_exp(s), 1025 - shell_exp(s) }
static __constant__ ShellFix c_shell_fix[8] = {LBM_SHELL_FIX(0), LBM_SHELL_FIX(1), LBM_SHELL_FIX(2),
                                               LBM_SHELL_FIX(3), LBM_SHELL_FIX(4), LBM_SHELL_FIX(5),
                                               LBM_SHELL_FIX(6), LBM_SHELL_FIX(7)};
#undef LBM_SHELL_FIX

// 8-byte asynchronous global -> shared copy (sm_80+ LDGSTS), cached in L1.
__device__ __forceinline__ void cp_async8(double* smem_dst, const double* gmem_src) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// The moment loop is unrolled completely, with the pairs' velocities and shells as
// compile-time constants; the relaxation loop takes 2 pairs per iteration from the
// constant-memory tables (measured on GB300: +4 % and +2 % over 2 and 3 per iteration
// from the tables; unrolling the relaxation loop completely overflows the instruction
// cache and loses 11 %).
#ifndef LBM_FIX64_UNROLL_RELAX
#define LBM_FIX64_UNROLL_RELAX 2
#endif
constexpr int kFixUnrollRelax = LBM_FIX64_UNROLL_RELAX;

template <bool B>
struct BoolConst {
  static constexpr bool value = B;
};

// Calls f(pair, j) for j = J .. NPAIR with the pair's data as compile-time constants: a
// fully unrolled pair loop in which velocity multiples fold into adds.
template <int J, class F>
__device__ __forceinline__ void for_pairs_ct(F&& f) {
  constexpr PairFix p = {rep_vx(J), rep_vy(J), rep_vx(J) * rep_vx(J) + rep_vy(J) * rep_vy(J), shell(J)};
  f(p, J);
  if constexpr (J < NPAIR) for_pairs_ct<J + 1>(f);
}
// Shell constants as compile-time values (for the unrolled loop).
__device__ __forceinline__ constexpr ShellFix shell_ct(int s) {
  return ShellFix{kCw(s), kCq(s), kCq2(s), kCw6(s), shell_exp(s), 1025 - shell_exp(s)};
}

// Shared staging: one warp holds sf[i * 32 + lane] for its 32 sites.
constexpr int kFixWarps = 4;  // warps per block (block = 32 x 4 threads)

// Pull-gather address of population i for the lane's row yc (interior warps).
template <bool PERIODIC>
__device__ __forceinline__ const double* gather_src(const double* fin, const StepScalars& a, int x, int yc, int i) {
  const long long col = (long long)wrap_index(x - vx(i), a.lx) * a.pitch;
  const int ys = PERIODIC ? wrap_index(yc - vy(i), a.ly) : yc - vy(i);
  return fin + i * a.pop + col + ys;
}

// The float64 collision of one interior site on values loaded again from global memory:
// the path of sites outside the fixed-point range.  Not inlined, so that its 37 live
// float64 values do not weigh on the register allocation of the fixed-point path.
template <bool PERIODIC, class Ld>
__device__ __noinline__ void collide_site_reloaded(const double* __restrict__ fin, double* __restrict__ fout,
                                                   const StepScalars& a, int x, int yc, unsigned self) {
  const Ld ld;
  double f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] = ld(gather_src<PERIODIC>(fin, a, x, yc, i));
  collide_site(f, a.cc, [&](int i, double val) { __stcs(fout + i * a.pop + self, val); });
}

// The float64 strip of a warp next to a wall, not inlined for the same reason.
template <bool PERIODIC, class Ld>
__device__ __noinline__ void wall_strip_fp64(const double* __restrict__ fin, double* __restrict__ fout,
                                             const StepScalars& a, const StepWalls& w, int x, int y0) {
  step_strip_fp64<PERIODIC>(fin, fout, a, w, x, y0, Ld());
}

// Whether the strip at rows y0 .. y0 + 31 runs the float64 wall strip (its pulls reach a
// ghost row).
template <bool PERIODIC>
__device__ __forceinline__ bool fix64_wall_strip(const StepScalars& a, int y0) {
  return !PERIODIC && (y0 < 3 || y0 + 32 > a.ly - 3);
}

// 1. The pull-gather of an interior strip into its shared-memory slots sf[i * 32 + lane]:
// asynchronous copies when Ld caches in L1 (the caller waits for them), loads otherwise.
template <bool PERIODIC, class Ld>
__device__ __forceinline__ void stage_strip_fix64(const double* __restrict__ fin, const StepScalars& a, int x, int y0,
                                                  Ld ld, double* __restrict__ sf) {
  const int lane = threadIdx.x & 31;
  const int y = y0 + lane;
  const int yc = y < a.ly ? y : a.ly - 1;
  unsigned off[7];  // column x_s, row yc within a population plane (planes < 2^32 elements)
#pragma unroll
  for (int d = 0; d < 7; ++d) off[d] = (unsigned)((long long)wrap_index(x - (d - 3), a.lx) * a.pitch + yc);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const double* src = PERIODIC ? fin + i * a.pop + (off[vx(i) + 3] - yc) + wrap_index(yc - vy(i), a.ly)
                                 : fin + i * a.pop + (off[vx(i) + 3] - vy(i));
    if (Ld::kL1) cp_async8(sf + i * 32 + lane, src);
    else sf[i * 32 + lane] = ld(src);
  }
}

template <bool PERIODIC, class Ld>
__device__ __forceinline__ void compute_strip_fix64(const double* __restrict__ fin, double* __restrict__ fout,
                                                    const StepScalars& a, int x, int y0, double* __restrict__ sf);

template <bool PERIODIC, class Ld>
__device__ __forceinline__ void step_strip_fix64(const double* __restrict__ fin, double* __restrict__ fout,
                                                 const StepScalars& a, const StepWalls& w, int x, int y0, Ld ld,
                                                 double* __restrict__ sf) {
  if (fix64_wall_strip<PERIODIC>(a, y0)) {
    wall_strip_fp64<PERIODIC, Ld>(fin, fout, a, w, x, y0);
    return;
  }
  stage_strip_fix64<PERIODIC>(fin, a, x, y0, ld, sf);
  if (Ld::kL1) cp_async_wait_all();
  __syncwarp();
  compute_strip_fix64<PERIODIC, Ld>(fin, fout, a, x, y0, sf);
}

// 2.-4. The collision of an interior strip from its staged populations.
template <bool PERIODIC, class Ld>
__device__ __forceinline__ void compute_strip_fix64(const double* __restrict__ fin, double* __restrict__ fout,
                                                    const StepScalars& a, int x, int y0, double* __restrict__ sf) {
  const int lane = threadIdx.x & 31;
  const int y = y0 + lane;
  const bool active = y < a.ly;
  const int yc = active ? y : a.ly - 1;
  sf += lane;
  long long* const sx = reinterpret_cast<long long*>(sf);  // the same slots, as fixed point
  // 2. every population to fixed point f' = f 2^(59 + e_s), written back in place, and the
  //    moments from f' rounded to 2^-56: rho, j and sum |v|^2 f stay below 2^4 there for
  //    every state in range.  In range, 2^-7 <= f 2^e_s < 8, f 2^(59 + e_s) is an integer
  //    (its significand shifted left by 0 to 9 places), so the conversion is exact; one
  //    unsigned compare of the exponent field flags everything else (negative, zero,
  //    small, large, non-finite), and such a site takes the float64 collision.
  bool out;
  long long R, Ei = 0, Jx = 0, Jy = 0;
  {
    constexpr int e = shell_exp(0);
    const double f0 = sf[0];
    unsigned sh0;
    out = !fx_exact_shift(f0, e, sh0);
    const long long q0 = fx_from_double_shifted(f0, sh0);
    sx[0] = q0;
    R = (q0 + (1LL << (2 + e))) >> (3 + e);
  }
  const auto moment_pair = [&](const PairFix pk, const int k) {
    const int vxk = pk.vx, vyk = pk.vy;
    const ShellFix c = shell_ct(pk.sh);
    const double fa = sf[k * 32], fb = sf[(k + NPAIR) * 32];
    unsigned sha, shb;
    out |= !fx_exact_shift(fa, c.e, sha) | !fx_exact_shift(fb, c.e, shb);
    const long long qa = fx_from_double_shifted(fa, sha), qb = fx_from_double_shifted(fb, shb);
    sx[k * 32] = qa;
    sx[(k + NPAIR) * 32] = qb;
    const int sh = 3 + c.e;
    const long long half = 1LL << (sh - 1);
    const long long va = (qa + half) >> sh, vb = (qb + half) >> sh;
    const long long P = va + vb, M = va - vb;
    R += P;
    Ei += (long long)pk.v2 * P;
    Jx += (long long)vxk * M;
    Jy += (long long)vyk * M;
  };
  for_pairs_ct<1>(moment_pair);
  if (!active) return;
  const unsigned self = (unsigned)((long long)x * a.pitch + y);
  const auto store = [&](int i, double val) { __stcs(fout + i * a.pop + self, val); };
  // 3. site scalars in float64; sites out of range (populations outside [2^-7, 8) 2^-e_s,
  //    fast or hot fluid) take the float64 collision
  const SiteScalars v = scalars_from_moments(fx_to_double_dp_pos(R, 56), fx_to_double_dp_pos(Jx, 56),
                                             fx_to_double_dp_pos(Jy, 56), fx_to_double_dp_pos(Ei, 56), a.cc);
  if (out || !fixed_range_ok(v)) {
    collide_site_reloaded<PERIODIC, Ld>(fin, fout, a, x, yc, self);
    return;
  }
  // 4. fixed-point relaxation.  Inputs: omega rho, c u_s and t = T_s - 1 from the float64
  //    stage; everything after them is integer arithmetic.
  bool unused = false;  // the range check rules overflow out
  const unsigned long long Rf = (unsigned long long)fx_from_double(v.R, 61, 64, unused);  // < 3
  // |1 - omega| < 1 with 63 fraction bits; its sign is the same for every site, so the
  // relaxation loop below is instantiated for each sign and multiplies unsigned values
  const unsigned long long om1u = (unsigned long long)fx_from_double(fabs(a.cc.om1), 63, 64, unused);
  const long long X1 = fx_from_double(v.Ux, 63, 64, unused), Y1 = fx_from_double(v.Uy, 63, 64, unused);
  const HermiteFix h = hermite_fix(X1, Y1, v.t);
  // A = omega rho a (the product with R at 61 bits takes 3 off each)
  const long long A00 = fx_mulhi_su(h.a00, Rf);  // 58
  const long long A01 = fx_mulhi_su(h.a01, Rf);  // 62
  const long long A02 = fx_mulhi_su(h.a02, Rf);  // 66
  const long long A10 = fx_mulhi_su(h.a10, Rf);  // 59
  const long long A11 = fx_mulhi_su(h.a11, Rf);  // 62 (A21: the same integer at 63)
  const long long A20 = fx_mulhi_su(h.a20, Rf);  // 60
  const auto relax = [&](auto neg) {
    constexpr bool NEG = decltype(neg)::value;
    const auto add_r = [](long long v, unsigned long long r) { return NEG ? v - (long long)r : v + (long long)r; };
    {
      constexpr int e = shell_exp(0);
      const long long K0 = fx_mulhi_su(A00, kCw(0)) * 2 + 1;
      store(0, fx_to_double_dp_pos(add_r(K0 + (NEG ? 0 : 1), fx_umulhi(om1u, sx[0])), 58 + e));
    }
    // K0 (58 bits) = w' (A00 + q A01 + q^2 A02), K1 (59) = w' (A10 + q A11),
    // K2 (60) = w' (A20 + q A21), K3 (61) = omega rho w' / 6, formed at the first pair of
    // each shell (pairs come grouped by shell).  The s^4 / 24 term's factor
    // omega rho w' s^2 / 24 is a quarter of K3 s^2 and takes no product of its own.
    int cur = -1, e = 0;
    long long K0 = 0, K1 = 0, K2 = 0;
    unsigned long long K3 = 0;
    const auto shell_setup = [&](const ShellFix& c) {
      K0 = (fx_mulhi_su(A00, c.cw) + fx_mulhi_su(A01, c.cq) + fx_mulhi_su(A02, c.cq2)) * 2 + 3;
      K1 = fx_mulhi_su(A10, c.cw) * 2 + fx_mulhi_su(A11, c.cq) * 4 + 3;  // 58 -> 59, 57 -> 59
      K2 = fx_mulhi_su(A20, c.cw) * 2 + fx_mulhi_su(A11, c.cq) * 4 + 3;  // 59 -> 60, 58 -> 60
      K3 = fx_umulhi(Rf, c.cw6);
      e = c.e;
    };
    const auto pair_body = [&](const PairFix pj, const int j) {
      const int vxk = pj.vx, vyk = pj.vy;
      const long long s = vxk * X1 + vyk * Y1;                                  // 63 bits, |s| < 0.6
      const unsigned long long as = (unsigned long long)(s < 0 ? -s : s);
      // The products drop the low partial product and the carries of the low halves
      // (fx_umulhi_approx): 0 to 2 units below the floor of the exact high half, about
      // 1.25 below the exact product on average, far inside the outputs' 5 guard bits.
      const long long s2 = (long long)fx_umulhi_approx(as, as);                 // 62
      // omega rho w' s^2 / 6 at 59 bits; halved, omega rho w' s^2 / 24 at 60 bits
      const unsigned long long h3 = fx_umulhi_approx(K3, (unsigned long long)s2);
      const long long o1 = K1 + (long long)h3;                                   // 59
      const long long e1 = K2 + (long long)(h3 >> 1);                            // 60
      const long long Ev = K0 + fx_mulhi_su_approx(e1, (unsigned long long)s2); // 58
      const long long Ov = fx_mulhi_approx(o1, s);                              // 58
      const unsigned long long rp = fx_umulhi_approx(om1u, sx[j * 32]);         // 63 + 59 -> 58
      const unsigned long long rm = fx_umulhi_approx(om1u, sx[(j + NPAIR) * 32]);
      // re-centring: Ev, Ov and r each come out about 1.25 units low on average (r only
      // 1/2 when 1 - omega has at most 32 significant bits), and r enters with the sign
      // of 1 - omega; the offsets keep each output within about a unit of its exact value
      // on average (the mass-drift tests bound the effect).
      store(j, fx_to_double_dp_pos(add_r(Ev + Ov + (NEG ? 2 : 4), rp), 58 + e));
      store(j + NPAIR, fx_to_double_dp_pos(add_r(Ev - Ov + (NEG ? -1 : 1), rm), 58 + e));
    };
    const auto relax_pair = [&](const PairFix pj, const int j) {
      if (pj.sh != cur) {  // uniform across the warp
        cur = pj.sh;
        shell_setup(c_shell_fix[pj.sh]);
      }
      pair_body(pj, j);
    };
#pragma unroll kFixUnrollRelax
    for (int j = 1; j <= NPAIR; ++j) relax_pair(c_pair_fix[j], j);
  };
  if (a.cc.om1 < 0.0) relax(BoolConst<true>());
  else relax(BoolConst<false>());
}

}  // namespace d2q37
