// Hand-written adjoint (vector-Jacobian product) of the FP64 fused step, and of the
// equilibrium initialisation and the kinetic-energy observable.
//
// The step is S = C o B o P: pull propagate P and wall bc B are linear in f (a ghost value
// is rho_w(x_s) * w_i P_i(T_wall), rho_w a sum of the source column's wall-row
// populations); collide C acts site by site (Sec. 3, eqs. "lbequation", "macro").  For
// lambda' = dL/df^{n+1}:
//   1. (k_adj_collide) at every site z, recompute f~ = B P f^n and its moments, then
//        mu_i = lambda'_i,
//        out_i = (1 - w) mu_i + w (nu_rho + nu_J . xi_i + nu_E |xi_i|^2),   w = 1/tau,
//      where nu = (d f^eq / d(rho, J, E))^T mu through u = J/rho,
//      T = (E/rho - |u|^2)/D, the gravity shift u_s = u + tau g, T_s = T + tau(1-tau)|g|^2/D
//      and the fourth-order Hermite polynomial; the site's contribution to dL/dtau is
//        sum_i mu_i d f_i'/d tau = -(1/tau^2) sum_i mu_i (f^eq_i - f~_i)
//                                   + w [G_u . g + G_t (1 - 2 tau) |g|^2 / D];
//      and the transpose of the pull is applied on the way out, as a push: out_i(z) is
//      the value of lambda_i(z - v_i) when z - v_i is a fluid site.  When it is a ghost
//      (z was fed from the wall), out_i(z) goes to a per-column slot of the wall's source
//      column instead; entries lambda_i(x) with no fluid source x + v_i are set to zero
//      by their own site;
//   2. (k_adj_walls) the wall rows: every population of (x_s, 0) receives the sum of the
//      bottom slots of column x_s, each times its ghost's weight w_i P_i(T_wall) (the
//      transpose of rho_w = sum_j f_j(x_s, 0)), and likewise at the top.
// dL/dtau partials are summed per block and then in a fixed order (deterministic).
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lbm_d2q37.h"
#include "adjoint_fix64.cuh"
#include "kernels.h"
#include "step_fp64.cuh"

namespace d2q37 {

static_assert(D == 2.0, "nu_E = g_t / D is formed as an exact halving");

namespace {

// Vector-Jacobian product of the equilibrium f^eq_i = w_i rho P_i(s_i, U, t),
// s_i = xi_i . u_s, U = |u_s|^2, t = T_s - 1, against mu: returns
//   Grho = sum mu_i w_i P_i,            (d/d rho at fixed u_s, t)
//   Gu   = rho sum mu_i w_i (dP/ds xi_i + 2 dP/dU u_s),
//   Gt   = rho sum mu_i w_i dP/dt.
struct EqVjp {
  double Grho, Gux, Guy, Gt;
};

// Computed one opposite pair (v, -v) at a time: with s = xi_v . u_s,
// P(+-s) = E +- O, dP/ds(+-s) = Pse +- Pso, dP/dU(+-s) = PUe +- PUo, dP/dt(+-s) = Pte +- Pto,
// and S = mu_v + mu_-v, Dm = mu_v - mu_-v, the pair contributes
//   Grho: w (S E + Dm O);  Gu: w [xi (Dm Pse + S Pso) + 2 u_s (S PUe + Dm PUo)];
//   Gt: w (S Pte + Dm Pto)   (the factor rho of Gu, Gt applied at the end).
// `mu(i)` returns mu_i (read on demand, so the 37 values need not stay in registers).
template <class Mu>
__device__ __forceinline__ EqVjp eq_vjp_pairs(double rho, double usx, double usy, double t, Mu&& mu) {
  const double U = fma(usx, usx, usy * usy);
  const double Ux = C * usx, Uy = C * usy;  // s = v . (Ux, Uy)
  double Gr, Gx, Gy, Gt;
  {  // rest population: s = 0, xi = 0
    const double c0 = 1.0 - 0.5 * U - 0.5 * t * D + 0.125 * U * U + 0.25 * t * U * (D + 2.0) +
                      0.125 * t * t * D * (D + 2.0);
    const double pue = -0.5 + 0.25 * U + 0.25 * t * (D + 2.0);
    const double pt0 = -0.5 * D + 0.25 * U * (D + 2.0) + 0.25 * t * D * (D + 2.0);
    const double m = mu(0) * weight(0);
    Gr = m * c0;
    Gx = m * (2.0 * pue * usx);
    Gy = m * (2.0 * pue * usy);
    Gt = m * pt0;
  }
#pragma unroll
  for (int k = 1; k <= NPAIR; ++k) {
    const double q = C2 * (double)v2(k);
    const double xix = C * (double)rep_vx(k), xiy = C * (double)rep_vy(k);
    const double c2 = 0.5 - 0.25 * U + 0.25 * t * (q - D - 4.0);
    const double c1 = 1.0 - 0.5 * U + 0.5 * t * (q - D - 2.0);
    const double c0 = 1.0 - 0.5 * U + 0.5 * t * (q - D) + 0.125 * U * U + 0.25 * t * U * (D + 2.0 - q) +
                      0.125 * t * t * (q * q - 2.0 * (D + 2.0) * q + D * (D + 2.0));
    const double pue0 = -0.5 + 0.25 * U + 0.25 * t * (D + 2.0 - q);
    const double pt0 = 0.5 * (q - D) + 0.25 * U * (D + 2.0 - q) +
                       0.25 * t * (q * q - 2.0 * (D + 2.0) * q + D * (D + 2.0));
    const double s = fma((double)rep_vx(k), Ux, (double)rep_vy(k) * Uy);
    const double s2 = s * s;
    const double E = fma(s2, fma(s2, 1.0 / 24.0, c2), c0);
    const double O = s * fma(s2, 1.0 / 6.0, c1);
    const double Pse = fma(0.5, s2, c1);
    const double Pso = s * fma(s2, 1.0 / 6.0, 2.0 * c2);
    const double PUe = fma(-0.25, s2, pue0);
    const double PUo = -0.5 * s;
    const double Pte = fma(0.25 * (q - D - 4.0), s2, pt0);
    const double Pto = 0.5 * (q - D - 2.0) * s;
    const double w = weight(k);
    const double mp = mu(k), mm = mu(k + NPAIR);
    const double S = (mp + mm) * w, Dm = (mp - mm) * w;
    Gr = fma(S, E, fma(Dm, O, Gr));
    const double xiPart = fma(Dm, Pse, S * Pso);
    const double uPart = 2.0 * fma(S, PUe, Dm * PUo);
    Gx = fma(xix, xiPart, fma(uPart, usx, Gx));
    Gy = fma(xiy, xiPart, fma(uPart, usy, Gy));
    Gt = fma(S, Pte, fma(Dm, Pto, Gt));
  }
  return {Gr, rho * Gx, rho * Gy, rho * Gt};
}

// The float64 VJP for sites outside the fixed-point range, not inlined so that its
// unrolled arithmetic does not weigh on the register allocation of the fixed-point path.
__device__ __noinline__ EqVjp eq_vjp_float64(double rho, double usx, double usy, double t, const double* mu_staged) {
  return eq_vjp_pairs(rho, usx, usy, t, [&](int i) { return mu_staged[i * 32]; });
}

__device__ __forceinline__ double block_sum_128(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __shared__ double ws[4];
  const int w = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
  if ((threadIdx.x & 31) == 0) ws[w] = v;
  __syncthreads();
  return (ws[0] + ws[1]) + (ws[2] + ws[3]);
}

// Ghost slots of one column: population i with vy_i > 0 fed rows 0 .. vy_i - 1 of column
// x_s + vx_i from the bottom ghosts of column x_s; those entries take bottom slots
// ghost_base(i, +1) + row of column x_s.  The top mirrors it with -vy_i and row ly - 1 - y.
__host__ __device__ constexpr int ghost_base_calc(int i, int sign) {
  int n = 0;
  for (int j = 0; j < i; ++j) n += sign * vy(j) > 0 ? sign * vy(j) : 0;
  return n;
}
constexpr int kGhostSlots = ghost_base_calc(Q, 1);  // 26 for D2Q37, the same at the top
static_assert(ghost_base_calc(Q, -1) == kGhostSlots, "the velocity set is symmetric in y");
__host__ __device__ constexpr int ghost_base(int i, int sign) {
  constexpr int b[Q] = {ghost_base_calc(0, 1),  ghost_base_calc(1, 1),  ghost_base_calc(2, 1),  ghost_base_calc(3, 1),
                        ghost_base_calc(4, 1),  ghost_base_calc(5, 1),  ghost_base_calc(6, 1),  ghost_base_calc(7, 1),
                        ghost_base_calc(8, 1),  ghost_base_calc(9, 1),  ghost_base_calc(10, 1), ghost_base_calc(11, 1),
                        ghost_base_calc(12, 1), ghost_base_calc(13, 1), ghost_base_calc(14, 1), ghost_base_calc(15, 1),
                        ghost_base_calc(16, 1), ghost_base_calc(17, 1), ghost_base_calc(18, 1), ghost_base_calc(19, 1),
                        ghost_base_calc(20, 1), ghost_base_calc(21, 1), ghost_base_calc(22, 1), ghost_base_calc(23, 1),
                        ghost_base_calc(24, 1), ghost_base_calc(25, 1), ghost_base_calc(26, 1), ghost_base_calc(27, 1),
                        ghost_base_calc(28, 1), ghost_base_calc(29, 1), ghost_base_calc(30, 1), ghost_base_calc(31, 1),
                        ghost_base_calc(32, 1), ghost_base_calc(33, 1), ghost_base_calc(34, 1), ghost_base_calc(35, 1),
                        ghost_base_calc(36, 1)};
  constexpr int t[Q] = {ghost_base_calc(0, -1),  ghost_base_calc(1, -1),  ghost_base_calc(2, -1),  ghost_base_calc(3, -1),
                        ghost_base_calc(4, -1),  ghost_base_calc(5, -1),  ghost_base_calc(6, -1),  ghost_base_calc(7, -1),
                        ghost_base_calc(8, -1),  ghost_base_calc(9, -1),  ghost_base_calc(10, -1), ghost_base_calc(11, -1),
                        ghost_base_calc(12, -1), ghost_base_calc(13, -1), ghost_base_calc(14, -1), ghost_base_calc(15, -1),
                        ghost_base_calc(16, -1), ghost_base_calc(17, -1), ghost_base_calc(18, -1), ghost_base_calc(19, -1),
                        ghost_base_calc(20, -1), ghost_base_calc(21, -1), ghost_base_calc(22, -1), ghost_base_calc(23, -1),
                        ghost_base_calc(24, -1), ghost_base_calc(25, -1), ghost_base_calc(26, -1), ghost_base_calc(27, -1),
                        ghost_base_calc(28, -1), ghost_base_calc(29, -1), ghost_base_calc(30, -1), ghost_base_calc(31, -1),
                        ghost_base_calc(32, -1), ghost_base_calc(33, -1), ghost_base_calc(34, -1), ghost_base_calc(35, -1),
                        ghost_base_calc(36, -1)};
  return sign > 0 ? b[i] : t[i];
}

// The pull-gather of a warp's strip into its shared-memory slots sf[i * 32 + lane] through
// registers (wall bc and periodic wrap included); not inlined, so that its 37 live values
// do not weigh on the register allocation of the collide kernel.
template <bool PERIODIC>
__device__ __noinline__ void gather_to_shared(const double* __restrict__ fin, const StepArgs& a, int x, int y0,
                                              int yc, double* sf) {
  double f[Q];
  gather_strip_fp64<PERIODIC>(fin, a, a, x, y0, yc, f, LdReadOnly());
#pragma unroll
  for (int i = 0; i < Q; ++i) sf[i * 32] = f[i];
}

// Float64 moments of a staged site (populations sf[i * 32]), for sites outside the
// fixed-point sums' range; not inlined, so the common path keeps its registers.
__device__ __noinline__ void moments_float64_staged(const double* sf, double& rho, double& jx, double& jy,
                                                     double& e) {
  moments_float64([&](int i) { return sf[i * 32]; }, rho, jx, jy, e);
}

__device__ __forceinline__ void cp_async8_adj(double* smem_dst, const double* gmem_src) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(gmem_src) : "memory");
}

}  // namespace

// The lattice-wide scalars of the adjoint collision, formed once on the host.
struct AdjConsts {
  double tau;
  double om, om2;       // w = 1/tau, w^2
  double om1;           // 1 - w
  double om_c, om_c2;   // w c, w c^2
  double tgx, tgy;      // the gravity shift of the velocity, tau g
  double tshift;        // tau (1 - tau) |g|^2 / D - 1:  t = T + tshift
  double gx, gy;
  double dts_dtau;      // d T_s / d tau = (1 - 2 tau) |g|^2 / D
};

// Step 1: per-site adjoint of the collision with the transposed propagate as its store
// (block 32 x 4 as the forward kernels).  `side` holds 2 * lx * kGhostSlots doubles: the
// bottom slots of every column, then the top slots.
#ifndef LBM_ADJ_MIN_BLOCKS
#define LBM_ADJ_MIN_BLOCKS 5  // 96 registers, 20 warps per SM (with 37.9 KB of staging per block)
#endif
template <bool PERIODIC>
__global__ void __launch_bounds__(128, LBM_ADJ_MIN_BLOCKS) k_adj_collide(const double* __restrict__ fin,
                                                     const double* __restrict__ lam_next, double* __restrict__ lam_out,
                                                     double* __restrict__ side, double* __restrict__ dtau_part,
                                                     StepArgs a, AdjConsts k) {
  const int x = blockIdx.y * 4 + threadIdx.y;
  const int y0 = blockIdx.x * 32;
  const int y = y0 + threadIdx.x;
  double contrib = 0.0;
  if (x < a.lx) {  // uniform per warp
    const bool active = y < a.ly;
    const int yc = active ? y : a.ly - 1;
    // the strip's pull-gather staged in shared memory (9.5 KB per warp): no registers held
    // for it, which lets 5 blocks of 4 warps share an SM (389 against 399 us per step with
    // the gather in registers at 4 blocks)
    __shared__ double staged[4][Q * 32];
    double* const sf = &staged[threadIdx.y][0] + (threadIdx.x & 31);
    if (PERIODIC || y0 < 3 || y0 + 32 > a.ly - 3) {
      gather_to_shared<PERIODIC>(fin, a, x, y0, yc, sf);
    } else {
      unsigned off[7];  // column x_s, row yc within a population plane
#pragma unroll
      for (int d = 0; d < 7; ++d) off[d] = (unsigned)((long long)wrap_index(x - (d - 3), a.lx) * a.pitch + yc);
#pragma unroll
      for (int i = 0; i < Q; ++i) cp_async8_adj(sf + i * 32, fin + i * a.pop + (off[vx(i) + 3] - vy(i)));
      asm volatile("cp.async.wait_all;\n" ::: "memory");
    }
    const auto fget = [&](int i) { return sf[i * 32]; };
    if (active) {
      double rho, jx, jy, e;
      moments_get_or(fget, rho, jx, jy, e, [](int, int) {},
                     [&](double& r, double& mx, double& my, double& me) { moments_float64_staged(sf, r, mx, my, me); });
      const double inv = 1.0 / rho;
      const double Jx = C * jx, Jy = C * jy, E = C2 * e;  // xi-unit moments
      const double ux = Jx * inv, uy = Jy * inv;
      const double uu = fma(ux, ux, uy * uy);
      const double TD = fma(E, inv, -uu);  // D T
      const double usx = ux + k.tgx, usy = uy + k.tgy;
      const double t = fma(TD, 1.0 / D, k.tshift);
      const long long o = (long long)x * a.pitch + y;
      const double* lam = lam_next + o;
      // sum_i mu_i f~_i; each staging slot, once its f~_i is read, takes mu_i = lambda_i, so
      // the three later passes over mu (the VJP's exponent scan and conversion, the outputs)
      // read shared memory instead of re-reading lambda, whose 37.9 KB per block do not stay
      // in the L1 that the staging leaves
      double mu_ft = 0.0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const double l = __ldg(lam + i * a.pop);
        mu_ft = fma(l, fget(i), mu_ft);
        sf[i * 32] = l;
      }
      const auto mu = [&](int i) { return sf[i * 32]; };
      // the VJP in fixed point (adjoint_fix64.cuh), in float64 outside its range, per unit
      // density: g = G / rho for G_u and G_t (G_rho has no factor rho)
      double gr, gux, guy, gt;
      {
        VjpSums V;
        if (eq_vjp_sums_fix(usx, usy, t, mu, V)) {
          gr = V.Gr;
          const double Wu2 = pow2_scale(V.Wu, 1);  // 2 Wu, exactly
          gux = fma(C, V.Ax, usx * Wu2);
          guy = fma(C, V.Ay, usy * Wu2);
          gt = V.Gt;
        } else {
          const EqVjp G = eq_vjp_float64(1.0, usx, usy, t, sf);
          gr = G.Grho;
          gux = G.Gux;
          guy = G.Guy;
          gt = G.Gt;
        }
      }
      // nu = (d f^eq / d(rho, J, E))^T mu through u = J / rho, T = (E / rho - |u|^2) / D:
      // the factors rho of G and 1 / rho of the chain rule cancel, and E / rho = D T + |u|^2
      const double nuE = pow2_scale(gt, -1);      // gt / D, D = 2 (exact scalings on the integer pipe)
      const double m2nuE = pow2_scale(-nuE, 1);   // -2 nuE
      const double nuJx = fma(ux, m2nuE, gux);
      const double nuJy = fma(uy, m2nuE, guy);
      const double nuR = fma(nuE, uu - TD, gr - fma(gux, ux, guy * uy));
      // out_i(z) is lambda_i(z - v_i) of the previous step (the transposed pull), or the
      // wall slot of its source column when z - v_i is a ghost
      // (the destination is selected, not branched on, to keep the kernel's code small)
      const auto push = [&](int i, double val) {
        const int xs = wrap_index(x - vx(i), a.lx), yd = y - vy(i);
        const long long in_fluid = i * a.pop + (long long)xs * a.pitch + (PERIODIC ? wrap_index(yd, a.ly) : yd);
        bool ghost = false;
        long long slot = 0;
        if (!PERIODIC && vy(i) > 0) {
          ghost = yd < 0;
          slot = (long long)xs * kGhostSlots + ghost_base(i, 1) + y;
        } else if (!PERIODIC && vy(i) < 0) {
          ghost = yd >= a.ly;
          slot = ((long long)a.lx + xs) * kGhostSlots + ghost_base(i, -1) + (a.ly - 1 - y);
        }
        // only the selected address is formed (the other offset may be out of its buffer)
        __stcs(ghost ? side + slot : lam_out + in_fluid, val);
      };
      // out_{+-v} = (1-w) mu + A_s +- B_v with A_s = w (nuR + nuE c^2 |v|^2) (one per shell)
      // and B_v = w c nuJ . v (from the multiples of w c nuJ)
      const double om1 = k.om1;
      const double wR = k.om * nuR, wE = k.om_c2 * nuE;
      const Multiples wJ = make_multiples(k.om_c * nuJx, k.om_c * nuJy);
      push(0, fma(om1, mu(0), wR));
#pragma unroll
      for (int j = 1; j <= NPAIR; ++j) {
        const double A = fma(wE, (double)v2(j), wR);
        const double B = dot_v(wJ, rep_vx(j), rep_vy(j));
        push(j, fma(om1, mu(j), A + B));
        push(j + NPAIR, fma(om1, mu(j + NPAIR), A - B));
      }
      // entries of this site whose source z + v_i lies beyond a wall get no push
      if (!PERIODIC && (y < 3 || y >= a.ly - 3)) {
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          const int ys = y + vy(i);
          if (ys < 0 || ys >= a.ly) __stcs(lam_out + i * a.pop + o, 0.0);
        }
      }
      // sum_i mu_i f^eq_i = rho * Grho
      contrib = fma(-k.om2, fma(rho, gr, -mu_ft), (k.om * rho) * fma(gux, k.gx, fma(guy, k.gy, gt * k.dts_dtau)));
    }
  }
  const double s = block_sum_128(contrib);
  if (threadIdx.x == 0 && threadIdx.y == 0) dtau_part[blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// Adds sum(part[0..n)) to *acc in a fixed order; one block of 256 threads.
__device__ __forceinline__ void reduce_add_256(const double* __restrict__ part, long long n, double* acc) {
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += 256) s += part[i];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += ws[w];
    *acc += t;
  }
}

// Step 2: the wall rows' share of the transposed bc, after step 1 has written every
// lambda entry: lambda_j(x, 0) += sum over the bottom slots of column x of the slot's value
// times its ghost's weight w_i P_i(T_bottom), for all j (the ghost values' dependence on
// rho_w(x) = sum_j f_j(x, 0)), and likewise for row ly - 1.  One thread per column, wall and
// population j: each forms its column's wall sum in the same fixed order (so the 37 entries
// of a column receive the same value; the column's 26 slots are read from cache) and adds
// it to its own entry, so the launch spreads over the GPU instead of running 37 dependent
// updates per column on a few blocks.  The grid's last block adds the step's dL/dtau
// partials to *dtau (the reduction needs step 1 complete too, so it shares this launch).
__global__ void __launch_bounds__(256) k_adj_walls(const double* __restrict__ side, double* __restrict__ lam,
                                                   StepArgs a, const double* __restrict__ part, long long n_part,
                                                   double* dtau) {
  if (blockIdx.x == gridDim.x - 1) {  // uniform per block
    reduce_add_256(part, n_part, dtau);
    return;
  }
  const long long item = (long long)blockIdx.x * 256 + threadIdx.x;  // (top * lx + x) * Q + j
  if (item >= 2LL * a.lx * Q) return;
  const int j = (int)(item % Q);
  const long long col = item / Q;  // top * lx + x: the slot column of `side`
  const int top = (int)(col / a.lx);
  const int x = (int)(col - (long long)top * a.lx);
  const double* src = side + col * kGhostSlots;
  double wall = 0.0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {  // rows in increasing y, then the ghost's weight
    double t = 0.0;
    if (top) {
      for (int r = -vy(i) - 1; r >= 0; --r) t += src[ghost_base(i, -1) + r];
      wall = vy(i) < 0 ? fma(t, a.wall_t[i], wall) : wall;
    } else {
      for (int r = 0; r < vy(i); ++r) t += src[ghost_base(i, 1) + r];
      wall = vy(i) > 0 ? fma(t, a.wall_b[i], wall) : wall;
    }
  }
  lam[j * a.pop + (long long)x * a.pitch + (top ? a.ly - 1 : 0)] += wall;
}

// Adds sum(part[0..n)) to *acc in a fixed order (one block of 256 threads).
__global__ void __launch_bounds__(256) k_reduce_add(const double* __restrict__ part, long long n, double* acc) {
  reduce_add_256(part, n, acc);
}

// dE/df_i for E = sum 1/2 |J|^2 / rho:  -|u|^2/2 + u . xi_i.
__global__ void __launch_bounds__(128) k_ke_grad(const double* __restrict__ f, double* __restrict__ lam, StepArgs a) {
  const int x = blockIdx.y * 4 + threadIdx.y;
  const int y = blockIdx.x * 32 + threadIdx.x;
  if (x >= a.lx || y >= a.ly) return;
  const long long o = (long long)x * a.pitch + y;
  double g[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) g[i] = __ldg(f + o + i * a.pop);
  double rho, jx, jy, e;
  moments_int(g, rho, jx, jy, e);
  const double ux = C * jx / rho, uy = C * jy / rho;
  const double h = -0.5 * fma(ux, ux, uy * uy);
#pragma unroll
  for (int i = 0; i < Q; ++i) lam[o + i * a.pop] = h + C * (ux * (double)vx(i) + uy * (double)vy(i));
}

// Gradient of f^0 = f^eq(rho, u, T) with respect to the four fields, against lambda^0.
__global__ void __launch_bounds__(128) k_init_adjoint(const double* __restrict__ rho, const double* __restrict__ ux,
                                                      const double* __restrict__ uy, const double* __restrict__ T,
                                                      const double* __restrict__ lam, double* __restrict__ g_rho,
                                                      double* __restrict__ g_ux, double* __restrict__ g_uy,
                                                      double* __restrict__ g_T, StepArgs a) {
  const int x = blockIdx.y * 4 + threadIdx.y;
  const int y = blockIdx.x * 32 + threadIdx.x;
  if (x >= a.lx || y >= a.ly) return;
  const long long fi = (long long)x * a.ly + y;
  const long long o = (long long)x * a.pitch + y;
  const EqVjp G = eq_vjp_pairs(rho[fi], ux[fi], uy[fi], T[fi] - 1.0, [&](int i) { return __ldg(lam + o + i * a.pop); });
  g_rho[fi] = G.Grho;
  g_ux[fi] = G.Gux;
  g_uy[fi] = G.Guy;
  g_T[fi] = G.Gt;
}

static inline dim3 site_grid(const StepArgs& a) { return dim3((a.ly + 31) / 32, (a.lx + 3) / 4); }

long long adjoint_partial_count(const StepArgs& a) {
  const dim3 g = site_grid(a);
  return (long long)g.x * g.y;
}

long long adjoint_side_count(const StepArgs& a) { return 2LL * a.lx * kGhostSlots; }

cudaError_t launch_adjoint_step(const double* fin, const double* lam_next, double* lam, double* side, double* part,
                                double* dtau, const StepArgs& a, double tau, double gx, double gy, cudaStream_t s) {
  const dim3 blk(32, 4);
  AdjConsts k;
  k.tau = tau;
  k.om = 1.0 / tau;
  k.om2 = k.om * k.om;
  k.om1 = 1.0 - k.om;
  k.om_c = k.om * C;
  k.om_c2 = k.om * C2;
  k.tgx = tau * gx;
  k.tgy = tau * gy;
  const double gg = gx * gx + gy * gy;
  k.tshift = tau * (1.0 - tau) * gg / D - 1.0;
  k.gx = gx;
  k.gy = gy;
  k.dts_dtau = (1.0 - 2.0 * tau) * gg / D;
  if (a.periodic) {
    k_adj_collide<true><<<site_grid(a), blk, 0, s>>>(fin, lam_next, lam, side, part, a, k);
  } else {
    k_adj_collide<false><<<site_grid(a), blk, 0, s>>>(fin, lam_next, lam, side, part, a, k);
    const long long items = 2LL * a.lx * Q;  // (column, wall, population), plus one block for the dtau sum
    k_adj_walls<<<(unsigned)((items + 255) / 256) + 1, 256, 0, s>>>(side, lam, a, part, adjoint_partial_count(a),
                                                                    dtau);
    return cudaGetLastError();
  }
  k_reduce_add<<<1, 256, 0, s>>>(part, adjoint_partial_count(a), dtau);
  return cudaGetLastError();
}

cudaError_t launch_ke_grad(const double* f, double* lam, const StepArgs& a, cudaStream_t s) {
  k_ke_grad<<<site_grid(a), dim3(32, 4), 0, s>>>(f, lam, a);
  return cudaGetLastError();
}

cudaError_t launch_init_adjoint(const double* rho, const double* ux, const double* uy, const double* T,
                                const double* lam, double* g_rho, double* g_ux, double* g_uy, double* g_T,
                                const StepArgs& a, cudaStream_t s) {
  k_init_adjoint<<<site_grid(a), dim3(32, 4), 0, s>>>(rho, ux, uy, T, lam, g_rho, g_ux, g_uy, g_T, a);
  return cudaGetLastError();
}

}  // namespace d2q37

using namespace d2q37;

namespace {

int32_t status_of(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ECUDA; }

bool a16(const void* p) { return p && ((uintptr_t)p % 16) == 0; }
bool a8(const void* p) { return p && ((uintptr_t)p % 8) == 0; }

}  // namespace

extern "C" {

int64_t lbm_adjoint_work_bytes(const lbm_params* p) {
  if (!params_valid(p) || p->precision != LBM_FP64) return -1;
  const StepArgs a = make_step_args(p);
  return (adjoint_side_count(a) + adjoint_partial_count(a)) * (int64_t)sizeof(double);
}

int32_t lbm_adjoint_step(const lbm_params* p, const void* f_n, const void* lam_next, void* lam_n, double* dtau_accum,
                         void* work, size_t work_bytes, void* stream) {
  if (!params_valid(p) || p->precision != LBM_FP64 || !a16(f_n) || !a16(lam_next) || !a16(lam_n) ||
      !a8(dtau_accum) || !a16(work))
    return LBM_EINVAL;
  const int64_t need = lbm_adjoint_work_bytes(p);
  if ((int64_t)work_bytes < need || lam_next == lam_n || f_n == lam_n) return LBM_EINVAL;
  const StepArgs a = make_step_args(p);
  double* side = (double*)work;
  double* part = side + adjoint_side_count(a);
  return status_of(launch_adjoint_step((const double*)f_n, (const double*)lam_next, (double*)lam_n, side, part,
                                       dtau_accum, a, p->tau, p->gx, p->gy, (cudaStream_t)stream));
}

int32_t lbm_kinetic_energy_grad(const lbm_params* p, const void* f, void* lam, void* stream) {
  if (!params_valid(p) || p->precision != LBM_FP64 || !a16(f) || !a16(lam) || f == lam) return LBM_EINVAL;
  const StepArgs a = make_step_args(p);
  return status_of(launch_ke_grad((const double*)f, (double*)lam, a, (cudaStream_t)stream));
}

int32_t lbm_init_adjoint(const lbm_params* p, const double* rho, const double* ux, const double* uy, const double* T,
                         const void* lam0, double* g_rho, double* g_ux, double* g_uy, double* g_T, void* stream) {
  if (!params_valid(p) || p->precision != LBM_FP64 || !a8(rho) || !a8(ux) || !a8(uy) || !a8(T) || !a16(lam0) ||
      !a8(g_rho) || !a8(g_ux) || !a8(g_uy) || !a8(g_T))
    return LBM_EINVAL;
  const StepArgs a = make_step_args(p);
  return status_of(launch_init_adjoint(rho, ux, uy, T, (const double*)lam0, g_rho, g_ux, g_uy, g_T, a,
                                       (cudaStream_t)stream));
}

}  // extern "C"
