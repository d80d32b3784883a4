// 64-bit fixed-point arithmetic on the integer pipes.
//
// GB300 executes float64 at 2 operations per clock per SM, 1/64 of its float32 rate, while
// its integer pipes issue 64 operations per clock per SM.  A signed or unsigned 64 x 64 ->
// high-64 product (a handful of IMAD instructions) then costs a fraction of one DFMA.  The
// helpers below move values between float64 and signed 64-bit fixed point (value = X * 2^-k)
// with integer instructions, except fx_to_double_dp, which uses the float64 pipe's I2F on
// purpose (that pipe is otherwise idle in the fixed-point kernels).
#pragma once
#include <stdint.h>

namespace d2q37 {

// round(v * 2^k) for a float64 v, as a signed 64-bit integer; integer instructions only.
// v * 2^k = m * 2^sh with m the 53-bit significand.  Left shifts (sh >= 0) are exact;
// right shifts round half away from zero.  The result is valid for sh <= 10, i.e.
// |v| * 2^k < 2^63 (callers guarantee it); `ovf` is set when sh > max_sh, for callers that
// check a tighter format bound instead.  Zeros and subnormals give 0.
__host__ __device__ __forceinline__ long long fx_from_double(double v, int k, int max_sh, bool& ovf) {
#ifdef __CUDA_ARCH__
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
#else
  unsigned long long b;
  __builtin_memcpy(&b, &v, 8);
#endif
  const int E = (int)((b >> 52) & 0x7ffu);
  const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
  const int sh = E - 1075 + k;
  ovf |= sh > max_sh;
  const int l = sh < 0 ? 0 : (sh < 10 ? sh : 10);
  const int r = sh < 0 ? (-sh < 62 ? -sh : 62) : 0;
  const long long half = r > 0 ? (1LL << (r - 1)) : 0;
  long long x = ((m + half) >> r) << l;
  x = E == 0 ? 0 : x;
  const long long s = (long long)b >> 63;  // 0 or -1
  return (x ^ s) - s;
}

// X * 2^-k as a float64, rounded half up in magnitude; integer instructions only.  (The
// kernels use fx_to_double_dp below, which balances their pipes better; this form is the
// integer-pipe alternative.)
// Valid for 0 < 1086 - clz(|X|) - k < 2047 (normal results), which holds for every use here.
__host__ __device__ __forceinline__ double fx_to_double(long long X, int k) {
  const long long s = X >> 63;
  const unsigned long long A = (unsigned long long)((X ^ s) - s);
#ifdef __CUDA_ARCH__
  const int lz = __clzll((long long)A);
#else
  const int lz = A ? __builtin_clzll(A) : 64;
#endif
  const unsigned long long M = A << (lz & 63);
  const unsigned long long mant = ((M >> 10) + 1) >> 1;  // 53 bits, may carry to 2^53
  const unsigned long long e = (unsigned long long)(1086 - lz - k - 1);
  unsigned long long bits = (e << 52) + mant;
  bits |= (unsigned long long)s & 0x8000000000000000ull;
  bits = A == 0 ? 0ull : bits;
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)bits);
#else
  double d;
  __builtin_memcpy(&d, &bits, 8);
  return d;
#endif
}

// X * 2^-k through the float64 pipe: one I2F (exact round to nearest) and an integer
// subtraction from the exponent field.  Valid for normal results; 0 stays 0.  Used to move
// part of the conversion work from the integer pipes to the otherwise idle float64 pipe.
__device__ __forceinline__ double fx_to_double_dp(long long X, int k) {
  const long long b = __double_as_longlong(__ll2double_rn(X)) - ((long long)k << 52);
  return X == 0 ? 0.0 : __longlong_as_double(b);
}

// The same for 0 <= k <= 1022 without a test for zero: the I2F result's high word h is 0
// for X = 0 and at least 0x3FF00000 otherwise (|X| >= 1; a sign bit makes it larger
// still), so subtracting min(h, k << 20) leaves 0 at 0 and lowers the exponent field of
// every other value by k.
// (The host build, for the tests, converts with the host's round-to-nearest cast.)
__host__ __device__ __forceinline__ double fx_to_double_dp_pos(long long X, int k) {
#ifdef __CUDA_ARCH__
  const double d = __ll2double_rn(X);
  const unsigned h = (unsigned)__double2hiint(d), K = (unsigned)k << 20;
  return __hiloint2double((int)(h - min(h, K)), __double2loint(d));
#else
  const double d = (double)X;
  unsigned long long b;
  __builtin_memcpy(&b, &d, 8);
  const unsigned h = (unsigned)(b >> 32), K = (unsigned)k << 20;
  b = ((unsigned long long)(h - (h < K ? h : K)) << 32) | (b & 0xFFFFFFFFull);
  double r;
  __builtin_memcpy(&r, &b, 8);
  return r;
#endif
}

// f' = f 2^(59 + e) for a population whose value is an integer there: with the exponent
// field E, sh = E - 1016 + e is the left shift of the 53-bit significand, and
// 2^-7 <= f 2^e < 8 is 0 <= sh <= 9 (one unsigned compare, which also fails for negative
// values, zeros, subnormals and non-finite ones).  fx_exact_shift returns whether f is in
// that range; fx_from_double_shifted forms the integer with two funnel shifts.
__host__ __device__ __forceinline__ unsigned fx_hi_word(double f) {
#ifdef __CUDA_ARCH__
  return (unsigned)__double2hiint(f);
#else
  unsigned long long b;
  __builtin_memcpy(&b, &f, 8);
  return (unsigned)(b >> 32);
#endif
}
__host__ __device__ __forceinline__ unsigned fx_lo_word(double f) {
#ifdef __CUDA_ARCH__
  return (unsigned)__double2loint(f);
#else
  unsigned long long b;
  __builtin_memcpy(&b, &f, 8);
  return (unsigned)b;
#endif
}
__host__ __device__ __forceinline__ bool fx_exact_shift(double f, int e, unsigned& sh) {
  sh = (fx_hi_word(f) >> 20) + (unsigned)e - 1016u;
  return sh <= 9u;
}
__host__ __device__ __forceinline__ long long fx_from_double_shifted(double f, unsigned sh) {
  const unsigned lo = fx_lo_word(f);
  const unsigned mh = (fx_hi_word(f) & 0xFFFFFu) | 0x100000u;
#ifdef __CUDA_ARCH__
  const unsigned xh = __funnelshift_l(lo, mh, sh);
#else
  const unsigned xh = (unsigned)((((unsigned long long)mh << 32) | lo) << (sh & 31u) >> 32);
#endif
  const unsigned xl = lo << (sh & 31u);  // sh <= 9 in range
  return (long long)(((unsigned long long)xh << 32) | xl);
}

// High 64 bits of the 128-bit products.
__host__ __device__ __forceinline__ long long fx_mulhi(long long a, long long b) {
#ifdef __CUDA_ARCH__
  return __mul64hi(a, b);
#else
  return (long long)(((__int128)a * (__int128)b) >> 64);
#endif
}
__host__ __device__ __forceinline__ unsigned long long fx_umulhi(unsigned long long a, unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (unsigned long long)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
#endif
}
// The high 64 bits of a b without the low partial product a0 b0 and without the carries
// out of the low halves of the two cross products (a = a1 2^32 + a0, b = b1 2^32 + b0):
// a1 b1 + hi(a1 b0) + hi(a0 b1), which is the floor of a b / 2^64 minus 0, 1 or 2
// (about 3/4 on average for uniform operands: the floor of the sum of the two dropped
// low halves and a0 b0 / 2^64).
__host__ __device__ __forceinline__ unsigned long long fx_umulhi_approx(unsigned long long a, unsigned long long b) {
  const unsigned a0 = (unsigned)a, a1 = (unsigned)(a >> 32), b0 = (unsigned)b, b1 = (unsigned)(b >> 32);
  const unsigned h1 = (unsigned)(((unsigned long long)a1 * b0) >> 32);
  const unsigned h2 = (unsigned)(((unsigned long long)a0 * b1) >> 32);
  return (unsigned long long)a1 * b1 + h1 + h2;
}
__host__ __device__ __forceinline__ long long fx_mulhi_su_approx(long long a, unsigned long long b) {
  const unsigned long long h = fx_umulhi_approx((unsigned long long)a, b);
  return (long long)(a < 0 ? h - b : h);
}
__host__ __device__ __forceinline__ long long fx_mulhi_approx(long long a, long long b) {
  unsigned long long h = fx_umulhi_approx((unsigned long long)a, (unsigned long long)b);
  h -= a < 0 ? (unsigned long long)b : 0ull;
  h -= b < 0 ? (unsigned long long)a : 0ull;
  return (long long)h;
}
// Signed a times b with 0 <= b < 2^63: the unsigned product of a's bit pattern is
// (a + 2^64) b when a < 0, whose high half exceeds that of a b by exactly b.
__host__ __device__ __forceinline__ long long fx_mulhi_su(long long a, unsigned long long b) {
  const unsigned long long h = fx_umulhi((unsigned long long)a, b);
  return (long long)(a < 0 ? h - b : h);
}

}  // namespace d2q37
