// Host build of the fixed-point helpers of the FP64 fixed-point relaxation, for the CPU
// tests: reads commands from stdin and prints results, one per line.
//   from <v as hex bits> <k>        -> fx_from_double(v, k) (decimal)
//   to <X decimal> <k>              -> fx_to_double(X, k) (hex bits)
//   top <X decimal> <k>             -> fx_to_double_dp_pos(X, k) (hex bits)
//   exact <v as hex bits> <e>       -> in-range flag and fx_from_double_shifted (decimal)
//   mulsu <a decimal> <b decimal>   -> fx_mulhi_su(a, b)
//   mul <a decimal> <b decimal>     -> fx_mulhi(a, b)
//   umul <a decimal> <b decimal>    -> fx_umulhi(a, b)
//   uapx <a decimal> <b decimal>    -> fx_umulhi_approx(a, b)
//   sapx <a decimal> <b decimal>    -> fx_mulhi_approx(a, b)
//   suapx <a decimal> <b decimal>   -> fx_mulhi_su_approx(a, b)
//   const                           -> the shell constants, one shell per line
//   rn <X decimal> <k>              -> fix_to_double_rn(X, k) (hex bits)
//   p2 <v as hex bits> <k>          -> pow2_scale(v, k) (hex bits)
#include <cstdio>
#include <cstring>
#include <cstdlib>

#include "../../paper_1703_04594_gb300/csrc/collide_fix64.cuh"

using namespace d2q37;

int main() {
  char cmd[16];
  while (std::scanf("%15s", cmd) == 1) {
    if (!std::strcmp(cmd, "from")) {
      unsigned long long bits;
      int k;
      std::scanf("%llx %d", &bits, &k);
      double v;
      std::memcpy(&v, &bits, 8);
      bool ovf = false;
      const long long r = fx_from_double(v, k, 64, ovf);
      std::printf("%lld\n", r);
    } else if (!std::strcmp(cmd, "to")) {
      long long X;
      int k;
      std::scanf("%lld %d", &X, &k);
      const double d = fx_to_double(X, k);
      unsigned long long bits;
      std::memcpy(&bits, &d, 8);
      std::printf("%016llx\n", bits);
    } else if (!std::strcmp(cmd, "rn")) {
      long long X;
      int k;
      std::scanf("%lld %d", &X, &k);
      const double d = fix_to_double_rn(X, k);
      unsigned long long bits;
      std::memcpy(&bits, &d, 8);
      std::printf("%llx\n", bits);
    } else if (!std::strcmp(cmd, "p2")) {
      unsigned long long vb;
      int k;
      std::scanf("%llx %d", &vb, &k);
      double v;
      std::memcpy(&v, &vb, 8);
      const double d = pow2_scale(v, k);
      unsigned long long bits;
      std::memcpy(&bits, &d, 8);
      std::printf("%llx\n", bits);
    } else if (!std::strcmp(cmd, "top")) {
      long long X;
      int k;
      std::scanf("%lld %d", &X, &k);
      const double d = fx_to_double_dp_pos(X, k);
      unsigned long long bits;
      std::memcpy(&bits, &d, 8);
      std::printf("%016llx\n", bits);
    } else if (!std::strcmp(cmd, "exact")) {
      unsigned long long bits;
      int e;
      std::scanf("%llx %d", &bits, &e);
      double v;
      std::memcpy(&v, &bits, 8);
      unsigned sh;
      const bool ok = fx_exact_shift(v, e, sh);
      std::printf("%d %lld\n", ok ? 1 : 0, ok ? fx_from_double_shifted(v, sh) : 0LL);
    } else if (!std::strcmp(cmd, "mulsu")) {
      long long a;
      unsigned long long b;
      std::scanf("%lld %llu", &a, &b);
      std::printf("%lld\n", fx_mulhi_su(a, b));
    } else if (!std::strcmp(cmd, "mul")) {
      long long a, b;
      std::scanf("%lld %lld", &a, &b);
      std::printf("%lld\n", fx_mulhi(a, b));
    } else if (!std::strcmp(cmd, "umul")) {
      unsigned long long a, b;
      std::scanf("%llu %llu", &a, &b);
      std::printf("%llu\n", fx_umulhi(a, b));
    } else if (!std::strcmp(cmd, "uapx")) {
      unsigned long long a, b;
      std::scanf("%llu %llu", &a, &b);
      std::printf("%llu\n", fx_umulhi_approx(a, b));
    } else if (!std::strcmp(cmd, "sapx")) {
      long long a, b;
      std::scanf("%lld %lld", &a, &b);
      std::printf("%lld\n", fx_mulhi_approx(a, b));
    } else if (!std::strcmp(cmd, "suapx")) {
      long long a;
      unsigned long long b;
      std::scanf("%lld %llu", &a, &b);
      std::printf("%lld\n", fx_mulhi_su_approx(a, b));
    } else if (!std::strcmp(cmd, "const")) {
      for (int s = 0; s < 8; ++s)
        std::printf("%d %d %lld %lld %lld %llu\n", s, shell_exp(s), kCw(s), kCq(s), kCq2(s), kCw6(s));
    } else {
      return 2;
    }
  }
  return 0;
}
