// Compares the integer-pipe binary64 addition and multiplication of
// lbm_fp64emu.cuh with the host's own binary64 arithmetic, bit for bit, on
// operands drawn from families that reach every path: random bit patterns
// (zeros, subnormals, infinities, NaNs), normal operands at every exponent
// distance, cancelling sums, exact ties of both operations, products at the
// edges of the normal range, and values of the lattice's magnitudes.
//
//   fp64emu_check <cases per family> <seed>
// prints one line per family and exits 1 on the first mismatch.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <utility>

#include "lbm_fp64emu.cuh"

using olbm::emu::bits_of;
using olbm::emu::double_of;

namespace {

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double make(uint64_t sign, int e, uint64_t frac) {
  return double_of((sign << 63) | ((uint64_t)e << 52) | (frac & 0x000FFFFFFFFFFFFFull));
}

bool same(double x, double y) {
  if (std::isnan(x) && std::isnan(y)) return true;  // any NaN is a NaN
  return bits_of(x) == bits_of(y);
}

int check(const char* what, double a, double b) {
  volatile double va = a, vb = b;
  const double s = va + vb, p = va * vb;
  const double es = olbm::emu::add64(a, b), ep = olbm::emu::mul64(a, b);
  if (!same(s, es)) {
    std::printf("MISMATCH %s add a=%a b=%a host=%a emu=%a\n", what, a, b, s, es);
    return 1;
  }
  if (!same(p, ep)) {
    std::printf("MISMATCH %s mul a=%a b=%a host=%a emu=%a\n", what, a, b, p, ep);
    return 1;
  }
  // the product without its fallback: the same bits, or a NaN outside the fast path
  // (never for normal operands whose product lies well inside the normal range)
  const double eu = olbm::emu::mul64<false>(a, b), ez = olbm::emu::mul64<false, true>(a, b);
  const bool inside = std::isnormal(a) && std::isnormal(b) && std::fabs(p) > 0x1p-1020 && std::fabs(p) < 0x1p+1022;
  const bool zero_in = (a == 0 && (std::isnormal(b) || b == 0)) || (b == 0 && std::isnormal(a));
  if (!(same(p, eu) || (std::isnan(eu) && !inside))) {
    std::printf("MISMATCH %s unchecked mul a=%a b=%a host=%a emu=%a\n", what, a, b, p, eu);
    return 1;
  }
  if (!(same(p, ez) || (std::isnan(ez) && !inside && !zero_in))) {
    std::printf("MISMATCH %s unchecked mul with zeros a=%a b=%a host=%a emu=%a\n", what, a, b, p, ez);
    return 1;
  }
  return 0;
}

}  // namespace

int main(int argc, char** argv) {
  const long n = argc > 1 ? std::atol(argv[1]) : 1000000;
  uint64_t st = argc > 2 ? std::strtoull(argv[2], nullptr, 10) : 1;
  const int kFamilies = 10;
  const char* names[kFamilies] = {"random bits", "normal, any distance", "cancelling", "add ties",
                                  "mul ties and exact", "range edges", "lattice magnitudes", "near one",
                                  "zeros and specials", "special pairs"};
  const double special[] = {0.0, -0.0, 1.0, -1.0, 0.5, 3.0, -0.1, 1e-300, -1e300, 0x1p-1022, -0x1p-1022,
                            0x1p-1074, -0x1p-1074, 0x1.8p-1060, 0x1.fffffffffffffp+1023, -0x1.fffffffffffffp+1023,
                            HUGE_VAL, -HUGE_VAL, NAN, -NAN};
  const int nspecial = (int)(sizeof special / sizeof special[0]);
  for (int fam = 0; fam < kFamilies; ++fam) {
    for (long i = 0; i < n; ++i) {
      const uint64_t r0 = splitmix(st), r1 = splitmix(st), r2 = splitmix(st);
      double a = 0, b = 0;
      switch (fam) {
        case 0:
          a = double_of(r0), b = double_of(r1);
          break;
        case 1: {
          const int ea = 1 + (int)(r2 % 2046);
          const int d = (int)((r2 >> 16) % 72);
          const int eb = ea - d >= 1 ? ea - d : 1;
          a = make(r0 >> 63, ea, r0), b = make(r1 >> 63, eb, r1);
          if (r2 >> 63) std::swap(a, b);
          break;
        }
        case 2: {
          // b = -(a with a few low bits changed), or a neighbour one exponent down
          const int ea = 2 + (int)(r2 % 2040);
          const uint64_t flip = r1 & ((1ull << ((r2 >> 12) % 53)) - 1);
          a = make(r0 >> 63, ea, r0);
          b = make((r0 >> 63) ^ 1, (r2 >> 40) & 1 ? ea - 1 : ea, r0 ^ flip);
          break;
        }
        case 3: {
          // b sits at half an ulp of a, or at an odd multiple of it
          const int ea = 60 + (int)(r2 % 1900);
          const int d = 52 + (int)((r2 >> 20) % 4);
          const uint64_t fb = (r2 >> 30) & 1 ? 0 : (r1 & 0xFFFFull) << 36;
          a = make(r0 >> 63, ea, r0), b = make(r1 >> 63, ea - d, fb);
          break;
        }
        case 4: {
          // significands of at most 27 bits: products of 54 bits or fewer, exact or exact ties
          const int k = 1 + (int)(r2 % 27);
          const uint64_t ma = (r0 >> (64 - k)) | 1u, mb = (r1 >> (64 - k)) | 1u;
          const int ea = 700 + (int)((r2 >> 8) % 600), eb = 700 + (int)((r2 >> 24) % 600);
          a = make(r0 & 1, ea, ma << (52 - k + 1)), b = make(r1 & 1, eb, mb << (52 - k + 1));
          break;
        }
        case 5: {
          // exponents whose product lands near the bottom or the top of the normal range
          const int lowhigh = (int)(r2 & 1);
          const int ea = 1 + (int)((r2 >> 4) % 2046);
          int eb = lowhigh ? 2046 + 1023 - ea + (int)((r2 >> 20) % 5) - 2 : 1023 + 1 - ea + (int)((r2 >> 20) % 5) - 2;
          eb = eb < 1 ? 1 : (eb > 2046 ? 2046 : eb);
          a = make(r0 >> 63, ea, r0), b = make(r1 >> 63, eb, r1);
          if ((r2 >> 40) & 1) b = -a * 0.75;  // sums at the edges too
          break;
        }
        case 6: {
          // populations, moments, velocities and their products in the step
          const double u0 = (double)(r0 >> 11) * 0x1p-53, u1 = (double)(r1 >> 11) * 0x1p-53;
          const double scale[4] = {1.0, 0.5, 0.1, 0.01};
          a = (u0 - 0.25) * scale[r2 & 3];
          b = (u1 - 0.5) * scale[(r2 >> 2) & 3];
          if ((r2 >> 8) % 5 == 0) b = -a + (u1 - 0.5) * 1e-9;
          break;
        }
        case 7: {
          const double u0 = (double)(r0 >> 11) * 0x1p-53;
          a = 1.0 + (u0 - 0.5) * 1e-6;
          b = (r2 & 1) ? -1.0 : 1.0 / 3.0;
          break;
        }
        case 8: {
          // a special value against a random normal one
          a = special[r2 % nspecial];
          b = make(r1 >> 63, 1 + (int)((r1 >> 20) % 2046), r0);
          break;
        }
        case 9: {
          // every pair of special values
          a = special[i % nspecial];
          b = special[(i / nspecial) % nspecial];
          break;
        }
      }
      if (check(names[fam], a, b) || check(names[fam], b, a)) return 1;
    }
    std::printf("%-22s %ld cases: all equal\n", names[fam], n);
  }
  return 0;
}
